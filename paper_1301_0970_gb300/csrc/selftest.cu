// Self-test of the bounded-wait error path (an execution aid, not part of
// the paper's method).  One CTA waits on an mbarrier that nothing completes,
// with a short limit in clock cycles; when the limit runs out it records the
// timeout in the context's error word and returns -- what the TMA kernels do
// when a copy never lands.  Nothing faults or hangs: the wait is bounded.
#include "runtime_internal.hpp"
#include "tma.cuh"

using namespace cgdir;
using namespace cgdir::rt;

namespace {

__global__ void k_wait_timeout(long long limit_cycles, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        bool ok = mbar_try_wait(&bar, 0);
        while (!ok && clock64() - t0 <= limit_cycles) ok = mbar_try_wait(&bar, 0);
        if (!ok) atomicExch(err, 1);
    }
}

}  // namespace

extern "C" int cgdir_selftest_wait_timeout(cgdir_ctx *ctx, int limit_us) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->err.clear();
    if (limit_us < 1 || limit_us > 2000000) return fail(ctx, CGDIR_EINVAL, "selftest: limit_us must be 1..2000000");
    DeviceGuard g(ctx->device);
    // at most 2.1 GHz: the wait lasts at least limit_us
    const long long cycles = (long long)limit_us * 2100;
    k_wait_timeout<<<1, 32, 0, ctx->stream>>>(cycles, ctx->err_word);
    note_launch();
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return check_err_word(ctx);
}
