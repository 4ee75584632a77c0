// RMS-ID over the UROI without any device allocation.
//
// Some callers cannot call cudaMalloc at all: hosts that own every byte of
// device memory through their own pool (a framework's caching allocator, a
// treatment-planning system with a fixed device budget) and loops where
// allocation is forbidden.  cgdir_rms_id needs a context, whose workspace is
// allocated; this entry point instead keeps its scratch -- the per-CTA
// partial sums, a completion counter and the result -- in a file-scope
// __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.  The caller still passes the inputs.
//
// Host code must not use the array's name as a device address (it is a host
// stand-in for the symbol): the array's real address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call on that
// device and again whenever the device's current CUDA context is not the one
// the address was taken in (cudaDeviceReset, or another context made
// current, can load the module at another address).  Every call shares the
// one array, so calls whose work overlaps on the GPU (two streams, two
// threads) race and give undefined results; calls on one stream are ordered
// and safe.  The counter is cleared at the start of every call.
#include "cgdir_internal.cuh"

#include <cuda.h>

#include <cmath>
#include <mutex>

namespace {

constexpr int kNT = 256;
constexpr int kMaxBlocks = 4096;                 // partials held in the array
constexpr int kVoxelsPerThread = 64;             // voxels per thread at the largest volume
constexpr long long kMaxVoxels = (long long)kMaxBlocks * kNT * kVoxelsPerThread;   // 67,108,864
// layout (doubles): [0, 4*kMaxBlocks) partials {ssd, count, -, -};
// [4*kMaxBlocks] completion counter (as unsigned); [4*kMaxBlocks + 2 ..] result {ssd, count}
constexpr int kCounterSlot = 4 * kMaxBlocks;
constexpr int kResultSlot = 4 * kMaxBlocks + 2;
constexpr int kScratchDoubles = 4 * kMaxBlocks + 8;

static __device__ __align__(256) double g_rms_scratch[kScratchDoubles];

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kNT) k_rms_noalloc(const float *__restrict__ I0, const float *__restrict__ T0,
                                                     const float *__restrict__ u,
                                                     const uint8_t *__restrict__ uroi, int nx, int ny, int nz,
                                                     double *scratch) {
    const size_t N = (size_t)nx * ny * nz;
    double ssd = 0.0;                            // FP64 per thread, like the block and grid sums
    int cnt = 0;
    for (size_t i = (size_t)blockIdx.x * kNT + threadIdx.x; i < N; i += (size_t)gridDim.x * kNT) {
        if (uroi && !uroi[i]) continue;
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const cgdir::Corners c = cgdir::corners((float)x + __ldg(u + i), (float)y + __ldg(u + N + i),
                                                (float)z + __ldg(u + 2 * N + i), nx, ny, nz);
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int cx = (q & 1) ? c.x1 : c.x0, cy = (q & 2) ? c.y1 : c.y0, cz = (q & 4) ? c.z1 : c.z0;
            const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                            ((q & 4) ? c.wz : 1.f - c.wz);
            acc = fmaf(w, __ldg(I0 + cgdir::vox(cx, cy, cz, nx, ny)), acc);
        }
        const double r = (double)(__ldg(T0 + i) - acc);
        ssd = fma(r, r, ssd);
        cnt += 1;
    }
    // fixed-order block sum in FP64
    __shared__ double ws[kNT / 32], wc[kNT / 32];
    __shared__ int last;
    double s = warp_sum_d(ssd), k = warp_sum_d((double)cnt);
    if ((threadIdx.x & 31) == 0) { ws[threadIdx.x >> 5] = s; wc[threadIdx.x >> 5] = k; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < kNT / 32; ++w) { a += ws[w]; b += wc[w]; }
        scratch[4 * blockIdx.x] = a;
        scratch[4 * blockIdx.x + 1] = b;
        __threadfence();
        unsigned *counter = reinterpret_cast<unsigned *>(scratch + kCounterSlot);
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the CTA that completes the grid sums the partials in block order
    __threadfence();
    __shared__ double ts[kNT], tc[kNT];
    double a = 0, b = 0;
    for (unsigned blk = threadIdx.x; blk < gridDim.x; blk += kNT) {
        a += __ldcg(scratch + 4 * blk);
        b += __ldcg(scratch + 4 * blk + 1);
    }
    ts[threadIdx.x] = a;
    tc[threadIdx.x] = b;
    __syncthreads();
    for (int h = kNT / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) { ts[threadIdx.x] += ts[threadIdx.x + h]; tc[threadIdx.x] += tc[threadIdx.x + h]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[kResultSlot] = ts[0];
        scratch[kResultSlot + 1] = tc[0];
    }
}

// Current context's unique id through the driver entry points (resolved once).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

bool current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr, *q = nullptr;
        cudaDriverEntryPointQueryResult r1, r2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1) == cudaSuccess &&
            r1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2) == cudaSuccess &&
            r2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
            get_id = reinterpret_cast<CtxGetIdFn>(q);
        } else {
            cudaGetLastError();
        }
    });
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || c == nullptr) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_rms_scratch per device, with the id of the context it
// was looked up in; looked up again when the current context differs.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    double *ptr = nullptr;
    unsigned long long ctx_id = 0;
};
std::mutex g_mu;
ScratchAddr g_addr[kMaxDevices];

int scratch_for_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CGDIR_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr &a = g_addr[dev];
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);   // false before the runtime binds a context
    if (!a.ptr || !have_id || id != a.ctx_id) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_rms_scratch);   // binds the device's context
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            a.ptr = nullptr;
            return CGDIR_ECUDA;
        }
        if (!current_context_id(&id)) return CGDIR_ECUDA;
        a.ptr = static_cast<double *>(p);
        a.ctx_id = id;
    }
    *out = a.ptr;
    return CGDIR_OK;
}

}  // namespace

extern "C" int cgdir_rms_id_noalloc(const float *I0, const float *T0, const float *u, const uint8_t *uroi,
                                    int nx, int ny, int nz, void *stream, double *rms_host,
                                    long long *count_host) {
    if (!I0 || !T0 || !u || !rms_host || nx < 1 || ny < 1 || nz < 1) return CGDIR_EINVAL;
    const long long N = (long long)nx * ny * nz;
    if (N > kMaxVoxels) return CGDIR_EINVAL;           // beyond the fixed scratch: rejected
    double *scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st != CGDIR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long blocks = (N + (long long)kNT * 16 - 1) / ((long long)kNT * 16);
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    if (blocks < 1) blocks = 1;
    // the completion counter must start at zero; the result slots are rewritten
    if (cudaMemsetAsync(scratch + kCounterSlot, 0, 2 * sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return CGDIR_ECUDA;
    }
    k_rms_noalloc<<<(unsigned)blocks, kNT, 0, s>>>(I0, T0, u, uroi, nx, ny, nz, scratch);
    cgdir::note_launch();
    if (cudaGetLastError() != cudaSuccess) return CGDIR_ECUDA;
    double res[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(res, scratch + kResultSlot, sizeof res, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return CGDIR_ECUDA;
    }
    *rms_host = res[1] > 0 ? std::sqrt(res[0] / res[1]) : 0.0;
    if (count_host) *count_host = (long long)res[1];
    return CGDIR_OK;
}
