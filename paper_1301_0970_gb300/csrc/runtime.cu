// Runtime and C ABI of the CG-DIR library (include/cgdir.h): contexts,
// device workspace, the image pyramid, and Algorithm A (Sec. 2.2) driven as
// a fixed sequence of kernel launches on the context's stream.
//
// The per-iteration sequence at a level (u stays in one buffer):
//   force(u -> du) ; finalize(delta^n, stop test) ;
//   smooth+compose(du, u -> du2) ; smooth(du2 -> u)
// and after the level's cap a metric pass gives delta^cap.  The stopping
// decision is taken on the device (finalize sets the level's stop flag and
// every later kernel of the level returns at once), so a level never waits
// for the host.
#include "cgdir_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace cgdir;

struct WsBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct ProfPending {
    int cls, level;
    cudaEvent_t a, b;
};

// Event pairs recorded around profiled launches, with the events they use.
struct ProfList {
    std::vector<ProfPending> recs;
    std::vector<cudaEvent_t> pool;
    void release() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        pool.clear();
        recs.clear();
    }
};

// One instantiated CUDA graph of the device part of a registration.
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    ProfList prof;
    unsigned long long launches = 0;
};

struct cgdir_ctx {
    unsigned prof_mask = 0;
    ProfList eager;
    std::map<std::pair<int, int>, std::pair<long long, double>> prof;
    bool use_graphs = true;
    unsigned long long ws_generation = 0;
    std::map<std::string, GraphEntry> graphs;
    int device = 0;
    bool plain_kernels = false;   // CGDIR_KERNELS=plain at creation: no TMA kernels
    int *err_word = nullptr;      // device word set by a kernel whose bounded wait ran out
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream the graphs are captured on
    bool own_stream = false;
    size_t budget = 0;
    size_t in_use = 0;
    std::string err;
    std::map<std::string, WsBuf> ws;
    std::vector<double> h_hist;
    std::vector<int> h_meta;
};

namespace cgdir {
static std::atomic<unsigned long long> g_launches{0};
void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int sm_count() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev] = n;
    return n;
}

int pick_zchunk(int nz, long xy_ctas, int resident_per_sm, int waves) {
    const long target = (long)waves * resident_per_sm * sm_count();
    long chunks = (target + xy_ctas - 1) / (xy_ctas > 0 ? xy_ctas : 1);
    if (chunks < 1) chunks = 1;
    if (chunks > nz) chunks = nz;
    return (int)((nz + chunks - 1) / chunks);
}

cudaError_t ensure_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &have = done[{func, dev}];
    if (have >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}
}  // namespace cgdir

namespace {

// Event pair around one launch of class `cls` when that class is profiled.
struct ProfScope {
    ProfList *list = nullptr;
    cudaStream_t stream;
    int idx = -1;
    ProfScope(ProfList *l, unsigned mask, cudaStream_t s, int cls, int level) : stream(s) {
        if (!(mask & (1u << cls))) return;
        const size_t need = 2 * (l->recs.size() + 1);
        while (l->pool.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
            l->pool.push_back(e);
        }
        ProfPending p{cls, level, l->pool[need - 2], l->pool[need - 1]};
        // External: inside a stream capture this becomes an event-record node
        cudaEventRecordWithFlags(p.a, s, cudaEventRecordExternal);
        l->recs.push_back(p);
        list = l;
        idx = (int)l->recs.size() - 1;
    }
    ~ProfScope() {
        if (idx >= 0) cudaEventRecordWithFlags(list->recs[idx].b, stream, cudaEventRecordExternal);
    }
};

// After the stream has drained: fold the recorded pairs into the totals.
void prof_collect(cgdir_ctx *ctx, const ProfList &l) {
    for (const ProfPending &p : l.recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto &t = ctx->prof[{p.cls, p.level}];
            t.first += 1;
            t.second += ms;
        } else {
            cudaGetLastError();
        }
    }
}

void drop_graphs(cgdir_ctx *ctx) {
    for (auto &kv : ctx->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        kv.second.prof.release();
    }
    ctx->graphs.clear();
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(cgdir_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(expr)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, CGDIR_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                 \
    do {                          \
        int r_ = (expr);          \
        if (r_ != CGDIR_OK) return r_; \
    } while (0)

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Grow-only named device buffers.  Growing frees the old buffer after the
// stream has drained, so callers must re-fetch pointers after any ws_get.
int ws_get(cgdir_ctx *ctx, const char *name, size_t bytes, void **out) {
    WsBuf &b = ctx->ws[name];
    if (bytes == 0) bytes = 256;
    if (b.p && b.cap >= bytes) { *out = b.p; return CGDIR_OK; }
    const size_t cap = round_up(bytes, (size_t)1 << 21);
    const size_t after = ctx->in_use - b.cap + cap;
    if (ctx->budget && after > ctx->budget)
        return fail(ctx, CGDIR_ENOMEM, std::string("device budget exceeded growing '") + name + "'");
    if (b.p) {
        cudaStreamSynchronize(ctx->stream);
        drop_graphs(ctx);              // cached graphs hold the old address
        cudaFree(b.p);
        ctx->in_use -= b.cap;
        b = WsBuf{};
    }
    ++ctx->ws_generation;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, CGDIR_ENOMEM, std::string("cudaMalloc '") + name + "': " + cudaGetErrorString(e));
    }
    b.p = p;
    b.cap = cap;
    ctx->in_use += cap;
    *out = p;
    return CGDIR_OK;
}

bool dims_ok(int nx, int ny, int nz) { return nx >= 1 && ny >= 1 && nz >= 1; }

// Error word handed to kernels with bounded waits; nullptr selects the
// plain-load kernels.
int *kerr(cgdir_ctx *ctx) { return ctx->plain_kernels ? nullptr : ctx->err_word; }

// After the stream has drained: a kernel wait that ran out is a timeout.
int check_err_word(cgdir_ctx *ctx) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, ctx->err_word, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(ctx, CGDIR_ECUDA, std::string("error word: ") + cudaGetErrorString(e));
    if (h) {
        cudaMemset(ctx->err_word, 0, sizeof(int));
        return fail(ctx, CGDIR_ETIMEDOUT, "a bounded wait inside a kernel ran out (TMA load not completed)");
    }
    return CGDIR_OK;
}

bool sigma_ok(float s) { return std::isfinite(s) && s >= 0.f && s <= CGDIR_MAX_SIGMA; }

size_t elem_size(int dtype) { return dtype == CGDIR_F32 ? 4 : 2; }

int fill_force_args(cgdir_ctx *ctx, ForceArgs &a, int k, const float *lambda, const int8_t *sign,
                    float offset, int contour) {
    if (k < 0 || k > kMaxMasks) return fail(ctx, CGDIR_EINVAL, "mask count must be 0..8");
    if (!std::isfinite(offset)) return fail(ctx, CGDIR_EINVAL, "intensity offset must be finite");
    a.k = k;
    a.contour = contour ? 1 : 0;
    a.offset = offset;
    for (int j = 0; j < kMaxMasks; ++j) { a.lambda[j] = 0.f; a.half_sign[j] = 0.5f; }
    for (int j = 0; j < k; ++j) {
        const float l = lambda ? lambda[j] : 1e-3f;
        if (!(std::isfinite(l) && l >= 0.f)) return fail(ctx, CGDIR_EINVAL, "lambda must be finite and >= 0");
        a.lambda[j] = l;
        if (sign && sign[j] != 1 && sign[j] != -1)
            return fail(ctx, CGDIR_EINVAL, "sign must be +1 or -1 for the primitives");
        a.half_sign[j] = sign ? 0.5f * (float)sign[j] : 0.5f;
    }
    return CGDIR_OK;
}

}  // namespace

// ======================================================================
extern "C" {

void cgdir_default_params(cgdir_params *p) {
    if (!p) return;
    static const int kIters[2] = {100, 50};
    std::memset(p, 0, sizeof(*p));
    p->levels = 2;
    p->iters = kIters;
    p->sigma_fluid = 1.f;
    p->sigma_diff = 1.f;
    p->lambda = nullptr;
    p->sign = nullptr;
    p->contour_level_mask = 1u << 1;
    p->stop_mode = CGDIR_STOP_WINDOW10;
    p->eps = 1e-4;
    p->spacing_mm[0] = 1.97;
    p->spacing_mm[1] = 1.97;
    p->spacing_mm[2] = 2.5;
    p->margin_mm = 10.0;
    p->intensity_offset = 1000.f;
    p->compose_mode = CGDIR_COMPOSE;
    p->init_dvf = nullptr;
    p->init_dvf_where = CGDIR_DEVICE;
    p->storage_dtype = CGDIR_STORAGE_AUTO;
}

const char *cgdir_strerror(int s) {
    switch (s) {
        case CGDIR_OK: return "ok";
        case CGDIR_EINVAL: return "invalid argument";
        case CGDIR_ENOMEM: return "out of device memory or budget";
        case CGDIR_ECUDA: return "CUDA error";
        case CGDIR_ETIMEDOUT: return "timed out";
        case CGDIR_ECANCELED: return "cancelled";
        case CGDIR_EBUSY: return "busy";
        default: return "unknown status";
    }
}

const char *cgdir_last_error(const cgdir_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t cgdir_mem_in_use(const cgdir_ctx *ctx) { return ctx ? ctx->in_use : 0; }

unsigned long long cgdir_launch_count(void) { return g_launches.load(); }

int cgdir_sync(cgdir_ctx *ctx) {
    if (!ctx) return CGDIR_EINVAL;
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    return check_err_word(ctx);
}

int cgdir_profile(cgdir_ctx *ctx, unsigned kernel_mask) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->prof_mask = kernel_mask & ((1u << CGDIR_K_COUNT) - 1u);
    ctx->prof.clear();
    return CGDIR_OK;
}

int cgdir_profile_read(const cgdir_ctx *ctx, cgdir_kernel_time *out, int cap) {
    if (!ctx || (cap > 0 && !out)) return -CGDIR_EINVAL;
    int n = 0;
    for (const auto &kv : ctx->prof) {
        if (n >= cap) break;
        out[n].kernel = kv.first.first;
        out[n].level = kv.first.second;
        out[n].launches = kv.second.first;
        out[n].total_ms = kv.second.second;
        ++n;
    }
    return n;
}

int cgdir_create(cgdir_ctx **out, const cgdir_config *cfg) {
    if (!out || !cfg) return CGDIR_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) { cudaGetLastError(); return CGDIR_ECUDA; }
    if (cfg->device < 0 || cfg->device >= n) return CGDIR_EINVAL;
    DeviceGuard g(cfg->device);
    cgdir_ctx *c = new cgdir_ctx();
    c->device = cfg->device;
    c->budget = cfg->mem_budget_bytes;
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return CGDIR_ECUDA;
        }
        c->own_stream = true;
    }
    const char *kern = std::getenv("CGDIR_KERNELS");
    c->plain_kernels = kern && std::strcmp(kern, "plain") == 0;
    const char *gr = std::getenv("CGDIR_GRAPHS");
    c->use_graphs = !(gr && std::strcmp(gr, "0") == 0);
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->use_graphs = false;
        c->cap_stream = nullptr;
    }
    if (cudaMalloc(&c->err_word, sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(c->err_word, 0, sizeof(int), c->stream) != cudaSuccess) {
        cudaGetLastError();
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return CGDIR_ECUDA;
    }
    *out = c;
    return CGDIR_OK;
}

void cgdir_destroy(cgdir_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->ws)
        if (kv.second.p) cudaFree(kv.second.p);
    drop_graphs(ctx);
    ctx->eager.release();
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->err_word) cudaFree(ctx->err_word);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// ---------------------------------------------------------------- primitives
int cgdir_pack_masks(cgdir_ctx *ctx, const uint8_t *const *masks, int k, size_t n, uint8_t *bits) {
    if (!ctx) return CGDIR_EINVAL;
    if (k < 0 || k > kMaxMasks || !bits || (k > 0 && !masks))
        return fail(ctx, CGDIR_EINVAL, "pack_masks: bad arguments");
    for (int j = 0; j < k; ++j)
        if (!masks[j]) return fail(ctx, CGDIR_EINVAL, "pack_masks: null mask pointer");
    DeviceGuard g(ctx->device);
    CK(launch_pack_masks(masks, k, n, bits, ctx->stream));
    return CGDIR_OK;
}

int cgdir_warp(cgdir_ctx *ctx, const float *f, const float *u, int nx, int ny, int nz, float *out) {
    if (!ctx) return CGDIR_EINVAL;
    if (!f || !u || !out || !dims_ok(nx, ny, nz)) return fail(ctx, CGDIR_EINVAL, "warp: bad arguments");
    DeviceGuard g(ctx->device);
    CK(launch_warp(f, u, nx, ny, nz, out, ctx->stream));
    return CGDIR_OK;
}

static int force_impl(cgdir_ctx *ctx, const ForceArgs &a, double *stats_host) {
    void *part = nullptr, *st = nullptr;
    ForceArgs b = a;
    const int zc = force_default_zchunk(a.nx, a.ny, a.nz);
    if (b.contour && b.k > 0 && !ctx->plain_kernels && b.mtex == nullptr) {
        // the TMA kernel gathers interleaved {I0, bits} texels
        const size_t N = (size_t)a.nx * a.ny * a.nz;
        void *tex = nullptr;
        TRY(ws_get(ctx, "force_tex", N * tex_elem_size(a.img_dtype), &tex));
        CK(launch_make_texels(a.I0, a.img_dtype, a.mbits, N, tex, ctx->stream));
        b.mtex = tex;
    }
    if (stats_host) {
        TRY(ws_get(ctx, "partial", force_partial_count(a.nx, a.ny, a.nz, zc) * kPartialStride * sizeof(double), &part));
        TRY(ws_get(ctx, "stats", 4 * sizeof(double), &st));
        b.partial = (double *)part;
    }
    int nb = 0;
    CK(launch_force(b, zc, &nb, ctx->stream, kerr(ctx)));
    if (stats_host) {
        LevelState ls{};
        CK(launch_finalize((double *)part, nb, ls, 0, 0, CGDIR_STOP_FIXED, 0.0, (double *)st, ctx->stream));
        CK(cudaMemcpyAsync(stats_host, st, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        TRY(check_err_word(ctx));
    }
    return CGDIR_OK;
}

int cgdir_force(cgdir_ctx *ctx, const float *I0, const float *T0, const uint8_t *mbits,
                const uint8_t *sbits, const uint8_t *uroi, int k, const float *lambda,
                const int8_t *sign, float offset, int contour, const float *u, int nx, int ny, int nz,
                float *du, float *warped, double *stats_host) {
    if (!ctx) return CGDIR_EINVAL;
    if (!I0 || !T0 || !u || !du || !dims_ok(nx, ny, nz))
        return fail(ctx, CGDIR_EINVAL, "force: bad arguments");
    const bool use_contour = contour && k > 0;
    if (use_contour && (!mbits || !sbits)) return fail(ctx, CGDIR_EINVAL, "force: mask bits required");
    ForceArgs a{};
    TRY(fill_force_args(ctx, a, k, lambda, sign, offset, use_contour));
    a.I0 = I0; a.T0 = T0; a.mbits = mbits; a.sbits = sbits; a.uroi = uroi; a.u = u; a.du = du;
    a.warped = warped; a.partial = nullptr; a.stop_flag = nullptr;
    a.nx = nx; a.ny = ny; a.nz = nz;
    DeviceGuard g(ctx->device);
    return force_impl(ctx, a, stats_host);
}

int cgdir_smooth(cgdir_ctx *ctx, const float *in, int ncomp, float sigma, int nx, int ny, int nz,
                 float *out) {
    if (!ctx) return CGDIR_EINVAL;
    if (!in || !out || in == out || ncomp < 1 || ncomp > 3 || !dims_ok(nx, ny, nz) || !sigma_ok(sigma))
        return fail(ctx, CGDIR_EINVAL, "smooth: bad arguments");
    DeviceGuard g(ctx->device);
    CK(launch_smooth(in, ncomp, sigma, nx, ny, nz, out, nullptr, ctx->stream, kerr(ctx)));
    return CGDIR_OK;
}

int cgdir_compose(cgdir_ctx *ctx, const float *u, const float *du, int mode, float sigma, int nx,
                  int ny, int nz, float *out) {
    if (!ctx) return CGDIR_EINVAL;
    if (!u || !du || !out || out == u || out == du || !dims_ok(nx, ny, nz) || !sigma_ok(sigma) ||
        (mode != CGDIR_COMPOSE && mode != CGDIR_ADDITIVE))
        return fail(ctx, CGDIR_EINVAL, "compose: bad arguments");
    DeviceGuard g(ctx->device);
    const size_t N = (size_t)nx * ny * nz;
    if (gauss_radius(sigma) == 0) {
        CK(launch_compose(u, du, mode, nx, ny, nz, out, nullptr, ctx->stream));
        return CGDIR_OK;
    }
    void *tmp = nullptr;
    TRY(ws_get(ctx, "field_tmp", 3 * N * sizeof(float), &tmp));
    CK(launch_compose(u, du, mode, nx, ny, nz, (float *)tmp, nullptr, ctx->stream));
    CK(launch_smooth((float *)tmp, 3, sigma, nx, ny, nz, out, nullptr, ctx->stream, kerr(ctx)));
    return CGDIR_OK;
}

int cgdir_iterate(cgdir_ctx *ctx, const float *I0, const float *T0, const uint8_t *mbits,
                  const uint8_t *sbits, const uint8_t *uroi, int k, const float *lambda,
                  const int8_t *sign, float offset, int contour, float sigma_fluid, float sigma_diff,
                  int compose_mode, const float *u_in, int nx, int ny, int nz, float *u_out,
                  float *du_out, double *stats_host) {
    if (!ctx) return CGDIR_EINVAL;
    if (!I0 || !T0 || !u_in || !u_out || u_in == u_out || !dims_ok(nx, ny, nz) ||
        !sigma_ok(sigma_fluid) || !sigma_ok(sigma_diff) ||
        (compose_mode != CGDIR_COMPOSE && compose_mode != CGDIR_ADDITIVE))
        return fail(ctx, CGDIR_EINVAL, "iterate: bad arguments");
    const bool use_contour = contour && k > 0;
    if (use_contour && (!mbits || !sbits)) return fail(ctx, CGDIR_EINVAL, "iterate: mask bits required");
    ForceArgs a{};
    TRY(fill_force_args(ctx, a, k, lambda, sign, offset, use_contour));
    DeviceGuard g(ctx->device);
    const size_t N = (size_t)nx * ny * nz;
    void *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
    TRY(ws_get(ctx, "iter_a", 3 * N * sizeof(float), &t1));
    TRY(ws_get(ctx, "iter_b", 3 * N * sizeof(float), &t2));
    TRY(ws_get(ctx, "iter_c", 3 * N * sizeof(float), &t3));
    float *du = (float *)t1, *un = (float *)t2;
    a.I0 = I0; a.T0 = T0; a.mbits = mbits; a.sbits = sbits; a.uroi = uroi; a.u = u_in; a.du = du;
    a.warped = nullptr; a.stop_flag = nullptr;
    a.nx = nx; a.ny = ny; a.nz = nz;
    TRY(force_impl(ctx, a, stats_host));
    if (du_out) {   // the smoothed du is wanted: steps 2 and 3 separately
        CK(launch_smooth(du, 3, sigma_fluid, nx, ny, nz, du_out, nullptr, ctx->stream, kerr(ctx)));
        CK(launch_compose(u_in, du_out, compose_mode, nx, ny, nz, un, nullptr, ctx->stream));
    } else {
        CK(launch_smooth_compose(du, u_in, compose_mode, sigma_fluid, nx, ny, nz, un, (float *)t3, nullptr,
                                 ctx->stream, kerr(ctx)));
    }
    CK(launch_smooth(un, 3, sigma_diff, nx, ny, nz, u_out, nullptr, ctx->stream, kerr(ctx)));
    return CGDIR_OK;
}

int cgdir_restrict_image(cgdir_ctx *ctx, const float *in, int nx, int ny, int nz, float *out) {
    if (!ctx) return CGDIR_EINVAL;
    if (!in || !out || !dims_ok(nx, ny, nz)) return fail(ctx, CGDIR_EINVAL, "restrict_image: bad arguments");
    DeviceGuard g(ctx->device);
    CK(launch_restrict_image(in, CGDIR_F32, nx, ny, nz, out, ctx->stream));
    return CGDIR_OK;
}

int cgdir_restrict_bits(cgdir_ctx *ctx, const uint8_t *in, int nx, int ny, int nz, uint8_t *out) {
    if (!ctx) return CGDIR_EINVAL;
    if (!in || !out || !dims_ok(nx, ny, nz)) return fail(ctx, CGDIR_EINVAL, "restrict_bits: bad arguments");
    DeviceGuard g(ctx->device);
    CK(launch_restrict_bits(in, nx, ny, nz, out, ctx->stream));
    return CGDIR_OK;
}

int cgdir_prolong(cgdir_ctx *ctx, const float *uc, int cx, int cy, int cz, int nx, int ny, int nz,
                  float *uf) {
    if (!ctx) return CGDIR_EINVAL;
    if (!uc || !uf || !dims_ok(cx, cy, cz) || !dims_ok(nx, ny, nz))
        return fail(ctx, CGDIR_EINVAL, "prolong: bad arguments");
    DeviceGuard g(ctx->device);
    CK(launch_prolong(uc, cx, cy, cz, nx, ny, nz, uf, ctx->stream));
    return CGDIR_OK;
}

int cgdir_uroi(cgdir_ctx *ctx, const uint8_t *sbits, int k, int nx, int ny, int nz,
               const double *spacing, double margin, uint8_t *out) {
    if (!ctx) return CGDIR_EINVAL;
    if (!out || !dims_ok(nx, ny, nz) || k < 0 || k > kMaxMasks || (k > 0 && (!sbits || !spacing)))
        return fail(ctx, CGDIR_EINVAL, "uroi: bad arguments");
    DeviceGuard g(ctx->device);
    void *rd = nullptr;
    TRY(ws_get(ctx, "rowdist", uroi_scratch_bytes((size_t)nx * ny * nz), &rd));
    const double sp1[3] = {1, 1, 1};
    cudaError_t e = launch_uroi(sbits, k, nx, ny, nz, spacing ? spacing : sp1, margin, (uint8_t *)rd, out,
                                ctx->stream);
    if (e == cudaErrorInvalidValue)
        return fail(ctx, CGDIR_EINVAL, "uroi: spacing must be > 0, margin >= 0, margin/spacing <= 15");
    CK(e);
    return CGDIR_OK;
}

static int auto_sign_impl(cgdir_ctx *ctx, const void *T0, int dtype, const uint8_t *sbits, int k, int nx,
                          int ny, int nz, int8_t *sign_host) {
    if (!ctx) return CGDIR_EINVAL;
    if (!T0 || !dims_ok(nx, ny, nz) || k < 0 || k > kMaxMasks || (k > 0 && (!sbits || !sign_host)))
        return fail(ctx, CGDIR_EINVAL, "auto_sign: bad arguments");
    if (k == 0) return CGDIR_OK;
    DeviceGuard g(ctx->device);
    const size_t N = (size_t)nx * ny * nz;
    void *ta = nullptr, *tb = nullptr, *part = nullptr, *sums = nullptr;
    TRY(ws_get(ctx, "sign_a", N, &ta));
    TRY(ws_get(ctx, "sign_b", N, &tb));
    TRY(ws_get(ctx, "sign_part", sign_partial_rows(N) * 4 * sizeof(double), &part));
    TRY(ws_get(ctx, "sign_sums", kMaxMasks * 4 * sizeof(double), &sums));
    CK(launch_sign_sums(T0, dtype, sbits, k, nx, ny, nz, (uint8_t *)ta, (uint8_t *)tb, (double *)part,
                        (double *)sums, ctx->stream));
    double h[kMaxMasks * 4];
    CK(cudaMemcpyAsync(h, sums, k * 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < k; ++j) {
        const double sin_ = h[4 * j], cin = h[4 * j + 1], ssh = h[4 * j + 2], csh = h[4 * j + 3];
        sign_host[j] = (cin == 0 || csh == 0) ? 1 : ((sin_ / cin >= ssh / csh) ? 1 : -1);
    }
    return CGDIR_OK;
}

int cgdir_auto_sign(cgdir_ctx *ctx, const float *T0, const uint8_t *sbits, int k, int nx, int ny,
                    int nz, int8_t *sign_host) {
    return auto_sign_impl(ctx, T0, CGDIR_F32, sbits, k, nx, ny, nz, sign_host);
}

int cgdir_rms_id(cgdir_ctx *ctx, const float *I0, const float *T0, const float *u,
                 const uint8_t *uroi, int nx, int ny, int nz, double *rms_host,
                 long long *count_host) {
    if (!ctx) return CGDIR_EINVAL;
    if (!I0 || !T0 || !u || !rms_host || !dims_ok(nx, ny, nz))
        return fail(ctx, CGDIR_EINVAL, "rms_id: bad arguments");
    DeviceGuard g(ctx->device);
    void *part = nullptr, *st = nullptr;
    TRY(ws_get(ctx, "partial_m", metric_partial_count(nx, ny, nz) * kPartialStride * sizeof(double), &part));
    TRY(ws_get(ctx, "stats", 4 * sizeof(double), &st));
    int nb = 0;
    CK(launch_metric(I0, T0, CGDIR_F32, u, uroi, nx, ny, nz, (double *)part, nullptr, &nb, ctx->stream));
    LevelState ls{};
    CK(launch_finalize((double *)part, nb, ls, 0, 0, CGDIR_STOP_FIXED, 0.0, (double *)st, ctx->stream));
    double h[3];
    CK(cudaMemcpyAsync(h, st, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *rms_host = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
    if (count_host) *count_host = (long long)h[1];
    return CGDIR_OK;
}

// ------------------------------------------------------------ registration
int cgdir_register(cgdir_ctx *ctx, const cgdir_volume *S, const cgdir_volume *M,
                   const cgdir_masks *SM, const cgdir_masks *MM, const cgdir_params *P,
                   float *dvf_out, int dvf_where, cgdir_level_stats *stats_out) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->err.clear();
    // ---- validation
    if (!S || !M || !P || !dvf_out) return fail(ctx, CGDIR_EINVAL, "register: null argument");
    if (!S->data || !M->data) return fail(ctx, CGDIR_EINVAL, "register: null image data");
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    if (!dims_ok(nx, ny, nz)) return fail(ctx, CGDIR_EINVAL, "register: image dimensions must be >= 1");
    if (M->nx != nx || M->ny != ny || M->nz != nz)
        return fail(ctx, CGDIR_EINVAL, "register: static and moving images differ in size");
    for (const cgdir_volume *v : {S, M}) {
        if (v->dtype != CGDIR_F32 && v->dtype != CGDIR_F16 && v->dtype != CGDIR_BF16)
            return fail(ctx, CGDIR_EINVAL, "register: unknown image dtype");
        if (v->where != CGDIR_HOST && v->where != CGDIR_DEVICE)
            return fail(ctx, CGDIR_EINVAL, "register: image 'where' must be HOST or DEVICE");
    }
    const int k = SM ? SM->count : 0;
    if ((MM ? MM->count : 0) != k) return fail(ctx, CGDIR_EINVAL, "register: static and moving mask counts differ");
    if (k < 0 || k > kMaxMasks) return fail(ctx, CGDIR_EINVAL, "register: mask count must be 0..8");
    for (const cgdir_masks *m : {SM, MM}) {
        if (k == 0) break;
        if (m->nx != nx || m->ny != ny || m->nz != nz)
            return fail(ctx, CGDIR_EINVAL, "register: masks must have the image size");
        if (m->where != CGDIR_HOST && m->where != CGDIR_DEVICE)
            return fail(ctx, CGDIR_EINVAL, "register: mask 'where' must be HOST or DEVICE");
        if (!m->data) return fail(ctx, CGDIR_EINVAL, "register: null mask array");
        for (int j = 0; j < k; ++j)
            if (!m->data[j]) return fail(ctx, CGDIR_EINVAL, "register: null mask pointer");
    }
    const int L = P->levels;
    if (L < 1 || L > CGDIR_MAX_LEVELS || !P->iters) return fail(ctx, CGDIR_EINVAL, "register: levels must be 1..8 with iters");
    int maxcap = 0;
    for (int l = 0; l < L; ++l) {
        if (P->iters[l] < 0 || P->iters[l] > 1000000) return fail(ctx, CGDIR_EINVAL, "register: iters must be 0..1e6");
        if (P->iters[l] > maxcap) maxcap = P->iters[l];
    }
    if (!sigma_ok(P->sigma_fluid) || !sigma_ok(P->sigma_diff))
        return fail(ctx, CGDIR_EINVAL, "register: sigma must be in [0, 2]");
    if (P->stop_mode < CGDIR_STOP_FIXED || P->stop_mode > CGDIR_STOP_PAPER_LITERAL || !std::isfinite(P->eps))
        return fail(ctx, CGDIR_EINVAL, "register: bad stop mode or eps");
    if (P->compose_mode != CGDIR_COMPOSE && P->compose_mode != CGDIR_ADDITIVE)
        return fail(ctx, CGDIR_EINVAL, "register: bad compose mode");
    for (int a = 0; a < 3; ++a)
        if (!(P->spacing_mm[a] > 0) || !std::isfinite(P->spacing_mm[a]))
            return fail(ctx, CGDIR_EINVAL, "register: spacing must be > 0");
    if (!(P->margin_mm >= 0) || !std::isfinite(P->margin_mm)) return fail(ctx, CGDIR_EINVAL, "register: margin must be >= 0");
    if (k > 0 && P->margin_mm / std::fmin(P->spacing_mm[0], std::fmin(P->spacing_mm[1], P->spacing_mm[2])) > 15.0)
        return fail(ctx, CGDIR_EINVAL, "register: UROI margin must be <= 15 voxels");
    if (dvf_where != CGDIR_HOST && dvf_where != CGDIR_DEVICE)
        return fail(ctx, CGDIR_EINVAL, "register: bad dvf_where");
    if (P->init_dvf && P->init_dvf_where != CGDIR_HOST && P->init_dvf_where != CGDIR_DEVICE)
        return fail(ctx, CGDIR_EINVAL, "register: bad init_dvf_where");
    if (P->storage_dtype < CGDIR_STORAGE_AUTO || P->storage_dtype > CGDIR_BF16)
        return fail(ctx, CGDIR_EINVAL, "register: bad storage_dtype");
    ForceArgs base{};
    {
        int8_t tmp_sign[kMaxMasks];
        for (int j = 0; j < kMaxMasks; ++j) tmp_sign[j] = 1;
        TRY(fill_force_args(ctx, base, k, P->lambda, tmp_sign, P->intensity_offset, 1));
    }

    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;

    // ---- sizes
    int dims[CGDIR_MAX_LEVELS][3];
    size_t Nl[CGDIR_MAX_LEVELS], off[CGDIR_MAX_LEVELS + 1];
    dims[L - 1][0] = nx; dims[L - 1][1] = ny; dims[L - 1][2] = nz;
    for (int l = L - 2; l >= 0; --l)
        for (int a = 0; a < 3; ++a) dims[l][a] = (dims[l + 1][a] + 1) / 2;
    off[0] = 0;
    for (int l = 0; l < L; ++l) {
        Nl[l] = (size_t)dims[l][0] * dims[l][1] * dims[l][2];
        off[l + 1] = off[l] + round_up(Nl[l], 64);
    }
    const size_t Nf = Nl[L - 1], Ntot = off[L];
    const int hcap = maxcap + 1;

    // ---- workspace
    void *p_img, *p_bits, *p_fields, *p_part, *p_state, *p_rowdist;
    // image storage type of the pyramid (float32, or 16-bit to halve the image bytes)
    const int sdt = P->storage_dtype >= 0 ? P->storage_dtype : (S->dtype == M->dtype ? S->dtype : CGDIR_F32);
    const size_t esz = img_elem_size(sdt), tsz = tex_elem_size(sdt);
    TRY(ws_get(ctx, "reg_img", 2 * Ntot * esz, &p_img));
    TRY(ws_get(ctx, "reg_bits", 3 * Ntot, &p_bits));
    void *p_tex = nullptr;
    TRY(ws_get(ctx, "reg_tex", Ntot * tsz, &p_tex));
    TRY(ws_get(ctx, "reg_fields", 4 * 3 * Nf * sizeof(float), &p_fields));
    size_t np = 0;
    for (int l = 0; l < L; ++l) {
        const size_t a = force_partial_count(dims[l][0], dims[l][1], dims[l][2],
                                             force_default_zchunk(dims[l][0], dims[l][1], dims[l][2]));
        const size_t b = metric_partial_count(dims[l][0], dims[l][1], dims[l][2]);
        np = std::max(np, std::max(a, b));
    }
    TRY(ws_get(ctx, "reg_partial", np * kPartialStride * sizeof(double), &p_part));
    const size_t state_bytes = (size_t)L * hcap * sizeof(double) + 5 * CGDIR_MAX_LEVELS * sizeof(int);
    TRY(ws_get(ctx, "reg_state", state_bytes, &p_state));
    TRY(ws_get(ctx, "rowdist", uroi_scratch_bytes(Nf), &p_rowdist));
    void *p_stage = nullptr;
    const bool need_stage = (S->where == CGDIR_HOST && S->dtype != sdt) ||
                            (M->where == CGDIR_HOST && M->dtype != sdt) ||
                            (k > 0 && (SM->where == CGDIR_HOST || MM->where == CGDIR_HOST));
    if (need_stage) TRY(ws_get(ctx, "reg_stage", std::max(Nf * 4, (size_t)k * Nf), &p_stage));
    // (re-fetch: a later ws_get may have reallocated an earlier name only if
    //  the same name was requested twice, which it is not)
    char *T[CGDIR_MAX_LEVELS], *I[CGDIR_MAX_LEVELS];          // images of type sdt
    uint8_t *SB[CGDIR_MAX_LEVELS], *MB[CGDIR_MAX_LEVELS], *UR[CGDIR_MAX_LEVELS];
    for (int l = 0; l < L; ++l) {
        T[l] = (char *)p_img + off[l] * esz;
        I[l] = (char *)p_img + (Ntot + off[l]) * esz;
        SB[l] = (uint8_t *)p_bits + off[l];
        MB[l] = (uint8_t *)p_bits + Ntot + off[l];
        UR[l] = (uint8_t *)p_bits + 2 * Ntot + off[l];
    }
    float *ua = (float *)p_fields, *ub = ua + 3 * Nf, *du = ub + 3 * Nf, *du2 = du + 3 * Nf;
    double *partial = (double *)p_part;
    double *hist = (double *)p_state;
    int *meta = (int *)((char *)p_state + (size_t)L * hcap * sizeof(double));
    int *hist_len = meta, *iters_run = meta + CGDIR_MAX_LEVELS, *reason = meta + 2 * CGDIR_MAX_LEVELS,
        *flags = meta + 3 * CGDIR_MAX_LEVELS;
    unsigned *done = (unsigned *)(meta + 4 * CGDIR_MAX_LEVELS);   // per-level completion counters

    // ---- ingest images (finest level)
    auto ingest = [&](const cgdir_volume *v, void *dst) -> int {
        const size_t bytes = Nf * elem_size(v->dtype);
        if (v->dtype == sdt) {
            CK(cudaMemcpyAsync(dst, v->data, bytes,
                               v->where == CGDIR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
        } else if (v->where == CGDIR_HOST) {
            CK(cudaMemcpyAsync(p_stage, v->data, bytes, cudaMemcpyHostToDevice, s));
            CK(launch_convert_image(p_stage, v->dtype, Nf, dst, sdt, s));
        } else {
            CK(launch_convert_image(v->data, v->dtype, Nf, dst, sdt, s));
        }
        return CGDIR_OK;
    };
    TRY(ingest(S, T[L - 1]));
    TRY(ingest(M, I[L - 1]));
    // ---- masks
    auto pack = [&](const cgdir_masks *m, uint8_t *dst) -> int {
        if (k == 0) { CK(cudaMemsetAsync(dst, 0, Nf, s)); return CGDIR_OK; }
        const uint8_t *ptrs[kMaxMasks];
        if (m->where == CGDIR_HOST) {
            for (int j = 0; j < k; ++j) {
                CK(cudaMemcpyAsync((uint8_t *)p_stage + (size_t)j * Nf, m->data[j], Nf, cudaMemcpyHostToDevice, s));
                ptrs[j] = (uint8_t *)p_stage + (size_t)j * Nf;
            }
        } else {
            for (int j = 0; j < k; ++j) ptrs[j] = m->data[j];
        }
        CK(launch_pack_masks(ptrs, k, Nf, dst, s));
        return CGDIR_OK;
    };
    TRY(pack(SM, SB[L - 1]));
    TRY(pack(MM, MB[L - 1]));
    // ---- signs (decided on the host before the device part is enqueued)
    int8_t sign[kMaxMasks];
    bool need_auto = false;
    for (int j = 0; j < k; ++j) {
        sign[j] = P->sign ? P->sign[j] : 0;
        if (sign[j] > 0) sign[j] = 1;
        else if (sign[j] < 0) sign[j] = -1;
        else need_auto = true;
    }
    if (need_auto) {
        int8_t autos[kMaxMasks];
        TRY(auto_sign_impl(ctx, T[L - 1], sdt, SB[L - 1], k, nx, ny, nz, autos));
        for (int j = 0; j < k; ++j)
            if (sign[j] == 0) sign[j] = autos[j];
    }
    for (int j = 0; j < k; ++j) base.half_sign[j] = 0.5f * (float)sign[j];

    const int first = P->init_dvf ? L - 1 : 0;
    if (P->init_dvf)
        CK(cudaMemcpyAsync(ua, P->init_dvf, 3 * Nf * sizeof(float),
                           P->init_dvf_where == CGDIR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    float *ufinal = ((L - 1 - first) % 2 == 0) ? ua : ub;

    // ---- the device part: pyramid, UROI, every level.  Its launches depend
    // only on the context's workspace, so it is captured once per shape and
    // parameter set into a CUDA graph and replayed.
    auto enqueue = [&](ProfList *pl, cudaStream_t s) -> int {
        for (int l = L - 2; l >= 0; --l) {
            const int *d = dims[l + 1];
            ProfScope ps(pl, ctx->prof_mask, s, CGDIR_K_SETUP, l);
            CK(launch_restrict_image(T[l + 1], sdt, d[0], d[1], d[2], T[l], s));
            CK(launch_restrict_image(I[l + 1], sdt, d[0], d[1], d[2], I[l], s));
            CK(launch_restrict_bits(SB[l + 1], d[0], d[1], d[2], SB[l], s));
            CK(launch_restrict_bits(MB[l + 1], d[0], d[1], d[2], MB[l], s));
        }
        for (int l = 0; l < L; ++l) {
            if (((P->contour_level_mask >> l) & 1u) && k > 0 && !ctx->plain_kernels) {
                ProfScope ps(pl, ctx->prof_mask, s, CGDIR_K_SETUP, l);
                CK(launch_make_texels(I[l], sdt, MB[l], Nl[l], (char *)p_tex + off[l] * tsz, s));
            }
            const double f = (double)(1 << (L - 1 - l));
            const double sp[3] = {P->spacing_mm[0] * f, P->spacing_mm[1] * f, P->spacing_mm[2] * f};
            ProfScope ps(pl, ctx->prof_mask, s, CGDIR_K_SETUP, l);
            CK(launch_uroi(SB[l], k, dims[l][0], dims[l][1], dims[l][2], sp, P->margin_mm,
                           (uint8_t *)p_rowdist, UR[l], s));
        }
        CK(cudaMemsetAsync(p_state, 0, state_bytes, s));
        float *ucur = ua, *uoth = ub;
        for (int l = first; l < L; ++l) {
            const int lx = dims[l][0], ly = dims[l][1], lz = dims[l][2];
            const size_t N = Nl[l];
            if (l == first) {
                if (!P->init_dvf) CK(cudaMemsetAsync(ucur, 0, 3 * N * sizeof(float), s));
            } else {
                ProfScope ps(pl, ctx->prof_mask, s, CGDIR_K_SETUP, l);
                CK(launch_prolong(ucur, dims[l - 1][0], dims[l - 1][1], dims[l - 1][2], lx, ly, lz, uoth, s));
                std::swap(ucur, uoth);
            }
            LevelState st{};
            st.hist = hist + (size_t)l * hcap;
            st.hist_len = hist_len + l;
            st.iters_run = iters_run + l;
            st.stop_reason = reason + l;
            st.stop_flag = flags + l;
            st.hist_cap = hcap;
            ForceArgs a = base;
            a.I0 = I[l]; a.T0 = T[l]; a.img_dtype = sdt; a.mbits = MB[l]; a.sbits = SB[l]; a.uroi = UR[l];
            a.mtex = ctx->plain_kernels ? nullptr : (const void *)((char *)p_tex + off[l] * tsz);
            a.u = ucur; a.du = du; a.warped = nullptr; a.partial = partial; a.stop_flag = flags + l;
            a.nx = lx; a.ny = ly; a.nz = lz;
            a.contour = ((P->contour_level_mask >> l) & 1u) && k > 0;
            const int zc = force_default_zchunk(lx, ly, lz);
            const int cap = P->iters[l];
            const unsigned m = ctx->prof_mask;
            a.fin.done = done + l;
            a.fin.st = st;
            a.fin.cap = cap;
            a.fin.stop_mode = P->stop_mode;
            a.fin.eps = P->eps;
            a.fin.stats_out = nullptr;
            for (int n = 0; n < cap; ++n) {
                int nb = 0;
                a.fin.n = n;   // the force kernel's last CTA reduces delta^n and runs the stop test
                { ProfScope ps(pl, m, s, CGDIR_K_FORCE, l); CK(launch_force(a, zc, &nb, s, kerr(ctx))); }
                { ProfScope ps(pl, m, s, CGDIR_K_SMOOTH_DU, l);   // steps 2 + 3
                  CK(launch_smooth_compose(du, ucur, P->compose_mode, P->sigma_fluid, lx, ly, lz, du2, uoth,
                                           flags + l, s, kerr(ctx))); }
                { ProfScope ps(pl, m, s, CGDIR_K_SMOOTH_U, l);    // step 4
                  CK(launch_smooth(du2, 3, P->sigma_diff, lx, ly, lz, ucur, flags + l, s, kerr(ctx))); }
            }
            int nb = 0;
            FinishArgs fm = a.fin;
            fm.n = cap;
            { ProfScope ps(pl, m, s, CGDIR_K_METRIC, l);
              CK(launch_metric(I[l], T[l], sdt, ucur, UR[l], lx, ly, lz, partial, flags + l, &nb, s, &fm)); }
        }
        return CGDIR_OK;
    };

    const ProfList *used = nullptr;
    if (ctx->use_graphs) {
        char key[1024];
        int len = std::snprintf(key, sizeof key, "%d %d %d|%d|%d %d %.9g %.9g %d %u %d %.17g %.17g %.17g %.17g "
                                "%.17g %.9g %d %d %llu %u %d|", nx, ny, nz, L, k, first, P->sigma_fluid, P->sigma_diff,
                                P->compose_mode, P->contour_level_mask, P->stop_mode, P->eps, P->spacing_mm[0],
                                P->spacing_mm[1], P->spacing_mm[2], P->margin_mm, P->intensity_offset,
                                (int)ctx->plain_kernels, maxcap, ctx->ws_generation, ctx->prof_mask, sdt);
        std::string skey(key, (size_t)len);
        for (int l = 0; l < L; ++l) skey += std::to_string(P->iters[l]) + ",";
        for (int j = 0; j < k; ++j) {
            char b[48];
            std::snprintf(b, sizeof b, "%.9g:%d,", base.lambda[j], (int)sign[j]);
            skey += b;
        }
        auto it = ctx->graphs.find(skey);
        if (it == ctx->graphs.end()) {
            GraphEntry ge;
            const unsigned long long before = g_launches.load();
            CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue(&ge.prof, ctx->cap_stream);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
            ge.launches = g_launches.load() - before;
            g_launches.fetch_sub(ge.launches);        // captured, not yet launched
            if (rc != CGDIR_OK) {
                if (graph) cudaGraphDestroy(graph);
                ge.prof.release();
                return rc;
            }
            if (ec != cudaSuccess) {
                ge.prof.release();
                return fail(ctx, CGDIR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
            }
            const cudaError_t ei = cudaGraphInstantiate(&ge.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) {
                ge.prof.release();
                return fail(ctx, CGDIR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
            }
            it = ctx->graphs.emplace(skey, std::move(ge)).first;
        }
        CK(cudaGraphLaunch(it->second.exec, s));
        note_launch((unsigned)it->second.launches);
        used = &it->second.prof;
    } else {
        ctx->eager.recs.clear();
        TRY(enqueue(&ctx->eager, s));
        used = &ctx->eager;
    }

    // ---- outputs
    CK(cudaMemcpyAsync(dvf_out, ufinal, 3 * Nf * sizeof(float),
                       dvf_where == CGDIR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    ctx->h_hist.assign((size_t)L * hcap, 0.0);
    ctx->h_meta.assign(4 * CGDIR_MAX_LEVELS, 0);
    CK(cudaMemcpyAsync(ctx->h_hist.data(), hist, (size_t)L * hcap * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_meta.data(), meta, 4 * CGDIR_MAX_LEVELS * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    prof_collect(ctx, *used);
    TRY(check_err_word(ctx));
    if (stats_out) {
        for (int l = 0; l < L; ++l) {
            cgdir_level_stats &o = stats_out[l];
            o.level = l;
            o.nx = dims[l][0]; o.ny = dims[l][1]; o.nz = dims[l][2];
            if (l < first) {
                o.iters_run = 0; o.stop_reason = CGDIR_REASON_SKIPPED; o.hist_len = 0; o.rms_id = nullptr;
                continue;
            }
            o.iters_run = ctx->h_meta[CGDIR_MAX_LEVELS + l];
            o.stop_reason = ctx->h_meta[2 * CGDIR_MAX_LEVELS + l];
            o.hist_len = ctx->h_meta[l];
            o.rms_id = ctx->h_hist.data() + (size_t)l * hcap;
        }
    }
    return CGDIR_OK;
}

}  // extern "C"
