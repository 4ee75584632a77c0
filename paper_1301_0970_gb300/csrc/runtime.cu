// Contexts, device workspace and the per-step primitives of the C ABI
// (include/cgdir.h).  The registration pipeline (Algorithm A, Sec. 2.2:
// single, batched and served) is in register.cu.
#include "runtime_internal.hpp"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

using namespace cgdir;
using namespace cgdir::rt;

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

namespace rt {

unsigned long long launches_now() { return g_launches.load(); }
void launches_sub(unsigned long long n) { g_launches.fetch_sub(n); }

void ProfList::release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    recs.clear();
}

size_t WsSet::bytes() const {
    size_t b = 0;
    for (const auto &kv : bufs) b += kv.second.cap;
    return b;
}

ProfScope::ProfScope(ProfList *l, unsigned mask, cudaStream_t s, int cls, int level) : stream(s) {
    // low 16 bits: kernel classes; high 16 bits: pyramid levels
    if (!(mask & (1u << cls)) || level < 0 || level >= 16 || !((mask >> 16) & (1u << level))) return;
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

ProfScope::~ProfScope() {
    if (idx >= 0) cudaEventRecordWithFlags(list->recs[idx].b, stream, cudaEventRecordExternal);
}

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

void drop_graphs(WsSet &ws) {
    for (auto &kv : ws.graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        kv.second.prof.release();
    }
    ws.graphs.clear();
}

DeviceGuard::DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) cudaSetDevice(d);
}
DeviceGuard::~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

int fail(cgdir_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int ws_get(cgdir_ctx *ctx, WsSet &ws, cudaStream_t sync, const char *name, size_t bytes, void **out) {
    WsBuf &b = ws.bufs[name];
    if (bytes == 0) bytes = 256;
    if (b.p && b.cap >= bytes) { *out = b.p; return CGDIR_OK; }
    const size_t cap = round_up(bytes, (size_t)1 << 21);
    const size_t after = ctx->in_use - b.cap + cap;
    if (ctx->budget && after > ctx->budget)
        return fail(ctx, CGDIR_ENOMEM, std::string("device budget exceeded growing '") + name + "'");
    if (b.p) {
        cudaStreamSynchronize(sync);
        drop_graphs(ws);               // cached graphs hold the old address
        cudaFree(b.p);
        ctx->in_use -= b.cap;
        b = WsBuf{};
    }
    ++ws.generation;
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

void ws_release(cgdir_ctx *ctx, WsSet &ws) {
    drop_graphs(ws);
    for (auto &kv : ws.bufs)
        if (kv.second.p) {
            cudaFree(kv.second.p);
            ctx->in_use -= kv.second.cap;
        }
    ws.bufs.clear();
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
    a.pass2_width = ctx->force_width;
    return CGDIR_OK;
}

}  // namespace rt
}  // namespace cgdir

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
    const unsigned k = kernel_mask & ((1u << CGDIR_K_COUNT) - 1u);
    ctx->prof_mask = k ? (k | 0xffff0000u) : 0u;
    ctx->prof.clear();
    return CGDIR_OK;
}

int cgdir_profile_levels(cgdir_ctx *ctx, unsigned level_mask) {
    if (!ctx) return CGDIR_EINVAL;
    const unsigned lv = level_mask & ((1u << CGDIR_MAX_LEVELS) - 1u);
    if (ctx->prof_mask & 0xffffu) ctx->prof_mask = (ctx->prof_mask & 0xffffu) | (lv << 16);
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
    c->fused_force = kern && std::strcmp(kern, "fused") == 0;
    const char *spr = std::getenv("CGDIR_SERVE_PRIORITY");
    c->serve_priority = !(spr && std::strcmp(spr, "0") == 0);
    const char *ssch = std::getenv("CGDIR_SERVE_SCHEDULE");
    c->serve_schedule = !ssch ? 2 : std::strcmp(ssch, "shared") == 0 ? 0 : std::strcmp(ssch, "alone") == 0 ? 1 : 2;
    const char *swc = std::getenv("CGDIR_SHARED_WIDE_CAP");
    if (swc) c->shared_wide_cap = std::atoi(swc);
    const char *fw = std::getenv("CGDIR_FORCE_WIDTH");
    c->force_width = fw && (std::strcmp(fw, "1") == 0 || std::strcmp(fw, "2") == 0) ? std::atoi(fw) : 0;
    const char *fz = std::getenv("CGDIR_FORCE_ZCHUNK");
    c->force_zchunk = fz ? std::atoi(fz) : 0;
    const char *sz = std::getenv("CGDIR_SMOOTH_ZCHUNK");
    c->smooth_zchunk = sz ? std::atoi(sz) : 0;
    const char *cm = std::getenv("CGDIR_COOP_MAX");
    c->coop_max_voxels = cm ? std::atol(cm) : 0;
    const char *sv = std::getenv("CGDIR_SMOOTH");
    c->smooth_variant = !sv ? SMOOTH_AUTO
                            : std::strcmp(sv, "tile") == 0 ? SMOOTH_TILE
                            : std::strcmp(sv, "march") == 0 ? SMOOTH_MARCH
                            : std::strcmp(sv, "march32") == 0 ? SMOOTH_MARCH_NARROW
                            : std::strcmp(sv, "split") == 0 ? SMOOTH_SPLIT
                            : std::strcmp(sv, "fused") == 0 ? SMOOTH_FUSED : SMOOTH_AUTO;
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
    for (auto &sl : ctx->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        ws_release(ctx, sl->ws);
        if (sl->own_stream && sl->stream) cudaStreamDestroy(sl->stream);
        if (sl->done) cudaEventDestroy(sl->done);
        if (sl->ready) cudaEventDestroy(sl->ready);
        if (sl->h_hist) cudaFreeHost(sl->h_hist);
        if (sl->h_meta) cudaFreeHost(sl->h_meta);
    }
    ctx->slots.clear();
    drop_graphs(ctx->batch);
    ws_release(ctx, ctx->ws);
    ctx->eager.release();
    for (cudaStream_t b : ctx->branch_streams) cudaStreamDestroy(b);
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

// Smoothing choice of the primitives: the context's forced variant, else by size.
static SmoothChoice prim_smooth(const cgdir_ctx *ctx) {
    SmoothChoice ch;
    ch.variant = ctx->smooth_variant;
    return ch;
}

static int force_impl(cgdir_ctx *ctx, const ForceArgs &a, double *stats_host) {
    void *part = nullptr, *st = nullptr;
    ForceArgs b = a;
    const int zc = force_zchunk_for(ctx, a.nx, a.ny, a.nz, a.contour && a.k > 0, a.img_dtype);
    b.pass2_width = force_width_for(ctx, a.nx, a.ny, a.nz, a.contour && a.k > 0, a.img_dtype);
    if (b.contour && b.k > 0 && !ctx->plain_kernels && b.mtex == nullptr) {
        // the TMA kernel gathers interleaved {I0, bits} texels
        const size_t N = (size_t)a.nx * a.ny * a.nz;
        void *tex = nullptr;
        TRY(ws_get(ctx, "force_tex", N * tex_elem_size(a.img_dtype), &tex));
        CK(launch_make_texels(a.I0, a.img_dtype, a.mbits, N, tex, ctx->stream));
        b.mtex = tex;
    }
    if (!ctx->plain_kernels && !ctx->fused_force) {
        const size_t N = (size_t)a.nx * a.ny * a.nz;
        void *scr = nullptr;
        TRY(ws_get(ctx, "force_scr", force_scratch_bytes(N, b.contour ? b.k : 0), &scr));
        force_scratch_assign(b, scr, N);
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
    void *scr = nullptr;
    if (ctx->smooth_variant == SMOOTH_SPLIT)
        TRY(ws_get(ctx, "smooth_scr", (size_t)ncomp * nx * ny * nz * sizeof(float), &scr));
    CK(launch_smooth(in, ncomp, sigma, nx, ny, nz, out, nullptr, ctx->stream, kerr(ctx), prim_smooth(ctx),
                     (float *)scr));
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
    CK(launch_smooth((float *)tmp, 3, sigma, nx, ny, nz, out, nullptr, ctx->stream, kerr(ctx), prim_smooth(ctx)));
    return CGDIR_OK;
}

int cgdir_smooth_compose(cgdir_ctx *ctx, const float *du, const float *u, int mode, float sigma, int nx, int ny,
                         int nz, float *out) {
    if (!ctx) return CGDIR_EINVAL;
    if (!u || !du || !out || out == u || out == du || !dims_ok(nx, ny, nz) || !sigma_ok(sigma) ||
        (mode != CGDIR_COMPOSE && mode != CGDIR_ADDITIVE))
        return fail(ctx, CGDIR_EINVAL, "smooth_compose: bad arguments");
    DeviceGuard g(ctx->device);
    if (gauss_radius(sigma) == 0) {
        CK(launch_compose(u, du, mode, nx, ny, nz, out, nullptr, ctx->stream));
        return CGDIR_OK;
    }
    void *tmp = nullptr;
    TRY(ws_get(ctx, "field_tmp", 3 * (size_t)nx * ny * nz * sizeof(float), &tmp));
    CK(launch_smooth_compose(du, u, mode, sigma, nx, ny, nz, out, (float *)tmp, nullptr, ctx->stream, kerr(ctx),
                             ctx->fused_force, prim_smooth(ctx)));
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
        CK(launch_smooth(du, 3, sigma_fluid, nx, ny, nz, du_out, nullptr, ctx->stream, kerr(ctx), prim_smooth(ctx)));
        CK(launch_compose(u_in, du_out, compose_mode, nx, ny, nz, un, nullptr, ctx->stream));
    } else {
        CK(launch_smooth_compose(du, u_in, compose_mode, sigma_fluid, nx, ny, nz, un, (float *)t3, nullptr,
                                 ctx->stream, kerr(ctx), ctx->fused_force, prim_smooth(ctx)));
    }
    CK(launch_smooth(un, 3, sigma_diff, nx, ny, nz, u_out, nullptr, ctx->stream, kerr(ctx), prim_smooth(ctx),
                     (float *)t3));
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

}  // extern "C"

int cgdir::rt::auto_sign_impl(cgdir_ctx *ctx, const void *T0, int dtype, const uint8_t *sbits, int k, int nx,
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

extern "C" {

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

}  // extern "C"
