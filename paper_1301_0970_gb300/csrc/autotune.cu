// Autotuner for the per-level kernel schedule (not part of the paper: an
// execution choice).  For one pyramid level shape it times, on synthetic
// data of that shape, the candidate launch configurations of the two
// kernels whose best configuration depends on the shape:
//   smoothing (with the composite update, i.e. steps 2-4 of an iteration):
//              the TMA z-march with its default z chunk, half, double and
//              four times that chunk (plus the separate update kernel), the 3-D
//              shared-memory tile kernel (idem), and the split xy + z
//              kernels with the update fused into the z pass;
//   force:     the stencil pass with the default z chunk, half, a quarter
//              and double;
// then the fused schedule (force stencil pass alone, 3-D tiles of G(du)
// with the update, 3-D tiles of G(u') with the next iteration's warp)
// against the best of those two, summed.
// The fastest of each is recorded in the context and used by every later
// registration of that shape (and baked into its CUDA graph).
#include "runtime_internal.hpp"

#include <algorithm>

using namespace cgdir;
using namespace cgdir::rt;

namespace {

__device__ __forceinline__ unsigned hash3(unsigned x, unsigned y, unsigned z, unsigned s) {
    unsigned h = x * 0x8da6b343u ^ y * 0xd8163841u ^ z * 0xcb1ab31fu ^ s * 0x165667b1u;
    h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12; h *= 0x297a2d39u; h ^= h >> 15;
    return h;
}

// Synthetic level shaped like a registration's: CT-like values with
// structure and noise, k compact structures (ellipsoids around the centre,
// the moving ones 2 voxels off the static ones, so a thin shell of voxels
// takes the mixed structure path as near real organ borders) and a smooth
// displacement field of up to 1.5 voxels.
template <typename IT>
__global__ void k_tune_fill(IT *I0, IT *T0, uint8_t *mbits, uint8_t *sbits, uint8_t *uroi, float *u, int nx,
                            int ny, int nz, int k) {
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const float base = 40.f * __sinf(0.11f * x) * __cosf(0.07f * y) + 30.f * __sinf(0.13f * z);
        const float n0 = (float)(hash3(x, y, z, 1) & 1023u) * (50.f / 1023.f);
        const float n1 = (float)(hash3(x, y, z, 2) & 1023u) * (50.f / 1023.f);
        I0[i] = from_f<IT>(base + n0);
        T0[i] = from_f<IT>(base + n1);
        const float fx = (x + 0.5f) / nx, fy = (y + 0.5f) / ny, fz = (z + 0.5f) / nz, sx = 2.f / nx;
        unsigned mb = 0, sb = 0;
        for (int j = 0; j < k; ++j) {
            const float a = 6.2831853f * j / (k > 0 ? k : 1);
            const float cx = 0.5f + 0.22f * __cosf(a), cy = 0.5f + 0.22f * __sinf(a);
            const float dy = (fy - cy) / 0.1f, dz = (fz - 0.5f) / 0.2f;
            const float ds = (fx - cx) / 0.1f, dm = (fx + sx - cx) / 0.1f;
            if (dm * dm + dy * dy + dz * dz <= 1.f) mb |= 1u << j;
            if (ds * ds + dy * dy + dz * dz <= 1.f) sb |= 1u << j;
        }
        mbits[i] = (uint8_t)mb;
        sbits[i] = (uint8_t)sb;
        uroi[i] = 1;
        for (int c = 0; c < 3; ++c)
            u[c * N + i] = 1.5f * __sinf(6.2831853f * (fx + 0.3f * c)) * __cosf(4.712389f * fy) * __cosf(3.1415927f * (fz - 0.5f));
    }
}

}  // namespace

namespace cgdir {
namespace rt {

int force_zchunk_min(int nx, int ny, int nz) { return std::max(1, force_default_zchunk(nx, ny, nz) / 4); }

static const TunedLevel *find_tuned(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt) {
    auto it = ctx->tuned.find(TuneKey{nx, ny, nz, contour ? 1 : 0, sdt});
    return it == ctx->tuned.end() ? nullptr : &it->second;
}

SmoothChoice smooth_choice(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt, bool allow_fused) {
    SmoothChoice ch;
    // registrations that share the GPU (batched, served) cap the wide z-march
    // at two CTAs per SM: three fill an SM's shared memory and registers and
    // starve the other registrations' kernels
    if (!allow_fused) ch.ctas_per_sm = ctx->shared_wide_cap;
    if (ctx->smooth_variant != SMOOTH_AUTO || ctx->smooth_zchunk > 0) {
        ch.variant = ctx->smooth_variant;
        ch.zchunk = ctx->smooth_zchunk;
        return ch;
    }
    if (const TunedLevel *t = find_tuned(ctx, nx, ny, nz, contour, sdt)) {
        ch.variant = t->fused && allow_fused ? SMOOTH_FUSED : t->smooth_variant;
        ch.zchunk = t->fused && allow_fused ? 0 : t->smooth_zchunk;
    }
    return ch;
}

bool use_level_coop(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt) {
    (void)contour; (void)sdt;
    return (long)nx * ny * nz <= ctx->coop_max_voxels;
}

// Voxels per thread of the force's stencil pass (0: the widest the shape
// and alignment allow).
int force_width_for(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt) {
    if (ctx->force_width > 0) return ctx->force_width;
    if (const TunedLevel *t = find_tuned(ctx, nx, ny, nz, contour, sdt)) return t->force_width;
    return 0;
}

// Never below force_zchunk_min: the registration's partial-sum buffer is
// sized for that chunk (a loaded table may hold any chunk).
int force_zchunk_for(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt) {
    const int lo = force_zchunk_min(nx, ny, nz);
    if (ctx->force_zchunk > 0) return std::max(lo, std::min(ctx->force_zchunk, nz));
    if (const TunedLevel *t = find_tuned(ctx, nx, ny, nz, contour, sdt))
        if (t->force_zchunk > 0) return std::max(lo, std::min(t->force_zchunk, nz));
    return force_default_zchunk(nx, ny, nz);
}

// Average time of `reps` launches of `body` after two untimed ones (ms).
template <typename Body>
static int time_ms(cgdir_ctx *ctx, cudaEvent_t a, cudaEvent_t b, int reps, float *ms, Body body) {
    cudaStream_t s = ctx->stream;
    for (int r = 0; r < 2; ++r) CK(body(s));
    CK(cudaEventRecord(a, s));
    for (int r = 0; r < reps; ++r) CK(body(s));
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, a, b));
    *ms = t / (float)reps;
    return CGDIR_OK;
}

int tune_level(cgdir_ctx *ctx, int nx, int ny, int nz, int k, int contour, int sdt, float sigma) {
    if (!dims_ok(nx, ny, nz) || k < 0 || k > kMaxMasks) return fail(ctx, CGDIR_EINVAL, "autotune: bad shape");
    if (ctx->plain_kernels || ctx->fused_force) return CGDIR_OK;     // nothing to choose
    contour = contour && k > 0;
    DeviceGuard g(ctx->device);
    const size_t N = (size_t)nx * ny * nz;
    const size_t esz = img_elem_size(sdt), tsz = tex_elem_size(sdt);
    void *img, *bits, *tex, *fields, *scr, *part, *state;
    TRY(ws_get(ctx, "tune_img", 2 * N * esz, &img));
    TRY(ws_get(ctx, "tune_bits", 3 * N, &bits));
    TRY(ws_get(ctx, "tune_tex", N * tsz, &tex));
    TRY(ws_get(ctx, "tune_fields", 4 * 3 * N * sizeof(float), &fields));
    TRY(ws_get(ctx, "tune_scr", force_scratch_bytes(N, contour ? k : 0), &scr));
    const size_t np = force_partial_count(nx, ny, nz, force_zchunk_min(nx, ny, nz));
    TRY(ws_get(ctx, "tune_part", np * kPartialStride * sizeof(double), &part));
    TRY(ws_get(ctx, "tune_state", 256, &state));
    cudaStream_t s = ctx->stream;
    char *I0 = (char *)img, *T0 = (char *)img + N * esz;
    uint8_t *mb = (uint8_t *)bits, *sb = mb + N, *ur = mb + 2 * N;
    float *u = (float *)fields, *du = u + 3 * N, *out = du + 3 * N, *sscr = out + 3 * N;
    const unsigned fg = (unsigned)std::min<size_t>((N + 255) / 256, 152 * 8);
    if (sdt == CGDIR_F16)
        k_tune_fill<__half><<<fg, 256, 0, s>>>((__half *)I0, (__half *)T0, mb, sb, ur, u, nx, ny, nz, k);
    else if (sdt == CGDIR_BF16)
        k_tune_fill<__nv_bfloat16><<<fg, 256, 0, s>>>((__nv_bfloat16 *)I0, (__nv_bfloat16 *)T0, mb, sb, ur, u, nx, ny,
                                                      nz, k);
    else
        k_tune_fill<float><<<fg, 256, 0, s>>>((float *)I0, (float *)T0, mb, sb, ur, u, nx, ny, nz, k);
    CK(cudaGetLastError());
    if (contour) CK(launch_make_texels(I0, sdt, mb, N, tex, s));
    CK(cudaMemsetAsync(state, 0, 256, s));
    CK(cudaMemsetAsync(du, 0, 3 * N * sizeof(float), s));

    // force with the fused reduction, as in a registration
    ForceArgs a{};
    {
        float lam[kMaxMasks];
        int8_t sg[kMaxMasks];
        for (int j = 0; j < kMaxMasks; ++j) { lam[j] = 1e-3f; sg[j] = (j & 1) ? -1 : 1; }
        TRY(fill_force_args(ctx, a, k, lam, sg, 1000.f, contour));
    }
    a.I0 = I0; a.T0 = T0; a.img_dtype = sdt; a.mbits = mb; a.sbits = sb; a.uroi = ur;
    a.mtex = contour ? tex : nullptr;
    a.u = u; a.du = du; a.partial = (double *)part; a.stop_flag = nullptr;
    a.nx = nx; a.ny = ny; a.nz = nz; a.contour = contour;
    force_scratch_assign(a, scr, N);
    double *hist = (double *)state;
    int *meta = (int *)((char *)state + 64);
    a.fin.done = (unsigned *)(meta + 8);
    a.fin.st.hist = hist; a.fin.st.hist_len = meta; a.fin.st.iters_run = meta + 1; a.fin.st.stop_reason = meta + 2;
    a.fin.st.stop_flag = meta + 3; a.fin.st.hist_cap = 1;
    a.fin.n = 0; a.fin.cap = 1 << 30; a.fin.stop_mode = CGDIR_STOP_FIXED; a.fin.eps = 0.0;

    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    TunedLevel best;
    const int reps = N > ((size_t)4 << 20) ? 5 : 20;
    int rc = CGDIR_OK;
    {
        const int d = force_default_zchunk(nx, ny, nz);
        const int cand[4] = {d, std::max(1, d / 2), std::max(1, d / 4), std::min(nz, 2 * d)};
        // the stencil pass's width: four voxels per thread (the default where
        // nx % 4 == 0) or two (twice the CTAs, for small levels)
        const int widths[2] = {0, 2};
        const int nw = (nx % 4 == 0 && ctx->force_width == 0) ? 2 : 1;
        float bt = 1e30f;
        for (int wi = 0; wi < nw && rc == CGDIR_OK; ++wi) {
            a.pass2_width = ctx->force_width > 0 ? ctx->force_width : widths[wi];
            for (int ci = 0; ci < 4 && rc == CGDIR_OK; ++ci) {
                bool seen = false;
                for (int cj = 0; cj < ci; ++cj) seen = seen || cand[cj] == cand[ci];
                if (seen) continue;
                float ms = 0.f;
                rc = time_ms(ctx, e0, e1, reps, &ms,
                             [&](cudaStream_t st) { return launch_force(a, cand[ci], nullptr, st, kerr(ctx)); });
                if (wi == 0 && ci == 0) best.default_force_ms = ms;
                if (rc == CGDIR_OK && ms < bt) {
                    bt = ms;
                    best.force_zchunk = cand[ci];
                    best.force_width = widths[wi];
                    best.force_ms = ms;
                }
            }
        }
        a.pass2_width = ctx->force_width > 0 ? ctx->force_width : best.force_width;
    }
    if (rc == CGDIR_OK) {
        float bt = 1e30f;
        const int d = smooth_default_zchunk(nx, ny, nz, 3);
        SmoothChoice cand[16];
        int nc = 0;
        auto add = [&](int variant, int zc) {
            for (int r = 0; r < nc; ++r)
                if (cand[r].variant == variant && cand[r].zchunk == zc) return;
            cand[nc].variant = variant;
            cand[nc++].zchunk = zc;
        };
        if (nx % 4 == 0) {
            // z chunks: the default and the volume cut into 1 .. 16 chunks
            // (longer chunks reload fewer halo planes; more chunks fill more
            // SMs, and the count of CTAs against whole waves decides which
            // wins); the 32 x 16 z-march with 2, 4 and 8 chunks where the
            // 64 x 16 one applies (more CTAs per chunk on small levels)
            add(SMOOTH_MARCH, d);
            const int nch[7] = {1, 2, 3, 4, 6, 8, 16};
            for (int q = 0; q < 7; ++q) add(SMOOTH_MARCH, (nz + nch[q] - 1) / nch[q]);
            if (nx % 8 == 0)
                for (int c = 2; c <= 8; c *= 2) add(SMOOTH_MARCH_NARROW, (nz + c - 1) / c);
        }
        cand[nc].variant = SMOOTH_TILE; cand[nc++].zchunk = 0;
        cand[nc].variant = SMOOTH_SPLIT; cand[nc++].zchunk = 0;
        const SmoothChoice dflt{smooth_auto_variant(nx, ny, nz), 0};
        for (int ci = 0; ci < nc && rc == CGDIR_OK; ++ci) {
            float ms = 0.f;
            // one iteration: the force step (so du and the caches are as in a
            // registration: timed alone on a level that fits in L2, the
            // smoothing favours other z chunks), G(du) with the composite
            // update, then G(u'); the force step's own time is taken off
            rc = time_ms(ctx, e0, e1, reps, &ms, [&](cudaStream_t st) {
                cudaError_t e = launch_force(a, best.force_zchunk, nullptr, st, kerr(ctx));
                if (e != cudaSuccess) return e;
                e = launch_smooth_compose(du, u, CGDIR_COMPOSE, sigma, nx, ny, nz, out, sscr, nullptr, st, kerr(ctx),
                                          false, cand[ci]);
                if (e != cudaSuccess) return e;
                return launch_smooth(out, 3, sigma, nx, ny, nz, du, nullptr, st, kerr(ctx), cand[ci], sscr);
            });
            ms = std::max(ms - best.force_ms, 0.f);
            const bool is_default = cand[ci].variant == dflt.variant &&
                                    (cand[ci].variant == SMOOTH_TILE || cand[ci].zchunk == d);
            if (is_default) best.default_smooth_ms = ms;
            if (rc == CGDIR_OK && ms < bt) {
                bt = ms;
                best.smooth_variant = cand[ci].variant;
                best.smooth_zchunk = cand[ci].zchunk;
                best.smooth_ms = ms;
            }
        }
    }
    // the fused schedule: force stencil pass only, then the two fused tile
    // kernels (G(du) + update; G(u') + the next warp)
    if (rc == CGDIR_OK && fused_schedule_ok(a) && gauss_taps(sigma).r > 0) {
        ForceArgs a2 = a;
        a2.skip_warp = 1;
        float f2 = 0.f, fs = 0.f;
        rc = time_ms(ctx, e0, e1, reps, &f2,
                     [&](cudaStream_t st) { return launch_force(a2, best.force_zchunk, nullptr, st, kerr(ctx)); });
        if (rc == CGDIR_OK)    // timed after the stencil pass, as in an iteration
            rc = time_ms(ctx, e0, e1, reps, &fs, [&](cudaStream_t st) {
                cudaError_t e = launch_force(a2, best.force_zchunk, nullptr, st, kerr(ctx));
                if (e != cudaSuccess) return e;
                e = launch_fused_smooth_compose(du, u, CGDIR_COMPOSE, sigma, nx, ny, nz, out, nullptr, kerr(ctx), st);
                if (e != cudaSuccess) return e;
                return launch_fused_smooth_warp(out, sigma, u, a2, kerr(ctx), st);
            });
        fs = std::max(fs - f2, 0.f);
        if (rc == CGDIR_OK && f2 + fs < best.force_ms + best.smooth_ms) {
            best.fused = 1;
            best.fused_smooth_ms = fs;
            best.fused_force_ms = f2;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(rc);
    TRY(check_err_word(ctx));
    // give the scratch back (a tuned shape may be large)
    CK(cudaStreamSynchronize(s));
    for (auto it = ctx->ws.bufs.begin(); it != ctx->ws.bufs.end();) {
        if (it->first.rfind("tune_", 0) == 0) {
            cudaFree(it->second.p);
            ctx->in_use -= it->second.cap;
            it = ctx->ws.bufs.erase(it);
        } else {
            ++it;
        }
    }
    ctx->tuned[TuneKey{nx, ny, nz, contour ? 1 : 0, sdt}] = best;
    ++ctx->tune_gen;
    return CGDIR_OK;
}

}  // namespace rt
}  // namespace cgdir

extern "C" {

int cgdir_autotune(cgdir_ctx *ctx, int nx, int ny, int nz, int k, int levels, unsigned contour_level_mask,
                   int storage_dtype, float sigma) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->err.clear();
    if (!dims_ok(nx, ny, nz) || levels < 1 || levels > CGDIR_MAX_LEVELS || k < 0 || k > kMaxMasks ||
        storage_dtype < CGDIR_F32 || storage_dtype > CGDIR_BF16 || !sigma_ok(sigma))
        return fail(ctx, CGDIR_EINVAL, "autotune: bad arguments");
    int d[3] = {nx, ny, nz};
    int dims[CGDIR_MAX_LEVELS][3];
    for (int l = levels - 1; l >= 0; --l) {
        for (int a = 0; a < 3; ++a) dims[l][a] = d[a];
        for (int a = 0; a < 3; ++a) d[a] = (d[a] + 1) / 2;
    }
    for (int l = 0; l < levels; ++l)
        TRY(tune_level(ctx, dims[l][0], dims[l][1], dims[l][2], k, (contour_level_mask >> l) & 1u,
                       level_storage(storage_dtype, l, levels), sigma));
    return CGDIR_OK;
}

int cgdir_set_autotune(cgdir_ctx *ctx, int on) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->autotune_on = on != 0;
    return CGDIR_OK;
}

int cgdir_tuning_read(const cgdir_ctx *ctx, cgdir_tuning *out, int cap) {
    if (!ctx || (cap > 0 && !out)) return -CGDIR_EINVAL;
    int n = 0;
    for (const auto &kv : ctx->tuned) {
        if (n < cap) {
            cgdir_tuning &o = out[n];
            o.nx = kv.first[0]; o.ny = kv.first[1]; o.nz = kv.first[2];
            o.contour = kv.first[3]; o.storage_dtype = kv.first[4];
            const TunedLevel &t = kv.second;
            o.smooth_variant = t.fused ? CGDIR_SMOOTH_FUSED : t.smooth_variant;
            o.smooth_zchunk = t.fused ? 0 : t.smooth_zchunk;
            o.force_zchunk = t.force_zchunk;
            o.smooth_ms = t.fused ? t.fused_smooth_ms : t.smooth_ms;
            o.force_ms = t.fused ? t.fused_force_ms : t.force_ms;
            o.default_smooth_ms = kv.second.default_smooth_ms; o.default_force_ms = kv.second.default_force_ms;
            o.force_width = t.force_width;
        }
        ++n;
    }
    return n;
}

int cgdir_tuning_load(cgdir_ctx *ctx, const cgdir_tuning *in, int n) {
    if (!ctx || n < 0 || (n > 0 && !in)) return CGDIR_EINVAL;
    ctx->err.clear();
    for (int i = 0; i < n; ++i) {
        const cgdir_tuning &t = in[i];
        if (!dims_ok(t.nx, t.ny, t.nz) || (t.contour != 0 && t.contour != 1) || t.storage_dtype < CGDIR_F32 ||
            t.storage_dtype > CGDIR_BF16 || t.smooth_variant < CGDIR_SMOOTH_MARCH ||
            t.smooth_variant > CGDIR_SMOOTH_MARCH32 || t.smooth_zchunk < 0 || t.smooth_zchunk > t.nz ||
            t.force_zchunk < 1 || t.force_zchunk > t.nz || t.force_width < 0 || t.force_width > 2)
            return fail(ctx, CGDIR_EINVAL, "tuning_load: bad entry");
    }
    for (int i = 0; i < n; ++i) {
        const cgdir_tuning &t = in[i];
        TunedLevel v;
        if (t.smooth_variant == CGDIR_SMOOTH_FUSED) {     // the per-step alternative was not saved: by size
            v.fused = 1;
            v.fused_smooth_ms = t.smooth_ms; v.fused_force_ms = t.force_ms;
        } else {
            v.smooth_variant = t.smooth_variant;
            v.smooth_zchunk = t.smooth_zchunk;
            v.smooth_ms = t.smooth_ms; v.force_ms = t.force_ms;
        }
        v.force_zchunk = t.force_zchunk;
        v.force_width = t.force_width;
        v.default_smooth_ms = t.default_smooth_ms; v.default_force_ms = t.default_force_ms;
        ctx->tuned[TuneKey{t.nx, t.ny, t.nz, t.contour, t.storage_dtype}] = v;
    }
    ++ctx->tune_gen;
    return CGDIR_OK;
}

}  // extern "C"
