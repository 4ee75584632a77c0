// The registration pipeline of the C ABI: Algorithm A (Sec. 2.2) over a
// coarse-to-fine pyramid, driven as a fixed sequence of kernel launches.
//
// A registration runs in a "slot" (its device buffers, cached graphs and
// host result buffers) in four phases:
//   plan_make     validate the arguments, size the pyramid;
//   plan_prepare  take the slot's buffers, copy the caller's images and
//                 masks in (pack the masks), decide automatic signs;
//   plan_enqueue  the device part: pyramid, UROI, every level's iterations.
//                 It only touches the slot's buffers, so it is captured once
//                 per shape / parameter set into a CUDA graph and replayed;
//   plan_outputs  copy the DVF and the RMS-ID histories out.
// The per-iteration sequence at a level (u stays in one buffer):
//   force(u -> du) [its last CTA reduces delta^n and runs the stop test] ;
//   smooth+compose(du, u -> du2) ; smooth(du2 -> u)
// and after the level's cap a metric pass gives delta^cap.  The stopping
// decision is a device flag that makes the level's remaining kernels return
// at once, so a level never waits for the host.
//
// cgdir_register runs one slot on the context stream; cgdir_register_batch
// captures one graph with a branch per case (the branches run concurrently);
// cgdir_submit runs each request in its own slot and stream, so requests
// that arrive while others run overlap on the device.
#include "runtime_internal.hpp"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <thread>

using namespace cgdir;
using namespace cgdir::rt;

namespace cgdir {
namespace rt {

struct RegPlan {
    const cgdir_volume *S = nullptr, *M = nullptr;
    const cgdir_masks *SM = nullptr, *MM = nullptr;
    int dvf_where = CGDIR_DEVICE;
    cgdir_params P{};
    std::vector<int> iters;
    int8_t sign[kMaxMasks] = {};
    int nx = 0, ny = 0, nz = 0, k = 0, L = 0, maxcap = 0, hcap = 0, first = 0, sdt = CGDIR_F32;
    int dims[CGDIR_MAX_LEVELS][3] = {};
    size_t Nl[CGDIR_MAX_LEVELS] = {}, off[CGDIR_MAX_LEVELS + 1] = {}, Nf = 0, Ntot = 0;
    int ldt[CGDIR_MAX_LEVELS] = {};                   // image type per level (level_storage)
    size_t ioff[CGDIR_MAX_LEVELS + 1] = {};           // byte offsets of the levels' images
    size_t toff[CGDIR_MAX_LEVELS + 1] = {};           // byte offsets of the levels' texels
    ForceArgs base{};
    // device buffers of the slot
    char *T[CGDIR_MAX_LEVELS] = {}, *I[CGDIR_MAX_LEVELS] = {};
    uint8_t *SB[CGDIR_MAX_LEVELS] = {}, *MB[CGDIR_MAX_LEVELS] = {}, *UR[CGDIR_MAX_LEVELS] = {};
    char *tex = nullptr;
    float *ua = nullptr, *ub = nullptr, *du = nullptr, *du2 = nullptr, *ufinal = nullptr;
    double *partial = nullptr;
    void *state = nullptr;
    size_t state_bytes = 0;
    double *hist = nullptr;
    int *meta = nullptr;
    uint8_t *rowdist = nullptr;
    void *stage = nullptr;
    void *fscr = nullptr;              // two-pass force scratch (null: one-pass kernels)
    bool shared_gpu = false;           // batched or served: the per-step schedule (throughput)
    unsigned long long generation = 0;
    // the slot buffers this plan needs: name and bytes (see plan_prepare)
    enum { B_IMG, B_BITS, B_TEX, B_FIELDS, B_PARTIAL, B_STATE, B_ROWDIST, B_STAGE, B_FSCR, B_COUNT };
    size_t need[B_COUNT] = {};
};

const char *const kBufName[RegPlan::B_COUNT] = {"img", "bits", "tex", "fields", "partial", "state", "rowdist",
                                                "stage", "fscr"};

// Bytes the slot's buffers must grow by to hold plan `pl` (ws_get rounding).
size_t plan_growth(const RegPlan &pl, const WsSet &ws) {
    size_t g = 0;
    for (int b = 0; b < RegPlan::B_COUNT; ++b) {
        if (!pl.need[b]) continue;
        const size_t cap = round_up(pl.need[b], (size_t)1 << 21);
        auto it = ws.bufs.find(kBufName[b]);
        const size_t have = it == ws.bufs.end() ? 0 : it->second.cap;
        if (have < pl.need[b]) g += cap - have;
    }
    return g;
}

void RegPlanDeleter::operator()(RegPlan *p) const { delete p; }

namespace {

int plan_make(cgdir_ctx *ctx, const cgdir_volume *S, const cgdir_volume *M, const cgdir_masks *SM,
              const cgdir_masks *MM, const cgdir_params *P, int dvf_where, RegPlan &pl) {
    if (!S || !M || !P) return fail(ctx, CGDIR_EINVAL, "register: null argument");
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
        maxcap = std::max(maxcap, P->iters[l]);
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
    {
        int8_t tmp_sign[kMaxMasks];
        for (int j = 0; j < kMaxMasks; ++j) tmp_sign[j] = 1;
        TRY(fill_force_args(ctx, pl.base, k, P->lambda, tmp_sign, P->intensity_offset, 1));
    }
    pl.S = S; pl.M = M; pl.SM = SM; pl.MM = MM; pl.dvf_where = dvf_where;
    pl.P = *P;
    pl.iters.assign(P->iters, P->iters + L);
    pl.P.iters = pl.iters.data();
    pl.P.lambda = nullptr;           // folded into base.lambda
    for (int j = 0; j < k; ++j) {
        const int8_t sj = P->sign ? P->sign[j] : 0;
        pl.sign[j] = sj > 0 ? 1 : (sj < 0 ? -1 : 0);
    }
    pl.P.sign = nullptr;
    pl.nx = nx; pl.ny = ny; pl.nz = nz; pl.k = k; pl.L = L; pl.maxcap = maxcap; pl.hcap = maxcap + 1;
    pl.first = P->init_dvf ? L - 1 : 0;
    pl.sdt = P->storage_dtype >= 0 ? P->storage_dtype : (S->dtype == M->dtype ? S->dtype : CGDIR_F32);
    pl.dims[L - 1][0] = nx; pl.dims[L - 1][1] = ny; pl.dims[L - 1][2] = nz;
    for (int l = L - 2; l >= 0; --l)
        for (int a = 0; a < 3; ++a) pl.dims[l][a] = (pl.dims[l + 1][a] + 1) / 2;
    pl.off[0] = 0;
    for (int l = 0; l < L; ++l) {
        pl.Nl[l] = (size_t)pl.dims[l][0] * pl.dims[l][1] * pl.dims[l][2];
        pl.off[l + 1] = pl.off[l] + round_up(pl.Nl[l], 64);
        pl.ldt[l] = level_storage(pl.sdt, l, L);
        pl.ioff[l + 1] = pl.ioff[l] + round_up(pl.Nl[l], 64) * img_elem_size(pl.ldt[l]);
        pl.toff[l + 1] = pl.toff[l] + round_up(pl.Nl[l], 64) * tex_elem_size(pl.ldt[l]);
    }
    pl.Nf = pl.Nl[L - 1];
    pl.Ntot = pl.off[L];
    // level histories, 5 ints per level, then 128 bytes per level for the
    // cooperative level kernel (RMS-ID sums and grid-barrier words)
    pl.state_bytes = (size_t)L * pl.hcap * sizeof(double) + 5 * CGDIR_MAX_LEVELS * sizeof(int) + 128 * CGDIR_MAX_LEVELS;
    size_t np = 0;
    for (int l = 0; l < L; ++l) {
        const int *d = pl.dims[l];
        np = std::max(np, std::max(force_partial_count(d[0], d[1], d[2], force_zchunk_min(d[0], d[1], d[2])),
                                   metric_partial_count(d[0], d[1], d[2])));
    }
    const size_t Ntot = pl.Ntot, Nf = pl.Nf;
    pl.need[RegPlan::B_IMG] = 2 * pl.ioff[L];
    pl.need[RegPlan::B_BITS] = 3 * Ntot;
    pl.need[RegPlan::B_TEX] = pl.toff[L];
    pl.need[RegPlan::B_FIELDS] = 4 * 3 * Nf * sizeof(float);
    pl.need[RegPlan::B_PARTIAL] = std::max<size_t>(np * kPartialStride * sizeof(double), 256);
    pl.need[RegPlan::B_STATE] = pl.state_bytes;
    pl.need[RegPlan::B_ROWDIST] = std::max<size_t>(uroi_scratch_bytes(Nf), 256);
    const bool need_stage = (S->where == CGDIR_HOST && S->dtype != pl.sdt) ||
                            (M->where == CGDIR_HOST && M->dtype != pl.sdt) ||
                            (k > 0 && (SM->where == CGDIR_HOST || MM->where == CGDIR_HOST));
    pl.need[RegPlan::B_STAGE] = need_stage ? std::max(Nf * 4, (size_t)k * Nf) : 0;
    // two-pass force scratch (sized for the finest level, reused by every level)
    pl.need[RegPlan::B_FSCR] = (ctx->plain_kernels || ctx->fused_force) ? 0 : force_scratch_bytes(Nf, k);
    return CGDIR_OK;
}

// Tune the level shapes of `pl` not seen before (when autotuning is on).
int plan_autotune(cgdir_ctx *ctx, const RegPlan &pl) {
    if (!ctx->autotune_on) return CGDIR_OK;
    for (int l = pl.first; l < pl.L; ++l) {
        const int contour = ((pl.P.contour_level_mask >> l) & 1u) && pl.k > 0;
        if (ctx->tuned.count(TuneKey{pl.dims[l][0], pl.dims[l][1], pl.dims[l][2], contour, pl.ldt[l]})) continue;
        TRY(tune_level(ctx, pl.dims[l][0], pl.dims[l][1], pl.dims[l][2], pl.k, contour, pl.ldt[l],
                       std::max(pl.P.sigma_fluid, pl.P.sigma_diff)));
    }
    return CGDIR_OK;
}

// Take the slot's buffers and copy the caller's inputs in (on stream s).
int plan_prepare(cgdir_ctx *ctx, Slot &sl, RegPlan &pl, cudaStream_t s) {
    const size_t Ntot = pl.Ntot, Nf = pl.Nf;
    const int L = pl.L, k = pl.k;
    void *p[RegPlan::B_COUNT] = {};
    WsSet &ws = sl.ws;
    for (int b = 0; b < RegPlan::B_COUNT; ++b)
        if (pl.need[b]) TRY(ws_get(ctx, ws, s, kBufName[b], pl.need[b], &p[b]));
    void *p_img = p[RegPlan::B_IMG], *p_bits = p[RegPlan::B_BITS], *p_tex = p[RegPlan::B_TEX],
         *p_fields = p[RegPlan::B_FIELDS], *p_part = p[RegPlan::B_PARTIAL], *p_state = p[RegPlan::B_STATE],
         *p_rowdist = p[RegPlan::B_ROWDIST], *p_stage = p[RegPlan::B_STAGE];
    pl.generation = ws.generation;
    for (int l = 0; l < L; ++l) {
        pl.T[l] = (char *)p_img + pl.ioff[l];
        pl.I[l] = (char *)p_img + pl.ioff[L] + pl.ioff[l];
        pl.SB[l] = (uint8_t *)p_bits + pl.off[l];
        pl.MB[l] = (uint8_t *)p_bits + Ntot + pl.off[l];
        pl.UR[l] = (uint8_t *)p_bits + 2 * Ntot + pl.off[l];
    }
    pl.tex = (char *)p_tex;
    pl.ua = (float *)p_fields; pl.ub = pl.ua + 3 * Nf; pl.du = pl.ub + 3 * Nf; pl.du2 = pl.du + 3 * Nf;
    pl.partial = (double *)p_part;
    pl.state = p_state;
    pl.hist = (double *)p_state;
    pl.meta = (int *)((char *)p_state + (size_t)L * pl.hcap * sizeof(double));
    pl.rowdist = (uint8_t *)p_rowdist;
    pl.stage = p_stage;
    pl.fscr = p[RegPlan::B_FSCR];
    pl.ufinal = ((L - 1 - pl.first) % 2 == 0) ? pl.ua : pl.ub;

    // images (finest level), converted to the storage type where needed
    auto ingest = [&](const cgdir_volume *v, void *dst) -> int {
        const size_t bytes = Nf * elem_size(v->dtype);
        if (v->dtype == pl.sdt) {
            CK(cudaMemcpyAsync(dst, v->data, bytes,
                               v->where == CGDIR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
        } else if (v->where == CGDIR_HOST) {
            CK(cudaMemcpyAsync(p_stage, v->data, bytes, cudaMemcpyHostToDevice, s));
            CK(launch_convert_image(p_stage, v->dtype, Nf, dst, pl.sdt, s));
        } else {
            CK(launch_convert_image(v->data, v->dtype, Nf, dst, pl.sdt, s));
        }
        return CGDIR_OK;
    };
    TRY(ingest(pl.S, pl.T[L - 1]));
    TRY(ingest(pl.M, pl.I[L - 1]));
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
    TRY(pack(pl.SM, pl.SB[L - 1]));
    TRY(pack(pl.MM, pl.MB[L - 1]));
    // automatic signs (decided on the host before the device part is enqueued)
    bool need_auto = false;
    for (int j = 0; j < k; ++j) need_auto |= pl.sign[j] == 0;
    if (need_auto) {
        int8_t autos[kMaxMasks];
        CK(cudaStreamSynchronize(s));
        TRY(auto_sign_impl(ctx, pl.T[L - 1], pl.sdt, pl.SB[L - 1], k, pl.nx, pl.ny, pl.nz, autos));
        for (int j = 0; j < k; ++j)
            if (pl.sign[j] == 0) pl.sign[j] = autos[j];
    }
    for (int j = 0; j < k; ++j) pl.base.half_sign[j] = 0.5f * (float)pl.sign[j];
    if (pl.P.init_dvf)
        CK(cudaMemcpyAsync(pl.ua, pl.P.init_dvf, 3 * Nf * sizeof(float),
                           pl.P.init_dvf_where == CGDIR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    return CGDIR_OK;
}

// The device part of a registration (capturable: touches the slot's buffers only).
int plan_enqueue(cgdir_ctx *ctx, const RegPlan &pl, cudaStream_t s, ProfList *prof) {
    const cgdir_params *P = &pl.P;
    const int L = pl.L, k = pl.k;
    const unsigned m = ctx->prof_mask;
    for (int l = L - 2; l >= 0; --l) {
        const int *d = pl.dims[l + 1];
        ProfScope ps(prof, m, s, CGDIR_K_SETUP, l);
        CK(launch_restrict_image(pl.T[l + 1], pl.ldt[l + 1], d[0], d[1], d[2], pl.T[l], pl.ldt[l], s));
        CK(launch_restrict_image(pl.I[l + 1], pl.ldt[l + 1], d[0], d[1], d[2], pl.I[l], pl.ldt[l], s));
        CK(launch_restrict_bits(pl.SB[l + 1], d[0], d[1], d[2], pl.SB[l], s));
        CK(launch_restrict_bits(pl.MB[l + 1], d[0], d[1], d[2], pl.MB[l], s));
    }
    for (int l = 0; l < L; ++l) {
        if (((P->contour_level_mask >> l) & 1u) && k > 0 && !ctx->plain_kernels) {
            ProfScope ps(prof, m, s, CGDIR_K_SETUP, l);
            CK(launch_make_texels(pl.I[l], pl.ldt[l], pl.MB[l], pl.Nl[l], pl.tex + pl.toff[l], s));
        }
        const double f = (double)(1 << (L - 1 - l));
        const double sp[3] = {P->spacing_mm[0] * f, P->spacing_mm[1] * f, P->spacing_mm[2] * f};
        ProfScope ps(prof, m, s, CGDIR_K_SETUP, l);
        CK(launch_uroi(pl.SB[l], k, pl.dims[l][0], pl.dims[l][1], pl.dims[l][2], sp, P->margin_mm, pl.rowdist,
                       pl.UR[l], s));
    }
    CK(cudaMemsetAsync(pl.state, 0, pl.state_bytes, s));
    int *hist_len = pl.meta, *iters_run = pl.meta + CGDIR_MAX_LEVELS, *reason = pl.meta + 2 * CGDIR_MAX_LEVELS,
        *flags = pl.meta + 3 * CGDIR_MAX_LEVELS;
    unsigned *done = (unsigned *)(pl.meta + 4 * CGDIR_MAX_LEVELS);   // per-level completion counters
    float *ucur = pl.ua, *uoth = pl.ub;
    for (int l = pl.first; l < L; ++l) {
        const int lx = pl.dims[l][0], ly = pl.dims[l][1], lz = pl.dims[l][2];
        const int sdt = pl.ldt[l];
        if (l == pl.first) {
            if (!P->init_dvf) CK(cudaMemsetAsync(ucur, 0, 3 * pl.Nl[l] * sizeof(float), s));
        } else {
            ProfScope ps(prof, m, s, CGDIR_K_SETUP, l);
            CK(launch_prolong(ucur, pl.dims[l - 1][0], pl.dims[l - 1][1], pl.dims[l - 1][2], lx, ly, lz, uoth, s));
            std::swap(ucur, uoth);
        }
        LevelState st{};
        st.hist = pl.hist + (size_t)l * pl.hcap;
        st.hist_len = hist_len + l;
        st.iters_run = iters_run + l;
        st.stop_reason = reason + l;
        st.stop_flag = flags + l;
        st.hist_cap = pl.hcap;
        ForceArgs a = pl.base;
        a.I0 = pl.I[l]; a.T0 = pl.T[l]; a.img_dtype = sdt;
        a.mbits = pl.MB[l]; a.sbits = pl.SB[l]; a.uroi = pl.UR[l];
        a.mtex = ctx->plain_kernels ? nullptr : (const void *)(pl.tex + pl.toff[l]);
        a.u = ucur; a.du = pl.du; a.warped = nullptr; a.partial = pl.partial; a.stop_flag = flags + l;
        a.nx = lx; a.ny = ly; a.nz = lz;
        a.contour = ((P->contour_level_mask >> l) & 1u) && k > 0;
        if (pl.fscr) force_scratch_assign(a, pl.fscr, pl.Nl[l]);
        const int zc = force_zchunk_for(ctx, lx, ly, lz, a.contour, sdt);
        a.pass2_width = force_width_for(ctx, lx, ly, lz, a.contour, sdt);
        const SmoothChoice sch = smooth_choice(ctx, lx, ly, lz, a.contour, sdt, !pl.shared_gpu);
        const int cap = P->iters[l];
        a.fin.done = done + l;
        a.fin.st = st;
        a.fin.cap = cap;
        a.fin.stop_mode = P->stop_mode;
        a.fin.eps = P->eps;
        a.fin.stats_out = nullptr;
        // small levels below the finest: all iterations in one cooperative launch
        const int coop_grid = (l < L - 1 && 2 * pl.Nl[l] <= pl.Nf && !ctx->plain_kernels && !ctx->fused_force &&
                               pl.fscr && use_level_coop(ctx, lx, ly, lz, a.contour, sdt))
                                  ? level_coop_grid(lx, ly, lz, a.contour, sdt) : 0;
        if (coop_grid > 0) {
            LevelCoopArgs c{};
            c.f = a;
            c.f.partial = nullptr;
            c.f.fin.done = nullptr;
            c.tmp1 = pl.du2;                                  // 3 N_l floats of 3 N_finest
            c.tmp2 = uoth;                                    // uoth holds 3 N_finest >= 6 N_l
            c.ub = uoth + 3 * pl.Nl[l];
            c.tf = gauss_taps(P->sigma_fluid);
            c.td = gauss_taps(P->sigma_diff);
            c.compose_mode = P->compose_mode;
            char *area = (char *)pl.meta + 5 * CGDIR_MAX_LEVELS * sizeof(int) + 128 * l;
            c.sums = (unsigned long long *)area;
            c.bar = (unsigned *)(area + 64);
            c.err = kerr(ctx);
            ProfScope ps(prof, m, s, CGDIR_K_LEVEL, l);
            CK(launch_level_coop(c, coop_grid, s));
            continue;
        }
        // fused schedule: the force runs its stencil pass only after the first
        // iteration; the smoothing of u' leaves the next warp behind it
        const bool fused = sch.variant == SMOOTH_FUSED && !ctx->plain_kernels && !ctx->fused_force &&
                           fused_schedule_ok(a) && gauss_taps(P->sigma_fluid).r > 0 &&
                           gauss_taps(P->sigma_diff).r > 0;
        for (int n = 0; n < cap; ++n) {
            int nb = 0;
            a.fin.n = n;   // the force kernel's last CTA reduces delta^n and runs the stop test
            a.skip_warp = fused && n > 0;
            { ProfScope ps(prof, m, s, CGDIR_K_FORCE, l); CK(launch_force(a, zc, &nb, s, kerr(ctx))); }
            if (fused) {
                { ProfScope ps(prof, m, s, CGDIR_K_SMOOTH_DU, l);   // steps 2 + 3
                  CK(launch_fused_smooth_compose(pl.du, ucur, P->compose_mode, P->sigma_fluid, lx, ly, lz, pl.du2,
                                                 flags + l, kerr(ctx), s)); }
                { ProfScope ps(prof, m, s, CGDIR_K_SMOOTH_U, l);    // step 4 + the next warp
                  CK(launch_fused_smooth_warp(pl.du2, P->sigma_diff, ucur, a, kerr(ctx), s)); }
                continue;
            }
            { ProfScope ps(prof, m, s, CGDIR_K_SMOOTH_DU, l);   // steps 2 + 3
              CK(launch_smooth_compose(pl.du, ucur, P->compose_mode, P->sigma_fluid, lx, ly, lz, pl.du2, uoth,
                                       flags + l, s, kerr(ctx), ctx->fused_force, sch)); }
            { ProfScope ps(prof, m, s, CGDIR_K_SMOOTH_U, l);    // step 4
              CK(launch_smooth(pl.du2, 3, P->sigma_diff, lx, ly, lz, ucur, flags + l, s, kerr(ctx), sch, uoth)); }
        }
        int nb = 0;
        FinishArgs fm = a.fin;
        fm.n = cap;
        { ProfScope ps(prof, m, s, CGDIR_K_METRIC, l);
          CK(launch_metric(pl.I[l], pl.T[l], sdt, ucur, pl.UR[l], lx, ly, lz, pl.partial, flags + l, &nb, s, &fm)); }
    }
    return CGDIR_OK;
}

std::string plan_key(cgdir_ctx *ctx, const RegPlan &pl) {
    const cgdir_params *P = &pl.P;
    char key[1024];
    const int len = std::snprintf(
        key, sizeof key, "%d %d %d|%d|%d %d %.9g %.9g %d %u %d %.17g %.17g %.17g %.17g %.17g %.9g %d %d %llu %u %d|",
        pl.nx, pl.ny, pl.nz, pl.L, pl.k, pl.first, P->sigma_fluid, P->sigma_diff, P->compose_mode,
        P->contour_level_mask, P->stop_mode, P->eps, P->spacing_mm[0], P->spacing_mm[1], P->spacing_mm[2],
        P->margin_mm, P->intensity_offset, (int)ctx->plain_kernels + 2 * (int)ctx->fused_force + 4 * ctx->smooth_variant + 16 * (int)ctx->tune_gen,
        pl.maxcap, pl.generation, ctx->prof_mask, pl.sdt);
    std::string s(key, (size_t)len);
    s += pl.shared_gpu ? "shared|" : "alone|";
    for (int l = 0; l < pl.L; ++l) s += std::to_string(P->iters[l]) + ",";
    for (int j = 0; j < pl.k; ++j) {
        char b[48];
        std::snprintf(b, sizeof b, "%.9g:%d,", pl.base.lambda[j], (int)pl.sign[j]);
        s += b;
    }
    return s;
}

// Capture `body` (which enqueues on the stream it is given) into a graph.
template <typename Body>
int capture(cgdir_ctx *ctx, GraphEntry &ge, Body body) {
    const unsigned long long before = launches_now();
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = body(ctx->cap_stream, &ge.prof);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
    ge.launches = launches_now() - before;
    launches_sub(ge.launches);        // captured, not yet launched
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
    return CGDIR_OK;
}

// Run the device part of one plan on stream s (graph replay or eager).
int plan_run(cgdir_ctx *ctx, Slot &sl, const RegPlan &pl, cudaStream_t s, const ProfList **used) {
    if (!ctx->use_graphs || !ctx->cap_stream) {
        ctx->eager.recs.clear();
        TRY(plan_enqueue(ctx, pl, s, &ctx->eager));
        *used = &ctx->eager;
        return CGDIR_OK;
    }
    const std::string key = plan_key(ctx, pl);
    auto it = sl.ws.graphs.find(key);
    if (it == sl.ws.graphs.end()) {
        GraphEntry ge;
        TRY(capture(ctx, ge, [&](cudaStream_t cs, ProfList *p) { return plan_enqueue(ctx, pl, cs, p); }));
        it = sl.ws.graphs.emplace(key, std::move(ge)).first;
    }
    CK(cudaGraphLaunch(it->second.exec, s));
    note_launch((unsigned)it->second.launches);
    *used = &it->second.prof;
    return CGDIR_OK;
}

int slot_host_buffers(cgdir_ctx *ctx, Slot &sl, size_t hist_doubles) {
    if (sl.h_hist && sl.h_hist_cap >= hist_doubles) return CGDIR_OK;
    if (sl.h_hist) cudaFreeHost(sl.h_hist);
    sl.h_hist = nullptr;
    CK(cudaMallocHost((void **)&sl.h_hist, hist_doubles * sizeof(double)));
    sl.h_hist_cap = hist_doubles;
    if (!sl.h_meta) CK(cudaMallocHost((void **)&sl.h_meta, 5 * CGDIR_MAX_LEVELS * sizeof(int)));
    return CGDIR_OK;
}

bool is_pinned_or_device(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Enqueue the copies of the result (the DVF unless deferred, the histories).
int plan_outputs(cgdir_ctx *ctx, Slot &sl, const RegPlan &pl, float *dvf_out, bool allow_defer, cudaStream_t s) {
    TRY(slot_host_buffers(ctx, sl, (size_t)pl.L * pl.hcap));
    sl.deferred_copy = false;
    sl.ufinal = pl.ufinal;
    sl.dvf_out = dvf_out;
    if (pl.dvf_where == CGDIR_DEVICE) {
        CK(cudaMemcpyAsync(dvf_out, pl.ufinal, 3 * pl.Nf * sizeof(float), cudaMemcpyDeviceToDevice, s));
    } else if (!allow_defer || is_pinned_or_device(dvf_out)) {
        CK(cudaMemcpyAsync(dvf_out, pl.ufinal, 3 * pl.Nf * sizeof(float), cudaMemcpyDeviceToHost, s));
    } else {
        sl.deferred_copy = true;       // pageable: copied when the request is collected
    }
    CK(cudaMemcpyAsync(sl.h_hist, pl.hist, (size_t)pl.L * pl.hcap * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(sl.h_meta, pl.meta, 4 * CGDIR_MAX_LEVELS * sizeof(int), cudaMemcpyDeviceToHost, s));
    return CGDIR_OK;
}

void plan_stats(const Slot &sl, const RegPlan &pl, cgdir_level_stats *out) {
    if (!out) return;
    for (int l = 0; l < pl.L; ++l) {
        cgdir_level_stats &o = out[l];
        o.level = l;
        o.nx = pl.dims[l][0]; o.ny = pl.dims[l][1]; o.nz = pl.dims[l][2];
        if (l < pl.first) {
            o.iters_run = 0; o.stop_reason = CGDIR_REASON_SKIPPED; o.hist_len = 0; o.rms_id = nullptr;
            continue;
        }
        o.iters_run = sl.h_meta[CGDIR_MAX_LEVELS + l];
        o.stop_reason = sl.h_meta[2 * CGDIR_MAX_LEVELS + l];
        o.hist_len = sl.h_meta[l];
        o.rms_id = sl.h_hist + (size_t)l * pl.hcap;
    }
}

Slot &slot_at(cgdir_ctx *ctx, size_t i) {
    while (ctx->slots.size() <= i) ctx->slots.emplace_back(new Slot());
    return *ctx->slots[i];
}

}  // namespace
}  // namespace rt
}  // namespace cgdir

extern "C" {

int cgdir_register(cgdir_ctx *ctx, const cgdir_volume *S, const cgdir_volume *M,
                   const cgdir_masks *SM, const cgdir_masks *MM, const cgdir_params *P,
                   float *dvf_out, int dvf_where, cgdir_level_stats *stats_out) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->err.clear();
    if (!dvf_out) return fail(ctx, CGDIR_EINVAL, "register: null dvf_out");
    RegPlan pl;
    TRY(plan_make(ctx, S, M, SM, MM, P, dvf_where, pl));
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    Slot &sl = slot_at(ctx, 0);
    if (sl.busy) return fail(ctx, CGDIR_EBUSY, "register: slot 0 is serving a request");
    TRY(plan_autotune(ctx, pl));
    TRY(plan_prepare(ctx, sl, pl, s));
    const ProfList *used = nullptr;
    TRY(plan_run(ctx, sl, pl, s, &used));
    TRY(plan_outputs(ctx, sl, pl, dvf_out, false, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    prof_collect(ctx, *used);
    TRY(check_err_word(ctx));
    plan_stats(sl, pl, stats_out);
    return CGDIR_OK;
}

int cgdir_register_batch(cgdir_ctx *ctx, int count, const cgdir_volume *statics, const cgdir_volume *movings,
                         const cgdir_masks *static_masks, const cgdir_masks *moving_masks,
                         const cgdir_params *params, float *const *dvf_outs, int dvf_where,
                         cgdir_level_stats *stats_out) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->err.clear();
    if (count < 1 || count > 1024 || !statics || !movings || !params || !dvf_outs)
        return fail(ctx, CGDIR_EINVAL, "register_batch: bad arguments");
    std::vector<RegPlan> pls(count);
    for (int i = 0; i < count; ++i) {
        if (!dvf_outs[i]) return fail(ctx, CGDIR_EINVAL, "register_batch: null dvf_out");
        TRY(plan_make(ctx, &statics[i], &movings[i], static_masks ? &static_masks[i] : nullptr,
                      moving_masks ? &moving_masks[i] : nullptr, &params[i], dvf_where, pls[i]));
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    for (int i = 0; i < count; ++i) {
        pls[i].shared_gpu = true;     // the branches share the GPU: throughput over latency
        TRY(plan_autotune(ctx, pls[i]));
    }
    for (int i = 0; i < count; ++i) {
        Slot &sl = slot_at(ctx, (size_t)i);
        if (sl.busy) return fail(ctx, CGDIR_EBUSY, "register_batch: a slot is serving a request");
        TRY(plan_prepare(ctx, sl, pls[i], s));
    }
    // one graph, one branch per case: the branches run concurrently
    std::string key = "batch|";
    for (int i = 0; i < count; ++i) key += plan_key(ctx, pls[i]) + "#";
    auto &cache = ctx->batch.graphs;
    const ProfList *used = nullptr;
    if (ctx->use_graphs && ctx->cap_stream) {
        while ((int)ctx->branch_streams.size() < count) {
            cudaStream_t b;
            CK(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
            ctx->branch_streams.push_back(b);
        }
        auto it = cache.find(key);
        if (it == cache.end()) {
            if (cache.size() >= 8) drop_graphs(ctx->batch);
            // fork / join events, made before the capture
            std::vector<cudaEvent_t> evs(count + 1, nullptr);
            int rc = CGDIR_OK;
            for (auto &e : evs)
                if (rc == CGDIR_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                    rc = fail(ctx, CGDIR_ECUDA, "register_batch: event creation failed");
            GraphEntry ge;
            if (rc == CGDIR_OK)
                rc = capture(ctx, ge, [&](cudaStream_t cs, ProfList *p) -> int {
                    CK(cudaEventRecord(evs[0], cs));
                    for (int i = 0; i < count; ++i) {
                        cudaStream_t b = ctx->branch_streams[i];
                        CK(cudaStreamWaitEvent(b, evs[0], 0));
                        TRY(plan_enqueue(ctx, pls[i], b, p));
                        CK(cudaEventRecord(evs[i + 1], b));
                        CK(cudaStreamWaitEvent(cs, evs[i + 1], 0));
                    }
                    return CGDIR_OK;
                });
            for (auto &e : evs)
                if (e) cudaEventDestroy(e);
            TRY(rc);
            it = cache.emplace(key, std::move(ge)).first;
        }
        CK(cudaGraphLaunch(it->second.exec, s));
        note_launch((unsigned)it->second.launches);
        used = &it->second.prof;
    } else {
        ctx->eager.recs.clear();
        for (int i = 0; i < count; ++i) TRY(plan_enqueue(ctx, pls[i], s, &ctx->eager));
        used = &ctx->eager;
    }
    for (int i = 0; i < count; ++i) TRY(plan_outputs(ctx, *ctx->slots[i], pls[i], dvf_outs[i], false, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    prof_collect(ctx, *used);
    TRY(check_err_word(ctx));
    if (stats_out)
        for (int i = 0; i < count; ++i) plan_stats(*ctx->slots[i], pls[i], stats_out + (size_t)i * pls[i].L);
    return CGDIR_OK;
}

// ---- serving ---------------------------------------------------------------
int cgdir_set_max_inflight(cgdir_ctx *ctx, int n) {
    if (!ctx || n < 1 || n > 256) return CGDIR_EINVAL;
    ctx->max_slots = n;
    return CGDIR_OK;
}

int cgdir_submit(cgdir_ctx *ctx, const cgdir_volume *S, const cgdir_volume *M, const cgdir_masks *SM,
                 const cgdir_masks *MM, const cgdir_params *P, float *dvf_out, int dvf_where,
                 long long *ticket) {
    if (!ctx) return CGDIR_EINVAL;
    ctx->err.clear();
    if (!dvf_out || !ticket) return fail(ctx, CGDIR_EINVAL, "submit: null argument");
    std::unique_ptr<RegPlan, RegPlanDeleter> pl(new RegPlan());
    TRY(plan_make(ctx, S, M, SM, MM, P, dvf_where, *pl));
    DeviceGuard g(ctx->device);
    // a request submitted while others run shares the GPU: the throughput
    // schedule (capped smoothing, per-step kernels); one that starts on an
    // idle GPU takes the latency schedule of cgdir_register.  Either gives
    // the same bits.  (Poisson arrivals of the 32-case mix at 16 requests/s,
    // FP16, 3 in flight: p50 / p99 47.8 / 164 ms against 51.0 / 160 with the
    // throughput schedule for every request and 48.1 / 200 with the latency one.)
    int running = 0;
    for (auto &o : ctx->slots)
        if (o->busy && o->done && cudaEventQuery(o->done) == cudaErrorNotReady) ++running;
    cudaGetLastError();
    pl->shared_gpu = ctx->serve_schedule == 0 || (ctx->serve_schedule == 2 && running > 0);
    TRY(plan_autotune(ctx, *pl));
    // a free slot (slot 0 is left to cgdir_register): first one that already
    // holds a graph for this request (no capture, no growth), else the one
    // whose buffers must grow least
    int pick = -1;
    size_t best = (size_t)-1;
    bool best_warm = false;
    for (int i = 1; i <= ctx->max_slots; ++i) {
        Slot &sl = slot_at(ctx, (size_t)i);
        if (sl.busy) continue;
        const size_t grow = plan_growth(*pl, sl.ws);
        bool warm = false;
        if (grow == 0 && ctx->use_graphs) {
            pl->generation = sl.ws.generation;
            warm = sl.ws.graphs.count(plan_key(ctx, *pl)) > 0;
        }
        if ((warm && !best_warm) || (warm == best_warm && grow < best)) {
            best = grow;
            best_warm = warm;
            pick = i;
        }
    }
    if (pick < 0) return fail(ctx, CGDIR_EBUSY, "submit: every slot is busy");
    Slot &sl = *ctx->slots[pick];
    // admission by the device-memory budget: what this request must add
    if (ctx->budget && ctx->in_use + best > ctx->budget)
        return fail(ctx, CGDIR_EBUSY, "submit: the device-memory budget cannot admit this request now");
    // the request's stream: ranked by age among the running requests (one
    // submitted while n others run is n priority levels below the highest),
    // so the device schedules the older requests' kernels first and the
    // younger ones fill the gaps; a graph runs at the priority of the stream
    // it is launched into
    int prio = 0;
    if (ctx->serve_priority) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        prio = std::min(least, greatest + running);
    }
    if (sl.stream && sl.own_stream && sl.priority != prio) {
        CK(cudaStreamDestroy(sl.stream));      // idle: its last request completed
        sl.stream = nullptr;
    }
    if (!sl.stream) {
        CK(cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio));
        sl.own_stream = true;
        sl.priority = prio;
    }
    if (!sl.done) CK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    if (!sl.ready) CK(cudaEventCreateWithFlags(&sl.ready, cudaEventDisableTiming));
    // inputs written on the context's stream are complete before the request reads them
    CK(cudaEventRecord(sl.ready, ctx->stream));
    CK(cudaStreamWaitEvent(sl.stream, sl.ready, 0));
    const int rc = [&]() -> int {
        TRY(plan_prepare(ctx, sl, *pl, sl.stream));
        const ProfList *used = nullptr;
        TRY(plan_run(ctx, sl, *pl, sl.stream, &used));
        TRY(plan_outputs(ctx, sl, *pl, dvf_out, true, sl.stream));
        CK(cudaEventRecord(sl.done, sl.stream));
        return CGDIR_OK;
    }();
    if (rc != CGDIR_OK) return rc;
    sl.busy = true;
    sl.ticket = ctx->next_ticket++;
    sl.plan = std::move(pl);
    sl.status = CGDIR_OK;
    *ticket = sl.ticket;
    return CGDIR_OK;
}

static Slot *find_ticket(cgdir_ctx *ctx, long long t) {
    for (auto &sl : ctx->slots)
        if (sl->busy && sl->ticket == t) return sl.get();
    return nullptr;
}

// Complete a finished request: deferred DVF copy, error word.
static int collect(cgdir_ctx *ctx, Slot &sl) {
    if (sl.deferred_copy) {
        CK(cudaMemcpy(sl.dvf_out, sl.ufinal, 3 * sl.plan->Nf * sizeof(float), cudaMemcpyDeviceToHost));
        sl.deferred_copy = false;
    }
    return check_err_word(ctx);
}

int cgdir_poll(cgdir_ctx *ctx, long long ticket) {
    if (!ctx) return CGDIR_EINVAL;
    Slot *sl = find_ticket(ctx, ticket);
    if (!sl) return fail(ctx, CGDIR_EINVAL, "poll: unknown or collected ticket");
    DeviceGuard g(ctx->device);
    const cudaError_t q = cudaEventQuery(sl->done);
    if (q == cudaErrorNotReady) return CGDIR_EBUSY;
    if (q != cudaSuccess) return fail(ctx, CGDIR_ECUDA, std::string("poll: ") + cudaGetErrorString(q));
    return collect(ctx, *sl);
}

int cgdir_wait(cgdir_ctx *ctx, long long ticket, int timeout_ms) {
    if (!ctx) return CGDIR_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int r = cgdir_poll(ctx, ticket);
        if (r != CGDIR_EBUSY) return r;
        if (timeout_ms >= 0 &&
            std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
            return fail(ctx, CGDIR_ETIMEDOUT, "wait: the request did not finish in time");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int cgdir_release(cgdir_ctx *ctx, long long ticket, cgdir_level_stats *stats_out) {
    if (!ctx) return CGDIR_EINVAL;
    Slot *sl = find_ticket(ctx, ticket);
    if (!sl) return fail(ctx, CGDIR_EINVAL, "release: unknown ticket");
    DeviceGuard g(ctx->device);
    const cudaError_t q = cudaEventQuery(sl->done);
    if (q == cudaErrorNotReady) return CGDIR_EBUSY;
    if (q != cudaSuccess) return fail(ctx, CGDIR_ECUDA, std::string("release: ") + cudaGetErrorString(q));
    if (sl->deferred_copy) TRY(collect(ctx, *sl));
    plan_stats(*sl, *sl->plan, stats_out);
    sl->busy = false;
    sl->ticket = -1;
    return CGDIR_OK;
}

int cgdir_cancel(cgdir_ctx *ctx, long long ticket) {
    if (!ctx) return CGDIR_EINVAL;
    Slot *sl = find_ticket(ctx, ticket);
    if (!sl) return fail(ctx, CGDIR_EINVAL, "cancel: unknown ticket");
    DeviceGuard g(ctx->device);
    // raise every level's stop flag: the request's remaining kernels return at once
    static const int ones[CGDIR_MAX_LEVELS] = {1, 1, 1, 1, 1, 1, 1, 1};
    int *flags = sl->plan->meta + 3 * CGDIR_MAX_LEVELS;
    CK(cudaMemcpyAsync(flags, ones, sizeof ones, cudaMemcpyHostToDevice, ctx->cap_stream));
    CK(cudaStreamSynchronize(ctx->cap_stream));
    CK(cudaEventSynchronize(sl->done));
    sl->deferred_copy = false;
    sl->busy = false;
    sl->ticket = -1;
    return CGDIR_OK;
}

}  // extern "C"
