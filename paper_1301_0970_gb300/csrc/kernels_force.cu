// Moving-vector kernel of CG-DIR (kernels 2, 3 and the image half of 4 in
// Sec. 2.2; Algorithm A steps 1, 5 and 6): warp of the moving image and of
// the structure terms, central-difference gradients, the amplitude v of
// Eq. 7 with beta = (T0 - I0~)^2, du = v n, and the per-block partial sums of
// the UROI RMS-ID.  Plus the metric-only warp and the deterministic FP64
// finalisation of the stopping metric.
//
// Structure terms without stored modified images: with J = I0 + offset and
// m_i(c) the moving mask bit at interpolation corner c,
//   I_i~ = sum_c w_c (1 + s_i m_i(c)/2) J(c) = J~ + (s_i/2) P_i,
//   P_i  = sum_c w_c m_i(c) J(c),
// and J~ = I0~ + offset, so grad I_i~ = grad I0~ + (s_i/2) grad P_i and
//   a_i = grad I_i~ . n = |grad I0~| + (s_i/2) grad P_i . n,
//   r_i = T_i - I_i~ = r0 + (s_i/2) (n_i (T0 + offset) - P_i).
// These are the quantities of Eq. 7 rearranged exactly; only P_i (k values)
// is interpolated per point besides I0~.
//
// Two versions share the tiling below.  The TMA version (used whenever the
// volume satisfies the tensor-map rules and fits 32-bit indexing) streams,
// per plane, the DVF tile with its halo and the static-side tiles (T0, mask
// bits, UROI) into a 4-stage shared-memory ring with cp.async.bulk.tensor,
// interpolates with 32-bit corner offsets, and takes a fast path where all
// 8 corners share the same mask bits (then P_i = bit_i (I0~ + offset) and,
// where the whole 7-point stencil agrees, grad P_i = bit_i grad I0~), so
// the per-structure work reduces to a few flops away from ROI borders.  The
// plain version keeps the per-corner accumulation everywhere.
//
// Tiling: a CTA owns a 32 x 8 column of voxels in x-y and marches along z
// over `zchunk` planes.  For each plane it interpolates I0~ and P_i at the
// (32+2) x (8+2) points of the tile plus a one-voxel halo into a three-plane
// ring in shared memory; the gradients of the middle plane are then read
// from the ring.  Halo points outside the volume take the clamped index,
// which reproduces the clamped central difference at the border.
#include <algorithm>

#include "cgdir_internal.cuh"
#include "tma.cuh"
#include "warp_corners.cuh"

namespace cgdir {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int HX = TX + 2, HY = TY + 2, HP = HX * HY;

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block reduction of (ssd, count, max) into partial[bid].  Each thread's
// SSD covers only its own column of a z-chunk (a few dozen non-negative
// terms) and is kept in FP32; it enters the block sum as an exact
// fixed-point integer (units of 2^-12 HU^2), so the in-block sum is exact
// and independent of order and needs no FP64 arithmetic (slow on this
// GPU).  The block total is exactly representable in FP64 and the
// cross-block sum (finalize_block) is FP64.
constexpr float kSsdScale = 4096.f;

template <int NTHREADS>
__device__ void block_partial(float ssd_f, int cnt_i, float mx, double *partial, int bid) {
    __shared__ unsigned long long rs[NTHREADS / 32];
    __shared__ double rd[NTHREADS / 32];
    __shared__ int rc[NTHREADS / 32];
    __shared__ float rm[NTHREADS / 32];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    // beyond 2^40 HU^2 per thread the fixed-point block sum could overflow:
    // such a block (never met by CT-range images) sums in FP64 instead
    const bool wide = __syncthreads_or(!(ssd_f <= 1.0995e12f));
    unsigned long long q = wide ? 0ull : __float2ull_rn(ssd_f * kSsdScale);
    double d = wide ? (double)ssd_f : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (wide) d += __shfl_xor_sync(0xffffffffu, d, o);
        else q += __shfl_xor_sync(0xffffffffu, q, o);
        cnt_i += __shfl_xor_sync(0xffffffffu, cnt_i, o);
    }
    mx = warp_max(mx);
    if ((tid & 31) == 0) { rs[tid >> 5] = q; rd[tid >> 5] = d; rc[tid >> 5] = cnt_i; rm[tid >> 5] = mx; }
    __syncthreads();
    if (tid == 0) {
        unsigned long long s = 0;
        double sd = 0.0;
        long long c = 0;
        float m = 0.f;
        for (int w = 0; w < NTHREADS / 32; ++w) { s += rs[w]; sd += rd[w]; c += rc[w]; m = fmaxf(m, rm[w]); }
        partial[(size_t)bid * kPartialStride + 0] = wide ? sd : (double)s * (1.0 / (double)kSsdScale);
        partial[(size_t)bid * kPartialStride + 1] = (double)c;
        partial[(size_t)bid * kPartialStride + 2] = (double)m;
        partial[(size_t)bid * kPartialStride + 3] = 0.0;
    }
}

// Stopping test of Sec. 2.2 on delta^n = dn and the earlier deltas it needs
// (same readings as the C ABI): WINDOW10 compares delta^(n-10), PAPER_LITERAL
// the steps delta^(n-1) -> delta^n and delta^(n-11) -> delta^(n-10).
struct PastDeltas {
    double d1, d10, d11;                 // delta^(n-1), delta^(n-10), delta^(n-11) (where n allows)
};
__device__ __forceinline__ PastDeltas past_deltas(const double *d, int n, int mode) {
    PastDeltas p{0.0, 0.0, 0.0};
    if (mode == CGDIR_STOP_WINDOW10 && n >= 10) p.d10 = d[n - 10];
    if (mode == CGDIR_STOP_PAPER_LITERAL && n >= 11) { p.d1 = d[n - 1]; p.d10 = d[n - 10]; p.d11 = d[n - 11]; }
    return p;
}
__device__ int stop_test(double dn, const PastDeltas &p, int n, int mode, double eps) {
    if (mode == CGDIR_STOP_WINDOW10) return (n >= 10) && (p.d10 - dn <= eps);
    if (mode == CGDIR_STOP_PAPER_LITERAL) {
        if (n < 11) return 0;
        const double ln = dn - p.d1, lm = p.d10 - p.d11;
        return (lm - ln) <= eps;
    }
    return 0;
}

// Fixed-order sum of the per-CTA partials, RMS-ID into the level history and
// the stop decision (kernel 5).  Run by one whole CTA (any shape, blockDim a
// multiple of 32, at most 1024 threads): each thread sums a fixed stride of
// partials, then warp shuffles and warp 0 combine them in a fixed order.
__device__ void finalize_block(const double *__restrict__ partial, int nblocks, const FinishArgs &f) {
    __shared__ double ws[32], wc[32], wm[32];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    double s = 0.0, c = 0.0, m = 0.0;
    // the earlier deltas of the stop test, read now so their latency overlaps the sums
    PastDeltas past{0.0, 0.0, 0.0};
    if (tid == 0 && f.st.hist) past = past_deltas(f.st.hist, f.n, f.stop_mode);
    // four partials in flight per thread, summed in the same (ascending) order
    constexpr int U = 4;
    int b = tid;
    for (; b + (U - 1) * nt < nblocks; b += U * nt) {
        double3 v[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const double *p = partial + (size_t)(b + q * nt) * kPartialStride;
            v[q] = make_double3(__ldcg(p), __ldcg(p + 1), __ldcg(p + 2));
        }
#pragma unroll
        for (int q = 0; q < U; ++q) { s += v[q].x; c += v[q].y; m = fmax(m, v[q].z); }
    }
    for (; b < nblocks; b += nt) {
        s += __ldcg(partial + (size_t)b * kPartialStride + 0);
        c += __ldcg(partial + (size_t)b * kPartialStride + 1);
        m = fmax(m, __ldcg(partial + (size_t)b * kPartialStride + 2));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((tid & 31) == 0) { ws[tid >> 5] = s; wc[tid >> 5] = c; wm[tid >> 5] = m; }
    __syncthreads();
    if (tid == 0) {
        double S = 0.0, C = 0.0, M = 0.0;
        for (int w = 0; w < nt / 32; ++w) { S += ws[w]; C += wc[w]; M = fmax(M, wm[w]); }
        if (f.stats_out) { f.stats_out[0] = S; f.stats_out[1] = C; f.stats_out[2] = M; }
        const LevelState &st = f.st;
        if (st.hist) {
            const double d = C > 0 ? sqrt(S / C) : 0.0;
            if (f.n < st.hist_cap) st.hist[f.n] = d;
            *st.hist_len = f.n + 1;
            if (stop_test(d, past, f.n, f.stop_mode, f.eps)) {
                *st.stop_flag = 1; *st.iters_run = f.n; *st.stop_reason = CGDIR_REASON_CONVERGED;
            } else if (f.n >= f.cap) {
                *st.stop_flag = 1; *st.iters_run = f.n; *st.stop_reason = CGDIR_REASON_CAP;
            }
        }
    }
}

// Called by every CTA after its partial is written: the CTA that completes
// the grid runs finalize_block and resets the counter for the next launch.
__device__ void finish_if_last(const double *partial, int nblocks, const FinishArgs &f) {
    __shared__ int last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(f.done, 1u) == (unsigned)(nblocks - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        finalize_block(partial, nblocks, f);
        if (tid == 0) *f.done = 0u;
    }
}

// Interpolate I0~ and the k structure sums P_i at the halo points of plane zz.
// slot layout: [1 + k][HP].
template <bool CONTOUR, typename IT>
__device__ __forceinline__ void force_plane(const ForceArgs &a, int zz, float *slot, int x0, int y0,
                                            int tid) {
    const IT *I0 = static_cast<const IT *>(a.I0);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const size_t N = (size_t)nx * ny * nz;
    const int gz = clampi(zz, 0, nz - 1);
    for (int p = tid; p < HP; p += NT) {
        const int hx = p % HX, hy = p / HX;
        const int gx = clampi(x0 - 1 + hx, 0, nx - 1), gy = clampi(y0 - 1 + hy, 0, ny - 1);
        const size_t i = vox(gx, gy, gz, nx, ny);
        const float ux = __ldg(a.u + i), uy = __ldg(a.u + N + i), uz = __ldg(a.u + 2 * N + i);
        const Corners c = corners((float)gx + ux, (float)gy + uy, (float)gz + uz, nx, ny, nz);
        float acc = 0.f;
        float P[kMaxMasks];
#pragma unroll
        for (int j = 0; j < kMaxMasks; ++j) P[j] = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int cx = (q & 1) ? c.x1 : c.x0;
            const int cy = (q & 2) ? c.y1 : c.y0;
            const int cz = (q & 4) ? c.z1 : c.z0;
            const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                            ((q & 4) ? c.wz : 1.f - c.wz);
            const size_t ci = vox(cx, cy, cz, nx, ny);
            const float v = ld_img<IT>(I0 + ci);
            acc = fmaf(w, v, acc);
            if (CONTOUR) {
                const unsigned b = __ldg(a.mbits + ci);
                const float wj = w * (v + a.offset);
#pragma unroll
                for (int j = 0; j < kMaxMasks; ++j)
                    if (j < a.k && ((b >> j) & 1u)) P[j] += wj;
            }
        }
        slot[p] = acc;
        if (CONTOUR) {
#pragma unroll
            for (int j = 0; j < kMaxMasks; ++j)
                if (j < a.k) slot[(1 + j) * HP + p] = P[j];
        }
    }
}

template <bool CONTOUR, typename IT>
__global__ void __launch_bounds__(NT) k_force(ForceArgs a, int zchunk) {
    if (a.stop_flag && *a.stop_flag) return;
    extern __shared__ float sm[];
    const int plane = (1 + (CONTOUR ? a.k : 0)) * HP;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const size_t N = (size_t)nx * ny * nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    const int c = (ty + 1) * HX + (tx + 1);

    force_plane<CONTOUR, IT>(a, zb - 1, sm, x0, y0, tid);
    force_plane<CONTOUR, IT>(a, zb, sm + plane, x0, y0, tid);
    float ssd = 0.f;
    int cnt = 0;
    float mx = 0.f;
    for (int z = zb; z < ze; ++z) {
        const int r = z - zb;
        float *Pm = sm + (r % 3) * plane, *Pc = sm + ((r + 1) % 3) * plane,
              *Pp = sm + ((r + 2) % 3) * plane;
        force_plane<CONTOUR, IT>(a, z + 1, Pp, x0, y0, tid);
        __syncthreads();
        if (act) {
            const size_t i = vox(x, y, z, nx, ny);
            const float w0 = Pc[c];
            const float gx = 0.5f * (Pc[c + 1] - Pc[c - 1]);
            const float gy = 0.5f * (Pc[c + HX] - Pc[c - HX]);
            const float gz = 0.5f * (Pp[c] - Pm[c]);
            const float T = ld_img<IT>(static_cast<const IT *>(a.T0) + i);
            const float r0 = T - w0;
            if (a.warped) a.warped[i] = w0;
            const float g2 = gx * gx + gy * gy + gz * gz;
            float dux = 0.f, duy = 0.f, duz = 0.f;
            if (g2 != 0.f) {
                const float gn = sqrtf(g2);
                const float inv = 1.f / gn;
                const float nxv = gx * inv, nyv = gy * inv, nzv = gz * inv;
                float num = gn * r0, den = gn * gn;
                if (CONTOUR) {
                    const unsigned sb = __ldg(a.sbits + i);
                    const float Toff = T + a.offset;
#pragma unroll
                    for (int j = 0; j < kMaxMasks; ++j) {
                        if (j < a.k) {
                            const float *Pjm = Pm + (1 + j) * HP, *Pjc = Pc + (1 + j) * HP,
                                        *Pjp = Pp + (1 + j) * HP;
                            const float dPx = 0.5f * (Pjc[c + 1] - Pjc[c - 1]);
                            const float dPy = 0.5f * (Pjc[c + HX] - Pjc[c - HX]);
                            const float dPz = 0.5f * (Pjp[c] - Pjm[c]);
                            const float hs = a.half_sign[j];
                            const float aj = gn + hs * (dPx * nxv + dPy * nyv + dPz * nzv);
                            const float inside = ((sb >> j) & 1u) ? Toff : 0.f;
                            const float rj = r0 + hs * (inside - Pjc[c]);
                            num = fmaf(a.lambda[j] * aj, rj, num);
                            den = fmaf(a.lambda[j] * aj, aj, den);
                        }
                    }
                }
                const float v = num / (den + r0 * r0);
                dux = v * nxv; duy = v * nyv; duz = v * nzv;
            }
            a.du[i] = dux;
            a.du[N + i] = duy;
            a.du[2 * N + i] = duz;
            if (a.uroi == nullptr || __ldg(a.uroi + i)) {
                ssd = fmaf(r0, r0, ssd);
                cnt += 1;
            }
            mx = fmaxf(mx, sqrtf(dux * dux + duy * duy + duz * duz));
        }
        __syncthreads();
    }
    if (a.partial) {
        block_partial<NT>(ssd, cnt, mx, a.partial,
                          (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
        if (a.fin.done) finish_if_last(a.partial, gridDim.x * gridDim.y * gridDim.z, a.fin);
    }
}


// ---- two-pass version --------------------------------------------------------
// Pass 1 (k_warp_pass): one thread per voxel, no halo and no barrier, so the
// eight independent corner gathers of many voxels are in flight at once.  It
// writes I0~, and for the structure terms the AND / OR of the corners' mask
// bits; P_j is stored only where the corners disagree on bit j -- elsewhere
// it is bit_j (I0~ + offset), rebuilt in pass 2 from I0~ and the bits.
// Pass 2 (k_force_pass): each thread marches its (x, y) column along z with
// the z-1, z, z+1 values in registers and the x / y neighbours from L1,
// forms the gradients, Eq. 7 and du, and the RMS-ID partials.  Pass 1 costs
// 6 + 4k bytes per voxel of extra traffic (written, then read once), but
// both passes keep all warps busy instead of waiting at per-plane barriers.
template <bool CONTOUR, typename IT>
__global__ void __launch_bounds__(NT, 4) k_warp_pass(ForceArgs a, int zw) {
    if (a.stop_flag && *a.stop_flag) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int nxy = nx * ny, N = nxy * nz;
    const int zb = blockIdx.z * zw, ze = min(zb + zw, nz);
    const float *__restrict__ u = a.u;
    // two planes at a time: both points' 16 corner loads are in flight
    // together, and the next two planes' displacements load meanwhile
    const int col = y * nx + x;
    auto disp = [&](int z, float &dx, float &dy, float &dz) {
        const int i = z * nxy + col;
        dx = __ldg(u + i); dy = __ldg(u + N + i); dz = __ldg(u + N + N + i);
    };
    float ax = 0.f, ay = 0.f, az = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    if (zb < ze) disp(zb, ax, ay, az);
    if (zb + 1 < ze) disp(zb + 1, bx, by, bz);
    int z = zb;
    for (; z + 1 < ze; z += 2) {
        CornerSet<IT> c0, c1;
        corner_load<CONTOUR, IT>(a, ax, ay, az, x, y, z, c0);
        corner_load<CONTOUR, IT>(a, bx, by, bz, x, y, z + 1, c1);
        if (z + 2 < ze) disp(z + 2, ax, ay, az);
        if (z + 3 < ze) disp(z + 3, bx, by, bz);
        corner_finish<CONTOUR, IT>(a, z * nxy + col, N, c0);
        corner_finish<CONTOUR, IT>(a, (z + 1) * nxy + col, N, c1);
    }
    if (z < ze) {
        CornerSet<IT> c0;
        corner_load<CONTOUR, IT>(a, ax, ay, az, x, y, z, c0);
        corner_finish<CONTOUR, IT>(a, z * nxy + col, N, c0);
    }
}

// Sums over a set m of structures (bit j = structure j), one table entry
// per m: Lam = sum lambda_j, H1 = sum lambda_j h_j, H2 = sum lambda_j
// (2 h_j + h_j^2), H3 = sum lambda_j h_j (1 + h_j), with h_j = s_j / 2.
// For a structure whose bits agree over the stencil (b_j: P_j =
// b_j (I0~ + offset); c_j = 1 + h_j b_j; n_j its static bit) the Eq. 7 terms
// are a_j = |g| c_j and r_j = r0 + h_j d_j with d_j = n_j T' - b_j J
// (T' = T0 + offset, J = I0~ + offset), so over a set U of such structures
//   sum lambda_j a_j r_j = |g| (r0 (Lam[U] + H1[b]) + (T' - J) H3[n & b]
//                               + T' H1[n & ~b] - J H3[b & ~n])
//   sum lambda_j a_j^2  = |g|^2 (Lam[U] + H2[b])
// (b, n restricted to U): table reads instead of a loop over the
// structures.  Identical images and masks give exactly r0 = 0, T' = J and
// n = b, hence exactly zero.
struct ContourTables {
    float lam[256], h1[256], h2[256], h3[256];
};

__device__ __forceinline__ void build_tables(const ForceArgs &a, ContourTables &t, int tid) {
    for (int m = tid; m < 256; m += NT) {
        float L = 0.f, A1 = 0.f, A2 = 0.f, A3 = 0.f;
        for (int j = 0; j < a.k; ++j) {
            if ((m >> j) & 1) {
                const float l = a.lambda[j], h = a.half_sign[j];
                L += l;
                A1 += l * h;
                A2 += l * (2.f * h + h * h);
                A3 += l * h * (1.f + h);
            }
        }
        t.lam[m] = L; t.h1[m] = A1; t.h2[m] = A2; t.h3[m] = A3;
    }
}

// P_j at a stencil point from pass 1's outputs.
__device__ __forceinline__ float p_at(const ForceArgs &a, int j, int N, int idx, float w, unsigned st) {
    const unsigned andb = st >> 8, orb = st & 0xffu;
    if ((((orb & ~andb) >> j) & 1u) != 0u) return __ldg(a.pfield + (size_t)j * N + idx);
    return ((andb >> j) & 1u) ? w + a.offset : 0.f;
}
// The same through L2-only loads (P_j written by the same kernel).
__device__ __forceinline__ float p_at_l2(const ForceArgs &a, int j, int N, int idx, float w, unsigned st) {
    const unsigned andb = st >> 8, orb = st & 0xffu;
    if ((((orb & ~andb) >> j) & 1u) != 0u) return __ldcg(a.pfield + (size_t)j * N + idx);
    return ((andb >> j) & 1u) ? w + a.offset : 0.f;
}

// As force_voxel below, with the stencil's corner-bit AND (A) and OR (O)
// over its seven points already formed by the caller.
template <bool CONTOUR, bool L2ONLY = false>
__device__ __forceinline__ void force_voxel_ao(const ForceArgs &a, const ContourTables &tab, int N, float w0,
                                               float Wxm, float Wxp, float Wym, float Wyp, float Wm, float Wp,
                                               float T, unsigned A, unsigned O, unsigned Sc, unsigned Sxm,
                                               unsigned Sxp, unsigned Sym, unsigned Syp, unsigned Sm, unsigned Sp,
                                               unsigned sb, int ic, int ixm, int ixp, int iym, int iyp, int im,
                                               int ip, float &dux, float &duy, float &duz, float &r0) {
    const float off = a.offset;
    const float gxv = 0.5f * (Wxp - Wxm), gyv = 0.5f * (Wyp - Wym), gzv = 0.5f * (Wp - Wm);
    r0 = T - w0;
    const float g2 = fmaf(gzv, gzv, fmaf(gyv, gyv, __fmul_rn(gxv, gxv)));
    dux = 0.f; duy = 0.f; duz = 0.f;
    // a vanishing gradient gives no force; below |g|^2 = 1e-30 (far below
    // the rounding of any image value) the gradient counts as vanishing, so
    // the reciprocal root never meets a subnormal argument
    if (!(g2 > 1e-30f)) return;
    const float inv = rsqrtf(g2);
    const float gn = __fmul_rn(g2, inv);
    const float nxv = __fmul_rn(gxv, inv), nyv = __fmul_rn(gyv, inv), nzv = __fmul_rn(gzv, inv);
    float num = __fmul_rn(gn, r0), den = __fmul_rn(gn, gn);
    if (CONTOUR && (O | sb) == 0u) {
        // no structure at any corner of the stencil nor at the static voxel:
        // every table entry below is entry 0 (all sums zero) but lam[all],
        // and the multiply-adds of zero sums change nothing, so this is the
        // same arithmetic without the lookups
        const float c1 = 1.f + tab.lam[(1u << a.k) - 1u];
        num = __fmul_rn(gn, __fmul_rn(r0, c1));
        den = __fmul_rn(__fmul_rn(gn, gn), c1);
    } else if (CONTOUR) {
        const float Toff = T + off;
        const unsigned kmask = (1u << a.k) - 1u;
        unsigned mixed = O & ~A & kmask;
        {
            const unsigned U = kmask & ~mixed, bU = A & U, nU = sb & U;
            const float J = w0 + off;
            const float cr = 1.f + tab.lam[U] + tab.h1[bU];
            float cn = __fmul_rn(r0, cr);
            cn = fmaf(Toff - J, tab.h3[nU & bU], cn);
            cn = fmaf(Toff, tab.h1[nU & ~bU], cn);
            cn = fmaf(-J, tab.h3[bU & ~nU], cn);
            num = __fmul_rn(gn, cn);
            den = __fmul_rn(__fmul_rn(gn, gn), 1.f + tab.lam[U] + tab.h2[bU]);
        }
        // near a structure border: P_j from pass 1 at the stencil points
        while (mixed) {
            const int j = __ffs(mixed) - 1;
            mixed &= mixed - 1u;
            const float hs = a.half_sign[j];
            const float inside = ((sb >> j) & 1u) ? Toff : 0.f;
            auto P = [&](int idx, float w, unsigned st) {
                return L2ONLY ? p_at_l2(a, j, N, idx, w, st) : p_at(a, j, N, idx, w, st);
            };
            const float dPx = 0.5f * (P(ixp, Wxp, Sxp) - P(ixm, Wxm, Sxm));
            const float dPy = 0.5f * (P(iyp, Wyp, Syp) - P(iym, Wym, Sym));
            const float dPz = 0.5f * (P(ip, Wp, Sp) - P(im, Wm, Sm));
            const float aj = fmaf(hs, fmaf(dPz, nzv, fmaf(dPy, nyv, __fmul_rn(dPx, nxv))), gn);
            const float rj = fmaf(hs, inside - P(ic, w0, Sc), r0);
            num = fmaf(a.lambda[j] * aj, rj, num);
            den = fmaf(a.lambda[j] * aj, aj, den);
        }
    }
    const float v = __fdividef(num, fmaf(r0, r0, den));
    dux = __fmul_rn(v, nxv); duy = __fmul_rn(v, nyv); duz = __fmul_rn(v, nzv);
}

// Eq. 7 at one voxel from its 7-point stencil of I0~ (w0 centre; x-, x+,
// y-, y+, z-, z+ neighbours) and corner-bit words, the static image T and
// bits sb; i* are the stencil points' indices (for the stored P_j).  Every
// multiply-add is written out (no compiler contraction), so the result does
// not depend on where this function is inlined.
template <bool CONTOUR, bool L2ONLY = false>
__device__ __forceinline__ void force_voxel(const ForceArgs &a, const ContourTables &tab, int N, float w0, float Wxm,
                                            float Wxp, float Wym, float Wyp, float Wm, float Wp, float T, unsigned Sc,
                                            unsigned Sxm, unsigned Sxp, unsigned Sym, unsigned Syp, unsigned Sm,
                                            unsigned Sp, unsigned sb, int ic, int ixm, int ixp, int iym, int iyp,
                                            int im, int ip, float &dux, float &duy, float &duz, float &r0) {
    const unsigned A = CONTOUR ? (Sc & Sxm & Sxp & Sym & Syp & Sm & Sp) >> 8 : 0u;
    const unsigned O = CONTOUR ? (Sc | Sxm | Sxp | Sym | Syp | Sm | Sp) & 0xffu : 0u;
    force_voxel_ao<CONTOUR, L2ONLY>(a, tab, N, w0, Wxm, Wxp, Wym, Wyp, Wm, Wp, T, A, O, Sc, Sxm, Sxp, Sym, Syp, Sm,
                                    Sp, sb, ic, ixm, ixp, iym, iyp, im, ip, dux, duy, duz, r0);
}

// Loads of one plane of pass 2 for one thread's column.  T0 stays raw (its
// bits) until the voxel's arithmetic: a conversion of a 16-bit value at the
// load would wait for the load in the prefetch.
template <bool CONTOUR, typename IT>
struct PlaneLoads {
    float wp, wxm, wxp, wym, wyp;
    unsigned t;
    unsigned sp, sxm, sxp, sym, syp, sb, ur;
};

// T0 of a voxel from its raw bits (plane loads), and of a voxel pair.
template <typename IT>
__device__ __forceinline__ float t_of(unsigned raw) { return from_raw16<IT>(raw); }
template <>
__device__ __forceinline__ float t_of<float>(unsigned raw) { return __uint_as_float(raw); }
template <typename IT>
__device__ __forceinline__ unsigned t_raw(const void *T0, int i) {
    return sizeof(IT) == 2 ? (unsigned)__ldg(static_cast<const unsigned short *>(T0) + i)
                           : __float_as_uint(__ldg(static_cast<const float *>(T0) + i));
}

// Issue every load of plane z (centre index ic) at once: one memory
// latency per plane, hidden behind the previous plane's arithmetic.
template <bool CONTOUR, typename IT>
__device__ __forceinline__ void plane_load(const ForceArgs &a, int ic, int ip, int oxm, int oxp, int oym, int oyp,
                                           PlaneLoads<CONTOUR, IT> &L) {
    const float *__restrict__ W = a.wfield;
    L.wp = __ldg(W + ip);
    L.wxm = __ldg(W + ic + oxm); L.wxp = __ldg(W + ic + oxp);
    L.wym = __ldg(W + ic + oym); L.wyp = __ldg(W + ic + oyp);
    L.t = t_raw<IT>(a.T0, ic);
    L.ur = a.uroi ? __ldg(a.uroi + ic) : 1u;
    if (CONTOUR) {
        const uint16_t *__restrict__ S = a.wstate;
        L.sp = __ldg(S + ip);
        L.sxm = __ldg(S + ic + oxm); L.sxp = __ldg(S + ic + oxp);
        L.sym = __ldg(S + ic + oym); L.syp = __ldg(S + ic + oyp);
        L.sb = __ldg(a.sbits + ic);
    }
}

template <bool CONTOUR, typename IT, bool MAXDU>
__global__ void __launch_bounds__(NT, 3) k_force_pass(ForceArgs a, int zchunk) {
    if (a.stop_flag && *a.stop_flag) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    const int nxy = nx * ny, N = nxy * nz;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    float ssd = 0.f, mx = 0.f;
    int cnt = 0;
    __shared__ ContourTables tab;
    if (CONTOUR) {
        build_tables(a, tab, threadIdx.y * TX + threadIdx.x);
        __syncthreads();
    }
    if (x < nx && y < ny) {
        float *__restrict__ du = a.du;
        const int col = y * nx + x;
        const int oxm = x > 0 ? -1 : 0, oxp = x < nx - 1 ? 1 : 0;
        const int oym = y > 0 ? -nx : 0, oyp = y < ny - 1 ? nx : 0;
        int ic = zb * nxy + col;
        int im = (zb > 0 ? zb - 1 : 0) * nxy + col;
        float Wm = __ldg(a.wfield + im), Wc = __ldg(a.wfield + ic);
        unsigned Sm = 0, Sc = 0;
        if (CONTOUR) { Sm = __ldg(a.wstate + im); Sc = __ldg(a.wstate + ic); }
        PlaneLoads<CONTOUR, IT> bufA, bufB;
        plane_load<CONTOUR, IT>(a, ic, zb < nz - 1 ? ic + nxy : ic, oxm, oxp, oym, oyp, bufA);
        int z = zb;
        // one plane: consumes `cur`, prefetches the next plane into `nxt`
        auto step = [&](const PlaneLoads<CONTOUR, IT> &cur, PlaneLoads<CONTOUR, IT> &nxt) {
            const int ip = z < nz - 1 ? ic + nxy : ic;
            if (z + 1 < ze)        // prefetch the next plane
                plane_load<CONTOUR, IT>(a, ic + nxy, z + 1 < nz - 1 ? ic + 2 * nxy : ic + nxy, oxm, oxp, oym,
                                        oyp, nxt);
            const float Wp = cur.wp;
            const unsigned Sp = CONTOUR ? cur.sp : 0u;
            if (a.warped) a.warped[ic] = Wc;
            float dux, duy, duz, r0;
            force_voxel<CONTOUR>(a, tab, N, Wc, cur.wxm, cur.wxp, cur.wym, cur.wyp, Wm, Wp, t_of<IT>(cur.t), Sc, cur.sxm,
                                 cur.sxp, cur.sym, cur.syp, Sm, Sp, CONTOUR ? cur.sb : 0u, ic, ic + oxm, ic + oxp,
                                 ic + oym, ic + oyp, im, ip, dux, duy, duz, r0);
            du[ic] = dux;
            du[N + ic] = duy;
            du[N + N + ic] = duz;
            if (cur.ur) {
                ssd = fmaf(r0, r0, ssd);
                cnt += 1;
            }
            if (MAXDU) mx = fmaxf(mx, dux * dux + duy * duy + duz * duz);
            Wm = Wc; Wc = Wp; im = ic;
            if (CONTOUR) { Sm = Sc; Sc = Sp; }
            ++z;
            ic += nxy;
        };
        // two planes per turn, the prefetch buffers alternating (no copies)
        for (; z + 1 < ze;) {
            step(bufA, bufB);
            step(bufB, bufA);
        }
        if (z < ze) step(bufA, bufB);
    }
    if (a.partial) {
        block_partial<NT>(ssd, cnt, sqrtf(mx), a.partial,
                          (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
        if (a.fin.done) finish_if_last(a.partial, gridDim.x * gridDim.y * gridDim.z, a.fin);
    }
}


// Pass 2 with two voxels per thread (columns x, x+1; x even): the stencil
// loads, the static-side loads and the du stores move as pairs, which halves
// their instruction count and address arithmetic.  Needs an even nx.
struct PlaneLoads2 {
    float2 wp, wym, wyp;       // I0~ pairs at z+1, y-1, y+1
    float wxm, wxp;            // I0~ at x-1 and x+2 (clamped)
    float t0, t1;              // T0 pair (float images)
    unsigned t16;              // T0 pair, raw (16-bit images; converted at use)
    unsigned sp, sym, syp;     // corner-bit word pairs (low half: x)
    unsigned sxm, sxp;         // corner-bit words at x-1 and x+2
    unsigned sb, ur;           // static bits / UROI byte pairs
};

// The T0 pair of a plane load as floats.
template <typename IT>
__device__ __forceinline__ void t_pair(const PlaneLoads2 &L, float &t0, float &t1) {
    t0 = from_raw16<IT>(L.t16 & 0xffffu);
    t1 = from_raw16<IT>(L.t16 >> 16);
}
template <>
__device__ __forceinline__ void t_pair<float>(const PlaneLoads2 &L, float &t0, float &t1) {
    t0 = L.t0;
    t1 = L.t1;
}

template <bool CONTOUR, typename IT>
__device__ __forceinline__ void plane_load2(const ForceArgs &a, int ic, int ip, int oxm, int oxp, int oym, int oyp,
                                            PlaneLoads2 &L) {
    const float *__restrict__ W = a.wfield;
    L.wp = __ldg(reinterpret_cast<const float2 *>(W + ip));
    L.wym = __ldg(reinterpret_cast<const float2 *>(W + ic + oym));
    L.wyp = __ldg(reinterpret_cast<const float2 *>(W + ic + oyp));
    L.wxm = __ldg(W + ic + oxm);
    L.wxp = __ldg(W + ic + oxp);
    if (sizeof(IT) == 2) {
        L.t16 = __ldg(reinterpret_cast<const unsigned *>(static_cast<const IT *>(a.T0) + ic));
        L.t0 = L.t1 = 0.f;
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(static_cast<const float *>(a.T0) + ic));
        L.t0 = t.x;
        L.t1 = t.y;
        L.t16 = 0u;
    }
    L.ur = a.uroi ? (unsigned)__ldg(reinterpret_cast<const unsigned short *>(a.uroi + ic)) : 0x0101u;
    if (CONTOUR) {
        const uint16_t *__restrict__ S = a.wstate;
        L.sp = __ldg(reinterpret_cast<const unsigned *>(S + ip));
        L.sym = __ldg(reinterpret_cast<const unsigned *>(S + ic + oym));
        L.syp = __ldg(reinterpret_cast<const unsigned *>(S + ic + oyp));
        L.sxm = __ldg(S + ic + oxm);
        L.sxp = __ldg(S + ic + oxp);
        L.sb = __ldg(reinterpret_cast<const unsigned short *>(a.sbits + ic));
    } else {
        L.sp = L.sym = L.syp = L.sxm = L.sxp = L.sb = 0u;
    }
}

template <bool CONTOUR, typename IT, bool MAXDU>
__global__ void __launch_bounds__(NT, 2) k_force_pass2(ForceArgs a, int zchunk) {
    if (a.stop_flag && *a.stop_flag) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = 2 * (blockIdx.x * TX + threadIdx.x), y = blockIdx.y * TY + threadIdx.y;
    const int nxy = nx * ny, N = nxy * nz;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    float ssd = 0.f, mx = 0.f;
    int cnt = 0;
    __shared__ ContourTables tab;
    if (CONTOUR) {
        build_tables(a, tab, threadIdx.y * TX + threadIdx.x);
        __syncthreads();
    }
    if (x < nx && y < ny) {
        float *__restrict__ du = a.du;
        const int col = y * nx + x;
        const int oxm = x > 0 ? -1 : 0, oxp = x + 2 < nx ? 2 : 1;
        const int oym = y > 0 ? -nx : 0, oyp = y < ny - 1 ? nx : 0;
        int ic = zb * nxy + col;
        int im = (zb > 0 ? zb - 1 : 0) * nxy + col;
        float2 Wm = __ldg(reinterpret_cast<const float2 *>(a.wfield + im));
        float2 Wc = __ldg(reinterpret_cast<const float2 *>(a.wfield + ic));
        unsigned Sm = 0, Sc = 0;
        if (CONTOUR) {
            Sm = __ldg(reinterpret_cast<const unsigned *>(a.wstate + im));
            Sc = __ldg(reinterpret_cast<const unsigned *>(a.wstate + ic));
        }
        PlaneLoads2 bufA, bufB;
        plane_load2<CONTOUR, IT>(a, ic, zb < nz - 1 ? ic + nxy : ic, oxm, oxp, oym, oyp, bufA);
        int z = zb;
        auto step = [&](const PlaneLoads2 &cur, PlaneLoads2 &nxt) {
            const int ip = z < nz - 1 ? ic + nxy : ic;
            if (z + 1 < ze)
                plane_load2<CONTOUR, IT>(a, ic + nxy, z + 1 < nz - 1 ? ic + 2 * nxy : ic + nxy, oxm, oxp, oym, oyp,
                                         nxt);
            if (a.warped) { a.warped[ic] = Wc.x; a.warped[ic + 1] = Wc.y; }
            float d0x, d0y, d0z, r00, d1x, d1y, d1z, r01, tv0, tv1;
            t_pair<IT>(cur, tv0, tv1);
            force_voxel<CONTOUR>(a, tab, N, Wc.x, cur.wxm, Wc.y, cur.wym.x, cur.wyp.x, Wm.x, cur.wp.x, tv0,
                                 Sc & 0xffffu, cur.sxm, Sc >> 16, cur.sym & 0xffffu, cur.syp & 0xffffu,
                                 Sm & 0xffffu, cur.sp & 0xffffu, cur.sb & 0xffu, ic, ic + oxm, ic + 1, ic + oym,
                                 ic + oyp, im, ip, d0x, d0y, d0z, r00);
            force_voxel<CONTOUR>(a, tab, N, Wc.y, Wc.x, cur.wxp, cur.wym.y, cur.wyp.y, Wm.y, cur.wp.y, tv1,
                                 Sc >> 16, Sc & 0xffffu, cur.sxp, cur.sym >> 16, cur.syp >> 16, Sm >> 16,
                                 cur.sp >> 16, (cur.sb >> 8) & 0xffu, ic + 1, ic, ic + oxp, ic + 1 + oym,
                                 ic + 1 + oyp, im + 1, ip + 1, d1x, d1y, d1z, r01);
            *reinterpret_cast<float2 *>(du + ic) = make_float2(d0x, d1x);
            *reinterpret_cast<float2 *>(du + N + ic) = make_float2(d0y, d1y);
            *reinterpret_cast<float2 *>(du + N + N + ic) = make_float2(d0z, d1z);
            if (cur.ur & 0xffu) { ssd = fmaf(r00, r00, ssd); cnt += 1; }
            if (cur.ur >> 8) { ssd = fmaf(r01, r01, ssd); cnt += 1; }
            if (MAXDU) mx = fmaxf(mx, fmaxf(d0x * d0x + d0y * d0y + d0z * d0z, d1x * d1x + d1y * d1y + d1z * d1z));
            Wm = Wc; Wc = cur.wp; im = ic;
            Sm = Sc; Sc = cur.sp;
            ++z;
            ic += nxy;
        };
        for (; z + 1 < ze;) {
            step(bufA, bufB);
            step(bufB, bufA);
        }
        if (z < ze) step(bufA, bufB);
    }
    if (a.partial) {
        block_partial<NT>(ssd, cnt, sqrtf(mx), a.partial,
                          (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
        if (a.fin.done) finish_if_last(a.partial, gridDim.x * gridDim.y * gridDim.z, a.fin);
    }
}


// Pass 2 with four voxels per thread (columns x .. x+3; x a multiple of 4):
// the stencil loads of I0~ and of the corner-bit words, the static-side
// loads and the du stores are 16-, 8- or 4-byte vectors, so a voxel takes a
// quarter of the one-voxel pass's load and address instructions.  Needs nx
// % 4 == 0 and 16-byte aligned fields (checked by the launcher).  The
// per-voxel arithmetic is force_voxel_ao, so the bits equal the other passes'.
struct PlaneLoads4 {
    float4 wp, wym, wyp;       // I0~ at z+1, y-1, y+1
    float wxm, wxp;            // I0~ at x-1 and x+4 (clamped)
    float4 t;                  // T0 (float images)
    uint2 t16;                 // T0, raw (16-bit images; converted at use)
    uint2 sp, sym, syp;        // corner-bit words (two per 32-bit half: low half the even voxel)
    unsigned sxm, sxp;         // corner-bit words at x-1 and x+4
    unsigned sb, ur;           // static bits / UROI bytes of the four voxels
};

template <bool CONTOUR, typename IT>
__device__ __forceinline__ void plane_load4(const ForceArgs &a, int ic, int ip, int oxm, int oxp, int oym, int oyp,
                                            PlaneLoads4 &L) {
    const float *__restrict__ W = a.wfield;
    L.wp = __ldg(reinterpret_cast<const float4 *>(W + ip));
    L.wym = __ldg(reinterpret_cast<const float4 *>(W + ic + oym));
    L.wyp = __ldg(reinterpret_cast<const float4 *>(W + ic + oyp));
    L.wxm = __ldg(W + ic + oxm);
    L.wxp = __ldg(W + ic + oxp);
    if (sizeof(IT) == 2) {
        L.t16 = __ldg(reinterpret_cast<const uint2 *>(static_cast<const IT *>(a.T0) + ic));
        L.t = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        L.t = __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(a.T0) + ic));
        L.t16 = make_uint2(0u, 0u);
    }
    L.ur = a.uroi ? __ldg(reinterpret_cast<const unsigned *>(a.uroi + ic)) : 0x01010101u;
    if (CONTOUR) {
        const uint16_t *__restrict__ S = a.wstate;
        L.sp = __ldg(reinterpret_cast<const uint2 *>(S + ip));
        L.sym = __ldg(reinterpret_cast<const uint2 *>(S + ic + oym));
        L.syp = __ldg(reinterpret_cast<const uint2 *>(S + ic + oyp));
        L.sxm = __ldg(S + ic + oxm);
        L.sxp = __ldg(S + ic + oxp);
        L.sb = __ldg(reinterpret_cast<const unsigned *>(a.sbits + ic));
    } else {
        L.sp = L.sym = L.syp = make_uint2(0u, 0u);
        L.sxm = L.sxp = L.sb = 0u;
    }
}

// T0 of the four voxels of a plane load.
template <typename IT>
__device__ __forceinline__ float4 t_quad(const PlaneLoads4 &L) {
    return make_float4(from_raw16<IT>(L.t16.x & 0xffffu), from_raw16<IT>(L.t16.x >> 16),
                       from_raw16<IT>(L.t16.y & 0xffffu), from_raw16<IT>(L.t16.y >> 16));
}
template <>
__device__ __forceinline__ float4 t_quad<float>(const PlaneLoads4 &L) { return L.t; }

// The corner-bit AND (high byte of each word) and OR (low byte) over the
// 7-point stencils of two adjacent voxels at once: c the pair's words (low
// half the left voxel), l the word left of the pair, r the word right of it.
__device__ __forceinline__ void pair_ao(unsigned c, unsigned l, unsigned r, unsigned ym, unsigned yp, unsigned zm,
                                        unsigned zp, unsigned &A0, unsigned &O0, unsigned &A1, unsigned &O1) {
    const unsigned side = (l & 0xffffu) | (r << 16);
    const unsigned swap = __byte_perm(c, 0u, 0x1032);
    const unsigned Ap = c & ym & yp & zm & zp & side & swap;
    const unsigned Op = c | ym | yp | zm | zp | side | swap;
    A0 = (Ap >> 8) & 0xffu; A1 = Ap >> 24;
    O0 = Op & 0xffu; O1 = (Op >> 16) & 0xffu;
}

template <bool CONTOUR, typename IT, bool MAXDU>
__global__ void __launch_bounds__(NT, 2) k_force_pass4(ForceArgs a, int zchunk) {
    if (a.stop_flag && *a.stop_flag) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = 4 * (blockIdx.x * TX + threadIdx.x), y = blockIdx.y * TY + threadIdx.y;
    const int nxy = nx * ny, N = nxy * nz;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    float ssd = 0.f, mx = 0.f;
    int cnt = 0;
    __shared__ ContourTables tab;
    if (CONTOUR) {
        build_tables(a, tab, threadIdx.y * TX + threadIdx.x);
        __syncthreads();
    }
    if (x < nx && y < ny) {
        float *__restrict__ du = a.du;
        const int col = y * nx + x;
        const int oxm = x > 0 ? -1 : 0, oxp = x + 4 < nx ? 4 : 3;
        const int oym = y > 0 ? -nx : 0, oyp = y < ny - 1 ? nx : 0;
        int ic = zb * nxy + col;
        int im = (zb > 0 ? zb - 1 : 0) * nxy + col;
        float4 Wm = __ldg(reinterpret_cast<const float4 *>(a.wfield + im));
        float4 Wc = __ldg(reinterpret_cast<const float4 *>(a.wfield + ic));
        uint2 Sm = make_uint2(0u, 0u), Sc = make_uint2(0u, 0u);
        if (CONTOUR) {
            Sm = __ldg(reinterpret_cast<const uint2 *>(a.wstate + im));
            Sc = __ldg(reinterpret_cast<const uint2 *>(a.wstate + ic));
        }
        PlaneLoads4 bufA, bufB;
        plane_load4<CONTOUR, IT>(a, ic, zb < nz - 1 ? ic + nxy : ic, oxm, oxp, oym, oyp, bufA);
        int z = zb;
        auto step = [&](const PlaneLoads4 &cur, PlaneLoads4 &nxt) {
            const int ip = z < nz - 1 ? ic + nxy : ic;
            if (z + 1 < ze)
                plane_load4<CONTOUR, IT>(a, ic + nxy, z + 1 < nz - 1 ? ic + 2 * nxy : ic + nxy, oxm, oxp, oym, oyp,
                                         nxt);
            if (a.warped) *reinterpret_cast<float4 *>(a.warped + ic) = Wc;
            unsigned A[4] = {0u, 0u, 0u, 0u}, O[4] = {0u, 0u, 0u, 0u};
            if (CONTOUR) {
                pair_ao(Sc.x, cur.sxm, Sc.y, cur.sym.x, cur.syp.x, Sm.x, cur.sp.x, A[0], O[0], A[1], O[1]);
                pair_ao(Sc.y, Sc.x >> 16, cur.sxp, cur.sym.y, cur.syp.y, Sm.y, cur.sp.y, A[2], O[2], A[3], O[3]);
            }
            const float4 T = t_quad<IT>(cur);
            const float w[6] = {cur.wxm, Wc.x, Wc.y, Wc.z, Wc.w, cur.wxp};
            const float wm[4] = {Wm.x, Wm.y, Wm.z, Wm.w}, wp[4] = {cur.wp.x, cur.wp.y, cur.wp.z, cur.wp.w};
            const float wym[4] = {cur.wym.x, cur.wym.y, cur.wym.z, cur.wym.w};
            const float wyp[4] = {cur.wyp.x, cur.wyp.y, cur.wyp.z, cur.wyp.w};
            const float tv[4] = {T.x, T.y, T.z, T.w};
            // corner-bit words of x-1 .. x+4, and of the y / z neighbours
            const unsigned sw[6] = {cur.sxm & 0xffffu, Sc.x & 0xffffu, Sc.x >> 16, Sc.y & 0xffffu, Sc.y >> 16,
                                    cur.sxp & 0xffffu};
            const unsigned sym[4] = {cur.sym.x & 0xffffu, cur.sym.x >> 16, cur.sym.y & 0xffffu, cur.sym.y >> 16};
            const unsigned syp[4] = {cur.syp.x & 0xffffu, cur.syp.x >> 16, cur.syp.y & 0xffffu, cur.syp.y >> 16};
            const unsigned smw[4] = {Sm.x & 0xffffu, Sm.x >> 16, Sm.y & 0xffffu, Sm.y >> 16};
            const unsigned spw[4] = {cur.sp.x & 0xffffu, cur.sp.x >> 16, cur.sp.y & 0xffffu, cur.sp.y >> 16};
            float dx[4], dy[4], dz[4], r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int xm = q == 0 ? ic + oxm : ic + q - 1, xp = q == 3 ? ic + oxp : ic + q + 1;
                force_voxel_ao<CONTOUR>(a, tab, N, w[q + 1], w[q], w[q + 2], wym[q], wyp[q], wm[q], wp[q], tv[q],
                                        A[q], O[q], sw[q + 1], sw[q], sw[q + 2], sym[q], syp[q], smw[q], spw[q],
                                        (cur.sb >> (8 * q)) & 0xffu, ic + q, xm, xp, ic + q + oym, ic + q + oyp,
                                        im + q, ip + q, dx[q], dy[q], dz[q], r[q]);
            }
            *reinterpret_cast<float4 *>(du + ic) = make_float4(dx[0], dx[1], dx[2], dx[3]);
            *reinterpret_cast<float4 *>(du + N + ic) = make_float4(dy[0], dy[1], dy[2], dy[3]);
            *reinterpret_cast<float4 *>(du + N + N + ic) = make_float4(dz[0], dz[1], dz[2], dz[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if ((cur.ur >> (8 * q)) & 0xffu) { ssd = fmaf(r[q], r[q], ssd); cnt += 1; }
                if (MAXDU) mx = fmaxf(mx, dx[q] * dx[q] + dy[q] * dy[q] + dz[q] * dz[q]);
            }
            Wm = Wc; Wc = cur.wp; im = ic;
            Sm = Sc; Sc = cur.sp;
            ++z;
            ic += nxy;
        };
        for (; z + 1 < ze;) {
            step(bufA, bufB);
            step(bufB, bufA);
        }
        if (z < ze) step(bufA, bufB);
    }
    if (a.partial) {
        block_partial<NT>(ssd, cnt, sqrtf(mx), a.partial,
                          (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
        if (a.fin.done) finish_if_last(a.partial, gridDim.x * gridDim.y * gridDim.z, a.fin);
    }
}


// ---- TMA-fed version -------------------------------------------------------
constexpr int kFStages = 5;
constexpr int UBX = TX + 8;           // DVF box width: x0-4 .. x0+35
constexpr int UBY = TY + 2;           // DVF box height: y0-1 .. y0+8
constexpr int U_BYTES = 3 * UBY * UBX * 4;                 // 4800
constexpr int T_OFF = (U_BYTES + 127) / 128 * 128;         // 4864
constexpr int SB_OFF = T_OFF + TX * TY * 4;                // 5888
constexpr int UR_OFF = SB_OFF + TX * TY;                   // 6144
constexpr int STAGE_BYTES = (UR_OFF + TX * TY + 127) / 128 * 128;   // 6400
constexpr int kRing = 4;              // warped planes kept (one barrier per plane)

struct ForceMaps {
    CUtensorMap u, t0, sb, ur;
};

__host__ __device__ constexpr size_t force2_smem_bytes(int nv) {
    return 128 + (size_t)kFStages * STAGE_BYTES + (size_t)kRing * nv * HP * 4 + (size_t)kRing * HP * 2 + 8 +
           kFStages * 8;
}

template <bool CONTOUR, typename IT>
__global__ void __launch_bounds__(NT) k_force_tma(const __grid_constant__ ForceMaps maps, ForceArgs a,
                                                  int zchunk, int *err) {
    using TT = typename TexOf<IT>::type;
    if (a.stop_flag && *a.stop_flag) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    unsigned char *stages = base;
    const int nv = CONTOUR ? 1 + a.k : 1;
    float *ring = reinterpret_cast<float *>(base + kFStages * STAGE_BYTES);      // [kRing][nv][HP]
    uint16_t *state = reinterpret_cast<uint16_t *>(ring + kRing * nv * HP);      // [kRing][HP]
    uint64_t *bar = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(state + kRing * HP) + 7) & ~uintptr_t(7));

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nxy = nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    const int P = (ze - zb) + 2;                   // planes zb-1 .. ze
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    const int cidx = (ty + 1) * HX + (tx + 1);
    const float off = a.offset;
    const uint32_t tx_bytes = (uint32_t)(U_BYTES + TX * TY * sizeof(IT) + (CONTOUR ? TX * TY : 0) +
                                         (a.uroi ? TX * TY : 0));

    auto issue = [&](int q) {
        const int sidx = q % kFStages;
        const int z = clampi(zb - 1 + q, 0, nz - 1);
        unsigned char *st = stages + sidx * STAGE_BYTES;
        mbar_expect_tx(&bar[sidx], tx_bytes);
        tma_load_4d(st, &maps.u, x0 - 4, y0 - 1, z, 0, &bar[sidx]);
        tma_load_3d(st + T_OFF, &maps.t0, x0, y0, z, &bar[sidx]);
        if (CONTOUR) tma_load_3d(st + SB_OFF, &maps.sb, x0, y0, z, &bar[sidx]);
        if (a.uroi) tma_load_3d(st + UR_OFF, &maps.ur, x0, y0, z, &bar[sidx]);
    };
    if (tid == 0) {
        for (int q = 0; q < kFStages; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0)
        for (; issued < kFStages && issued < P; ++issued) issue(issued);

    // halo points of this thread (the same in every plane): offset of the
    // DVF value in a stage (-1 = none) and the clamped voxel coordinates
    constexpr int PPT = (HP + NT - 1) / NT;
    int hp_u[PPT];
    float hp_gx[PPT], hp_gy[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = tid + q * NT;
        const int hx = p % HX, hy = p / HX;
        const int gx = clampi(x0 - 1 + hx, 0, nx - 1), gy = clampi(y0 - 1 + hy, 0, ny - 1);
        hp_u[q] = p < HP ? (gy - (y0 - 1)) * UBX + (gx - (x0 - 4)) : -1;
        hp_gx[q] = (float)gx;
        hp_gy[q] = (float)gy;
    }
    const float fxmax = (float)(nx - 1), fymax = (float)(ny - 1), fzmax = (float)(nz - 1);
    float ssd = 0.f;
    int cnt = 0;
    float mx = 0.f;
    int t = 0;
    for (; t < P; ++t) {
        const int sidx = t % kFStages;
        const bool ok = mbar_wait_bounded(&bar[sidx], (uint32_t)((t / kFStages) & 1));
        // ---- warp the halo points of plane zb-1+t into ring slot t % kRing
        {
            const float *U = reinterpret_cast<const float *>(stages + sidx * STAGE_BYTES);
            float *W = ring + (t % kRing) * nv * HP;
            uint16_t *Sg = state + (t % kRing) * HP;
            const float gzf = (float)clampi(zb - 1 + t, 0, nz - 1);
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (hp_u[q] < 0) continue;
                const int p = tid + q * NT;
                const float ux = U[hp_u[q]];
                const float uy = U[UBY * UBX + hp_u[q]];
                const float uz = U[2 * UBY * UBX + hp_u[q]];
                const float px = fminf(fmaxf(hp_gx[q] + ux, 0.f), fxmax);
                const float py = fminf(fmaxf(hp_gy[q] + uy, 0.f), fymax);
                const float pz = fminf(fmaxf(gzf + uz, 0.f), fzmax);
                const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
                const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
                const float wx = px - fx, wy = py - fy, wz = pz - fz;
                const int dx = ix < nx - 1 ? 1 : 0, dy = iy < ny - 1 ? nx : 0, dz = iz < nz - 1 ? nxy : 0;
                const int b0 = (iz * ny + iy) * nx + ix;
                float c000, c100, c010, c110, c001, c101, c011, c111;
                unsigned m000 = 0, m100 = 0, m010 = 0, m110 = 0, m001 = 0, m101 = 0, m011 = 0, m111 = 0;
                if (CONTOUR) {
                    const TT *q0 = static_cast<const TT *>(a.mtex) + b0;
                    tex_unpack<IT>(__ldg(q0), c000, m000);
                    tex_unpack<IT>(__ldg(q0 + dx), c100, m100);
                    tex_unpack<IT>(__ldg(q0 + dy), c010, m010);
                    tex_unpack<IT>(__ldg(q0 + dy + dx), c110, m110);
                    tex_unpack<IT>(__ldg(q0 + dz), c001, m001);
                    tex_unpack<IT>(__ldg(q0 + dz + dx), c101, m101);
                    tex_unpack<IT>(__ldg(q0 + dz + dy), c011, m011);
                    tex_unpack<IT>(__ldg(q0 + dz + dy + dx), c111, m111);
                } else {
                    const IT *q0 = static_cast<const IT *>(a.I0) + b0;
                    c000 = ld_img<IT>(q0); c100 = ld_img<IT>(q0 + dx); c010 = ld_img<IT>(q0 + dy);
                    c110 = ld_img<IT>(q0 + dy + dx); c001 = ld_img<IT>(q0 + dz); c101 = ld_img<IT>(q0 + dz + dx);
                    c011 = ld_img<IT>(q0 + dz + dy); c111 = ld_img<IT>(q0 + dz + dy + dx);
                }
                const float e00 = fmaf(wx, c100 - c000, c000), e10 = fmaf(wx, c110 - c010, c010);
                const float e01 = fmaf(wx, c101 - c001, c001), e11 = fmaf(wx, c111 - c011, c011);
                const float f0 = fmaf(wy, e10 - e00, e00), f1 = fmaf(wy, e11 - e01, e01);
                const float acc = fmaf(wz, f1 - f0, f0);
                W[p] = acc;
                if (CONTOUR) {
                    const unsigned andb = m000 & m100 & m010 & m110 & m001 & m101 & m011 & m111;
                    const unsigned orb = m000 | m100 | m010 | m110 | m001 | m101 | m011 | m111;
                    Sg[p] = (uint16_t)((andb << 8) | orb);
                    if (andb == orb) {
                        const float J = acc + off;
#pragma unroll
                        for (int j = 0; j < kMaxMasks; ++j)
                            if (j < a.k) W[(1 + j) * HP + p] = ((andb >> j) & 1u) ? J : 0.f;
                    } else {
                        const float ax = 1.f - wx, ay = 1.f - wy, az = 1.f - wz;
                        const float q000 = ax * ay * az * (c000 + off), q100 = wx * ay * az * (c100 + off);
                        const float q010 = ax * wy * az * (c010 + off), q110 = wx * wy * az * (c110 + off);
                        const float q001 = ax * ay * wz * (c001 + off), q101 = wx * ay * wz * (c101 + off);
                        const float q011 = ax * wy * wz * (c011 + off), q111 = wx * wy * wz * (c111 + off);
#pragma unroll
                        for (int j = 0; j < kMaxMasks; ++j) {
                            if (j < a.k) {
                                float pj = 0.f;
                                pj += ((m000 >> j) & 1u) ? q000 : 0.f;
                                pj += ((m100 >> j) & 1u) ? q100 : 0.f;
                                pj += ((m010 >> j) & 1u) ? q010 : 0.f;
                                pj += ((m110 >> j) & 1u) ? q110 : 0.f;
                                pj += ((m001 >> j) & 1u) ? q001 : 0.f;
                                pj += ((m101 >> j) & 1u) ? q101 : 0.f;
                                pj += ((m011 >> j) & 1u) ? q011 : 0.f;
                                pj += ((m111 >> j) & 1u) ? q111 : 0.f;
                                W[(1 + j) * HP + p] = pj;
                            }
                        }
                    }
                }
            }
        }
        if (__syncthreads_or(!ok)) break;
        if (tid == 0 && t >= 2 && issued < P) {
            fence_proxy_async();
            issue(issued);
            ++issued;
        }
        // ---- force for plane z = zb + t - 2 from warped slots t-2, t-1, t
        if (t >= 2 && act) {
            const int z = zb + t - 2;
            const unsigned char *st = stages + ((t - 1) % kFStages) * STAGE_BYTES;
            const float *Pm = ring + ((t - 2) % kRing) * nv * HP;
            const float *Pc = ring + ((t - 1) % kRing) * nv * HP;
            const float *Pp = ring + (t % kRing) * nv * HP;
            const size_t N = (size_t)nx * ny * nz;
            const size_t i = ((size_t)z * ny + y) * nx + x;
            const float w0 = Pc[cidx];
            const float gxv = 0.5f * (Pc[cidx + 1] - Pc[cidx - 1]);
            const float gyv = 0.5f * (Pc[cidx + HX] - Pc[cidx - HX]);
            const float gzv = 0.5f * (Pp[cidx] - Pm[cidx]);
            const float T = to_f<IT>(reinterpret_cast<const IT *>(st + T_OFF)[ty * TX + tx]);
            const float r0 = T - w0;
            if (a.warped) a.warped[i] = w0;
            const float g2 = gxv * gxv + gyv * gyv + gzv * gzv;
            float dux = 0.f, duy = 0.f, duz = 0.f;
            if (g2 != 0.f) {
                // approximate reciprocal root (well inside the 1e-5 parity bar);
                // exact path for subnormal g2, which the approximation flushes
                const float inv = g2 > 1e-30f ? rsqrtf(g2) : 1.f / sqrtf(g2);
                const float gn = g2 * inv;
                const float nxv = gxv * inv, nyv = gyv * inv, nzv = gzv * inv;
                float num = gn * r0, den = gn * gn;
                if (CONTOUR) {
                    const unsigned sb = st[SB_OFF + ty * TX + tx];
                    const float Toff = T + off;
                    const uint16_t *Sm = state + ((t - 2) % kRing) * HP;
                    const uint16_t *Sc = state + ((t - 1) % kRing) * HP;
                    const uint16_t *Sp = state + (t % kRing) * HP;
                    const unsigned s0 = Sc[cidx], s1 = Sc[cidx - 1], s2 = Sc[cidx + 1], s3 = Sc[cidx - HX],
                                   s4 = Sc[cidx + HX], s5 = Sm[cidx], s6 = Sp[cidx];
                    const unsigned A = (s0 & s1 & s2 & s3 & s4 & s5 & s6) >> 8;      // inside at every corner
                    const unsigned O = (s0 | s1 | s2 | s3 | s4 | s5 | s6) & 0xffu;   // inside at some corner
                    const unsigned mixed = O & ~A;                                   // needs the stored P_j
#pragma unroll
                    for (int j = 0; j < kMaxMasks; ++j) {
                        if (j < a.k) {
                            const float hs = a.half_sign[j];
                            const float inside = ((sb >> j) & 1u) ? Toff : 0.f;
                            float aj, rj;
                            if (!((mixed >> j) & 1u)) {
                                const float b = (float)((A >> j) & 1u);     // P_j = b (I0~ + offset) on the stencil
                                aj = fmaf(hs * b, gn, gn);
                                rj = fmaf(hs, inside - b * (w0 + off), r0);
                            } else {
                                const float *Pjm = Pm + (1 + j) * HP, *Pjc = Pc + (1 + j) * HP,
                                            *Pjp = Pp + (1 + j) * HP;
                                const float dPx = 0.5f * (Pjc[cidx + 1] - Pjc[cidx - 1]);
                                const float dPy = 0.5f * (Pjc[cidx + HX] - Pjc[cidx - HX]);
                                const float dPz = 0.5f * (Pjp[cidx] - Pjm[cidx]);
                                aj = gn + hs * (dPx * nxv + dPy * nyv + dPz * nzv);
                                rj = r0 + hs * (inside - Pjc[cidx]);
                            }
                            num = fmaf(a.lambda[j] * aj, rj, num);
                            den = fmaf(a.lambda[j] * aj, aj, den);
                        }
                    }
                }
                const float v = __fdividef(num, den + r0 * r0);
                dux = v * nxv; duy = v * nyv; duz = v * nzv;
            }
            a.du[i] = dux;
            a.du[N + i] = duy;
            a.du[2 * N + i] = duz;
            if (a.uroi == nullptr || st[UR_OFF + ty * TX + tx]) {
                ssd = fmaf(r0, r0, ssd);
                cnt += 1;
            }
            mx = fmaxf(mx, dux * dux + duy * duy + duz * duz);      // squared; root taken per block
        }
    }
    if (t < P) {
        if (tid == 0) {
            atomicExch(err, 1);
            for (int q = t; q < issued; ++q)
                mbar_wait_bounded(&bar[q % kFStages], (uint32_t)((q / kFStages) & 1));
        }
        __syncthreads();
        return;
    }
    if (a.partial) {
        block_partial<NT>(ssd, cnt, sqrtf(mx), a.partial,
                          (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
        if (a.fin.done) finish_if_last(a.partial, gridDim.x * gridDim.y * gridDim.z, a.fin);
    }
}

// ---- cooperative level kernel (small levels) --------------------------------
// All iterations of one level in one launch.  Each iteration is eight
// grid-wide phases separated by barriers: warp (pass 1), force + RMS-ID
// (pass 2), the stop decision, x / y / z passes of the Gaussian of du with
// the composite update fused into the z pass, and x / y / z passes of the
// Gaussian of u.  Every phase has the arithmetic of the per-iteration
// kernels (same formulas, same order of operations), so both give the same
// DVF.  Buffers written inside the kernel are read with L2-only loads
// (ld.global.cg): the L1 is not coherent across CTAs.  Every barrier wait is
// bounded; a CTA whose wait runs out records the error and returns.

// Sense-reversing grid barrier over `nb` resident CTAs; false if the wait
// ran out (about 1 s).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nb, int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        ok = 1;
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nb - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > kWaitLimitCycles) { atomicExch(err, 1); ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}


// One pass of the separable Gaussian along axis `stride` (1, nx or nx*ny)
// over all three components: out = sum_j w_j in[clamp(p + j - R)].
__device__ __forceinline__ void coop_pass(const float *in, float *out, const Taps &t, int stride, int n_axis,
                                          int nx, int nxy, int N, int gt, int gs, int axis) {
    const int R = t.r;
    for (int e = gt; e < 3 * N; e += gs) {
        const int c = e / N, i = e - c * N;
        const int pos = axis == 0 ? i % nx : axis == 1 ? (i / nx) % (nxy / nx) : i / nxy;
        const float *src = in + (size_t)c * N + i;
        float acc = 0.f;
        for (int j = 0; j <= 2 * R; ++j) {
            const int q = min(max(pos + j - R, 0), n_axis - 1);
            acc = fmaf(t.w[j], __ldcg(src + (q - pos) * stride), acc);
        }
        out[e] = acc;
    }
}

template <bool CONTOUR, typename IT>
__global__ void __launch_bounds__(NT, 2) k_level_coop(const __grid_constant__ LevelCoopArgs p) {
    const ForceArgs &a = p.f;
    const int nx = a.nx, ny = a.ny, nz = a.nz, nxy = nx * ny, N = nxy * nz;
    const int tid = threadIdx.y * TX + threadIdx.x, gt = blockIdx.x * NT + tid, gs = gridDim.x * NT;
    const unsigned nb = gridDim.x;
    const LevelState &st = a.fin.st;
    float *u = const_cast<float *>(a.u);
    __shared__ ContourTables tab;
    if (CONTOUR) {
        build_tables(a, tab, tid);
        __syncthreads();
    }
    for (int n = 0;; ++n) {
        // ---- pass 1: warp
        for (int i = gt; i < N; i += gs) {
            const int x = i % nx, y = (i / nx) % ny, z = i / nxy;
            CornerSet<IT> cs;
            corner_load<CONTOUR, IT>(a, __ldcg(u + i), __ldcg(u + N + i), __ldcg(u + N + N + i), x, y, z, cs);
            corner_finish<CONTOUR, IT>(a, i, N, cs);
        }
        if (!grid_barrier(p.bar, nb, p.err)) return;
        // ---- pass 2: force and the RMS-ID sums
        float ssd = 0.f;
        int cnt = 0;
        for (int i = gt; i < N; i += gs) {
            const int x = i % nx, y = (i / nx) % ny, z = i / nxy;
            const int oxm = x > 0 ? -1 : 0, oxp = x < nx - 1 ? 1 : 0;
            const int oym = y > 0 ? -nx : 0, oyp = y < ny - 1 ? nx : 0;
            const int ozm = z > 0 ? -nxy : 0, ozp = z < nz - 1 ? nxy : 0;
            const float *W = a.wfield;
            const float w0 = __ldcg(W + i);
            const float Wxm = __ldcg(W + i + oxm), Wxp = __ldcg(W + i + oxp);
            const float Wym = __ldcg(W + i + oym), Wyp = __ldcg(W + i + oyp);
            const float Wm = __ldcg(W + i + ozm), Wp = __ldcg(W + i + ozp);
            const float T = ld_img<IT>(static_cast<const IT *>(a.T0) + i);
            unsigned Sc = 0, Sxm = 0, Sxp = 0, Sym = 0, Syp = 0, Sm = 0, Sp = 0, sb = 0;
            if (CONTOUR) {
                const uint16_t *S = a.wstate;
                Sc = __ldcg(S + i); Sxm = __ldcg(S + i + oxm); Sxp = __ldcg(S + i + oxp);
                Sym = __ldcg(S + i + oym); Syp = __ldcg(S + i + oyp);
                Sm = __ldcg(S + i + ozm); Sp = __ldcg(S + i + ozp);
                sb = __ldg(a.sbits + i);
            }
            float dux, duy, duz, r0;
            force_voxel<CONTOUR, true>(a, tab, N, w0, Wxm, Wxp, Wym, Wyp, Wm, Wp, T, Sc, Sxm, Sxp, Sym, Syp, Sm, Sp,
                                       sb, i, i + oxm, i + oxp, i + oym, i + oyp, i + ozm, i + ozp, dux, duy, duz,
                                       r0);
            a.du[i] = dux;
            a.du[N + i] = duy;
            a.du[N + N + i] = duz;
            if (a.uroi == nullptr || __ldg(a.uroi + i)) {
                ssd = fmaf(r0, r0, ssd);
                cnt += 1;
            }
        }
        {
            // exact in-block sum (fixed point), then one atomic per CTA
            __shared__ unsigned long long rs[NT / 32];
            __shared__ int rc[NT / 32];
            unsigned long long q = __float2ull_rn(fminf(ssd, 1.0995e12f) * kSsdScale);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                q += __shfl_xor_sync(0xffffffffu, q, o);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            }
            if ((tid & 31) == 0) { rs[tid >> 5] = q; rc[tid >> 5] = cnt; }
            __syncthreads();
            if (tid == 0) {
                unsigned long long sq = 0, sc = 0;
                for (int w = 0; w < NT / 32; ++w) { sq += rs[w]; sc += (unsigned long long)rc[w]; }
                atomicAdd(p.sums + (n & 1) * 4 + 0, sq);
                atomicAdd(p.sums + (n & 1) * 4 + 1, sc);
            }
        }
        if (!grid_barrier(p.bar, nb, p.err)) return;
        // ---- the stop decision, taken identically by every CTA
        {
            const double S = (double)__ldcg(p.sums + (n & 1) * 4 + 0) * (1.0 / (double)kSsdScale);
            const double C = (double)__ldcg(p.sums + (n & 1) * 4 + 1);
            const double d = C > 0 ? sqrt(S / C) : 0.0;
            bool stop = false;
            if (a.fin.stop_mode == CGDIR_STOP_WINDOW10) {
                stop = n >= 10 && (__ldcg(st.hist + n - 10) - d <= a.fin.eps);
            } else if (a.fin.stop_mode == CGDIR_STOP_PAPER_LITERAL && n >= 11) {
                const double ln = d - __ldcg(st.hist + n - 1);
                const double lm = __ldcg(st.hist + n - 10) - __ldcg(st.hist + n - 11);
                stop = (lm - ln) <= a.fin.eps;
            }
            const bool cap = n >= a.fin.cap;
            if (blockIdx.x == 0 && tid == 0) {
                if (n < st.hist_cap) st.hist[n] = d;
                *st.hist_len = n + 1;
                p.sums[((n + 1) & 1) * 4 + 0] = 0ull;
                p.sums[((n + 1) & 1) * 4 + 1] = 0ull;
                if (stop || cap) {
                    *st.stop_flag = 1;
                    *st.iters_run = n;
                    *st.stop_reason = stop ? CGDIR_REASON_CONVERGED : CGDIR_REASON_CAP;
                }
            }
            if (stop || cap) return;
        }
        // ---- Gaussian of du (x, y), z pass with the composite update fused
        coop_pass(a.du, p.tmp1, p.tf, 1, nx, nx, nxy, N, gt, gs, 0);
        if (!grid_barrier(p.bar, nb, p.err)) return;
        coop_pass(p.tmp1, p.tmp2, p.tf, nx, ny, nx, nxy, N, gt, gs, 1);
        if (!grid_barrier(p.bar, nb, p.err)) return;
        for (int i = gt; i < N; i += gs) {
            const int x = i % nx, y = (i / nx) % ny, z = i / nxy;
            float s3[3];
            for (int c = 0; c < 3; ++c) {
                const float *src = p.tmp2 + (size_t)c * N + i;
                float acc = 0.f;
                for (int j = 0; j <= 2 * p.tf.r; ++j) {
                    const int q = min(max(z + j - p.tf.r, 0), nz - 1);
                    acc = fmaf(p.tf.w[j], __ldcg(src + (q - z) * nxy), acc);
                }
                s3[c] = acc;
            }
            float ax, ay, az;
            if (p.compose_mode == CGDIR_ADDITIVE) {
                ax = __ldcg(u + i); ay = __ldcg(u + N + i); az = __ldcg(u + N + N + i);
            } else {
                const float px = fminf(fmaxf((float)x + s3[0], 0.f), (float)(nx - 1));
                const float py = fminf(fmaxf((float)y + s3[1], 0.f), (float)(ny - 1));
                const float pz = fminf(fmaxf((float)z + s3[2], 0.f), (float)(nz - 1));
                const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
                const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
                const float wx = px - fx, wy = py - fy, wz = pz - fz;
                const int ddx = ix < nx - 1 ? 1 : 0, ddy = iy < ny - 1 ? nx : 0, ddz = iz < nz - 1 ? nxy : 0;
                const int b0 = iz * nxy + iy * nx + ix;
                const int o[8] = {0, ddx, ddy, ddy + ddx, ddz, ddz + ddx, ddz + ddy, ddz + ddy + ddx};
                float r3[3];
                for (int c = 0; c < 3; ++c) {
                    float cc[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) cc[q] = __ldcg(u + (size_t)c * N + b0 + o[q]);
                    const float e00 = fmaf(wx, cc[1] - cc[0], cc[0]), e10 = fmaf(wx, cc[3] - cc[2], cc[2]);
                    const float e01 = fmaf(wx, cc[5] - cc[4], cc[4]), e11 = fmaf(wx, cc[7] - cc[6], cc[6]);
                    const float f0 = fmaf(wy, e10 - e00, e00), f1 = fmaf(wy, e11 - e01, e01);
                    r3[c] = fmaf(wz, f1 - f0, f0);
                }
                ax = r3[0]; ay = r3[1]; az = r3[2];
            }
            p.ub[i] = s3[0] + ax;
            p.ub[N + i] = s3[1] + ay;
            p.ub[N + N + i] = s3[2] + az;
        }
        if (!grid_barrier(p.bar, nb, p.err)) return;
        // ---- Gaussian of u
        coop_pass(p.ub, p.tmp1, p.td, 1, nx, nx, nxy, N, gt, gs, 0);
        if (!grid_barrier(p.bar, nb, p.err)) return;
        coop_pass(p.tmp1, p.tmp2, p.td, nx, ny, nx, nxy, N, gt, gs, 1);
        if (!grid_barrier(p.bar, nb, p.err)) return;
        coop_pass(p.tmp2, u, p.td, nxy, nz, nx, nxy, N, gt, gs, 2);
        if (!grid_barrier(p.bar, nb, p.err)) return;
    }
}

// Metric-only pass: I0~ at every voxel and the UROI partial sums (the warp
// of Algorithm A step 5 after a level's last update).
constexpr int MT = 256;
template <typename IT>
__global__ void __launch_bounds__(MT) k_metric(const IT *__restrict__ I0,
                                               const IT *__restrict__ T0,
                                               const float *__restrict__ u,
                                               const uint8_t *__restrict__ uroi, int nx, int ny,
                                               int nz, double *partial, const int *stop_flag,
                                               FinishArgs fin) {
    if (stop_flag && *stop_flag) return;
    const size_t N = (size_t)nx * ny * nz;
    float ssd = 0.f;
    int cnt = 0;
    for (size_t i = (size_t)blockIdx.x * MT + threadIdx.x; i < N; i += (size_t)gridDim.x * MT) {
        if (uroi && !uroi[i]) continue;
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const Corners c = corners((float)x + __ldg(u + i), (float)y + __ldg(u + N + i),
                                  (float)z + __ldg(u + 2 * N + i), nx, ny, nz);
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int cx = (q & 1) ? c.x1 : c.x0, cy = (q & 2) ? c.y1 : c.y0, cz = (q & 4) ? c.z1 : c.z0;
            const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                            ((q & 4) ? c.wz : 1.f - c.wz);
            acc = fmaf(w, ld_img<IT>(I0 + vox(cx, cy, cz, nx, ny)), acc);
        }
        const float r = ld_img<IT>(T0 + i) - acc;
        ssd = fmaf(r, r, ssd);
        cnt += 1;
    }
    block_partial<MT>(ssd, cnt, 0.f, partial, blockIdx.x);
    if (fin.done) finish_if_last(partial, gridDim.x, fin);
}

// Plain warp of one image (interpolation kernel 4).
__global__ void k_warp(const float *__restrict__ f, const float *__restrict__ u, int nx, int ny,
                       int nz, float *__restrict__ out) {
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const Corners c = corners((float)x + __ldg(u + i), (float)y + __ldg(u + N + i),
                                  (float)z + __ldg(u + 2 * N + i), nx, ny, nz);
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int cx = (q & 1) ? c.x1 : c.x0, cy = (q & 2) ? c.y1 : c.y0, cz = (q & 4) ? c.z1 : c.z0;
            const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                            ((q & 4) ? c.wz : 1.f - c.wz);
            acc = fmaf(w, __ldg(f + vox(cx, cy, cz, nx, ny)), acc);
        }
        out[i] = acc;
    }
}

constexpr int FT = 256;
__global__ void __launch_bounds__(FT) k_finalize(const double *__restrict__ partial, int nblocks,
                                                 FinishArgs f) {
    if (f.st.stop_flag && *f.st.stop_flag) return;
    finalize_block(partial, nblocks, f);
}

}  // namespace

// z chunk of the force kernels: enough CTAs for about two waves of 4
// resident CTAs per SM; a chunk re-warps 2 halo planes, so big volumes keep
// long chunks and small ones get short, parallel marches.
// Where pass 2 takes four voxels per thread (nx % 4 == 0) its CTAs cover
// 128 x 8 columns at 2 per SM: about four waves of them, but at least 4
// planes (each chunk also reads the planes on either side).  512x512x160:
// 32 planes, 491 us per force step against 525 us with 80-plane chunks (the
// one-voxel pass's default, 1.7 waves of quad CTAs).
int force_default_zchunk(int nx, int ny, int nz) {
    if (nx % 4 == 0)
        return std::max(std::min(4, nz), pick_zchunk(nz, (long)((nx / 4 + TX - 1) / TX) * ((ny + TY - 1) / TY), 2, 4));
    return pick_zchunk(nz, (long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY), 4, 2);
}

// z chunks of pass 1 of the two-pass force: short, so the grid is several
// waves deep.
static int two_pass_zchunk(int nx, int ny, int nz) {
    return pick_zchunk(nz, (long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY), 8, 4);
}

size_t force_partial_count(int nx, int ny, int nz, int zchunk) {
    return (size_t)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * ((nz + zchunk - 1) / zchunk);
}

// Pass 2 takes four voxels per thread where nx % 4 == 0 and every field it
// reads or writes with vectors is aligned for them.
// (512x512x160, contour terms on: 525 against 548 us per force step with
// FP32 images, 482 against 507 with FP16, from twice the bytes in flight per
// thread at the same 2 CTAs per SM.)
static bool pass2_quad(const ForceArgs &a) {
    auto al = [](const void *p, unsigned b) { return p == nullptr || ((uintptr_t)p & (b - 1)) == 0; };
    const unsigned tb = a.img_dtype == CGDIR_F32 ? 16u : 8u;
    return a.nx % 4 == 0 && a.pass2_width == 0 && al(a.wfield, 16) && al(a.wstate, 8) && al(a.T0, tb) &&
           al(a.du, 16) && al(a.warped, 16) && al(a.uroi, 4) && al(a.sbits, 4);
}

template <typename IT>
static cudaError_t launch_force_t(const ForceArgs &a, int zchunk, dim3 grid, dim3 block, cudaStream_t s,
                                  int *err) {
    const bool contour = a.contour && a.k > 0;
    const size_t N = (size_t)a.nx * a.ny * a.nz;
    if (a.wfield != nullptr && N < (size_t)1 << 31) {
        const int zc = two_pass_zchunk(a.nx, a.ny, a.nz);
        dim3 g(grid.x, grid.y, (a.nz + zc - 1) / zc);
        // pass 2 marches the caller's (longer) z chunks: fewer CTAs, so fewer
        // end-of-block fences before the fused reduction
        const bool quad = pass2_quad(a);
        const bool paired = a.nx % 2 == 0 && a.pass2_width != 1;
        dim3 g2 = quad ? dim3((a.nx / 4 + TX - 1) / TX, grid.y, grid.z)
                       : paired ? dim3((a.nx / 2 + TX - 1) / TX, grid.y, grid.z) : grid;
        const bool warp = !a.skip_warp;
        // max |du| is reported by the primitive only (a registration's fused
        // reduction keeps the RMS-ID sums alone)
        const bool maxdu = a.partial != nullptr && (a.fin.done == nullptr || a.fin.stats_out != nullptr);
#define CGDIR_PASS2(C, M)                                                        \
    do {                                                                         \
        if (quad) k_force_pass4<C, IT, M><<<g2, block, 0, s>>>(a, zchunk);       \
        else if (paired) k_force_pass2<C, IT, M><<<g2, block, 0, s>>>(a, zchunk);\
        else k_force_pass<C, IT, M><<<grid, block, 0, s>>>(a, zchunk);           \
    } while (0)
        if (contour) {
            if (warp) k_warp_pass<true, IT><<<g, block, 0, s>>>(a, zc);
            if (maxdu) CGDIR_PASS2(true, true); else CGDIR_PASS2(true, false);
        } else {
            if (warp) k_warp_pass<false, IT><<<g, block, 0, s>>>(a, zc);
            if (maxdu) CGDIR_PASS2(false, true); else CGDIR_PASS2(false, false);
        }
#undef CGDIR_PASS2
        note_launch(warp ? 2 : 1);
        return cudaGetLastError();
    }
    if (err != nullptr && N < (size_t)1 << 31 && (!contour || a.mtex != nullptr)) {
        ForceMaps m;
        const uint64_t du4[4] = {(uint64_t)a.nx, (uint64_t)a.ny, (uint64_t)a.nz, 3};
        const uint64_t d3[3] = {(uint64_t)a.nx, (uint64_t)a.ny, (uint64_t)a.nz};
        const uint32_t ubox[4] = {UBX, UBY, 1, 3}, tbox[3] = {TX, TY, 1};
        bool ok = encode_tensor_map(&m.u, a.u, 4, du4, ubox, 4) &&
                  encode_tensor_map(&m.t0, a.T0, 3, d3, tbox, (int)sizeof(IT));
        if (ok && contour) ok = encode_tensor_map(&m.sb, a.sbits, 3, d3, tbox, 1);
        if (ok && a.uroi) ok = encode_tensor_map(&m.ur, a.uroi, 3, d3, tbox, 1);
        if (ok) {
            const size_t smem = force2_smem_bytes(contour ? 1 + a.k : 1);
            cudaError_t e;
            if (contour) {
                e = ensure_smem((const void *)k_force_tma<true, IT>, smem);
                if (e == cudaSuccess) k_force_tma<true, IT><<<grid, block, smem, s>>>(m, a, zchunk, err);
            } else {
                e = ensure_smem((const void *)k_force_tma<false, IT>, smem);
                if (e == cudaSuccess) k_force_tma<false, IT><<<grid, block, smem, s>>>(m, a, zchunk, err);
            }
            note_launch();
            return e != cudaSuccess ? e : cudaGetLastError();
        }
    }
    const size_t smem = 3u * (1 + (contour ? a.k : 0)) * HP * sizeof(float);
    if (contour) {
        ensure_smem((const void *)k_force<true, IT>, smem);
        k_force<true, IT><<<grid, block, smem, s>>>(a, zchunk);
    } else {
        k_force<false, IT><<<grid, block, smem, s>>>(a, zchunk);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_force(const ForceArgs &a, int zchunk, int *nblocks_out, cudaStream_t s, int *err) {
    if (zchunk <= 0) zchunk = force_default_zchunk(a.nx, a.ny, a.nz);
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + zchunk - 1) / zchunk);
    dim3 block(TX, TY);
    if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
    if (nblocks_out && a.wfield != nullptr && (size_t)a.nx * a.ny * a.nz < (size_t)1 << 31) {
        if (pass2_quad(a)) *nblocks_out = (int)(((a.nx / 4 + TX - 1) / TX) * grid.y * grid.z);
        else if (a.nx % 2 == 0 && a.pass2_width != 1)
            *nblocks_out = (int)(((a.nx / 2 + TX - 1) / TX) * grid.y * grid.z);   // paired pass 2
    }

    if (a.img_dtype == CGDIR_F16) return launch_force_t<__half>(a, zchunk, grid, block, s, err);
    if (a.img_dtype == CGDIR_BF16) return launch_force_t<__nv_bfloat16>(a, zchunk, grid, block, s, err);
    return launch_force_t<float>(a, zchunk, grid, block, s, err);
}

// At most 16 voxels per thread, so each thread's FP32 partial sum stays short.
static int metric_grid(int nx, int ny, int nz) {
    const size_t N = (size_t)nx * ny * nz;
    const size_t g = (N + MT * 16 - 1) / (MT * 16);
    return (int)(g > 0 ? g : 1);
}

size_t metric_partial_count(int nx, int ny, int nz) { return (size_t)metric_grid(nx, ny, nz); }

cudaError_t launch_metric(const void *I0, const void *T0, int img_dtype, const float *u,
                          const uint8_t *uroi, int nx, int ny, int nz, double *partial,
                          const int *stop_flag, int *nblocks_out, cudaStream_t s, const FinishArgs *fin) {
    const int g = metric_grid(nx, ny, nz);
    if (nblocks_out) *nblocks_out = g;
    FinishArgs f{};
    if (fin) f = *fin;
    if (img_dtype == CGDIR_F16)
        k_metric<__half><<<g, MT, 0, s>>>((const __half *)I0, (const __half *)T0, u, uroi, nx, ny, nz, partial,
                                          stop_flag, f);
    else if (img_dtype == CGDIR_BF16)
        k_metric<__nv_bfloat16><<<g, MT, 0, s>>>((const __nv_bfloat16 *)I0, (const __nv_bfloat16 *)T0, u, uroi,
                                                 nx, ny, nz, partial, stop_flag, f);
    else
        k_metric<float><<<g, MT, 0, s>>>((const float *)I0, (const float *)T0, u, uroi, nx, ny, nz, partial,
                                         stop_flag, f);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partial, int nblocks, LevelState st, int n, int cap,
                            int stop_mode, double eps, double *stats_out, cudaStream_t s) {
    FinishArgs f{};
    f.st = st; f.n = n; f.cap = cap; f.stop_mode = stop_mode; f.eps = eps; f.stats_out = stats_out;
    k_finalize<<<1, FT, 0, s>>>(partial, nblocks, f);
    note_launch();
    return cudaGetLastError();
}

template <bool CONTOUR, typename IT>
static int coop_blocks_per_sm() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cached[dev] == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level_coop<CONTOUR, IT>, NT, 0) != cudaSuccess) {
            cudaGetLastError();
            nb = -1;
        }
        cached[dev] = nb > 0 ? nb : -1;
    }
    return cached[dev] > 0 ? cached[dev] : 0;
}

int level_coop_grid(int nx, int ny, int nz, bool contour, int img_dtype) {
    const long N = (long)nx * ny * nz;
    if (N <= 0 || N >= (1L << 31) / 3) return 0;
    int per = 0;
    if (img_dtype == CGDIR_F16) per = contour ? coop_blocks_per_sm<true, __half>() : coop_blocks_per_sm<false, __half>();
    else if (img_dtype == CGDIR_BF16)
        per = contour ? coop_blocks_per_sm<true, __nv_bfloat16>() : coop_blocks_per_sm<false, __nv_bfloat16>();
    else per = contour ? coop_blocks_per_sm<true, float>() : coop_blocks_per_sm<false, float>();
    if (per <= 0) return 0;
    const long need = (N + NT - 1) / NT;
    return (int)std::max(1L, std::min(need, (long)per * sm_count()));
}

template <bool CONTOUR, typename IT>
static cudaError_t launch_coop_t(const LevelCoopArgs &p, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TX, TY);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_level_coop<CONTOUR, IT>, p);
}

cudaError_t launch_level_coop(const LevelCoopArgs &p, int grid, cudaStream_t s) {
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const bool contour = p.f.contour && p.f.k > 0;
    cudaError_t e;
    if (p.f.img_dtype == CGDIR_F16)
        e = contour ? launch_coop_t<true, __half>(p, grid, s) : launch_coop_t<false, __half>(p, grid, s);
    else if (p.f.img_dtype == CGDIR_BF16)
        e = contour ? launch_coop_t<true, __nv_bfloat16>(p, grid, s) : launch_coop_t<false, __nv_bfloat16>(p, grid, s);
    else
        e = contour ? launch_coop_t<true, float>(p, grid, s) : launch_coop_t<false, float>(p, grid, s);
    note_launch();
    return e;
}

cudaError_t launch_warp(const float *f, const float *u, int nx, int ny, int nz, float *out,
                        cudaStream_t s) {
    const size_t N = (size_t)nx * ny * nz;
    size_t g = (N + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    k_warp<<<(unsigned)g, 256, 0, s>>>(f, u, nx, ny, nz, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cgdir
