// Low-pass filter kernel of CG-DIR (kernel 1, Sec. 2.2; Algorithm A steps 2
// and 4) and the composite update (Algorithm A step 3, the vector half of
// kernel 4).
//
// Smoothing: the 3-D Gaussian is applied as x, y and z passes (the
// separability the paper uses) inside ONE kernel, so each component is read
// once and written once.  A CTA owns a 32 x 8 column in x-y and marches
// along z: every input plane of the column plus an R-voxel halo goes to
// shared memory, the x pass and the y pass run there, and each thread keeps
// the last 2R+1 xy-filtered values of its column in registers for the z
// pass.  Halo indices are clamped (clamp-to-edge).  All three components of
// a displacement field are filtered by the same CTA.
//
// Two versions of the smoothing kernel share that structure.  The TMA one
// (used whenever the field satisfies the tensor-map rules: nx a multiple of
// 4, 16-byte aligned base) streams each input plane of the column into a
// 4-stage shared-memory ring with cp.async.bulk.tensor, so the loads of the
// next planes are in flight while the current one is filtered; clamping at
// the volume border is done by index remapping in the x and y passes (the
// TMA box itself zero-fills outside the volume).  The plain one loads the
// halo with ordinary clamped loads.
//
// Every kernel here returns at once when the level's stop flag is set, so a
// level that converged early leaves its fields untouched.
#include "cgdir_internal.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cmath>

namespace cgdir {

int gauss_radius(float sigma) {
    if (!(sigma > 0.f)) return 0;
    return (int)std::ceil(3.0 * (double)sigma - 1e-9);
}

Taps gauss_taps(float sigma) {
    Taps t{};
    t.r = gauss_radius(sigma);
    if (t.r == 0) { t.w[0] = 1.f; return t; }
    double w[2 * kMaxRadius + 1], s = 0.0;
    for (int j = -t.r; j <= t.r; ++j) {
        w[j + t.r] = std::exp(-(double)(j * j) / (2.0 * (double)sigma * (double)sigma));
        s += w[j + t.r];
    }
    for (int j = 0; j <= 2 * t.r; ++j) t.w[j] = (float)(w[j] / s);
    return t;
}

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;

template <int R>
__global__ void __launch_bounds__(NT) k_smooth(const float *__restrict__ in,
                                               float *__restrict__ out, int ncomp, Taps taps,
                                               int nx, int ny, int nz, int zchunk,
                                               const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    constexpr int SX = TX + 2 * R, SY = TY + 2 * R, K = 2 * R + 1;
    __shared__ float S[3][SY][SX];
    __shared__ float X[3][SY][TX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const size_t N = (size_t)nx * ny * nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    float w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = taps.w[j];
    float ring[3][K];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < K; ++j) ring[c][j] = 0.f;

    for (int zi = zb - R; zi < ze + R; ++zi) {
        const int gz = clampi(zi, 0, nz - 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c >= ncomp) break;
            const float *src = in + c * N;
            for (int p = tid; p < SX * SY; p += NT) {
                const int hx = p % SX, hy = p / SX;
                const int gx = clampi(x0 - R + hx, 0, nx - 1), gy = clampi(y0 - R + hy, 0, ny - 1);
                S[c][hy][hx] = __ldg(src + vox(gx, gy, gz, nx, ny));
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c >= ncomp) break;
            for (int p = tid; p < SY * TX; p += NT) {
                const int hy = p / TX, xx = p % TX;
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) acc = fmaf(w[j], S[c][hy][xx + j], acc);
                X[c][hy][xx] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c >= ncomp) break;
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) acc = fmaf(w[j], X[c][ty + j][tx], acc);
#pragma unroll
            for (int j = 0; j < K - 1; ++j) ring[c][j] = ring[c][j + 1];
            ring[c][K - 1] = acc;
            const int zo = zi - R;
            if (zo >= zb && act) {
                float o = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) o = fmaf(w[j], ring[c][j], o);
                out[c * N + vox(x, y, zo, nx, ny)] = o;
            }
        }
    }
}

// ---- TMA-fed version ---------------------------------------------------
// A CTA (32 x 8 threads) filters NC components (NC = 1: one component per
// CTA; NC = 3: the three components of a DVF, needed by the composite-update
// epilogue) of a 32 x 16 column; each thread owns two adjacent output rows.
// Per input plane one TMA box (x from x0 - ML, ML = R rounded up to 4 so the
// start is 16-byte aligned; y from y0 - R) lands in a 4-stage ring.
// x pass: each task filters 4 adjacent outputs of one row from 16-byte
// shared loads; y pass: two rows from 2R+2 loads; z pass: a (2R+1)-deep
// register ring whose slots are fixed at compile time by unrolling the
// plane loop 2R+1 times.  One barrier per plane.
//
// COMPOSE (NC = 3): the z-pass result is the smoothed du at (x, y, z); the
// epilogue applies Algorithm A step 3 there, u_new = du + u(x + du), so the
// smoothed du never goes back to memory.
constexpr int SY = 16;                 // output rows per CTA (2 per thread)

template <int R, int NC>
struct SmoothGeom {
    static constexpr int ML = (R + 3) / 4 * 4;
    static constexpr int BXW = TX + 2 * ML;
    static constexpr int BY = SY + 2 * R;
    static constexpr int ST = NC == 1 ? 8 : 6;                      // pipeline stages
    static constexpr int STAGE = (NC * BY * BXW + 31) / 32 * 32;   // floats per stage
    static constexpr int NV = (4 + R + ML + 3) / 4;                // float4 per x task
    static constexpr int XB = NC * BY * TX;                          // floats per X buffer
    static constexpr int NTASK = NC * BY * (TX / 4);                 // x-pass tasks per plane
    static constexpr int TPT = (NTASK + NT - 1) / NT;                // tasks per thread
    static constexpr size_t bytes() {
        return sizeof(float) * ((size_t)ST * STAGE + 2 * XB) + ST * sizeof(uint64_t) + 128;
    }
};

__device__ __forceinline__ float trilinear_at(const float *__restrict__ f, size_t b0, int ddx, int ddy,
                                              int ddz, float wx, float wy, float wz) {
    const float c000 = __ldg(f + b0), c100 = __ldg(f + b0 + ddx), c010 = __ldg(f + b0 + ddy),
                c110 = __ldg(f + b0 + ddy + ddx), c001 = __ldg(f + b0 + ddz), c101 = __ldg(f + b0 + ddz + ddx),
                c011 = __ldg(f + b0 + ddz + ddy), c111 = __ldg(f + b0 + ddz + ddy + ddx);
    const float e00 = fmaf(wx, c100 - c000, c000), e10 = fmaf(wx, c110 - c010, c010);
    const float e01 = fmaf(wx, c101 - c001, c001), e11 = fmaf(wx, c111 - c011, c011);
    const float f0 = fmaf(wy, e10 - e00, e00), f1 = fmaf(wy, e11 - e01, e01);
    return fmaf(wz, f1 - f0, f0);
}

template <int R, int NC, bool COMPOSE>
__global__ void __launch_bounds__(NT) k_smooth_tma(const __grid_constant__ CUtensorMap tin,
                                                   const float *__restrict__ ucomp, int mode,
                                                   float *__restrict__ out, int ncomp, Taps taps,
                                                   int nx, int ny, int nz, int zchunk,
                                                   const int *stop_flag, int *err) {
    if (stop_flag && *stop_flag) return;
    using G = SmoothGeom<R, NC>;
    constexpr int BY = G::BY, BXW = G::BXW, ML = G::ML, STAGE = G::STAGE, NV = G::NV, K = 2 * R + 1;
    constexpr int ST = G::ST, TPT = G::TPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stage = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *Xb = stage + ST * STAGE;                                 // [2][NC][BY][TX]
    uint64_t *bar = reinterpret_cast<uint64_t *>(Xb + 2 * G::XB);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const size_t N = (size_t)nx * ny * nz, nxy = (size_t)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * SY;
    const int nchunks = (nz + zchunk - 1) / zchunk;
    const int chunk = (int)blockIdx.z % nchunks;
    const int comp = NC == 1 ? (int)blockIdx.z / nchunks : 0;      // component of an NC=1 CTA
    const int zb = chunk * zchunk, ze = min(zb + zchunk, nz);
    const int P = (ze - zb) + 2 * R;
    const int x = x0 + tx, ya = y0 + 2 * ty;                        // rows ya, ya + 1
    const bool acta = x < nx && ya < ny, actb = x < nx && ya + 1 < ny;
    const bool xin = (x0 - R >= 0) && (x0 + TX + R <= nx);
    const uint32_t tx_bytes = (uint32_t)(NC * BY * BXW * sizeof(float));
    (void)ncomp;

    float2 w2[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w2[j] = make_float2(taps.w[j], taps.w[j]);
    float2 ring[NC][K];                                             // {row ya, row ya+1}
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int j = 0; j < K; ++j) ring[c][j] = make_float2(0.f, 0.f);

    // x-pass tasks of this thread (the same in every plane): row offset in a
    // stage, first column of its 4 outputs, destination offset in X
    int t_row[TPT], t_g4[TPT], t_dst[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int task = tid + q * NT;
        const int g = task & (TX / 4 - 1), row = task >> 3;         // row = c * BY + hy
        const int c = NC == 1 ? 0 : row / BY, hy = row - c * BY;
        const int ly = clampi(y0 - R + hy, 0, ny - 1) - (y0 - R);
        t_row[q] = task < G::NTASK ? (c * BY + ly) * BXW : -1;
        t_g4[q] = 4 * g;
        t_dst[q] = row * TX + 4 * g;
    }
    const int xlim = nx - x0 + ML;        // first local column beyond the volume's last x
    float *outp[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) outp[c] = out + (size_t)(comp + c) * N + (size_t)ya * nx + x;

    auto issue = [&](int q) {
        const int sidx = q % ST;
        const int z = clampi(zb - R + q, 0, nz - 1);
        mbar_expect_tx(&bar[sidx], tx_bytes);
        tma_load_4d(stage + sidx * STAGE, &tin, x0 - ML, y0 - R, z, comp, &bar[sidx]);
    };
    if (tid == 0) {
        for (int q = 0; q < ST; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0)
        for (; issued < ST && issued < P; ++issued) issue(issued);

    bool aborted = false;
    int tw = 0;                         // plane being waited for
    int sidx = 0;                       // its stage
    uint32_t par = 0;                   // and the phase parity of that stage
    for (int t0 = 0; t0 < P && !aborted; t0 += K) {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int t = t0 + r;
            if (t >= P) break;
            tw = t;
            const bool ok = mbar_wait_bounded(&bar[sidx], par);
            const float *S = stage + sidx * STAGE;
            float *X = Xb + (t & 1) * G::XB;
            // x pass: 4 adjacent outputs per task, paired FMAs
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                if (t_row[q] < 0) continue;
                const float *src = S + t_row[q];
                float2 o01 = make_float2(0.f, 0.f), o23 = make_float2(0.f, 0.f);
                float v[4 * NV];
#pragma unroll
                for (int h = 0; h < NV; ++h) {
                    const float4 f = reinterpret_cast<const float4 *>(src + t_g4[q])[h];
                    v[4 * h] = f.x; v[4 * h + 1] = f.y; v[4 * h + 2] = f.z; v[4 * h + 3] = f.w;
                }
                if (!xin) {
                    // the box crosses an x border of the volume (its copy holds
                    // zeros there): the taps outside take the border value
#pragma unroll
                    for (int g = 0; g < ML; g += 4)            // left: x0 = 0, the first ML / 4 tasks of a row
                        if (x0 == 0 && t_g4[q] == g) {
#pragma unroll
                            for (int k = 0; k < ML - g; ++k) v[k] = v[ML - g];
                        }
                    if (t_g4[q] + 4 * NV > xlim) {             // right: columns from xlim on lie beyond nx - 1
                        const float b = src[xlim - 1];
#pragma unroll
                        for (int k = 0; k < 4 * NV; ++k) v[k] = t_g4[q] + k >= xlim ? b : v[k];
                    }
                }
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    if ((j + ML - R) % 2 == 0) {       // operand pairs register-aligned: paired FMAs
                        o01 = __ffma2_rn(w2[j], make_float2(v[j + ML - R], v[j + 1 + ML - R]), o01);
                        o23 = __ffma2_rn(w2[j], make_float2(v[j + 2 + ML - R], v[j + 3 + ML - R]), o23);
                    } else {                           // odd offset: scalar FMAs (same rounding, no moves)
                        o01.x = fmaf(w2[j].x, v[j + ML - R], o01.x);
                        o01.y = fmaf(w2[j].x, v[j + 1 + ML - R], o01.y);
                        o23.x = fmaf(w2[j].x, v[j + 2 + ML - R], o23.x);
                        o23.y = fmaf(w2[j].x, v[j + 3 + ML - R], o23.y);
                    }
                }
                reinterpret_cast<float4 *>(X + t_dst[q])[0] = make_float4(o01.x, o01.y, o23.x, o23.y);
            }
            if (__syncthreads_or(!ok)) { aborted = true; break; }
            if (tid == 0 && issued < P) {
                fence_proxy_async();
                issue(issued);
                ++issued;
            }
            if (++sidx == ST) { sidx = 0; par ^= 1u; }
            // y pass into the ring slot of this plane, z pass for plane t - 2R
            float2 res[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float *col = X + (c * BY + 2 * ty) * TX + tx;
                float yin[K + 1];
#pragma unroll
                for (int j = 0; j <= K; ++j) yin[j] = col[j * TX];
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    if (j % 2 == 0) {
                        a = __ffma2_rn(w2[j], make_float2(yin[j], yin[j + 1]), a);
                    } else {
                        a.x = fmaf(w2[j].x, yin[j], a.x);
                        a.y = fmaf(w2[j].x, yin[j + 1], a.y);
                    }
                }
                ring[c][r] = a;
                float2 o = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < K; ++j) o = __ffma2_rn(w2[j], ring[c][(r + 1 + j) % K], o);
                res[c] = o;
            }
            if (t >= 2 * R) {
                const int zo = zb + t - 2 * R;
                const size_t zoff = (size_t)zo * nxy;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!(h == 0 ? acta : actb)) continue;
                    const size_t off = zoff + (size_t)h * nx;
                    if (COMPOSE) {
                        const int y = ya + h;
                        const size_t i = off + (size_t)ya * nx + x;
                        const float dx = h ? res[0].y : res[0].x;
                        const float dy = NC > 1 ? (h ? res[NC > 1 ? 1 : 0].y : res[NC > 1 ? 1 : 0].x) : 0.f;
                        const float dz = NC > 2 ? (h ? res[NC > 2 ? 2 : 0].y : res[NC > 2 ? 2 : 0].x) : 0.f;
                        float ax, ay, az;
                        if (mode == CGDIR_ADDITIVE) {
                            ax = __ldg(ucomp + i); ay = __ldg(ucomp + N + i); az = __ldg(ucomp + 2 * N + i);
                        } else {
                            const Corners cc = corners((float)x + dx, (float)y + dy, (float)zo + dz, nx, ny, nz);
                            const int ddx = cc.x1 - cc.x0, ddy = (cc.y1 - cc.y0) * nx, ddz = (cc.z1 - cc.z0) * nx * ny;
                            const size_t b0 = ((size_t)cc.z0 * ny + cc.y0) * nx + cc.x0;
                            ax = trilinear_at(ucomp, b0, ddx, ddy, ddz, cc.wx, cc.wy, cc.wz);
                            ay = trilinear_at(ucomp + N, b0, ddx, ddy, ddz, cc.wx, cc.wy, cc.wz);
                            az = trilinear_at(ucomp + 2 * N, b0, ddx, ddy, ddz, cc.wx, cc.wy, cc.wz);
                        }
                        outp[0][off] = dx + ax;
                        outp[0][N + off] = dy + ay;
                        outp[0][2 * N + off] = dz + az;
                    } else {
#pragma unroll
                        for (int c = 0; c < NC; ++c) outp[c][off] = h ? res[c].y : res[c].x;
                    }
                }
            }
        }
    }
    if (aborted) {
        // a wait ran out: record it, drain the loads still in flight (bounded), leave
        if (tid == 0) {
            atomicExch(err, 1);
            for (int q = tw; q < issued; ++q)
                mbar_wait_bounded(&bar[q % ST], (uint32_t)((q / ST) & 1));
        }
        __syncthreads();
    }
}

// ---- wide-tile z-march (one component per CTA, nx % 8 == 0, R <= 4) -----
// The same passes and the same order of operations as k_smooth_tma (so the
// same bits), on a 64 x 16 output tile with less work per output:
//  * per input plane one TMA box (x from x0 - 4, 72 wide; y from y0 - R)
//    lands in a ring of stages; the ring and the x-pass buffers are indexed
//    from the kernel's own shared array, so every access is a shared-memory
//    load or store;
//  * x pass: a task is 8 adjacent outputs of one box row (four 16-byte
//    loads, 56 FMAs, half of them paired); the clamp at the volume's x
//    borders is a select on the loaded values (the box is zero-filled
//    there), the clamp in y a remapped row, in z a clamped plane;
//  * y pass: a thread takes a column pair and two rows: 8-byte loads of the
//    pair, paired FMAs only;
//  * z pass: the last 2R+1 y-pass results of those four outputs stay in
//    registers (slots fixed at compile time by unrolling the plane loop
//    2R+1 times), paired FMAs; 8-byte stores.
// One barrier per PB planes (PB x-pass buffers, double-buffered); the
// launcher takes PB = 1 (two to four planes per barrier measured slower:
// 262-332 against 218 us at 512 x 512 x 160).  The plane count of a step is
// the runtime min(PB, planes left) even for PB = 1: written with a
// compile-time 1 instead (same bits), the kernel took 265 us.
// Box rows are 76 floats wide (x0 - 4 .. x0 + 71; the last 4 columns are
// not used) and so are the x-pass buffer's rows: 19 16-byte units, so the
// x-pass tasks below (task q: box row q % BY, column group q / BY) hit
// distinct bank groups in every quarter-warp, for their 16-byte loads and
// stores alike (unit 19 row + 2 group = 3 q mod 8 when BY = 6 mod 8).
constexpr int WX = 64, WY = 16, WML = 4, WBX = 76;

template <int R>
struct WideGeom {
    static constexpr int BY = WY + 2 * R;                       // box rows
    static constexpr int ST = 8;                                // pipeline stages
    static constexpr int STAGE = (BY * WBX + 31) / 32 * 32;     // floats per stage (128-byte multiple)
    static constexpr int XB = BY * WBX;                         // floats per x-pass buffer
    static constexpr int NTASK = BY * (WX / 8);                 // x-pass tasks per plane
    static constexpr size_t bytes(int pb) {
        return sizeof(float) * ((size_t)ST * STAGE + 2 * (size_t)pb * XB) + ST * sizeof(uint64_t) + 128;
    }
};

template <int R, int PB>
__global__ void __launch_bounds__(NT, 2) k_smooth_wide(const __grid_constant__ CUtensorMap tin,
                                                       float *__restrict__ out, Taps taps, int nx, int ny,
                                                       int nz, int zchunk, const int *stop_flag, int *err) {
    if (stop_flag && *stop_flag) return;
    using G = WideGeom<R>;
    constexpr int K = 2 * R + 1, BY = G::BY, ST = G::ST, STAGE = G::STAGE, XB = G::XB;
    static_assert(R >= 1 && R <= 4, "8-output x tasks read 16 loaded values");
    static_assert(PB >= 1 && PB <= 4, "planes per barrier");
    extern __shared__ __align__(128) float wsm[];
    // 128-byte aligned base for the TMA stages, still a shared-memory pointer
    const int pad = (int)(((128u - (smem_u32(wsm) & 127u)) & 127u) >> 2);
    float *stage0 = wsm + pad;                                   // [ST][STAGE]
    float *xbuf = stage0 + ST * STAGE;                           // [2][PB][BY][WBX]
    uint64_t *bar = reinterpret_cast<uint64_t *>(xbuf + 2 * PB * XB);

    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x0 = blockIdx.x * WX, y0 = blockIdx.y * WY;
    const int nchunks = (nz + zchunk - 1) / zchunk;
    const int chunk = (int)blockIdx.z % nchunks, comp = (int)blockIdx.z / nchunks;
    const int zb = chunk * zchunk, ze = min(zb + zchunk, nz);
    const int P = (ze - zb) + 2 * R;
    const uint32_t tx_bytes = (uint32_t)(BY * WBX * sizeof(float));

    float2 w2[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w2[j] = make_float2(taps.w[j], taps.w[j]);

    // x-pass task of this thread (fixed for every plane): box row and column group
    const bool xtask = tid < G::NTASK;
    const int xrow = tid % BY, xg = tid / BY;
    const int srow = clampi(y0 - R + xrow, 0, ny - 1) - (y0 - R);    // clamped source row in the box
    const int xsrc = srow * WBX + 8 * xg;                            // first loaded float
    const int xdst = xrow * WBX + 8 * xg;
    const bool pleft = x0 == 0 && xg == 0;                            // taps left of x = 0
    const bool pright = x0 + 8 * xg + 8 == nx;                        // taps right of x = nx - 1
    const bool xedge = x0 == 0 || x0 + WX >= nx;                      // the same for the whole CTA
    // y / z pass: column pair (x, x + 1) and rows (y, y + 1) of this thread
    const int yc = 2 * (tid & 31), yr = 2 * (tid >> 5);
    const int gx = x0 + yc, gy = y0 + yr;
    const bool act0 = gx < nx && gy < ny, act1 = gx < nx && gy + 1 < ny;
    const size_t nxy = (size_t)nx * ny;
    float *optr = out + (size_t)comp * nxy * nz + (size_t)zb * nxy + (size_t)gy * nx + gx;

    auto issue = [&](int q) {
        const int sidx = q % ST;
        const int z = clampi(zb - R + q, 0, nz - 1);
        mbar_expect_tx(&bar[sidx], tx_bytes);
        tma_load_4d(stage0 + sidx * STAGE, &tin, x0 - WML, y0 - R, z, comp, &bar[sidx]);
    };
    if (tid == 0) {
        for (int q = 0; q < ST; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int q = 0; q < ST && q < P; ++q) issue(q);

    float2 ring[2][K];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < K; ++j) ring[h][j] = make_float2(0.f, 0.f);

    // x pass of the plane in stage sidx into x-pass buffer dst
    auto xpass = [&](int sidx, float *dst) {
        const float *src = stage0 + sidx * STAGE + xsrc;
        float v[16];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float4 f = *reinterpret_cast<const float4 *>(src + 4 * h);
            v[4 * h] = f.x; v[4 * h + 1] = f.y; v[4 * h + 2] = f.z; v[4 * h + 3] = f.w;
        }
        if (xedge) {                   // CTAs at an x border of the volume only
#pragma unroll
            for (int k = WML - R; k < WML; ++k) v[k] = pleft ? v[WML] : v[k];
#pragma unroll
            for (int k = 8 + WML; k < 8 + WML + R; ++k) v[k] = pright ? v[7 + WML] : v[k];
        }
        float2 o[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) o[m] = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            constexpr int B = WML - R;
            if ((B + j) % 2 == 0) {            // operand pairs register-aligned
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    o[m] = __ffma2_rn(w2[j], make_float2(v[B + j + 2 * m], v[B + j + 2 * m + 1]), o[m]);
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    o[m].x = fmaf(w2[j].x, v[B + j + 2 * m], o[m].x);
                    o[m].y = fmaf(w2[j].x, v[B + j + 2 * m + 1], o[m].y);
                }
            }
        }
        float *d = dst + xdst;
        *reinterpret_cast<float4 *>(d) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        *reinterpret_cast<float4 *>(d + 4) = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
    };

    int tw = -1;                        // plane whose wait ran out (-1: none)
    int sidx = 0, xo = 0;               // stage of plane t, x-pass buffer offset
    uint32_t par = 0;                   // phase parity of that stage
    for (int t0 = 0; t0 < P && tw < 0; t0 += PB * K) {
#pragma unroll
        for (int rr = 0; rr < PB * K; rr += PB) {
            const int t = t0 + rr;
            if (t >= P) break;
            const int np = min(PB, P - t);                // planes this step (the same for every thread)
            bool ok = true;
            if (xtask) {
                int si = sidx;
                uint32_t pa = par;
#pragma unroll
                for (int e = 0; e < PB; ++e) {
                    if (e >= np) break;
                    ok = ok && mbar_wait_bounded(&bar[si], pa);
                    xpass(si, xbuf + xo + e * XB);
                    if (++si == ST) { si = 0; pa ^= 1u; }
                }
            }
            if (__syncthreads_or(!ok)) { tw = t; break; }
            if (tid == 0) {                    // the stages just consumed take planes t + e + ST
                fence_proxy_async();
                for (int e = 0; e < np; ++e)
                    if (t + e + ST < P) issue(t + e + ST);
            }
            for (int e = 0; e < np; ++e)
                if (++sidx == ST) { sidx = 0; par ^= 1u; }
            // y pass into the planes' ring slots, z pass for planes t + e - 2R
#pragma unroll
            for (int e = 0; e < PB; ++e) {
                if (e >= np) break;
                const int te = t + e, re = (rr + e) % K;
                const float *col = xbuf + xo + e * XB + yr * WBX + yc;
                float2 yin[K + 1];
#pragma unroll
                for (int j = 0; j <= K; ++j) yin[j] = *reinterpret_cast<const float2 *>(col + j * WBX);
                float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    a0 = __ffma2_rn(w2[j], yin[j], a0);
                    a1 = __ffma2_rn(w2[j], yin[j + 1], a1);
                }
                ring[0][re] = a0;
                ring[1][re] = a1;
                if (te >= 2 * R) {
                    float2 o0 = make_float2(0.f, 0.f), o1 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        o0 = __ffma2_rn(w2[j], ring[0][(re + 1 + j) % K], o0);
                        o1 = __ffma2_rn(w2[j], ring[1][(re + 1 + j) % K], o1);
                    }
                    if (act0) *reinterpret_cast<float2 *>(optr) = o0;
                    if (act1) *reinterpret_cast<float2 *>(optr + nx) = o1;
                    optr += nxy;
                }
            }
            xo ^= PB * XB;
        }
    }
    if (tw >= 0) {
        // a wait ran out: record it, drain the loads still in flight (planes
        // tw .. tw + ST + PB - 2 were issued at most; bounded waits), leave
        if (tid == 0) {
            atomicExch(err, 1);
            for (int q = tw; q < min(tw + ST + PB - 1, P); ++q)
                mbar_wait_bounded(&bar[q % ST], (uint32_t)((q / ST) & 1));
        }
        __syncthreads();
    }
}

// Composite update u_new = du + u(x + du) (trilinear, clamped) or u + du,
// one voxel per thread along x-y tiles marching a few planes in z.  The
// update is bound by the latency of its 24 gathers per voxel, which resident
// warps hide: 5 CTAs per SM (40 warps) rather than 4.
__global__ void __launch_bounds__(NT, 5) k_compose_tiles(const float *__restrict__ u, const float *__restrict__ du,
                                                         int mode, int nx, int ny, int nz, int zc,
                                                         float *__restrict__ out, const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int zb = blockIdx.z * zc, ze = min(zb + zc, nz);
    const size_t nxy = (size_t)nx * ny, N = nxy * nz;
    const float fxmax = (float)(nx - 1), fymax = (float)(ny - 1), fzmax = (float)(nz - 1);
    const size_t col = (size_t)y * nx + x;
    // the next plane's du loads while this plane's corners are gathered
    float nx0 = 0.f, ny0 = 0.f, nz0 = 0.f;
    if (zb < ze) {
        const size_t i = (size_t)zb * nxy + col;
        nx0 = __ldg(du + i); ny0 = __ldg(du + N + i); nz0 = __ldg(du + 2 * N + i);
    }
    for (int z = zb; z < ze; ++z) {
        const size_t i = (size_t)z * nxy + col;
        const float dx = nx0, dy = ny0, dz = nz0;
        if (mode == CGDIR_ADDITIVE) {
            if (z + 1 < ze) { nx0 = __ldg(du + i + nxy); ny0 = __ldg(du + N + i + nxy); nz0 = __ldg(du + 2 * N + i + nxy); }
            out[i] = __ldg(u + i) + dx;
            out[N + i] = __ldg(u + N + i) + dy;
            out[2 * N + i] = __ldg(u + 2 * N + i) + dz;
            continue;
        }
        const float px = fminf(fmaxf((float)x + dx, 0.f), fxmax);
        const float py = fminf(fmaxf((float)y + dy, 0.f), fymax);
        const float pz = fminf(fmaxf((float)z + dz, 0.f), fzmax);
        const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
        const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        const float wx = px - fx, wy = py - fy, wz = pz - fz;
        const int ddx = ix < nx - 1 ? 1 : 0, ddy = iy < ny - 1 ? nx : 0;
        const size_t ddz = iz < nz - 1 ? nxy : 0;
        const size_t b0 = (size_t)iz * nxy + (size_t)iy * nx + ix;
        float cx[8], cy[8], cz[8];
        const size_t o[8] = {0, (size_t)ddx, (size_t)ddy, (size_t)(ddy + ddx), ddz, ddz + ddx, ddz + ddy,
                             ddz + ddy + ddx};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            cx[q] = __ldg(u + b0 + o[q]);
            cy[q] = __ldg(u + N + b0 + o[q]);
            cz[q] = __ldg(u + 2 * N + b0 + o[q]);
        }
        if (z + 1 < ze) { nx0 = __ldg(du + i + nxy); ny0 = __ldg(du + N + i + nxy); nz0 = __ldg(du + 2 * N + i + nxy); }
        auto tri = [&](const float *c) {
            const float e00 = fmaf(wx, c[1] - c[0], c[0]), e10 = fmaf(wx, c[3] - c[2], c[2]);
            const float e01 = fmaf(wx, c[5] - c[4], c[4]), e11 = fmaf(wx, c[7] - c[6], c[6]);
            const float f0 = fmaf(wy, e10 - e00, e00), f1 = fmaf(wy, e11 - e01, e01);
            return fmaf(wz, f1 - f0, f0);
        };
        out[i] = dx + tri(cx);
        out[N + i] = dy + tri(cy);
        out[2 * N + i] = dz + tri(cz);
    }
}

// The composite update for volumes below 2^31 voxels: the same arithmetic
// with 32-bit indices from per-component base pointers (one multiply-add
// per gather address, 48 registers at 5 CTAs per SM without spills).
// 512x512x160: 313 us per launch against 345 us for the 64-bit kernel at 4
// CTAs per SM; 6 CTAs per SM (40 registers) measured slower.
__global__ void __launch_bounds__(NT, 5) k_compose_tiles32(const float *__restrict__ u,
                                                                       const float *__restrict__ du, int nx, int ny,
                                                                       int nz, int zc, float *__restrict__ out,
                                                                       const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int zb = blockIdx.z * zc, ze = min(zb + zc, nz);
    const int nxy = nx * ny, N = nxy * nz;
    const float *__restrict__ ux = u, *__restrict__ uy = u + N, *__restrict__ uz = uy + N;
    const float *__restrict__ dx_ = du, *__restrict__ dy_ = du + N, *__restrict__ dz_ = dy_ + N;
    float *__restrict__ ox = out, *__restrict__ oy = out + N, *__restrict__ oz = oy + N;
    const float fxmax = (float)(nx - 1), fymax = (float)(ny - 1), fzmax = (float)(nz - 1);
    int i = zb * nxy + y * nx + x;
    float nx0 = 0.f, ny0 = 0.f, nz0 = 0.f;
    if (zb < ze) { nx0 = __ldg(dx_ + i); ny0 = __ldg(dy_ + i); nz0 = __ldg(dz_ + i); }
    for (int z = zb; z < ze; ++z, i += nxy) {
        const float dx = nx0, dy = ny0, dz = nz0;
        const float px = fminf(fmaxf((float)x + dx, 0.f), fxmax);
        const float py = fminf(fmaxf((float)y + dy, 0.f), fymax);
        const float pz = fminf(fmaxf((float)z + dz, 0.f), fzmax);
        const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
        const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        const float wx = px - fx, wy = py - fy, wz = pz - fz;
        const int ddx = ix < nx - 1 ? 1 : 0, ddy = iy < ny - 1 ? nx : 0, ddz = iz < nz - 1 ? nxy : 0;
        const int b0 = iz * nxy + iy * nx + ix;
        const int o[8] = {b0, b0 + ddx, b0 + ddy, b0 + ddy + ddx, b0 + ddz, b0 + ddz + ddx, b0 + ddz + ddy,
                          b0 + ddz + ddy + ddx};
        float cx[8], cy[8], cz[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            cx[q] = __ldg(ux + o[q]);
            cy[q] = __ldg(uy + o[q]);
            cz[q] = __ldg(uz + o[q]);
        }
        if (z + 1 < ze) { nx0 = __ldg(dx_ + i + nxy); ny0 = __ldg(dy_ + i + nxy); nz0 = __ldg(dz_ + i + nxy); }
        auto tri = [&](const float *c) {
            const float e00 = fmaf(wx, c[1] - c[0], c[0]), e10 = fmaf(wx, c[3] - c[2], c[2]);
            const float e01 = fmaf(wx, c[5] - c[4], c[4]), e11 = fmaf(wx, c[7] - c[6], c[6]);
            const float f0 = fmaf(wy, e10 - e00, e00), f1 = fmaf(wy, e11 - e01, e01);
            return fmaf(wz, f1 - f0, f0);
        };
        ox[i] = dx + tri(cx);
        oy[i] = dy + tri(cy);
        oz[i] = dz + tri(cz);
    }
}

// ---- 3-D tile version (small volumes) ------------------------------------
// A CTA loads a 16 x 16 x 8 output tile of one component with its R-voxel
// halo into shared memory (clamped indices) and runs the x, y and z passes
// there; no z march, so a small level's whole volume is filtered in one
// short wave instead of a long chain of plane steps.
constexpr int QX = 16, QY = 16, QZ = 8;

template <int R>
struct TileGeom {
    static constexpr int AX = QX + 2 * R, AY = QY + 2 * R, AZ = QZ + 2 * R;
    static constexpr int IN = AX * AY * AZ;            // input with halo
    static constexpr int XO = QX * AY * AZ;            // after the x pass
    static constexpr int YO = QX * QY * AZ;            // after the y pass (reuses the input buffer)
    static constexpr size_t bytes() { return sizeof(float) * ((size_t)IN + XO); }
};

template <int R>
__global__ void __launch_bounds__(NT) k_smooth_tile(const float *__restrict__ in, float *__restrict__ out,
                                                    Taps taps, int nx, int ny, int nz, int tiles_z,
                                                    const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    using G = TileGeom<R>;
    constexpr int K = 2 * R + 1, AX = G::AX, AY = G::AY;
    extern __shared__ float sm[];
    float *A = sm, *B = sm + G::IN;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int comp = blockIdx.z / tiles_z, tz = blockIdx.z % tiles_z;
    const int x0 = blockIdx.x * QX, y0 = blockIdx.y * QY, z0 = tz * QZ;
    const size_t nxy = (size_t)nx * ny;
    const float *src = in + (size_t)comp * nxy * nz;
    // batches of loads in flight before their stores (a load-then-store loop
    // would wait out one memory latency per element)
    constexpr int kBatch = 16;
    for (int p0 = 0; p0 < G::IN; p0 += kBatch * NT) {
        float v[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int p = p0 + b * NT + tid;
            if (p < G::IN) {
                const int hx = p % AX, hy = (p / AX) % AY, hz = p / (AX * AY);
                const int gx = clampi(x0 - R + hx, 0, nx - 1), gy = clampi(y0 - R + hy, 0, ny - 1),
                          gz = clampi(z0 - R + hz, 0, nz - 1);
                v[b] = __ldg(src + (size_t)gz * nxy + (size_t)gy * nx + gx);
            }
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int p = p0 + b * NT + tid;
            if (p < G::IN) A[p] = v[b];
        }
    }
    __syncthreads();
    for (int p = tid; p < G::XO; p += NT) {            // x pass: [AZ][AY][QX]
        const int ox = p % QX, r = p / QX;
        const float *row = A + r * AX + ox;
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc = fmaf(taps.w[j], row[j], acc);
        B[p] = acc;
    }
    __syncthreads();
    for (int p = tid; p < G::YO; p += NT) {            // y pass: [AZ][QY][QX] into A
        const int ox = p % QX, oy = (p / QX) % QY, hz = p / (QX * QY);
        const float *colp = B + (hz * AY + oy) * QX + ox;
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc = fmaf(taps.w[j], colp[j * QX], acc);
        A[p] = acc;
    }
    __syncthreads();
    float *dst = out + (size_t)comp * nxy * nz;
    for (int p = tid; p < QX * QY * QZ; p += NT) {      // z pass to memory
        const int ox = p % QX, oy = (p / QX) % QY, oz = p / (QX * QY);
        const int gx = x0 + ox, gy = y0 + oy, gz = z0 + oz;
        if (gx >= nx || gy >= ny || gz >= nz) continue;
        const float *colp = A + (oz * QY + oy) * QX + ox;
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc = fmaf(taps.w[j], colp[j * QX * QY], acc);
        dst[(size_t)gz * nxy + (size_t)gy * nx + gx] = acc;
    }
}

// ---- split version: xy pass and z pass as two kernels ------------------------
// k_smooth_xy filters planes in x and y: a CTA takes a 32 x 32 output tile
// of one component over a few consecutive planes; each plane's tile plus its
// R-voxel halo is loaded (clamped indices, positions precomputed once; the
// next plane's loads are issued before the current plane is filtered) into
// shared memory, filtered along x in 4-output register blocks and along y in
// 4-row register blocks.  k_smooth_z marches each (x, y) column through z
// with the three components' last 2R+1 values in registers and, for the
// du field, applies the composite update (Algorithm A step 3) on the spot:
// the z pass is where all three smoothed components of a voxel first meet,
// so the update costs no extra pass over memory.
constexpr int XYT = 32;                // xy output tile (32 x 32)
constexpr int XYZ = 4;                 // planes per CTA in the xy pass

template <int R>
__global__ void __launch_bounds__(NT) k_smooth_xy(const float *__restrict__ in, float *__restrict__ out, Taps taps,
                                                  int nx, int ny, int nz, int zgroups, const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    constexpr int K = 2 * R + 1, AX = XYT + 2 * R, AY = XYT + 2 * R, NA = AX * AY;
    constexpr int LPT = (NA + NT - 1) / NT;          // loads per thread per plane
    constexpr int XT = AY * (XYT / 4);               // x-pass tasks (4 outputs each)
    __shared__ float A[NA];
    __shared__ __align__(16) float B[AY * XYT];
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x0 = blockIdx.x * XYT, y0 = blockIdx.y * XYT;
    const int comp = blockIdx.z / zgroups, zb = (blockIdx.z % zgroups) * XYZ, ze = min(zb + XYZ, nz);
    const size_t nxy = (size_t)nx * ny, N = nxy * nz;
    const float *src = in + (size_t)comp * N;
    float *dst = out + (size_t)comp * N;
    int loff[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
        const int pidx = tid + q * NT;
        const int hy = pidx / AX, hx = pidx - hy * AX;
        const int gx = clampi(x0 - R + hx, 0, nx - 1), gy = clampi(y0 - R + hy, 0, ny - 1);
        loff[q] = pidx < NA ? gy * nx + gx : -1;
    }
    float pre[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) pre[q] = loff[q] >= 0 ? __ldg(src + (size_t)zb * nxy + loff[q]) : 0.f;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int z = zb; z < ze; ++z) {
#pragma unroll
        for (int q = 0; q < LPT; ++q)
            if (loff[q] >= 0) A[tid + q * NT] = pre[q];
        __syncthreads();
        if (z + 1 < ze) {                            // next plane's loads fly during the passes
#pragma unroll
            for (int q = 0; q < LPT; ++q) pre[q] = loff[q] >= 0 ? __ldg(src + (size_t)(z + 1) * nxy + loff[q]) : 0.f;
        }
        for (int task = tid; task < XT; task += NT) {   // x pass: row, 4 outputs
            const int row = task >> 3, xs = (task & 7) * 4;
            const float *a = A + row * AX + xs;
            float v[4 + 2 * R];
#pragma unroll
            for (int i = 0; i < 4 + 2 * R; ++i) v[i] = a[i];
            float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                o0 = fmaf(taps.w[j], v[j], o0);
                o1 = fmaf(taps.w[j], v[j + 1], o1);
                o2 = fmaf(taps.w[j], v[j + 2], o2);
                o3 = fmaf(taps.w[j], v[j + 3], o3);
            }
            *reinterpret_cast<float4 *>(B + row * XYT + xs) = make_float4(o0, o1, o2, o3);
        }
        __syncthreads();
        {                                              // y pass: column tx, rows 4ty .. 4ty+3
            float c[4 + 2 * R];
#pragma unroll
            for (int i = 0; i < 4 + 2 * R; ++i) c[i] = B[(4 * ty + i) * XYT + tx];
            float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int m = 0; m < 4; ++m) o[m] = fmaf(taps.w[j], c[j + m], o[m]);
            const int x = x0 + tx;
            if (x < nx) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int y = y0 + 4 * ty + m;
                    if (y < ny) dst[(size_t)z * nxy + (size_t)y * nx + x] = o[m];
                }
            }
        }
        // the next plane overwrites A only after every thread has left the x pass
    }
}

template <int R, int NC, bool COMPOSE>
__global__ void __launch_bounds__(NT) k_smooth_z(const float *__restrict__ in, const float *__restrict__ u, int mode,
                                                 float *__restrict__ out, Taps taps, int nx, int ny, int nz,
                                                 int zchunk, const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    constexpr int K = 2 * R + 1;
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int nchunks = (nz + zchunk - 1) / zchunk;
    const int comp = NC == 1 ? (int)blockIdx.z / nchunks : 0;
    const int zb = ((int)blockIdx.z % nchunks) * zchunk, ze = min(zb + zchunk, nz);
    const int P = (ze - zb) + 2 * R;
    const size_t nxy = (size_t)nx * ny, N = nxy * nz, col = (size_t)y * nx + x;
    const float *src = in + (size_t)comp * N + col;
    float *dst = out + (size_t)comp * N + col;
    float ring[NC][K];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int j = 0; j < K; ++j) ring[c][j] = 0.f;
    float nxt[NC];
    {
        const size_t zo = (size_t)clampi(zb - R, 0, nz - 1) * nxy;
#pragma unroll
        for (int c = 0; c < NC; ++c) nxt[c] = __ldg(src + c * N + zo);
    }
    const float fxmax = (float)(nx - 1), fymax = (float)(ny - 1), fzmax = (float)(nz - 1);
    for (int t0 = 0; t0 < P; t0 += K) {
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int t = t0 + r;
            if (t >= P) break;
#pragma unroll
            for (int c = 0; c < NC; ++c) ring[c][r] = nxt[c];
            if (t + 1 < P) {
                const size_t zo = (size_t)clampi(zb - R + t + 1, 0, nz - 1) * nxy;
#pragma unroll
                for (int c = 0; c < NC; ++c) nxt[c] = __ldg(src + c * N + zo);
            }
            if (t < 2 * R) continue;
            const int z = zb + t - 2 * R;
            float sv[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) acc = fmaf(taps.w[j], ring[c][(r + 1 + j) % K], acc);
                sv[c] = acc;
            }
            const size_t i = (size_t)z * nxy;
            if (COMPOSE) {
                float a0, a1, a2;
                if (mode == CGDIR_ADDITIVE) {
                    a0 = __ldg(u + i + col); a1 = __ldg(u + N + i + col); a2 = __ldg(u + 2 * N + i + col);
                } else {
                    const float px = fminf(fmaxf((float)x + sv[0], 0.f), fxmax);
                    const float py = fminf(fmaxf((float)y + sv[NC > 1 ? 1 : 0], 0.f), fymax);
                    const float pz = fminf(fmaxf((float)z + sv[NC > 2 ? 2 : 0], 0.f), fzmax);
                    const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
                    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
                    const float wx = px - fx, wy = py - fy, wz = pz - fz;
                    const int ddx = ix < nx - 1 ? 1 : 0, ddy = iy < ny - 1 ? nx : 0;
                    const size_t ddz = iz < nz - 1 ? nxy : 0;
                    const size_t b0 = (size_t)iz * nxy + (size_t)iy * nx + ix;
                    a0 = trilinear_at(u, b0, ddx, ddy, (int)ddz, wx, wy, wz);
                    a1 = trilinear_at(u + N, b0, ddx, ddy, (int)ddz, wx, wy, wz);
                    a2 = trilinear_at(u + 2 * N, b0, ddx, ddy, (int)ddz, wx, wy, wz);
                }
                dst[i] = sv[0] + a0;
                dst[N + i] = sv[NC > 1 ? 1 : 0] + a1;
                dst[2 * N + i] = sv[NC > 2 ? 2 : 0] + a2;
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) dst[c * N + i] = sv[c];
            }
        }
    }
}

__global__ void k_copy(const float *__restrict__ in, float *__restrict__ out, size_t n,
                       const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

// z chunk of the smoothing kernels: about two waves of resident CTAs (4 per
// SM for one component per CTA, 2 for the three-component compose variant).
int smooth_zchunk(int nx, int ny, int nz, int rows, int comp_ctas, int resident) {
    return pick_zchunk(nz, (long)((nx + TX - 1) / TX) * ((ny + rows - 1) / rows) * comp_ctas, resident, 2);
}

unsigned flat_grid(size_t n) {
    size_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g ? g : 1);
}

}  // namespace

template <int R, int NC, bool COMPOSE>
static cudaError_t smooth_tma_r(const float *in, const float *ucomp, int mode, float *out, int ncomp,
                                const Taps &t, int nx, int ny, int nz, const int *stop_flag, int *err,
                                cudaStream_t s, bool *launched, int zc_override) {
    using G = SmoothGeom<R, NC>;
    CUtensorMap m;
    const uint64_t dims[4] = {(uint64_t)nx, (uint64_t)ny, (uint64_t)nz, (uint64_t)ncomp};
    const uint32_t box[4] = {(uint32_t)G::BXW, (uint32_t)G::BY, 1u, (uint32_t)NC};
    *launched = false;
    if (!encode_tensor_map(&m, in, 4, dims, box, 4)) return cudaSuccess;
    const int zc = zc_override > 0 ? std::min(zc_override, nz)
                                   : smooth_zchunk(nx, ny, nz, SY, NC == 1 ? ncomp : 1, NC == 1 ? 4 : 2);
    const int nchunks = (nz + zc - 1) / zc;
    dim3 grid((nx + TX - 1) / TX, (ny + SY - 1) / SY, nchunks * (NC == 1 ? ncomp : 1)), block(TX, TY);
    const size_t smem = G::bytes();
    cudaError_t e = ensure_smem((const void *)k_smooth_tma<R, NC, COMPOSE>, smem);
    if (e != cudaSuccess) return e;
    k_smooth_tma<R, NC, COMPOSE><<<grid, block, smem, s>>>(m, ucomp, mode, out, ncomp, t, nx, ny, nz, zc,
                                                          stop_flag, err);
    *launched = true;
    note_launch();
    return cudaGetLastError();
}

// z chunk of the wide-tile z-march: about four waves of 3 resident CTAs per SM.
static int wide_default_zchunk(int nx, int ny, int nz, int ncomp) {
    return pick_zchunk(nz, (long)((nx + WX - 1) / WX) * ((ny + WY - 1) / WY) * ncomp, 3, 4);
}

// The wide-tile z-march for one component per CTA (nx % 8 == 0, R <= 4).
template <int R>
static cudaError_t smooth_wide_r(const float *in, float *out, int ncomp, const Taps &t, int nx, int ny, int nz,
                                 const int *stop_flag, int *err, cudaStream_t s, bool *launched, int zc_override,
                                 int cap) {
    using G = WideGeom<R>;
    CUtensorMap m;
    const uint64_t dims[4] = {(uint64_t)nx, (uint64_t)ny, (uint64_t)nz, (uint64_t)ncomp};
    const uint32_t box[4] = {(uint32_t)WBX, (uint32_t)G::BY, 1u, 1u};
    *launched = false;
    if (!encode_tensor_map(&m, in, 4, dims, box, 4)) return cudaSuccess;
    const int zc = zc_override > 0 ? std::min(zc_override, nz) : wide_default_zchunk(nx, ny, nz, ncomp);
    const int nchunks = (nz + zc - 1) / zc;
    dim3 grid((nx + WX - 1) / WX, (ny + WY - 1) / WY, nchunks * ncomp), block(TX, TY);
    constexpr int PB = 1;       // planes per barrier: 2 to 4 measured slower (more x-pass buffers)
    // a cap on CTAs per SM is a shared-memory request above 1/(cap+1) of the SM's 228 KB
    const size_t smem = std::max(G::bytes(PB), cap > 0 ? (size_t)(228 << 10) / (cap + 1) + 1024 : (size_t)0);
    cudaError_t e = ensure_smem((const void *)k_smooth_wide<R, PB>, smem);
    if (e != cudaSuccess) return e;
    k_smooth_wide<R, PB><<<grid, block, smem, s>>>(m, out, t, nx, ny, nz, zc, stop_flag, err);
    *launched = true;
    note_launch();
    return cudaGetLastError();
}

static cudaError_t smooth_wide(const float *in, float *out, int ncomp, const Taps &t, int nx, int ny, int nz,
                               const int *stop_flag, int *err, cudaStream_t s, bool *launched, int zc = 0,
                               int cap = 0) {
    *launched = false;
    if (nx % 8 != 0) return cudaSuccess;
    switch (t.r) {
        case 1: return smooth_wide_r<1>(in, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc, cap);
        case 2: return smooth_wide_r<2>(in, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc, cap);
        case 3: return smooth_wide_r<3>(in, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc, cap);
        case 4: return smooth_wide_r<4>(in, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc, cap);
        default: return cudaSuccess;
    }
}

template <int NC, bool COMPOSE>
static cudaError_t smooth_tma(const float *in, const float *ucomp, int mode, float *out, int ncomp,
                              const Taps &t, int nx, int ny, int nz, const int *stop_flag, int *err,
                              cudaStream_t s, bool *launched, int zc = 0) {
    switch (t.r) {
        case 1: return smooth_tma_r<1, NC, COMPOSE>(in, ucomp, mode, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc);
        case 2: return smooth_tma_r<2, NC, COMPOSE>(in, ucomp, mode, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc);
        case 3: return smooth_tma_r<3, NC, COMPOSE>(in, ucomp, mode, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc);
        case 4: return smooth_tma_r<4, NC, COMPOSE>(in, ucomp, mode, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc);
        case 5: return smooth_tma_r<5, NC, COMPOSE>(in, ucomp, mode, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc);
        case 6: return smooth_tma_r<6, NC, COMPOSE>(in, ucomp, mode, out, ncomp, t, nx, ny, nz, stop_flag, err, s, launched, zc);
        default: *launched = false; return cudaErrorInvalidValue;
    }
}

template <int R>
static cudaError_t smooth_tile_r(const float *in, int ncomp, const Taps &t, int nx, int ny, int nz, float *out,
                                 const int *stop_flag, cudaStream_t s) {
    const int tz = (nz + QZ - 1) / QZ;
    dim3 grid((nx + QX - 1) / QX, (ny + QY - 1) / QY, tz * ncomp), block(TX, TY);
    const size_t smem = TileGeom<R>::bytes();
    cudaError_t e = ensure_smem((const void *)k_smooth_tile<R>, smem);
    if (e != cudaSuccess) return e;
    k_smooth_tile<R><<<grid, block, smem, s>>>(in, out, t, nx, ny, nz, tz, stop_flag);
    note_launch();
    return cudaGetLastError();
}

static cudaError_t smooth_tile(const float *in, int ncomp, const Taps &t, int nx, int ny, int nz, float *out,
                               const int *stop_flag, cudaStream_t s) {
    switch (t.r) {
        case 1: return smooth_tile_r<1>(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
        case 2: return smooth_tile_r<2>(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
        case 3: return smooth_tile_r<3>(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
        case 4: return smooth_tile_r<4>(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
        case 5: return smooth_tile_r<5>(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
        case 6: return smooth_tile_r<6>(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
        default: return cudaErrorInvalidValue;
    }
}

static cudaError_t smooth_plain(const float *in, int ncomp, const Taps &t, int nx, int ny, int nz,
                                float *out, const int *stop_flag, cudaStream_t s) {
    const int zc = smooth_zchunk(nx, ny, nz, TY, 1, 4);
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + zc - 1) / zc), block(TX, TY);
    switch (t.r) {
        case 1: k_smooth<1><<<grid, block, 0, s>>>(in, out, ncomp, t, nx, ny, nz, zc, stop_flag); break;
        case 2: k_smooth<2><<<grid, block, 0, s>>>(in, out, ncomp, t, nx, ny, nz, zc, stop_flag); break;
        case 3: k_smooth<3><<<grid, block, 0, s>>>(in, out, ncomp, t, nx, ny, nz, zc, stop_flag); break;
        case 4: k_smooth<4><<<grid, block, 0, s>>>(in, out, ncomp, t, nx, ny, nz, zc, stop_flag); break;
        case 5: k_smooth<5><<<grid, block, 0, s>>>(in, out, ncomp, t, nx, ny, nz, zc, stop_flag); break;
        case 6: k_smooth<6><<<grid, block, 0, s>>>(in, out, ncomp, t, nx, ny, nz, zc, stop_flag); break;
        default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

int smooth_auto_variant(int nx, int ny, int nz) {
    return (size_t)nx * ny * nz < ((size_t)2 << 20) ? SMOOTH_TILE : SMOOTH_MARCH;
}

template <int R>
static cudaError_t smooth_split_r(const float *in, const float *u, int mode, bool compose, int ncomp, const Taps &t,
                                  int nx, int ny, int nz, float *out, float *scratch, int zc_override,
                                  const int *stop_flag, cudaStream_t s) {
    const int zgroups = (nz + XYZ - 1) / XYZ;
    dim3 g1((nx + XYT - 1) / XYT, (ny + XYT - 1) / XYT, zgroups * ncomp), block(TX, TY);
    k_smooth_xy<R><<<g1, block, 0, s>>>(in, scratch, t, nx, ny, nz, zgroups, stop_flag);
    const long tiles = (long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
    const int zc = zc_override > 0 ? std::min(zc_override, nz) : pick_zchunk(nz, tiles, 8, 1);
    const int nch = (nz + zc - 1) / zc;
    if (compose) {
        dim3 g2((nx + TX - 1) / TX, (ny + TY - 1) / TY, nch);
        k_smooth_z<R, 3, true><<<g2, block, 0, s>>>(scratch, u, mode, out, t, nx, ny, nz, zc, stop_flag);
    } else if (ncomp == 3) {
        dim3 g2((nx + TX - 1) / TX, (ny + TY - 1) / TY, nch);
        k_smooth_z<R, 3, false><<<g2, block, 0, s>>>(scratch, nullptr, 0, out, t, nx, ny, nz, zc, stop_flag);
    } else {
        dim3 g2((nx + TX - 1) / TX, (ny + TY - 1) / TY, nch * ncomp);
        k_smooth_z<R, 1, false><<<g2, block, 0, s>>>(scratch, nullptr, 0, out, t, nx, ny, nz, zc, stop_flag);
    }
    note_launch(2);
    return cudaGetLastError();
}

static cudaError_t smooth_split(const float *in, const float *u, int mode, bool compose, int ncomp, const Taps &t,
                                int nx, int ny, int nz, float *out, float *scratch, int zc, const int *stop_flag,
                                cudaStream_t s) {
    switch (t.r) {
        case 1: return smooth_split_r<1>(in, u, mode, compose, ncomp, t, nx, ny, nz, out, scratch, zc, stop_flag, s);
        case 2: return smooth_split_r<2>(in, u, mode, compose, ncomp, t, nx, ny, nz, out, scratch, zc, stop_flag, s);
        case 3: return smooth_split_r<3>(in, u, mode, compose, ncomp, t, nx, ny, nz, out, scratch, zc, stop_flag, s);
        case 4: return smooth_split_r<4>(in, u, mode, compose, ncomp, t, nx, ny, nz, out, scratch, zc, stop_flag, s);
        case 5: return smooth_split_r<5>(in, u, mode, compose, ncomp, t, nx, ny, nz, out, scratch, zc, stop_flag, s);
        case 6: return smooth_split_r<6>(in, u, mode, compose, ncomp, t, nx, ny, nz, out, scratch, zc, stop_flag, s);
        default: return cudaErrorInvalidValue;
    }
}

int smooth_default_zchunk(int nx, int ny, int nz, int ncomp) {
    if (nx % 8 == 0) return wide_default_zchunk(nx, ny, nz, ncomp);
    return smooth_zchunk(nx, ny, nz, SY, ncomp, 4);
}

cudaError_t launch_smooth(const float *in, int ncomp, float sigma, int nx, int ny, int nz,
                          float *out, const int *stop_flag, cudaStream_t s, int *err, SmoothChoice ch, float *scratch) {
    int variant = ch.variant;
    const Taps t = gauss_taps(sigma);
    const size_t N = (size_t)nx * ny * nz;
    if (t.r == 0) {
        k_copy<<<flat_grid(N * ncomp), 256, 0, s>>>(in, out, N * ncomp, stop_flag);
        note_launch();
        return cudaGetLastError();
    }
    if (err != nullptr) {
        // small volumes: the 3-D tile kernel (one short wave); large: the
        // TMA z-march, whose plane pipeline needs long chunks to pay off
        if (variant == SMOOTH_AUTO) variant = smooth_auto_variant(nx, ny, nz);
        if (variant == SMOOTH_FUSED) variant = SMOOTH_TILE;     // nothing to fuse with here
        if (variant == SMOOTH_TILE) return smooth_tile(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
        if (variant == SMOOTH_SPLIT && scratch != nullptr && scratch != in && scratch != out)
            return smooth_split(in, nullptr, 0, false, ncomp, t, nx, ny, nz, out, scratch, ch.zchunk, stop_flag, s);
        bool launched = false;
        if (variant != SMOOTH_MARCH_NARROW) {      // the wide-tile z-march where it applies
            cudaError_t e = smooth_wide(in, out, ncomp, t, nx, ny, nz, stop_flag, err, s, &launched, ch.zchunk,
                                        ch.ctas_per_sm);
            if (e != cudaSuccess || launched) return e;
        }
        cudaError_t e =
            smooth_tma<1, false>(in, nullptr, 0, out, ncomp, t, nx, ny, nz, stop_flag, err, s, &launched, ch.zchunk);
        if (e != cudaSuccess || launched) return e;
    }
    return smooth_plain(in, ncomp, t, nx, ny, nz, out, stop_flag, s);
}

cudaError_t launch_smooth_compose(const float *du, const float *u, int mode, float sigma, int nx, int ny,
                                  int nz, float *out, float *tmp, const int *stop_flag, cudaStream_t s,
                                  int *err, bool one_pass, SmoothChoice ch) {
    const Taps t = gauss_taps(sigma);
    if (!one_pass && t.r > 0 && err != nullptr) {
        int variant = ch.variant == SMOOTH_AUTO ? smooth_auto_variant(nx, ny, nz) : ch.variant;
        if (variant == SMOOTH_SPLIT)   // x/y pass, then the z pass with the composite update fused
            return smooth_split(du, u, mode, true, 3, t, nx, ny, nz, out, tmp, ch.zchunk, stop_flag, s);
        if (variant == SMOOTH_FUSED && (size_t)nx * ny * nz < (size_t)1 << 31)   // one 3-D tile kernel
            return launch_fused_smooth_compose(du, u, mode, sigma, nx, ny, nz, out, stop_flag, err, s);
    }
    if (one_pass && t.r > 0 && err != nullptr) {
        bool launched = false;
        cudaError_t e = smooth_tma<3, true>(du, u, mode, out, 3, t, nx, ny, nz, stop_flag, err, s, &launched);
        if (e != cudaSuccess || launched) return e;
    }
    // smooth du into tmp, then compose
    if (ch.variant == SMOOTH_SPLIT) ch.variant = SMOOTH_MARCH;
    cudaError_t e = launch_smooth(du, 3, sigma, nx, ny, nz, tmp, stop_flag, s, err, ch);
    if (e != cudaSuccess) return e;
    return launch_compose(u, tmp, mode, nx, ny, nz, out, stop_flag, s);
}

cudaError_t launch_compose(const float *u, const float *du, int mode, int nx, int ny, int nz,
                           float *out, const int *stop_flag, cudaStream_t s) {
    const long tiles = (long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
    const int zc = pick_zchunk(nz, tiles, 8, 4);
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + zc - 1) / zc), block(TX, TY);
    if (mode != CGDIR_ADDITIVE && (size_t)nx * ny * nz < ((size_t)1 << 31)) {
        k_compose_tiles32<<<grid, block, 0, s>>>(u, du, nx, ny, nz, zc, out, stop_flag);
        note_launch();
        return cudaGetLastError();
    }
    k_compose_tiles<<<grid, block, 0, s>>>(u, du, mode, nx, ny, nz, zc, out, stop_flag);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cgdir
