// Fused iteration schedule for small and medium pyramid levels.
//
// At a coarse level an iteration of Algorithm A (Sec. 2.2) is five short
// kernels (warp, force stencil, G(du), composite update, G(u)), each bound
// by launch and memory latency rather than bandwidth.  Two kernels here
// take four of those steps:
//
//   k_fused_smooth_compose  G_fluid(du) (step 2) and the composite update
//                           du + u(x + du) or u + du (step 3) -> u'
//   k_fused_smooth_warp     G_diff(u') -> u (step 4), then the warp of the
//                           moving image and the structure terms at the new
//                           u: the first pass of the next iteration's force
//
// so an iteration becomes the force stencil pass plus these two.  A CTA
// owns an 8 x 8 x 8 output tile of all three components: the tile plus its
// R-voxel halo (R = ceil(3 sigma)) is brought into shared memory, filtered
// along x (a row per task), then y (a column per task), then z (a z column
// per task), and each thread then takes its output voxels' three smoothed
// components from shared memory for the update (or the warp), with no
// further pass over memory.  Every tap sum runs in the same order as the
// other smoothing kernels (x, y, z; taps in ascending offset; every
// multiply-add a separately rounded FMA), the update has the update
// kernel's arithmetic and the warp is the force's own warp function, so
// the fused schedule gives the same bits as the unfused one.
#include "cgdir_internal.cuh"
#include "tma.cuh"
#include "warp_corners.cuh"

namespace cgdir {

namespace {

constexpr int FT = 256;     // threads per CTA
constexpr int FQ = 8;       // output tile edge

// Shared-memory plan of one CTA (all three components):
//   S  the input box, W x A x A per component (x fastest), as one TMA box
//      (x from x0 - ML, ML = R rounded up to 4, so the start is 16-byte
//      aligned; y and z from y0 - R and z0 - R; zero fill outside the
//      volume) or, when no tensor map is possible, loaded with clamped
//      indices;
//   X  the x pass, [c][hz][hy][8] with row stride XS and plane stride XP;
//   Y  the y pass, [c][hz][oy][8] with plane stride YP (over S);
//   Z  the z pass, [c][oz][oy][ox] (over X).
// Clamping at the volume border: the x pass reads, for a halo row outside
// the volume, the clamped row of S, so X, Y and Z hold exactly the clamped
// filter; in x, tiles whose halo leaves the volume read clamped columns.
// W / 4 odd, XS = 12 and XP, YP = 8 mod 32 make the row-per-thread and
// column-per-thread accesses free of bank conflicts.
template <int R>
struct FusedTile {
    static constexpr int A = FQ + 2 * R;                 // haloed edge in y and z
    static constexpr int ML = (R + 3) / 4 * 4;           // x margin of the box
    static constexpr int WMIN = ML + FQ + R;
    static constexpr int W = ((WMIN + 3) / 4 % 2 == 1) ? (WMIN + 3) / 4 * 4 : (WMIN + 3) / 4 * 4 + 4;
    static constexpr int XS = 12;
    static constexpr int XP = (A * XS + 23) / 32 * 32 + 8;
    static constexpr int YP = 72;
    static constexpr int SN = 3 * A * A * W;            // floats of the input box
    // u around the tile for the composite update (x from x0 - 4, 16 wide;
    // y, z from -UH, 8 + 2 UH), landing beside Y in the S region while the
    // y and z passes run
    static constexpr int UH = 2, UW = 16, UA = FQ + 2 * UH;
    static constexpr int UN = 3 * UA * UA * UW;
    static constexpr int UOFF = (3 * A * 72 + 31) / 32 * 32;          // after Y
    static constexpr int SREG = SN > UOFF + UN ? SN : UOFF + UN;      // floats of the S region
    static constexpr int XN = 3 * A * XP;               // floats of X (at S + SREG)
    static constexpr int ROWS = 3 * A * A;              // x-pass tasks
    static constexpr int COLS = 3 * A * FQ;             // y-pass tasks
    static constexpr int ZCOLS = 3 * FQ * FQ;           // z-pass tasks
    static constexpr size_t bytes() { return 128 + sizeof(float) * ((size_t)SREG + XN) + 16; }
    static_assert(3 * A * YP <= SN && 3 * FQ * FQ * FQ <= XN, "overlays");
    static_assert(XP % 32 == 8 && XP >= A * XS, "x-pass layout");
};

// G(in) over the CTA's tile into Z (smem), all three components.  Returns
// false (every thread) if the TMA wait ran out; the error word is then set.
// With umap, the u tile's TMA copy (completing on bar[1]) is issued as soon
// as the input box has been read.
template <int R>
__device__ __forceinline__ bool tile_smooth(const CUtensorMap *tin, bool use_tma, const float *__restrict__ in,
                                            const Taps &t, int nx, int ny, int nz, int x0, int y0, int z0,
                                            float *S, float *X, uint64_t *bar, int *err, int tid,
                                            const CUtensorMap *umap = nullptr) {
    using G = FusedTile<R>;
    constexpr int K = 2 * R + 1, A = G::A, ML = G::ML, W = G::W, XS = G::XS, XP = G::XP, YP = G::YP;
    float2 w2[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w2[j] = make_float2(t.w[j], t.w[j]);
    if (use_tma) {
        if (tid == 0) {
            mbar_init(bar, 1);
            if (umap) mbar_init(bar + 1, 1);
            fence_mbar_init();
            mbar_expect_tx(bar, (uint32_t)(G::SN * sizeof(float)));
            tma_load_4d(S, tin, x0 - ML, y0 - R, z0 - R, 0, bar);
        }
        __syncthreads();
        const bool ok = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(bar, 0);              // let the copy land before leaving
            }
            __syncthreads();
            return false;
        }
    } else {
        const int nxy = nx * ny, N = nxy * nz;
        constexpr int kBatch = 16;
        for (int p0 = 0; p0 < G::SN; p0 += kBatch * FT) {
            float v[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int p = p0 + b * FT + tid;
                if (p < G::SN) {
                    const int i = p % W, row = p / W;
                    const int c = row / (A * A), rem = row - c * (A * A), hz = rem / A, hy = rem - hz * A;
                    const int gx = clampi(x0 - ML + i, 0, nx - 1), gy = clampi(y0 - R + hy, 0, ny - 1),
                              gz = clampi(z0 - R + hz, 0, nz - 1);
                    v[b] = __ldg(in + (size_t)c * N + gz * nxy + gy * nx + gx);
                }
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int p = p0 + b * FT + tid;
                if (p < G::SN) S[p] = v[b];
            }
        }
        __syncthreads();
    }
    // x pass: one row (8 outputs) per task
    const bool xfast = !use_tma || (x0 - R >= 0 && x0 + FQ + R <= nx);
    for (int task = tid; task < G::ROWS; task += FT) {
        const int c = task / (A * A), rem = task - c * (A * A), hz = rem / A, hy = rem - hz * A;
        const int hzc = clampi(z0 - R + hz, 0, nz - 1) - (z0 - R), hyc = clampi(y0 - R + hy, 0, ny - 1) - (y0 - R);
        const float *src = S + ((c * A + hzc) * A + hyc) * W;
        float *dst = X + (c * A + hz) * XP + hy * XS;
        float o[FQ];
        if (xfast) {
            constexpr int F0 = (ML - R) / 4, F1 = (ML + FQ + R - 1) / 4;   // float4s holding the taps
            float v[4 * (F1 + 1)];
#pragma unroll
            for (int h = F0; h <= F1; ++h) {
                const float4 f = reinterpret_cast<const float4 *>(src)[h];
                v[4 * h] = f.x; v[4 * h + 1] = f.y; v[4 * h + 2] = f.z; v[4 * h + 3] = f.w;
            }
#pragma unroll
            for (int q = 0; q < FQ; q += 2) {
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    if ((ML - R + j) % 2 == 0) {       // operand pair register-aligned: paired FMA
                        a = __ffma2_rn(w2[j], make_float2(v[ML - R + q + j], v[ML - R + q + 1 + j]), a);
                    } else {                           // odd offset: scalar FMAs (same rounding, no moves)
                        a.x = fmaf(w2[j].x, v[ML - R + q + j], a.x);
                        a.y = fmaf(w2[j].x, v[ML - R + q + 1 + j], a.y);
                    }
                }
                o[q] = a.x; o[q + 1] = a.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < FQ; ++q) {
                float a = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) a = fmaf(t.w[j], src[clampi(x0 + q + j - R, 0, nx - 1) - (x0 - ML)], a);
                o[q] = a;
            }
        }
        reinterpret_cast<float4 *>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<float4 *>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
    __syncthreads();
    if (umap && tid == 0) {                                // S has been read: bring u's tile in
        fence_proxy_async();
        mbar_expect_tx(bar + 1, (uint32_t)(G::UN * sizeof(float)));
        tma_load_4d(S + G::UOFF, umap, x0 - 4, y0 - G::UH, z0 - G::UH, 0, bar + 1);
    }
    float *Y = S;                                          // S is free now
    for (int task = tid; task < G::COLS; task += FT) {     // y pass: one column (8 outputs) per task
        const int ch = task >> 3, ox = task & 7;           // ch = c * A + hz
        const float *col = X + ch * XP + ox;
        float yin[A];
#pragma unroll
        for (int h = 0; h < A; ++h) yin[h] = col[h * XS];
        float *dst = Y + ch * YP + ox;
#pragma unroll
        for (int q = 0; q < FQ; q += 2) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (j % 2 == 0) {
                    a = __ffma2_rn(w2[j], make_float2(yin[q + j], yin[q + 1 + j]), a);
                } else {
                    a.x = fmaf(w2[j].x, yin[q + j], a.x);
                    a.y = fmaf(w2[j].x, yin[q + 1 + j], a.y);
                }
            }
            dst[q * FQ] = a.x;
            dst[(q + 1) * FQ] = a.y;
        }
    }
    __syncthreads();
    float *Z = X;                                          // X is free now
    for (int task = tid; task < G::ZCOLS; task += FT) {    // z pass: one z column per task
        const int c = task >> 6, oyx = task & 63;
        const float *col = Y + c * A * YP + oyx;
        float zin[A];
#pragma unroll
        for (int h = 0; h < A; ++h) zin[h] = col[h * YP];
        float *dst = Z + c * (FQ * FQ * FQ) + oyx;
#pragma unroll
        for (int q = 0; q < FQ; q += 2) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (j % 2 == 0) {
                    a = __ffma2_rn(w2[j], make_float2(zin[q + j], zin[q + 1 + j]), a);
                } else {
                    a.x = fmaf(w2[j].x, zin[q + j], a.x);
                    a.y = fmaf(w2[j].x, zin[q + 1 + j], a.y);
                }
            }
            dst[q * FQ * FQ] = a.x;
            dst[(q + 1) * FQ * FQ] = a.y;
        }
    }
    __syncthreads();
    return true;
}

template <int R>
struct TileSmem {
    float *S, *X;
    uint64_t *bar;
    __device__ explicit TileSmem(unsigned char *raw) {
        using G = FusedTile<R>;
        S = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
        X = S + G::SREG;
        bar = reinterpret_cast<uint64_t *>(X + G::XN);
    }
};

constexpr int kVoxPerThread = FQ * FQ * FQ / FT;          // 2

template <int R>
__global__ void __launch_bounds__(FT, 3) k_fused_smooth_compose(const __grid_constant__ CUtensorMap tin, int use_tma,
                                                              const __grid_constant__ CUtensorMap umap,
                                                              const float *__restrict__ du,
                                                              const float *__restrict__ u, int mode, Taps t,
                                                              int nx, int ny, int nz, float *__restrict__ out,
                                                              const int *stop_flag, int *err) {
    if (stop_flag && *stop_flag) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileSmem<R> sm(smem_raw);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * FQ, y0 = blockIdx.y * FQ, z0 = blockIdx.z * FQ;
    const bool utile = use_tma != 0 && mode != CGDIR_ADDITIVE;
    if (!tile_smooth<R>(&tin, use_tma != 0, du, t, nx, ny, nz, x0, y0, z0, sm.S, sm.X, sm.bar, err, tid,
                        utile ? &umap : nullptr))
        return;
    const float *Z = sm.X;
    const int nxy = nx * ny, N = nxy * nz;
    const float fxmax = (float)(nx - 1), fymax = (float)(ny - 1), fzmax = (float)(nz - 1);
    // both output voxels' smoothed values, then both voxels' 24 gathers in flight together
    float s[kVoxPerThread][3];
    int xv[kVoxPerThread], yv[kVoxPerThread], zv[kVoxPerThread];
    bool in_vol[kVoxPerThread];
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v) {
        const int p = tid + v * FT;
        xv[v] = x0 + (p & 7); yv[v] = y0 + ((p >> 3) & 7); zv[v] = z0 + (p >> 6);
        in_vol[v] = xv[v] < nx && yv[v] < ny && zv[v] < nz;
#pragma unroll
        for (int c = 0; c < 3; ++c) s[v][c] = Z[c * (FQ * FQ * FQ) + p];
    }
    if (mode == CGDIR_ADDITIVE) {
#pragma unroll
        for (int v = 0; v < kVoxPerThread; ++v) {
            if (!in_vol[v]) continue;
            const int i = zv[v] * nxy + yv[v] * nx + xv[v];
#pragma unroll
            for (int c = 0; c < 3; ++c) out[(size_t)c * N + i] = __ldg(u + (size_t)c * N + i) + s[v][c];
        }
        return;
    }
    using G = FusedTile<R>;
    float cc[kVoxPerThread][3][8];
    float wx[kVoxPerThread], wy[kVoxPerThread], wz[kVoxPerThread];
    bool in_tile[kVoxPerThread];
    int lb[kVoxPerThread], lo[kVoxPerThread][3];
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v) {
        if (!in_vol[v]) continue;
        const float px = fminf(fmaxf((float)xv[v] + s[v][0], 0.f), fxmax);
        const float py = fminf(fmaxf((float)yv[v] + s[v][1], 0.f), fymax);
        const float pz = fminf(fmaxf((float)zv[v] + s[v][2], 0.f), fzmax);
        const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
        const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        wx[v] = px - fx; wy[v] = py - fy; wz[v] = pz - fz;
        const int ddx = ix < nx - 1 ? 1 : 0, ddy = iy < ny - 1 ? nx : 0, ddz = iz < nz - 1 ? nxy : 0;
        // corners inside u's tile come from shared memory (the same values)
        const int lx = ix - (x0 - 4), ly = iy - (y0 - G::UH), lz = iz - (z0 - G::UH);
        if (utile && lx >= 0 && lx + 1 < G::UW && ly >= 0 && ly + 1 < G::UA && lz >= 0 && lz + 1 < G::UA) {
            in_tile[v] = true;
            lb[v] = (lz * G::UA + ly) * G::UW + lx;
            lo[v][0] = ddx ? 1 : 0;
            lo[v][1] = ddy ? G::UW : 0;
            lo[v][2] = ddz ? G::UA * G::UW : 0;
            continue;
        }
        in_tile[v] = false;
        const int b0 = iz * nxy + iy * nx + ix;
        const int o[8] = {0, ddx, ddy, ddy + ddx, ddz, ddz + ddx, ddz + ddy, ddz + ddy + ddx};
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 8; ++q) cc[v][c][q] = __ldg(u + (size_t)c * N + b0 + o[q]);
    }
    if (utile) {
        const bool ok = mbar_wait_bounded(sm.bar + 1, 0);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(sm.bar + 1, 0);
            }
            __syncthreads();
            return;
        }
        const float *U = sm.S + G::UOFF;
#pragma unroll
        for (int v = 0; v < kVoxPerThread; ++v) {
            if (!in_vol[v] || !in_tile[v]) continue;
            const int o[8] = {0, lo[v][0], lo[v][1], lo[v][1] + lo[v][0], lo[v][2], lo[v][2] + lo[v][0],
                              lo[v][2] + lo[v][1], lo[v][2] + lo[v][1] + lo[v][0]};
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < 8; ++q) cc[v][c][q] = U[c * (G::UA * G::UA * G::UW) + lb[v] + o[q]];
        }
    }
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v) {
        if (!in_vol[v]) continue;
        const int i = zv[v] * nxy + yv[v] * nx + xv[v];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float *q = cc[v][c];
            const float e00 = fmaf(wx[v], q[1] - q[0], q[0]), e10 = fmaf(wx[v], q[3] - q[2], q[2]);
            const float e01 = fmaf(wx[v], q[5] - q[4], q[4]), e11 = fmaf(wx[v], q[7] - q[6], q[6]);
            const float f0 = fmaf(wy[v], e10 - e00, e00), f1 = fmaf(wy[v], e11 - e01, e01);
            out[(size_t)c * N + i] = s[v][c] + fmaf(wz[v], f1 - f0, f0);
        }
    }
}

template <int R, bool CONTOUR, typename IT>
__global__ void __launch_bounds__(FT) k_fused_smooth_warp(const __grid_constant__ CUtensorMap tin, int use_tma,
                                                           const float *__restrict__ in, Taps t,
                                                           float *__restrict__ u, ForceArgs a, int *err) {
    if (a.stop_flag && *a.stop_flag) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileSmem<R> sm(smem_raw);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * FQ, y0 = blockIdx.y * FQ, z0 = blockIdx.z * FQ;
    if (!tile_smooth<R>(&tin, use_tma != 0, in, t, nx, ny, nz, x0, y0, z0, sm.S, sm.X, sm.bar, err, tid)) return;
    const float *Z = sm.X;
    const int nxy = nx * ny, N = nxy * nz;
    CornerSet<IT> cs[kVoxPerThread];
    int iv[kVoxPerThread];
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v) {
        const int p = tid + v * FT;
        const int x = x0 + (p & 7), y = y0 + ((p >> 3) & 7), z = z0 + (p >> 6);
        iv[v] = -1;
        if (x >= nx || y >= ny || z >= nz) continue;
        const int i = z * nxy + y * nx + x;
        iv[v] = i;
        const float sx = Z[p], sy = Z[FQ * FQ * FQ + p], sz = Z[2 * FQ * FQ * FQ + p];
        u[i] = sx;
        u[N + i] = sy;
        u[N + N + i] = sz;
        corner_load<CONTOUR, IT>(a, sx, sy, sz, x, y, z, cs[v]);
    }
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v)
        if (iv[v] >= 0) corner_finish<CONTOUR, IT>(a, iv[v], N, cs[v]);
}

// Tensor map of a [3][nz][ny][nx] field for the tile box; false if TMA
// cannot be used (nx % 4 != 0, misaligned base): the kernels then load
// with clamped indices.
template <int R>
bool tile_map(CUtensorMap *m, const float *f, int nx, int ny, int nz) {
    using G = FusedTile<R>;
    const uint64_t dims[4] = {(uint64_t)nx, (uint64_t)ny, (uint64_t)nz, 3};
    const uint32_t box[4] = {(uint32_t)G::W, (uint32_t)G::A, (uint32_t)G::A, 3};
    return encode_tensor_map(m, f, 4, dims, box, 4);
}

template <int R>
cudaError_t compose_r(const float *du, const float *u, int mode, const Taps &t, int nx, int ny, int nz,
                      float *out, const int *stop_flag, int *err, cudaStream_t s) {
    const size_t smem = FusedTile<R>::bytes();
    cudaError_t e = ensure_smem((const void *)k_fused_smooth_compose<R>, smem);
    if (e != cudaSuccess) return e;
    CUtensorMap m{}, mu{};
    int use_tma = tile_map<R>(&m, du, nx, ny, nz) ? 1 : 0;
    if (use_tma) {
        using G = FusedTile<R>;
        const uint64_t dims[4] = {(uint64_t)nx, (uint64_t)ny, (uint64_t)nz, 3};
        const uint32_t box[4] = {(uint32_t)G::UW, (uint32_t)G::UA, (uint32_t)G::UA, 3};
        if (!encode_tensor_map(&mu, u, 4, dims, box, 4)) use_tma = 0;
    }
    dim3 grid((nx + FQ - 1) / FQ, (ny + FQ - 1) / FQ, (nz + FQ - 1) / FQ);
    k_fused_smooth_compose<R><<<grid, FT, smem, s>>>(m, use_tma, mu, du, u, mode, t, nx, ny, nz, out, stop_flag, err);
    note_launch();
    return cudaGetLastError();
}

template <int R, bool CONTOUR, typename IT>
cudaError_t warp_rt(const float *in, const Taps &t, float *u, const ForceArgs &a, int *err, cudaStream_t s) {
    const size_t smem = FusedTile<R>::bytes();
    cudaError_t e = ensure_smem((const void *)k_fused_smooth_warp<R, CONTOUR, IT>, smem);
    if (e != cudaSuccess) return e;
    CUtensorMap m{};
    const int use_tma = tile_map<R>(&m, in, a.nx, a.ny, a.nz) ? 1 : 0;
    dim3 grid((a.nx + FQ - 1) / FQ, (a.ny + FQ - 1) / FQ, (a.nz + FQ - 1) / FQ);
    k_fused_smooth_warp<R, CONTOUR, IT><<<grid, FT, smem, s>>>(m, use_tma, in, t, u, a, err);
    note_launch();
    return cudaGetLastError();
}

template <int R>
cudaError_t warp_r(const float *in, const Taps &t, float *u, const ForceArgs &a, int *err, cudaStream_t s) {
    const bool contour = a.contour && a.k > 0;
    if (a.img_dtype == CGDIR_F16)
        return contour ? warp_rt<R, true, __half>(in, t, u, a, err, s) : warp_rt<R, false, __half>(in, t, u, a, err, s);
    if (a.img_dtype == CGDIR_BF16)
        return contour ? warp_rt<R, true, __nv_bfloat16>(in, t, u, a, err, s)
                       : warp_rt<R, false, __nv_bfloat16>(in, t, u, a, err, s);
    return contour ? warp_rt<R, true, float>(in, t, u, a, err, s) : warp_rt<R, false, float>(in, t, u, a, err, s);
}

}  // namespace

bool fused_schedule_ok(const ForceArgs &a) {
    return a.wfield != nullptr && (size_t)a.nx * a.ny * a.nz < (size_t)1 << 31;
}

cudaError_t launch_fused_smooth_compose(const float *du, const float *u, int mode, float sigma, int nx, int ny,
                                        int nz, float *out, const int *stop_flag, int *err, cudaStream_t s) {
    if ((size_t)nx * ny * nz >= (size_t)1 << 31) return cudaErrorInvalidValue;
    const Taps t = gauss_taps(sigma);
    switch (t.r) {
        case 1: return compose_r<1>(du, u, mode, t, nx, ny, nz, out, stop_flag, err, s);
        case 2: return compose_r<2>(du, u, mode, t, nx, ny, nz, out, stop_flag, err, s);
        case 3: return compose_r<3>(du, u, mode, t, nx, ny, nz, out, stop_flag, err, s);
        case 4: return compose_r<4>(du, u, mode, t, nx, ny, nz, out, stop_flag, err, s);
        case 5: return compose_r<5>(du, u, mode, t, nx, ny, nz, out, stop_flag, err, s);
        case 6: return compose_r<6>(du, u, mode, t, nx, ny, nz, out, stop_flag, err, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_smooth_warp(const float *in, float sigma, float *u, const ForceArgs &a, int *err,
                                     cudaStream_t s) {
    if (!fused_schedule_ok(a)) return cudaErrorInvalidValue;
    const Taps t = gauss_taps(sigma);
    switch (t.r) {
        case 1: return warp_r<1>(in, t, u, a, err, s);
        case 2: return warp_r<2>(in, t, u, a, err, s);
        case 3: return warp_r<3>(in, t, u, a, err, s);
        case 4: return warp_r<4>(in, t, u, a, err, s);
        case 5: return warp_r<5>(in, t, u, a, err, s);
        case 6: return warp_r<6>(in, t, u, a, err, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cgdir
