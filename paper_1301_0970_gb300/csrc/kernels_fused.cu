// Fused iteration schedule for small and medium pyramid levels.
//
// At a coarse level an iteration of Algorithm A (Sec. 2.2) is five short
// kernels (warp, force stencil, G(du), composite update, G(u)), each bound
// by launch and memory latency rather than bandwidth.  Two kernels here
// take four of those steps:
//
//   k_fused_smooth_compose  G_fluid(du) (steps 2) and the composite update
//                           du + u(x + du) or u + du (step 3) -> u'
//   k_fused_smooth_warp     G_diff(u') -> u (step 4), then the warp of the
//                           moving image and the structure terms at the new
//                           u: the first pass of the next iteration's force
//
// so an iteration becomes the force stencil pass plus these two.  A CTA
// owns an 8 x 8 x 8 output tile of all three components: the tile plus its
// R-voxel halo (clamped indices, R = ceil(3 sigma)) is loaded into shared
// memory, filtered along x, then y, then z, and each thread takes the z
// pass of its output voxels for all three components, so the update (or
// the warp) follows in registers with no further pass over memory.  Every
// tap sum runs in the same order as the other smoothing kernels (x, y, z;
// taps in ascending offset; explicit FMAs), the update has the update
// kernel's arithmetic and the warp is the force's own warp function, so
// the fused schedule gives the same bits as the unfused one.
#include "cgdir_internal.cuh"
#include "warp_corners.cuh"

namespace cgdir {

namespace {

constexpr int FT = 256;     // threads per CTA
constexpr int FQ = 8;       // output tile edge

template <int R>
struct FusedTile {
    static constexpr int A = FQ + 2 * R;                 // haloed edge
    static constexpr int IN = A * A * A;                 // haloed input      [z][y][x]
    static constexpr int XO = FQ * A * A;                // after the x pass  [z][y][FQ]
    static constexpr int YO = FQ * FQ * A;               // after the y pass  [z][FQ][FQ] (over the input)
    static constexpr int OUT = FQ * FQ * FQ;
    static constexpr int PER = IN + XO;                  // floats per component
    static constexpr size_t bytes() { return 3 * sizeof(float) * (size_t)PER; }
    static_assert(OUT % FT == 0, "outputs per thread");
};

// Load the haloed tile of the three components of `in` ([3][N]) and run the
// x and y passes; afterwards component c's y-pass output is at sm + c*PER.
template <int R>
__device__ __forceinline__ void tile_xy(const float *__restrict__ in, const Taps &t, int nx, int ny, int nz,
                                        int x0, int y0, int z0, float *sm, int tid) {
    using G = FusedTile<R>;
    constexpr int K = 2 * R + 1, A = G::A;
    const int nxy = nx * ny, N = nxy * nz;
    for (int p = tid; p < 3 * G::IN; p += FT) {
        const int c = p / G::IN, q = p - c * G::IN;
        const int hx = q % A, hy = (q / A) % A, hz = q / (A * A);
        const int gx = clampi(x0 - R + hx, 0, nx - 1), gy = clampi(y0 - R + hy, 0, ny - 1),
                  gz = clampi(z0 - R + hz, 0, nz - 1);
        sm[c * G::PER + q] = __ldg(in + (size_t)c * N + gz * nxy + gy * nx + gx);
    }
    __syncthreads();
    for (int p = tid; p < 3 * G::XO; p += FT) {           // x pass
        const int c = p / G::XO, q = p - c * G::XO;
        const int ox = q % FQ, r = q / FQ;
        const float *row = sm + c * G::PER + r * A + ox;
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc = fmaf(t.w[j], row[j], acc);
        sm[c * G::PER + G::IN + q] = acc;
    }
    __syncthreads();
    for (int p = tid; p < 3 * G::YO; p += FT) {           // y pass, over the input
        const int c = p / G::YO, q = p - c * G::YO;
        const int ox = q % FQ, oy = (q / FQ) % FQ, hz = q / (FQ * FQ);
        const float *colp = sm + c * G::PER + G::IN + (hz * A + oy) * FQ + ox;
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc = fmaf(t.w[j], colp[j * FQ], acc);
        sm[c * G::PER + q] = acc;
    }
    __syncthreads();
}

// z pass of component c at output (ox, oy, oz) of the tile.
template <int R>
__device__ __forceinline__ float tile_z(const float *sm, const Taps &t, int c, int ox, int oy, int oz) {
    using G = FusedTile<R>;
    constexpr int K = 2 * R + 1;
    const float *colp = sm + c * G::PER + (oz * FQ + oy) * FQ + ox;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) acc = fmaf(t.w[j], colp[j * FQ * FQ], acc);
    return acc;
}

constexpr int kVoxPerThread = FQ * FQ * FQ / FT;          // 2

template <int R>
__global__ void __launch_bounds__(FT, 2) k_fused_smooth_compose(const float *__restrict__ du,
                                                                 const float *__restrict__ u, int mode, Taps t,
                                                                 int nx, int ny, int nz, float *__restrict__ out,
                                                                 const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    extern __shared__ float sm[];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * FQ, y0 = blockIdx.y * FQ, z0 = blockIdx.z * FQ;
    tile_xy<R>(du, t, nx, ny, nz, x0, y0, z0, sm, tid);
    const int nxy = nx * ny, N = nxy * nz;
    const float fxmax = (float)(nx - 1), fymax = (float)(ny - 1), fzmax = (float)(nz - 1);
    // both output voxels' smoothed values, then both voxels' 24 gathers in flight together
    float s[kVoxPerThread][3];
    int xv[kVoxPerThread], yv[kVoxPerThread], zv[kVoxPerThread];
    bool in_vol[kVoxPerThread];
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v) {
        const int p = tid + v * FT;
        const int ox = p % FQ, oy = (p / FQ) % FQ, oz = p / (FQ * FQ);
        xv[v] = x0 + ox; yv[v] = y0 + oy; zv[v] = z0 + oz;
        in_vol[v] = xv[v] < nx && yv[v] < ny && zv[v] < nz;
#pragma unroll
        for (int c = 0; c < 3; ++c) s[v][c] = tile_z<R>(sm, t, c, ox, oy, oz);
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
    float cc[kVoxPerThread][3][8];
    float wx[kVoxPerThread], wy[kVoxPerThread], wz[kVoxPerThread];
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
        const int b0 = iz * nxy + iy * nx + ix;
        const int o[8] = {0, ddx, ddy, ddy + ddx, ddz, ddz + ddx, ddz + ddy, ddz + ddy + ddx};
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 8; ++q) cc[v][c][q] = __ldg(u + (size_t)c * N + b0 + o[q]);
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
__global__ void __launch_bounds__(FT, 2) k_fused_smooth_warp(const float *__restrict__ in, Taps t,
                                                              float *__restrict__ u, ForceArgs a) {
    if (a.stop_flag && *a.stop_flag) return;
    extern __shared__ float sm[];
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * FQ, y0 = blockIdx.y * FQ, z0 = blockIdx.z * FQ;
    tile_xy<R>(in, t, nx, ny, nz, x0, y0, z0, sm, tid);
    const int nxy = nx * ny, N = nxy * nz;
    CornerSet<IT> cs[kVoxPerThread];
    int iv[kVoxPerThread];
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v) {
        const int p = tid + v * FT;
        const int ox = p % FQ, oy = (p / FQ) % FQ, oz = p / (FQ * FQ);
        const int x = x0 + ox, y = y0 + oy, z = z0 + oz;
        iv[v] = -1;
        if (x >= nx || y >= ny || z >= nz) continue;
        const int i = z * nxy + y * nx + x;
        iv[v] = i;
        const float sx = tile_z<R>(sm, t, 0, ox, oy, oz), sy = tile_z<R>(sm, t, 1, ox, oy, oz),
                    sz = tile_z<R>(sm, t, 2, ox, oy, oz);
        u[i] = sx;
        u[N + i] = sy;
        u[N + N + i] = sz;
        corner_load<CONTOUR, IT>(a, sx, sy, sz, x, y, z, cs[v]);
    }
#pragma unroll
    for (int v = 0; v < kVoxPerThread; ++v)
        if (iv[v] >= 0) corner_finish<CONTOUR, IT>(a, iv[v], N, cs[v]);
}

template <int R>
cudaError_t compose_r(const float *du, const float *u, int mode, const Taps &t, int nx, int ny, int nz,
                      float *out, const int *stop_flag, cudaStream_t s) {
    const size_t smem = FusedTile<R>::bytes();
    cudaError_t e = ensure_smem((const void *)k_fused_smooth_compose<R>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((nx + FQ - 1) / FQ, (ny + FQ - 1) / FQ, (nz + FQ - 1) / FQ);
    k_fused_smooth_compose<R><<<grid, FT, smem, s>>>(du, u, mode, t, nx, ny, nz, out, stop_flag);
    note_launch();
    return cudaGetLastError();
}

template <int R, bool CONTOUR, typename IT>
cudaError_t warp_rt(const float *in, const Taps &t, float *u, const ForceArgs &a, cudaStream_t s) {
    const size_t smem = FusedTile<R>::bytes();
    cudaError_t e = ensure_smem((const void *)k_fused_smooth_warp<R, CONTOUR, IT>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + FQ - 1) / FQ, (a.ny + FQ - 1) / FQ, (a.nz + FQ - 1) / FQ);
    k_fused_smooth_warp<R, CONTOUR, IT><<<grid, FT, smem, s>>>(in, t, u, a);
    note_launch();
    return cudaGetLastError();
}

template <int R>
cudaError_t warp_r(const float *in, const Taps &t, float *u, const ForceArgs &a, cudaStream_t s) {
    const bool contour = a.contour && a.k > 0;
    if (a.img_dtype == CGDIR_F16)
        return contour ? warp_rt<R, true, __half>(in, t, u, a, s) : warp_rt<R, false, __half>(in, t, u, a, s);
    if (a.img_dtype == CGDIR_BF16)
        return contour ? warp_rt<R, true, __nv_bfloat16>(in, t, u, a, s)
                       : warp_rt<R, false, __nv_bfloat16>(in, t, u, a, s);
    return contour ? warp_rt<R, true, float>(in, t, u, a, s) : warp_rt<R, false, float>(in, t, u, a, s);
}

}  // namespace

bool fused_schedule_ok(const ForceArgs &a) {
    return a.wfield != nullptr && (size_t)a.nx * a.ny * a.nz < (size_t)1 << 31;
}

cudaError_t launch_fused_smooth_compose(const float *du, const float *u, int mode, float sigma, int nx, int ny,
                                        int nz, float *out, const int *stop_flag, cudaStream_t s) {
    if ((size_t)nx * ny * nz >= (size_t)1 << 31) return cudaErrorInvalidValue;
    const Taps t = gauss_taps(sigma);
    switch (t.r) {
        case 1: return compose_r<1>(du, u, mode, t, nx, ny, nz, out, stop_flag, s);
        case 2: return compose_r<2>(du, u, mode, t, nx, ny, nz, out, stop_flag, s);
        case 3: return compose_r<3>(du, u, mode, t, nx, ny, nz, out, stop_flag, s);
        case 4: return compose_r<4>(du, u, mode, t, nx, ny, nz, out, stop_flag, s);
        case 5: return compose_r<5>(du, u, mode, t, nx, ny, nz, out, stop_flag, s);
        case 6: return compose_r<6>(du, u, mode, t, nx, ny, nz, out, stop_flag, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_smooth_warp(const float *in, float sigma, float *u, const ForceArgs &a, cudaStream_t s) {
    if (!fused_schedule_ok(a)) return cudaErrorInvalidValue;
    const Taps t = gauss_taps(sigma);
    switch (t.r) {
        case 1: return warp_r<1>(in, t, u, a, s);
        case 2: return warp_r<2>(in, t, u, a, s);
        case 3: return warp_r<3>(in, t, u, a, s);
        case 4: return warp_r<4>(in, t, u, a, s);
        case 5: return warp_r<5>(in, t, u, a, s);
        case 6: return warp_r<6>(in, t, u, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cgdir
