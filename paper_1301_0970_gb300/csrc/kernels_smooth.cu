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
constexpr int kStages = 4;

// Box of one plane: x from x0 - ML (ML = R rounded up to 4, so the start is a
// 16-byte multiple) over TX + 2 ML columns, y from y0 - R over TY + 2R rows.
// Each stage starts on a 128-byte boundary.
template <int R>
struct SmoothSmem {
    static constexpr int ML = (R + 3) / 4 * 4;
    static constexpr int BXW = TX + 2 * ML;
    static constexpr int BY = TY + 2 * R;
    static constexpr int STAGE = (3 * BY * BXW + 31) / 32 * 32;   // floats per stage (3 components)
    static constexpr size_t bytes() {
        return sizeof(float) * (kStages * STAGE + 2 * 3 * BY * TX) + kStages * sizeof(uint64_t) + 128;
    }
};

template <int R>
__global__ void __launch_bounds__(NT) k_smooth_tma(const __grid_constant__ CUtensorMap tin,
                                                   float *__restrict__ out, int ncomp, Taps taps,
                                                   int nx, int ny, int nz, int zchunk,
                                                   const int *stop_flag, int *err) {
    if (stop_flag && *stop_flag) return;
    constexpr int BY = SmoothSmem<R>::BY, STAGE = SmoothSmem<R>::STAGE, K = 2 * R + 1;
    constexpr int ML = SmoothSmem<R>::ML, BXW = SmoothSmem<R>::BXW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stage = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *Xb = stage + kStages * STAGE;                       // [2][3][BY][TX]
    uint64_t *bar = reinterpret_cast<uint64_t *>(Xb + 2 * 3 * BY * TX);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const size_t N = (size_t)nx * ny * nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    const int P = (ze - zb) + 2 * R;                           // input planes
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    const bool xin = (x0 - R >= 0) && (x0 + TX + R <= nx);
    const uint32_t tx_bytes = (uint32_t)(ncomp * BY * BXW * sizeof(float));

    float w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = taps.w[j];
    float ring[3][K];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < K; ++j) ring[c][j] = 0.f;

    auto issue = [&](int q) {
        const int s = q % kStages;
        const int z = clampi(zb - R + q, 0, nz - 1);
        mbar_expect_tx(&bar[s], tx_bytes);
        tma_load_4d(stage + s * STAGE, &tin, x0 - ML, y0 - R, z, 0, &bar[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int q = 0; q < kStages && q < P; ++q) issue(q);

    int t = 0;
    for (; t < P; ++t) {
        const int s = t % kStages;
        const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((t / kStages) & 1));
        const float *S = stage + s * STAGE;
        float *X = Xb + (t & 1) * 3 * BY * TX;
        // x pass over every (clamped) row of the box
        for (int p = tid; p < BY * TX; p += NT) {
            const int hy = p / TX, xx = p % TX;
            const int ly = clampi(y0 - R + hy, 0, ny - 1) - (y0 - R);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (c >= ncomp) break;
                const float *row = S + (c * BY + ly) * BXW;
                float acc = 0.f;
                if (xin) {
#pragma unroll
                    for (int j = 0; j < K; ++j) acc = fmaf(w[j], row[xx + j + ML - R], acc);
                } else {
#pragma unroll
                    for (int j = 0; j < K; ++j)
                        acc = fmaf(w[j], row[clampi(x0 + xx + j - R, 0, nx - 1) - x0 + ML], acc);
                }
                X[(c * BY + hy) * TX + xx] = acc;
            }
        }
        if (__syncthreads_or(!ok)) break;
        if (tid == 0 && t + kStages < P) {
            fence_proxy_async();
            issue(t + kStages);
        }
        // y pass, z ring, output
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c >= ncomp) break;
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) acc = fmaf(w[j], X[(c * BY + ty + j) * TX + tx], acc);
#pragma unroll
            for (int j = 0; j < K - 1; ++j) ring[c][j] = ring[c][j + 1];
            ring[c][K - 1] = acc;
            if (t >= 2 * R && act) {
                float o = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) o = fmaf(w[j], ring[c][j], o);
                out[c * N + vox(x, y, zb + t - 2 * R, nx, ny)] = o;
            }
        }
    }
    if (t < P) {
        // a wait ran out: record it, drain the loads still in flight (bounded), leave
        if (tid == 0) {
            atomicExch(err, 1);
            for (int q = t; q < P && q < t + kStages; ++q)
                mbar_wait_bounded(&bar[q % kStages], (uint32_t)((q / kStages) & 1));
        }
        __syncthreads();
    }
}

__global__ void k_copy(const float *__restrict__ in, float *__restrict__ out, size_t n,
                       const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

// u_new(x) = du(x) + u(x + du(x)) (trilinear, clamped), or u + du.
__global__ void k_compose(const float *__restrict__ u, const float *__restrict__ du, int mode,
                          int nx, int ny, int nz, float *__restrict__ out, const int *stop_flag) {
    if (stop_flag && *stop_flag) return;
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const float dx = __ldg(du + i), dy = __ldg(du + N + i), dz = __ldg(du + 2 * N + i);
        if (mode == CGDIR_ADDITIVE) {
            out[i] = __ldg(u + i) + dx;
            out[N + i] = __ldg(u + N + i) + dy;
            out[2 * N + i] = __ldg(u + 2 * N + i) + dz;
            continue;
        }
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const Corners c = corners((float)x + dx, (float)y + dy, (float)z + dz, nx, ny, nz);
        float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int cx = (q & 1) ? c.x1 : c.x0, cy = (q & 2) ? c.y1 : c.y0, cz = (q & 4) ? c.z1 : c.z0;
            const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                            ((q & 4) ? c.wz : 1.f - c.wz);
            const size_t ci = vox(cx, cy, cz, nx, ny);
            ax = fmaf(w, __ldg(u + ci), ax);
            ay = fmaf(w, __ldg(u + N + ci), ay);
            az = fmaf(w, __ldg(u + 2 * N + ci), az);
        }
        out[i] = dx + ax;
        out[N + i] = dy + ay;
        out[2 * N + i] = dz + az;
    }
}

int smooth_zchunk(int nx, int ny, int nz) {
    const long tiles = (long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
    const long target = 152L * 8;
    long chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int zc = (int)((nz + chunks - 1) / chunks);
    if (zc < 8) zc = 8;
    return zc > nz ? nz : zc;
}

unsigned flat_grid(size_t n) {
    size_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g ? g : 1);
}

}  // namespace

template <int R>
static cudaError_t smooth_tma_r(const CUtensorMap &m, float *out, int ncomp, const Taps &t, int nx,
                                int ny, int nz, int zc, const int *stop_flag, int *err, dim3 grid,
                                dim3 block, cudaStream_t s) {
    const size_t smem = SmoothSmem<R>::bytes();
    cudaError_t e = ensure_smem((const void *)k_smooth_tma<R>, smem);
    if (e != cudaSuccess) return e;
    k_smooth_tma<R><<<grid, block, smem, s>>>(m, out, ncomp, t, nx, ny, nz, zc, stop_flag, err);
    return cudaGetLastError();
}

cudaError_t launch_smooth(const float *in, int ncomp, float sigma, int nx, int ny, int nz,
                          float *out, const int *stop_flag, cudaStream_t s, int *err) {
    const Taps t = gauss_taps(sigma);
    const size_t N = (size_t)nx * ny * nz;
    if (t.r == 0) {
        k_copy<<<flat_grid(N * ncomp), 256, 0, s>>>(in, out, N * ncomp, stop_flag);
        note_launch();
        return cudaGetLastError();
    }
    const int zc = smooth_zchunk(nx, ny, nz);
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + zc - 1) / zc), block(TX, TY);
    if (err != nullptr) {
        CUtensorMap m;
        const uint64_t dims[4] = {(uint64_t)nx, (uint64_t)ny, (uint64_t)nz, (uint64_t)ncomp};
        const uint32_t ml = (uint32_t)((t.r + 3) / 4 * 4);
        const uint32_t box[4] = {(uint32_t)TX + 2 * ml, (uint32_t)(TY + 2 * t.r), 1u, (uint32_t)ncomp};
        if (encode_tensor_map(&m, in, 4, dims, box, 4)) {
            cudaError_t e;
            switch (t.r) {
                case 1: e = smooth_tma_r<1>(m, out, ncomp, t, nx, ny, nz, zc, stop_flag, err, grid, block, s); break;
                case 2: e = smooth_tma_r<2>(m, out, ncomp, t, nx, ny, nz, zc, stop_flag, err, grid, block, s); break;
                case 3: e = smooth_tma_r<3>(m, out, ncomp, t, nx, ny, nz, zc, stop_flag, err, grid, block, s); break;
                case 4: e = smooth_tma_r<4>(m, out, ncomp, t, nx, ny, nz, zc, stop_flag, err, grid, block, s); break;
                case 5: e = smooth_tma_r<5>(m, out, ncomp, t, nx, ny, nz, zc, stop_flag, err, grid, block, s); break;
                case 6: e = smooth_tma_r<6>(m, out, ncomp, t, nx, ny, nz, zc, stop_flag, err, grid, block, s); break;
                default: return cudaErrorInvalidValue;
            }
            note_launch();
            return e;
        }
    }
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

cudaError_t launch_compose(const float *u, const float *du, int mode, int nx, int ny, int nz,
                           float *out, const int *stop_flag, cudaStream_t s) {
    const size_t N = (size_t)nx * ny * nz;
    k_compose<<<flat_grid(N), 256, 0, s>>>(u, du, mode, nx, ny, nz, out, stop_flag);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cgdir
