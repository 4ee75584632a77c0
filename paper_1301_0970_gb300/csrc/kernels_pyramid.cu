// Set-up kernels of CG-DIR: mask bit-packing, the factor-2 image pyramid and
// the prolongation of the DVF between levels (multi-scale strategy,
// Sec. 2.2), the UROI map of the stopping criterion (Sec. 2.2), the sums
// behind the automatic sign of the modified images (Sec. 2.1) and image
// type conversion.  None of these run per iteration.
#include "cgdir_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace cgdir {

namespace {

unsigned flat_grid(size_t n, size_t cap = 152 * 16) {
    size_t g = (n + 255) / 256;
    if (g > cap) g = cap;
    return (unsigned)(g ? g : 1);
}

// Row launches: a CTA covers RB consecutive x of one (y, z) row, so no
// index is recovered by division (the grid-stride loops above divide a
// 64-bit index per voxel).  Volumes with ny or nz above the grid limit keep
// the grid-stride kernels.
constexpr int RB = 128;
bool rows_ok(int ny, int nz) { return ny <= 65535 && nz <= 65535; }
dim3 row_grid(int nx, int ny, int nz) { return dim3((unsigned)((nx + RB - 1) / RB), (unsigned)ny, (unsigned)nz); }

struct MaskPtrs {
    const uint8_t *p[kMaxMasks];
};

// Four voxels per thread: one 32-bit load per mask, a byte-wise nonzero test.
__global__ void k_pack4(MaskPtrs m, int k, size_t n4, uint32_t *__restrict__ bits) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        uint32_t b = 0;
#pragma unroll
        for (int j = 0; j < kMaxMasks; ++j)
            if (j < k) b |= __vcmpne4(__ldg(reinterpret_cast<const uint32_t *>(m.p[j]) + i), 0u) & (0x01010101u << j);
        bits[i] = b;
    }
}

__global__ void k_pack(MaskPtrs m, int k, size_t n, uint8_t *__restrict__ bits) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        unsigned b = 0;
#pragma unroll
        for (int j = 0; j < kMaxMasks; ++j)
            if (j < k && __ldg(m.p[j] + i)) b |= 1u << j;
        bits[i] = (uint8_t)b;
    }
}

// 2x2x2 box mean, source indices clamped (odd sizes replicate the border),
// accumulated in float32 and stored in the output level's image type.
template <typename IT, typename OT>
__global__ void k_restrict_image(const IT *__restrict__ in, int nx, int ny, int nz,
                                 OT *__restrict__ out) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    const size_t Nc = (size_t)cx * cy * cz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < Nc;
         i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % cx), Y = (int)((i / cx) % cy), Z = (int)(i / ((size_t)cx * cy));
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int x = min(2 * X + (q & 1), nx - 1), y = min(2 * Y + ((q >> 1) & 1), ny - 1),
                      z = min(2 * Z + ((q >> 2) & 1), nz - 1);
            s += ld_img<IT>(in + vox(x, y, z, nx, ny));
        }
        out[i] = from_f<OT>(s * 0.125f);
    }
}

// The same box mean per coarse row (X = thread, Y, Z = grid).
template <typename IT, typename OT>
__global__ void k_restrict_image_rows(const IT *__restrict__ in, int nx, int ny, int nz, OT *__restrict__ out) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2;
    const int X = blockIdx.x * RB + threadIdx.x, Y = blockIdx.y, Z = blockIdx.z;
    if (X >= cx) return;
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int x = min(2 * X + (q & 1), nx - 1), y = min(2 * Y + ((q >> 1) & 1), ny - 1),
                  z = min(2 * Z + ((q >> 2) & 1), nz - 1);
        s += ld_img<IT>(in + vox(x, y, z, nx, ny));
    }
    out[vox(X, Y, Z, cx, cy)] = from_f<OT>(s * 0.125f);
}

// Per bit: inside if at least 4 of the 8 source voxels are inside.
__global__ void k_restrict_bits(const uint8_t *__restrict__ in, int nx, int ny, int nz,
                                uint8_t *__restrict__ out) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    const size_t Nc = (size_t)cx * cy * cz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < Nc;
         i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % cx), Y = (int)((i / cx) % cy), Z = (int)(i / ((size_t)cx * cy));
        int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int x = min(2 * X + (q & 1), nx - 1), y = min(2 * Y + ((q >> 1) & 1), ny - 1),
                      z = min(2 * Z + ((q >> 2) & 1), nz - 1);
            const unsigned b = __ldg(in + vox(x, y, z, nx, ny));
#pragma unroll
            for (int j = 0; j < 8; ++j) cnt[j] += (b >> j) & 1u;
        }
        unsigned o = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) o |= (cnt[j] >= 4 ? 1u : 0u) << j;
        out[i] = (uint8_t)o;
    }
}

// u_f(x) = 2 u_c((x + 0.5)/2 - 0.5), trilinear with clamped coordinates.
__global__ void k_restrict_bits_rows(const uint8_t *__restrict__ in, int nx, int ny, int nz,
                                     uint8_t *__restrict__ out) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2;
    const int X = blockIdx.x * RB + threadIdx.x, Y = blockIdx.y, Z = blockIdx.z;
    if (X >= cx) return;
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int x = min(2 * X + (q & 1), nx - 1), y = min(2 * Y + ((q >> 1) & 1), ny - 1),
                  z = min(2 * Z + ((q >> 2) & 1), nz - 1);
        const unsigned b = __ldg(in + vox(x, y, z, nx, ny));
#pragma unroll
        for (int j = 0; j < 8; ++j) cnt[j] += (b >> j) & 1u;
    }
    unsigned o = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) o |= (cnt[j] >= 4 ? 1u : 0u) << j;
    out[vox(X, Y, Z, cx, cy)] = (uint8_t)o;
}

// Prolongation over 64 x 8 x 8 fine tiles: the coarse values the tile's
// interpolations read (34 x 6 x 6 per component, indices clamped) are staged
// in shared memory once, then each thread forms two x-adjacent fine voxels per
// row and plane with the same corners and the same order of multiply-adds as
// k_prolong (same bits), and stores them as a pair.  Replaces 24 cached
// gathers per fine voxel by shared-memory reads.
constexpr int PX = 64, PY = 8, PZ = 8;
constexpr int PCX = PX / 2 + 2, PCY = PY / 2 + 2, PCZ = PZ / 2 + 2;
__global__ void __launch_bounds__(256) k_prolong_tile(const float *__restrict__ uc, int cx, int cy, int cz, int nx,
                                                      int ny, int nz, float *__restrict__ uf) {
    __shared__ float t[3][PCZ][PCY][PCX];
    const int x0 = blockIdx.x * PX, y0 = blockIdx.y * PY, z0 = blockIdx.z * PZ;
    const int bx = x0 / 2 - 1, by = y0 / 2 - 1, bz = z0 / 2 - 1;      // coarse origin of the tile
    const size_t Nc = (size_t)cx * cy * cz, N = (size_t)nx * ny * nz;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int e = tid; e < 3 * PCZ * PCY * PCX; e += blockDim.x * blockDim.y) {
        const int i = e % PCX, j = (e / PCX) % PCY, k = (e / (PCX * PCY)) % PCZ, comp = e / (PCX * PCY * PCZ);
        const int gx = clampi(bx + i, 0, cx - 1), gy = clampi(by + j, 0, cy - 1), gz = clampi(bz + k, 0, cz - 1);
        t[comp][k][j][i] = __ldg(uc + comp * Nc + ((size_t)gz * cy + gy) * cx + gx);
    }
    __syncthreads();
    const int y = y0 + threadIdx.y, xa = x0 + 2 * threadIdx.x;
    if (y >= ny || xa >= nx) return;
    const bool two = xa + 1 < nx;
    for (int dz = 0; dz < PZ; ++dz) {
        const int z = z0 + dz;
        if (z >= nz) break;
        float out[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = xa + h;
            const Corners c = corners((x + 0.5f) * 0.5f - 0.5f, (y + 0.5f) * 0.5f - 0.5f, (z + 0.5f) * 0.5f - 0.5f,
                                      cx, cy, cz);
            float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int qx = (q & 1) ? c.x1 : c.x0, qy = (q & 2) ? c.y1 : c.y0, qz = (q & 4) ? c.z1 : c.z0;
                const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                                ((q & 4) ? c.wz : 1.f - c.wz);
#pragma unroll
                for (int comp = 0; comp < 3; ++comp)
                    acc[comp] = fmaf(w, t[comp][qz - bz][qy - by][qx - bx], acc[comp]);
            }
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) out[h][comp] = 2.f * acc[comp];
        }
        const size_t i = vox(xa, y, z, nx, ny);
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            float *o = uf + comp * N + i;
            if (two && (reinterpret_cast<uintptr_t>(o) & 7u) == 0) {
                *reinterpret_cast<float2 *>(o) = make_float2(out[0][comp], out[1][comp]);
            } else {
                o[0] = out[0][comp];
                if (two) o[1] = out[1][comp];
            }
        }
    }
}

__global__ void k_prolong(const float *__restrict__ uc, int cx, int cy, int cz, int nx, int ny,
                          int nz, float *__restrict__ uf) {
    const size_t N = (size_t)nx * ny * nz, Nc = (size_t)cx * cy * cz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const Corners c = corners((x + 0.5f) * 0.5f - 0.5f, (y + 0.5f) * 0.5f - 0.5f,
                                  (z + 0.5f) * 0.5f - 0.5f, cx, cy, cz);
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            const float *f = uc + comp * Nc;
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int qx = (q & 1) ? c.x1 : c.x0, qy = (q & 2) ? c.y1 : c.y0, qz = (q & 4) ? c.z1 : c.z0;
                const float w = ((q & 1) ? c.wx : 1.f - c.wx) * ((q & 2) ? c.wy : 1.f - c.wy) *
                                ((q & 4) ? c.wz : 1.f - c.wz);
                acc = fmaf(w, __ldg(f + vox(qx, qy, qz, cx, cy)), acc);
            }
            uf[comp * N + i] = 2.f * acc;
        }
    }
}

// ---- UROI: exact ellipsoidal dilation in three passes -----------------
// pass 1: per voxel, the distance |dx| (voxels) to the nearest union voxel of
// its x-row within rx, 255 if none.  pass 2: per voxel (x, y, z') and per
// z offset dz, bit dz+rz says that some row (y+dy, z') holds a union voxel
// within the x extent the ellipsoid allows at (dy, dz).  pass 3: voxel
// (x, y, z) is in the UROI if bit dz+rz of pass 2 at (x, y, z+dz) is set for
// some dz.  The extents are computed on the host with the same double
// expression as the definition, so the decision equals the brute-force test
// voxel by voxel.
constexpr int kMaxUroiRadius = 15;
struct UroiTable {
    int rx, ry, rz;
    int8_t ext[2 * kMaxUroiRadius + 1][2 * kMaxUroiRadius + 1];   // [dz][dy], -1 = none
};

__global__ void k_uroi_rows(const uint8_t *__restrict__ sbits, unsigned mask, int rx, int nx,
                            int ny, int nz, uint8_t *__restrict__ rowdist) {
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        int d = 255;
        for (int dx = -rx; dx <= rx; ++dx) {
            const int xx = x + dx;
            if (xx < 0 || xx >= nx) continue;
            if (__ldg(sbits + i - x + xx) & mask) d = min(d, abs(dx));
        }
        rowdist[i] = (uint8_t)d;
    }
}

__global__ void k_uroi_planes(const uint8_t *__restrict__ rowdist, UroiTable t, int nx, int ny, int nz,
                              uint32_t *__restrict__ zbits) {
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)((i / nx) % ny);
        uint32_t b = 0;
        for (int dy = -t.ry; dy <= t.ry; ++dy) {
            const int yy = y + dy;
            if (yy < 0 || yy >= ny) continue;
            const int r = __ldg(rowdist + i + (ptrdiff_t)dy * nx);
            if (r == 255) continue;
            for (int dz = -t.rz; dz <= t.rz; ++dz)
                if (r <= t.ext[dz + t.rz][dy + t.ry]) b |= 1u << (dz + t.rz);
        }
        zbits[i] = b;
    }
}

__global__ void k_uroi_dilate(const uint32_t *__restrict__ zbits, int rz, int nx, int ny, int nz,
                              uint8_t *__restrict__ out) {
    const size_t N = (size_t)nx * ny * nz, nxy = (size_t)nx * ny;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i / nxy);
        uint32_t hit = 0;
        for (int dz = -rz; dz <= rz; ++dz) {
            const int zz = z + dz;
            if (zz < 0 || zz >= nz) continue;
            hit |= ((uint32_t)__ldg(zbits + i + (ptrdiff_t)dz * (ptrdiff_t)nxy) >> (dz + rz)) & 1u;
        }
        out[i] = (uint8_t)hit;
    }
}

// Row versions of the three UROI passes.  Pass 1 stages the row's mask bits
// (with an rx halo) in shared memory; pass 2 takes, per y offset, the z
// offsets whose extent admits the row distance r from a table built on the
// host (bit dz + rz of zsets[dy + ry][r] set iff r <= ext[dz][dy]), the same
// decisions as the loop over dz.
struct UroiZsets {
    uint32_t zs[2 * kMaxUroiRadius + 1][kMaxUroiRadius + 1];
};

__global__ void k_uroi_rows_r(const uint8_t *__restrict__ sbits, unsigned mask, int rx, int nx, int ny, int nz,
                              uint8_t *__restrict__ rowdist) {
    __shared__ uint8_t row[RB + 2 * kMaxUroiRadius];
    const int x0 = blockIdx.x * RB, y = blockIdx.y, z = blockIdx.z;
    const size_t rb = vox(0, y, z, nx, ny);
    for (int p = threadIdx.x; p < RB + 2 * rx; p += RB) {
        const int xx = x0 - rx + p;
        row[p] = (xx >= 0 && xx < nx && (__ldg(sbits + rb + xx) & mask)) ? 1 : 0;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= nx) return;
    int d = 255;
    for (int dx = -rx; dx <= rx; ++dx)
        if (row[threadIdx.x + rx + dx]) d = min(d, abs(dx));
    rowdist[rb + x] = (uint8_t)d;
}

// W: the z-mask word, 16 bits where 2 rz + 1 <= 16 (half the bytes written
// here and read by the z pass), else 32.
template <typename W>
__global__ void k_uroi_planes_r(const uint8_t *__restrict__ rowdist, const __grid_constant__ UroiZsets t, int ry,
                                int nx, int ny, int nz, W *__restrict__ zbits) {
    const int x = blockIdx.x * RB + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const size_t i = vox(x, y, z, nx, ny);
    uint32_t b = 0;
    for (int dy = -ry; dy <= ry; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= ny) continue;
        const int r = __ldg(rowdist + i + (ptrdiff_t)dy * nx);
        if (r != 255) b |= t.zs[dy + ry][r];
    }
    zbits[i] = (W)b;
}

// Pass 3 marching z: a thread owns an x position of a row and takes kUroiZc
// consecutive planes, so each z-mask word it reads for one plane is read
// again, from L1, for the next 2 rz planes.
constexpr int kUroiZc = 16;
template <typename W>
__global__ void k_uroi_dilate_r(const W *__restrict__ zbits, int rz, int nx, int ny, int nz,
                                uint8_t *__restrict__ out) {
    const int x = blockIdx.x * RB + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int zb = blockIdx.z * kUroiZc, ze = min(zb + kUroiZc, nz);
    const size_t nxy = (size_t)nx * ny;
    for (int z = zb; z < ze; ++z) {
        const size_t i = vox(x, y, z, nx, ny);
        uint32_t hit = 0;
        for (int dz = -rz; dz <= rz; ++dz) {
            const int zz = z + dz;
            if (zz < 0 || zz >= nz) continue;
            hit |= (__ldg(zbits + i + (ptrdiff_t)dz * (ptrdiff_t)nxy) >> (dz + rz)) & 1u;
        }
        out[i] = (uint8_t)hit;
    }
}

__global__ void k_fill_u8(uint8_t *p, size_t n, uint8_t v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---- automatic sign ---------------------------------------------------
// Chebyshev dilation by 2 voxels of all mask bits, one axis per launch.
__global__ void k_dilate_axis(const uint8_t *__restrict__ in, int axis, int nx, int ny, int nz,
                              uint8_t *__restrict__ out) {
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        unsigned b = 0;
        for (int d = -2; d <= 2; ++d) {
            int xx = x, yy = y, zz = z;
            if (axis == 0) xx += d; else if (axis == 1) yy += d; else zz += d;
            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
            b |= __ldg(in + vox(xx, yy, zz, nx, ny));
        }
        out[i] = (uint8_t)b;
    }
}

constexpr int ST = 256;
// Per block: {sum T0 inside j, count inside, sum T0 in shell, count shell}.
template <typename IT>
__global__ void __launch_bounds__(ST) k_sign_partial(const IT *__restrict__ T0,
                                                     const uint8_t *__restrict__ sbits,
                                                     const uint8_t *__restrict__ dil, int j,
                                                     size_t n, double *__restrict__ partial) {
    double a = 0, b = 0, c = 0, d = 0;
    for (size_t i = (size_t)blockIdx.x * ST + threadIdx.x; i < n; i += (size_t)gridDim.x * ST) {
        const bool in = (__ldg(sbits + i) >> j) & 1u;
        const bool sh = !in && ((__ldg(dil + i) >> j) & 1u);
        const double t = (double)ld_img<IT>(T0 + i);
        if (in) { a += t; b += 1.0; }
        if (sh) { c += t; d += 1.0; }
    }
    __shared__ double r[4][ST];
    r[0][threadIdx.x] = a; r[1][threadIdx.x] = b; r[2][threadIdx.x] = c; r[3][threadIdx.x] = d;
    __syncthreads();
    for (int h = ST / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int q = 0; q < 4; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[(size_t)blockIdx.x * 4 + threadIdx.x] = r[threadIdx.x][0];
}

__global__ void k_sum_rows4(const double *__restrict__ partial, int rows, double *__restrict__ out) {
    if (threadIdx.x < 4) {
        double s = 0;
        for (int b = 0; b < rows; ++b) s += partial[(size_t)b * 4 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

__global__ void k_make_texels_f32(const float *__restrict__ I0, const uint8_t *__restrict__ bits, size_t n,
                                  float2 *__restrict__ tex) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        tex[i] = make_float2(__ldg(I0 + i), __uint_as_float((unsigned)__ldg(bits + i)));
}

// 16-bit images: low half = the value's bits, bits 16..23 = the mask bits.
__global__ void k_make_texels_16(const unsigned short *__restrict__ I0, const uint8_t *__restrict__ bits,
                                 size_t n, uint32_t *__restrict__ tex) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        tex[i] = (uint32_t)__ldg(I0 + i) | ((uint32_t)__ldg(bits + i) << 16);
}

template <typename IN, typename OUT>
__global__ void k_convert(const IN *__restrict__ in, size_t n, OUT *__restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = from_f<OUT>(to_f<IN>(in[i]));
}

}  // namespace

cudaError_t launch_pack_masks(const uint8_t *const *masks, int k, size_t n, uint8_t *bits,
                              cudaStream_t s) {
    MaskPtrs m{};
    bool aligned = n % 4 == 0 && reinterpret_cast<uintptr_t>(bits) % 4 == 0;
    for (int j = 0; j < k && j < kMaxMasks; ++j) {
        m.p[j] = masks[j];
        aligned = aligned && reinterpret_cast<uintptr_t>(masks[j]) % 4 == 0;
    }
    if (aligned)
        k_pack4<<<flat_grid(n / 4), 256, 0, s>>>(m, k, n / 4, reinterpret_cast<uint32_t *>(bits));
    else
        k_pack<<<flat_grid(n), 256, 0, s>>>(m, k, n, bits);
    note_launch();
    return cudaGetLastError();
}

template <typename IT>
static void restrict_image_to(const void *in, int nx, int ny, int nz, void *out, int out_dtype, size_t Nc,
                              cudaStream_t s) {
    const IT *src = static_cast<const IT *>(in);
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    if (rows_ok(cy, cz)) {
        const dim3 g = row_grid(cx, cy, cz);
        if (out_dtype == CGDIR_F16)
            k_restrict_image_rows<IT, __half><<<g, RB, 0, s>>>(src, nx, ny, nz, (__half *)out);
        else if (out_dtype == CGDIR_BF16)
            k_restrict_image_rows<IT, __nv_bfloat16><<<g, RB, 0, s>>>(src, nx, ny, nz, (__nv_bfloat16 *)out);
        else
            k_restrict_image_rows<IT, float><<<g, RB, 0, s>>>(src, nx, ny, nz, (float *)out);
        return;
    }
    if (out_dtype == CGDIR_F16)
        k_restrict_image<IT, __half><<<flat_grid(Nc), 256, 0, s>>>(src, nx, ny, nz, (__half *)out);
    else if (out_dtype == CGDIR_BF16)
        k_restrict_image<IT, __nv_bfloat16><<<flat_grid(Nc), 256, 0, s>>>(src, nx, ny, nz, (__nv_bfloat16 *)out);
    else
        k_restrict_image<IT, float><<<flat_grid(Nc), 256, 0, s>>>(src, nx, ny, nz, (float *)out);
}

cudaError_t launch_restrict_image(const void *in, int in_dtype, int nx, int ny, int nz, void *out, int out_dtype,
                                  cudaStream_t s) {
    const size_t Nc = (size_t)((nx + 1) / 2) * ((ny + 1) / 2) * ((nz + 1) / 2);
    if (in_dtype == CGDIR_F16)
        restrict_image_to<__half>(in, nx, ny, nz, out, out_dtype, Nc, s);
    else if (in_dtype == CGDIR_BF16)
        restrict_image_to<__nv_bfloat16>(in, nx, ny, nz, out, out_dtype, Nc, s);
    else
        restrict_image_to<float>(in, nx, ny, nz, out, out_dtype, Nc, s);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_restrict_image(const void *in, int dtype, int nx, int ny, int nz, void *out,
                                  cudaStream_t s) {
    return launch_restrict_image(in, dtype, nx, ny, nz, out, dtype, s);
}

cudaError_t launch_restrict_bits(const uint8_t *in, int nx, int ny, int nz, uint8_t *out,
                                 cudaStream_t s) {
    const size_t Nc = (size_t)((nx + 1) / 2) * ((ny + 1) / 2) * ((nz + 1) / 2);
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    if (rows_ok(cy, cz))
        k_restrict_bits_rows<<<row_grid(cx, cy, cz), RB, 0, s>>>(in, nx, ny, nz, out);
    else
        k_restrict_bits<<<flat_grid(Nc), 256, 0, s>>>(in, nx, ny, nz, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prolong(const float *uc, int cx, int cy, int cz, int nx, int ny, int nz,
                           float *uf, cudaStream_t s) {
    if (rows_ok(ny, nz))
        k_prolong_tile<<<dim3((nx + PX - 1) / PX, (ny + PY - 1) / PY, (nz + PZ - 1) / PZ), dim3(32, 8), 0, s>>>(
            uc, cx, cy, cz, nx, ny, nz, uf);
    else
        k_prolong<<<flat_grid((size_t)nx * ny * nz), 256, 0, s>>>(uc, cx, cy, cz, nx, ny, nz, uf);
    note_launch();
    return cudaGetLastError();
}

// scratch: 5 N bytes (row distances, then per-voxel z masks at offset N
// rounded up to 4 bytes).
cudaError_t launch_uroi(const uint8_t *sbits, int k, int nx, int ny, int nz, const double *spacing,
                        double margin, uint8_t *scratch, uint8_t *out, cudaStream_t s) {
    const size_t N = (size_t)nx * ny * nz;
    if (k <= 0) {
        k_fill_u8<<<flat_grid(N), 256, 0, s>>>(out, N, 1); note_launch();
        return cudaGetLastError();
    }
    if (!(margin >= 0.0) || !(spacing[0] > 0) || !(spacing[1] > 0) || !(spacing[2] > 0))
        return cudaErrorInvalidValue;
    UroiTable t{};
    t.rx = (int)(margin / spacing[0]);
    t.ry = (int)(margin / spacing[1]);
    t.rz = (int)(margin / spacing[2]);
    if (t.rx > kMaxUroiRadius || t.ry > kMaxUroiRadius || t.rz > kMaxUroiRadius)
        return cudaErrorInvalidValue;
    for (int dz = -t.rz; dz <= t.rz; ++dz)
        for (int dy = -t.ry; dy <= t.ry; ++dy) {
            int e = -1;
            for (int dx = 0; dx <= t.rx; ++dx) {
                const double d2 = (dx * spacing[0]) * (dx * spacing[0]) + (dy * spacing[1]) * (dy * spacing[1]) +
                                  (dz * spacing[2]) * (dz * spacing[2]);
                if (d2 <= margin * margin) e = dx;
            }
            t.ext[dz + t.rz][dy + t.ry] = (int8_t)e;
        }
    const unsigned mask = (k >= 8) ? 0xffu : ((1u << k) - 1u);
    uint8_t *rowdist = scratch;
    uint32_t *zbits = reinterpret_cast<uint32_t *>(scratch + (N + 3) / 4 * 4);
    if (rows_ok(ny, nz)) {
        UroiZsets zt{};
        for (int dy = -t.ry; dy <= t.ry; ++dy)
            for (int r = 0; r <= t.rx; ++r) {
                uint32_t b = 0;
                for (int dz = -t.rz; dz <= t.rz; ++dz)
                    if (r <= t.ext[dz + t.rz][dy + t.ry]) b |= 1u << (dz + t.rz);
                zt.zs[dy + t.ry][r] = b;
            }
        const dim3 g = row_grid(nx, ny, nz);
        k_uroi_rows_r<<<g, RB, 0, s>>>(sbits, mask, t.rx, nx, ny, nz, rowdist); note_launch();
        const dim3 gz(g.x, g.y, (unsigned)((nz + kUroiZc - 1) / kUroiZc));
        if (2 * t.rz + 1 <= 16) {
            uint16_t *z16 = reinterpret_cast<uint16_t *>(zbits);
            k_uroi_planes_r<uint16_t><<<g, RB, 0, s>>>(rowdist, zt, t.ry, nx, ny, nz, z16); note_launch();
            k_uroi_dilate_r<uint16_t><<<gz, RB, 0, s>>>(z16, t.rz, nx, ny, nz, out); note_launch();
        } else {
            k_uroi_planes_r<uint32_t><<<g, RB, 0, s>>>(rowdist, zt, t.ry, nx, ny, nz, zbits); note_launch();
            k_uroi_dilate_r<uint32_t><<<gz, RB, 0, s>>>(zbits, t.rz, nx, ny, nz, out); note_launch();
        }
        return cudaGetLastError();
    }
    k_uroi_rows<<<flat_grid(N), 256, 0, s>>>(sbits, mask, t.rx, nx, ny, nz, rowdist); note_launch();
    k_uroi_planes<<<flat_grid(N), 256, 0, s>>>(rowdist, t, nx, ny, nz, zbits); note_launch();
    k_uroi_dilate<<<flat_grid(N), 256, 0, s>>>(zbits, t.rz, nx, ny, nz, out); note_launch();
    return cudaGetLastError();
}

size_t uroi_scratch_bytes(size_t n) { return (n + 3) / 4 * 4 + 4 * n; }

// sums: device [k][4]; tmp_a, tmp_b: N bytes each; partial: sign_partial_rows(N) x 4 doubles.
cudaError_t launch_sign_sums(const void *T0, int dtype, const uint8_t *sbits, int k, int nx, int ny,
                                int nz, uint8_t *tmp_a, uint8_t *tmp_b, double *partial,
                                double *sums, cudaStream_t s) {
    const size_t N = (size_t)nx * ny * nz;
    const unsigned g = flat_grid(N);
    k_dilate_axis<<<g, 256, 0, s>>>(sbits, 0, nx, ny, nz, tmp_a);
    k_dilate_axis<<<g, 256, 0, s>>>(tmp_a, 1, nx, ny, nz, tmp_b);
    k_dilate_axis<<<g, 256, 0, s>>>(tmp_b, 2, nx, ny, nz, tmp_a);
    note_launch(3);
    const unsigned gp = flat_grid(N, 152 * 4);
    for (int j = 0; j < k; ++j) {
        if (dtype == CGDIR_F16)
            k_sign_partial<__half><<<gp, ST, 0, s>>>((const __half *)T0, sbits, tmp_a, j, N, partial);
        else if (dtype == CGDIR_BF16)
            k_sign_partial<__nv_bfloat16><<<gp, ST, 0, s>>>((const __nv_bfloat16 *)T0, sbits, tmp_a, j, N, partial);
        else
            k_sign_partial<float><<<gp, ST, 0, s>>>((const float *)T0, sbits, tmp_a, j, N, partial);
        note_launch();
        k_sum_rows4<<<1, 32, 0, s>>>(partial, (int)gp, sums + 4 * j); note_launch();
    }
    return cudaGetLastError();
}

size_t sign_partial_rows(size_t n) { return flat_grid(n, 152 * 4); }

cudaError_t launch_make_texels(const void *I0, int dtype, const uint8_t *bits, size_t n, void *tex,
                               cudaStream_t s) {
    if (dtype == CGDIR_F32)
        k_make_texels_f32<<<flat_grid(n), 256, 0, s>>>((const float *)I0, bits, n, (float2 *)tex);
    else
        k_make_texels_16<<<flat_grid(n), 256, 0, s>>>((const unsigned short *)I0, bits, n, (uint32_t *)tex);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_convert_image(const void *in, int in_dtype, size_t n, void *out, int out_dtype,
                                 cudaStream_t s) {
    if (in_dtype == out_dtype)
        return cudaMemcpyAsync(out, in, n * img_elem_size(in_dtype), cudaMemcpyDeviceToDevice, s);
    const unsigned g = flat_grid(n);
#define CGDIR_CONV(IN, OUT) k_convert<IN, OUT><<<g, 256, 0, s>>>((const IN *)in, n, (OUT *)out)
    if (in_dtype == CGDIR_F32 && out_dtype == CGDIR_F16) CGDIR_CONV(float, __half);
    else if (in_dtype == CGDIR_F32 && out_dtype == CGDIR_BF16) CGDIR_CONV(float, __nv_bfloat16);
    else if (in_dtype == CGDIR_F16 && out_dtype == CGDIR_F32) CGDIR_CONV(__half, float);
    else if (in_dtype == CGDIR_BF16 && out_dtype == CGDIR_F32) CGDIR_CONV(__nv_bfloat16, float);
    else if (in_dtype == CGDIR_F16 && out_dtype == CGDIR_BF16) CGDIR_CONV(__half, __nv_bfloat16);
    else if (in_dtype == CGDIR_BF16 && out_dtype == CGDIR_F16) CGDIR_CONV(__nv_bfloat16, __half);
    else return cudaErrorInvalidValue;
#undef CGDIR_CONV
    note_launch();
    return cudaGetLastError();
}

}  // namespace cgdir
