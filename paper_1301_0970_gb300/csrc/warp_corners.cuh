// Trilinear warp of the moving image and of the structure terms at one
// point (the first pass of the two-pass force, Algorithm A steps 5-6 of
// Sec. 2.2): the eight corners' values and mask bits are loaded, then I0~,
// the corners' bit AND / OR and, where the corners disagree on bit j, P_j
// are written to the two-pass scratch of ForceArgs.  Shared by the force
// kernels and the fused smoothing + warp kernel, so both give the same bits.
#pragma once

#include "cgdir_internal.cuh"

namespace cgdir {

// The eight corners of one interpolation point, loaded (pass 1).  Values of
// 16-bit images stay raw until corner_finish converts them: a conversion at
// the load would wait for the load there, before the other gathers of the
// thread are issued.
//   c  values (float images)
//   h  raw 16-bit values (16-bit images without texels)
//   m  words whose bits sh .. sh + 7 are the corners' moving-mask bits
//      (mask_shift): for 16-bit texels the whole texel word (value in the
//      low half, sh = 16), otherwise the bits alone (sh = 0)
template <typename IT>
struct CornerSet {
    float c[8];
    unsigned short h[8];
    unsigned m[8];
    float wx, wy, wz;
};

template <bool CONTOUR, typename IT>
__device__ __forceinline__ int mask_shift(const ForceArgs &a) {
    return (CONTOUR && sizeof(IT) == 2 && a.mtex != nullptr) ? 16 : 0;
}

// The float value of a raw 16-bit image value (the low half of w).
template <typename IT>
__device__ __forceinline__ float from_raw16(unsigned w);
template <>
__device__ __forceinline__ float from_raw16<__half>(unsigned w) { return __half2float(__ushort_as_half((unsigned short)w)); }
template <>
__device__ __forceinline__ float from_raw16<__nv_bfloat16>(unsigned w) {
    return __uint_as_float(w << 16);        // a bfloat16 is the high half of a float
}
template <>
__device__ __forceinline__ float from_raw16<float>(unsigned w) { return __uint_as_float(w); }   // not used

// Clamp x + u, find the corners and issue their loads (texels when the
// structure terms are on and texels exist, else image values and mask bits).
template <bool CONTOUR, typename IT>
__device__ __forceinline__ void corner_load(const ForceArgs &a, float ux, float uy, float uz, int x, int y, int z,
                                            CornerSet<IT> &cs) {
    using TT = typename TexOf<IT>::type;
    const int nx = a.nx, ny = a.ny, nz = a.nz, nxy = nx * ny;
    const float px = fminf(fmaxf((float)x + ux, 0.f), (float)(nx - 1));
    const float py = fminf(fmaxf((float)y + uy, 0.f), (float)(ny - 1));
    const float pz = fminf(fmaxf((float)z + uz, 0.f), (float)(nz - 1));
    const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    cs.wx = px - fx; cs.wy = py - fy; cs.wz = pz - fz;
    const int dx = ix < nx - 1 ? 1 : 0, dy = iy < ny - 1 ? nx : 0, dz = iz < nz - 1 ? nxy : 0;
    const int b0 = iz * nxy + iy * nx + ix;
    const int o[8] = {0, dx, dy, dy + dx, dz, dz + dx, dz + dy, dz + dy + dx};
    if (CONTOUR && a.mtex != nullptr) {
        const TT *__restrict__ q0 = static_cast<const TT *>(a.mtex) + b0;
        if (sizeof(IT) == 2) {
#pragma unroll
            for (int q = 0; q < 8; ++q) cs.m[q] = (unsigned)__ldg(reinterpret_cast<const uint32_t *>(q0 + o[q]));
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 t = __ldg(reinterpret_cast<const float2 *>(q0 + o[q]));
                cs.c[q] = t.x;
                cs.m[q] = __float_as_uint(t.y);
            }
        }
    } else {
        const IT *__restrict__ q0 = static_cast<const IT *>(a.I0) + b0;
        if (sizeof(IT) == 2) {
#pragma unroll
            for (int q = 0; q < 8; ++q) cs.h[q] = __ldg(reinterpret_cast<const unsigned short *>(q0 + o[q]));
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) cs.c[q] = __ldg(reinterpret_cast<const float *>(q0 + o[q]));
        }
        if (CONTOUR) {
            const uint8_t *__restrict__ r0 = a.mbits + b0;
#pragma unroll
            for (int q = 0; q < 8; ++q) cs.m[q] = __ldg(r0 + o[q]);
        }
    }
}

// Interpolate I0~ from the loaded corners, write it, the corner bits'
// AND / OR and, where they disagree, P_j.
template <bool CONTOUR, typename IT>
__device__ __forceinline__ void corner_finish(const ForceArgs &a, int i, int N, const CornerSet<IT> &cs) {
    const float wx = cs.wx, wy = cs.wy, wz = cs.wz;
    float c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        c[q] = sizeof(IT) == 4 ? cs.c[q]
                               : (CONTOUR && a.mtex != nullptr ? from_raw16<IT>(cs.m[q]) : from_raw16<IT>(cs.h[q]));
    const float e00 = fmaf(wx, c[1] - c[0], c[0]), e10 = fmaf(wx, c[3] - c[2], c[2]);
    const float e01 = fmaf(wx, c[5] - c[4], c[4]), e11 = fmaf(wx, c[7] - c[6], c[6]);
    const float f0 = fmaf(wy, e10 - e00, e00), f1 = fmaf(wy, e11 - e01, e01);
    a.wfield[i] = fmaf(wz, f1 - f0, f0);
    if (CONTOUR) {
        const unsigned *m = cs.m;
        const int sh = mask_shift<CONTOUR, IT>(a);
        // the words hold nothing above the mask bits (texel bits 24-31 are zero)
        const unsigned andb = (m[0] & m[1] & m[2] & m[3] & m[4] & m[5] & m[6] & m[7]) >> sh;
        const unsigned orb = (m[0] | m[1] | m[2] | m[3] | m[4] | m[5] | m[6] | m[7]) >> sh;
        a.wstate[i] = (uint16_t)((andb << 8) | orb);
        unsigned mixed = orb & ~andb;
        if (mixed) {
            const float off = a.offset;
            const float ax = 1.f - wx, ay = 1.f - wy, az = 1.f - wz;
            // products rounded on their own (never contracted into the sums
            // below), so every kernel that inlines this gives the same bits
            auto w3 = [](float p, float q, float r, float v) { return __fmul_rn(__fmul_rn(__fmul_rn(p, q), r), v); };
            float q[8];
            q[0] = w3(ax, ay, az, c[0] + off); q[1] = w3(wx, ay, az, c[1] + off);
            q[2] = w3(ax, wy, az, c[2] + off); q[3] = w3(wx, wy, az, c[3] + off);
            q[4] = w3(ax, ay, wz, c[4] + off); q[5] = w3(wx, ay, wz, c[5] + off);
            q[6] = w3(ax, wy, wz, c[6] + off); q[7] = w3(wx, wy, wz, c[7] + off);
            while (mixed) {
                const int j = __ffs(mixed) - 1;
                mixed &= mixed - 1u;
                float pj = 0.f;
#pragma unroll
                for (int t = 0; t < 8; ++t) pj += ((m[t] >> (sh + j)) & 1u) ? q[t] : 0.f;
                a.pfield[(size_t)j * N + i] = pj;
            }
        }
    }
}

}  // namespace cgdir
