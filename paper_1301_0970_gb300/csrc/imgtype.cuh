// Image storage types of the pyramid: float32, float16 or bfloat16.  Every
// value is widened to float32 at load; all arithmetic is float32.
//
// Moving-image texels (image value + the moving mask bits, gathered together
// at each interpolation corner): {float value, uint32 bits} for float32
// images (8 bytes), and one 32-bit word for 16-bit images: the low half
// holds the value's bits, bits 16..23 the mask bits (4 bytes).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "cgdir.h"

namespace cgdir {

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__device__ __forceinline__ float ld_img(const T *p) { return to_f<T>(__ldg(p)); }

// 16-bit value of a half / bfloat16 as raw bits and back
template <typename T>
__device__ __forceinline__ float from_bits16(unsigned b);
template <>
__device__ __forceinline__ float from_bits16<__half>(unsigned b) { return __half2float(__ushort_as_half((unsigned short)b)); }
template <>
__device__ __forceinline__ float from_bits16<__nv_bfloat16>(unsigned b) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)b));
}

template <typename T>
struct TexOf { using type = uint32_t; };
template <>
struct TexOf<float> { using type = float2; };

template <typename T>
__device__ __forceinline__ void tex_unpack(typename TexOf<T>::type t, float &v, unsigned &bits) {
    v = from_bits16<T>(t & 0xffffu);
    bits = (t >> 16) & 0xffu;
}
template <>
__device__ __forceinline__ void tex_unpack<float>(float2 t, float &v, unsigned &bits) {
    v = t.x;
    bits = __float_as_uint(t.y);
}

inline size_t img_elem_size(int dtype) { return dtype == CGDIR_F32 ? 4 : 2; }
inline size_t tex_elem_size(int dtype) { return dtype == CGDIR_F32 ? 8 : 4; }

}  // namespace cgdir
