// Quad elements: four taps of a bilinear cell stored together, so that one
// aligned load fetches them.  F32 quads are float4 (16 B); BF16 / F16 quads
// are four 16-bit values in a uint2 (8 B).  The forward projector stores the
// four taps (f, f+1) x (m, m+1) of a volume plane; the backprojector the taps
// (c, c+1) x (r, r+1) of a detector image.
#pragma once

#include "common.cuh"

namespace tigre {

template <typename T> struct QuadOf;
template <> struct QuadOf<float> { using type = float4; };
template <> struct QuadOf<__nv_bfloat16> { using type = uint2; };
template <> struct QuadOf<__half> { using type = uint2; };

__device__ __forceinline__ float4 pack_quad(float a, float b, float c, float d)
{
    return make_float4(a, b, c, d);
}
__device__ __forceinline__ uint32_t bits16(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
__device__ __forceinline__ uint32_t bits16(__half v) { return __half_as_ushort(v); }
template <typename T>
__device__ __forceinline__ uint2 pack_quad16(T a, T b, T c, T d)
{
    return make_uint2(bits16(a) | (bits16(b) << 16), bits16(c) | (bits16(d) << 16));
}

__device__ __forceinline__ float4 load_quad(const float4* p, float*) { return __ldg(p); }
__device__ __forceinline__ float4 load_quad(const uint2* p, __nv_bfloat16*)
{
    const uint2 q = __ldg(p);
    return make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xffff0000u),
                       __uint_as_float(q.y << 16), __uint_as_float(q.y & 0xffff0000u));
}
__device__ __forceinline__ float4 load_quad(const uint2* p, __half*)
{
    const uint2 q = __ldg(p);
    return make_float4(__half2float(__ushort_as_half((unsigned short)(q.x & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(q.x >> 16))),
                       __half2float(__ushort_as_half((unsigned short)(q.y & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(q.y >> 16))));
}

}  // namespace tigre
