// Quad elements: one bilinear cell stored together, so that one aligned
// 16-byte load fetches it.  The forward projector's cells are (f, f+1) x
// (m, m+1) of a volume plane, the backprojector's (c, c+1) x (r, r+1) of a
// detector image.  Whatever the storage type of the volume or projections,
// an element holds the cell's four bilinear coefficients in FP32 (formed from
// the taps converted to FP32 when the layout is built), so the interpolation
// is three FMAs after one load.
#pragma once

#include "common.cuh"

namespace tigre {

template <typename T> struct QuadOf { using type = float4; };

__device__ __forceinline__ float4 load_quad(const float4* p) { return __ldg(p); }

}  // namespace tigre
