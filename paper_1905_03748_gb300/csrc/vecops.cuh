// Vector operations with FP64 device scalars (see vecops.cu).
#pragma once

#include "common.cuh"

namespace tigre {

// out[0] = sum partials (fixed order); with sqrt_out also out[1] = sqrt(out[0]).
tigre_status reduce_partials(const double* partials, double* out, int sqrt_out, cudaStream_t st);
// Load (under lazy module loading) the kernels of reduce_partials / of the
// TV steps on the current device, so that a later launch loads nothing.
tigre_status reduce_load_kernels();
tigre_status tv_load_kernels();
// y += sign * (num/den) x        (num, den: device doubles; den == 0 -> no-op)
tigre_status axpy_ratio(float* y, const float* x, int64_t n, const double* num, const double* den,
                        float sign, cudaStream_t st);
// same, and out[0] = ||y_new||^2, out[1] = ||y_new||
tigre_status axpy_ratio_norm(float* y, const float* x, int64_t n, const double* num,
                             const double* den, float sign, double* partials, double* out,
                             cudaStream_t st);
// y = x + (num/den) y
tigre_status xpay_ratio(float* y, const float* x, int64_t n, const double* num, const double* den,
                        cudaStream_t st);
// r = W (b - q) (W may be null = ones); out[0] = ||b - q||^2, out[1] = ||b - q||
tigre_status weighted_residual(const float* b, const float* q, const float* W, float* r, int64_t n,
                               double* partials, double* out, cudaStream_t st);
// Storage-typed: r = W (b - q) with b, q, r in dtype t; ||a - b|| for dtype t.
tigre_status weighted_residual_dt(tigre_dtype t, const void* b, const void* q, const float* W,
                                  void* r, int64_t n, double* partials, double* out,
                                  cudaStream_t st);
tigre_status diff_norm_dt(tigre_dtype t, const void* a, const void* b, int64_t n, double* partials,
                          double* out, cudaStream_t st);
// y = y > floor ? 1/y : 0
tigre_status guarded_reciprocal(float* y, int64_t n, float floor_, cudaStream_t st);
// out[0] = ||a - b||^2, out[1] = ||a - b||
tigre_status diff_norm(const float* a, const float* b, int64_t n, double* partials, double* out,
                       cudaStream_t st);
tigre_status copy_dscalar(double* dst, const double* src, cudaStream_t st);
// hist[*counter] = *v when *counter < cap; ++*counter (device-side index)
tigre_status record_dscalar(double* hist, int cap, int* counter, const double* v, cudaStream_t st);
// mode 0: dst = src; 1: dst += src; 2: dst = sqrt(src)
tigre_status combine_dscalar(double* dst, const double* src, int mode, cudaStream_t st);
tigre_status fill_f32(float* p, float v, int64_t n, cudaStream_t st);
// Storage-typed forms of dot_f64, axpy_ratio, axpy_ratio_norm, xpay_ratio
// (vectors in dtype t, FP32 arithmetic, FP64 sums; the norm is that of the
// stored, rounded vector).
tigre_status dot_f64_dt(tigre_dtype t, const void* a, const void* b, int64_t n, double* d_partials,
                        double* d_out, cudaStream_t st);
tigre_status axpy_ratio_dt(tigre_dtype t, void* y, const void* x, int64_t n, const double* num,
                           const double* den, float sign, cudaStream_t st);
tigre_status axpy_ratio_norm_dt(tigre_dtype t, void* y, const void* x, int64_t n,
                                const double* num, const double* den, float sign,
                                double* partials, double* out, cudaStream_t st);
tigre_status xpay_ratio_dt(tigre_dtype t, void* y, const void* x, int64_t n, const double* num,
                           const double* den, cudaStream_t st);
tigre_status scale_dscalar(double* dst, const double* src, double factor, cudaStream_t st);

}  // namespace tigre
