// Vector operations and deterministic FP64 reductions used by the solvers.
//
// Reductions: a fixed grid of kRedBlocks blocks walks the vector with a
// fixed stride, each thread accumulating in FP64 (a product of two FP32
// numbers is exact in FP64); blocks reduce in shared memory in a fixed tree
// order and write one partial each; a single block then adds the partials
// in a fixed order.  The result is therefore bitwise reproducible for a
// given n, independent of timing.
#include "vecops.cuh"

namespace tigre {

__device__ __forceinline__ double block_sum(double v, double* sh)
{
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) sh[t] += sh[t + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// The element-wise kernels below are templates on the storage type T of the
// vectors (F32, BF16 or F16): values are widened to FP32 for the arithmetic,
// sums are FP64, results are rounded once to T.  For T = float they are the
// plain FP32 kernels.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) dot_partials_kernel(const T* __restrict__ a,
                                                                   const T* __restrict__ b,
                                                                   int64_t n,
                                                                   double* __restrict__ partials)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        acc = fma((double)to_f32<T>(a[i]), (double)to_f32<T>(b[i]), acc);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out[0] = sum of partials (fixed order); if sqrt_out, also out[1] = sqrt.
__global__ void __launch_bounds__(kRedThreads) reduce_partials_kernel(
    const double* __restrict__ partials, int np, double* __restrict__ out, int sqrt_out)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        out[0] = s;
        if (sqrt_out) out[1] = sqrt(s);
    }
}

tigre_status reduce_load_kernels()
{
    cudaFuncAttributes fa;
    TIGRE_CUDA(cudaFuncGetAttributes(&fa, reduce_partials_kernel));
    return TIGRE_OK;
}

tigre_status reduce_partials(const double* partials, double* out, int sqrt_out, cudaStream_t st)
{
    reduce_partials_kernel<<<1, kRedThreads, 0, st>>>(partials, kRedBlocks, out, sqrt_out);
    TIGRE_LAUNCHED("reduce_partials_kernel");
    return TIGRE_OK;
}

tigre_status dot_f64(const float* a, const float* b, int64_t n, double* d_partials, double* d_out,
                     cudaStream_t st)
{
    dot_partials_kernel<float><<<kRedBlocks, kRedThreads, 0, st>>>(a, b, n, d_partials);
    TIGRE_LAUNCHED("dot_partials_kernel");
    return reduce_partials(d_partials, d_out, 0, st);
}

// Scalar num/den read from device memory; 0 when den is 0 (or either is not finite).
__device__ __forceinline__ double dev_ratio(const double* num, const double* den)
{
    const double d = *den;
    const double r = d != 0.0 ? *num / d : 0.0;
    return isfinite(r) ? r : 0.0;
}

// y += sign * (num/den) * x
template <typename T>
__global__ void axpy_ratio_kernel(T* __restrict__ y, const T* __restrict__ x, int64_t n,
                                  const double* num, const double* den, float sign)
{
    const float s = sign * (float)dev_ratio(num, den);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = from_f32<T>(fmaf(s, to_f32<T>(x[i]), to_f32<T>(y[i])));
}

// y += sign * (num/den) * x, and per-block partial sums of y_new^2.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) axpy_ratio_norm_kernel(
    T* __restrict__ y, const T* __restrict__ x, int64_t n, const double* num,
    const double* den, float sign, double* __restrict__ partials)
{
    __shared__ double sh[kRedThreads];
    const float s = sign * (float)dev_ratio(num, den);
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T v = from_f32<T>(fmaf(s, to_f32<T>(x[i]), to_f32<T>(y[i])));
        y[i] = v;
        const double vd = (double)to_f32<T>(v);  // the norm of the stored vector
        acc = fma(vd, vd, acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// y = x + (num/den) * y
template <typename T>
__global__ void xpay_ratio_kernel(T* __restrict__ y, const T* __restrict__ x, int64_t n,
                                  const double* num, const double* den)
{
    const float s = (float)dev_ratio(num, den);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = from_f32<T>(fmaf(s, to_f32<T>(y[i]), to_f32<T>(x[i])));
}

// r = W * (b - q), partial sums of (b - q)^2.
// (q and r may alias: each element is read before it is written.)
__global__ void __launch_bounds__(kRedThreads) weighted_residual_kernel(
    const float* __restrict__ b, const float* q, const float* __restrict__ W, float* r, int64_t n,
    double* __restrict__ partials)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float d = b[i] - q[i];
        r[i] = W ? W[i] * d : d;
        acc = fma((double)d, (double)d, acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// y = 1/y where y > floor, else 0.
__global__ void guarded_reciprocal_kernel(float* __restrict__ y, int64_t n, float floor_)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = y[i];
        y[i] = v > floor_ ? 1.0f / v : 0.0f;
    }
}

// partial sums of (a - b)^2
__global__ void __launch_bounds__(kRedThreads) diff_norm_partials_kernel(
    const float* __restrict__ a, const float* __restrict__ b, int64_t n,
    double* __restrict__ partials)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double d = (double)a[i] - (double)b[i];
        acc = fma(d, d, acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void fill_kernel(float* __restrict__ p, float v, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

__global__ void copy_dscalar_kernel(double* dst, const double* src) { *dst = *src; }

// mode 0: dst = src; 1: dst += src; 2: dst = sqrt(src)
__global__ void combine_dscalar_kernel(double* dst, const double* src, int mode)
{
    const double v = *src;
    *dst = mode == 0 ? v : mode == 1 ? *dst + v : sqrt(v);
}

__global__ void scale_dscalar_kernel(double* dst, const double* src, double factor)
{
    *dst = factor * *src;
}

// hist[*counter] = *v (if it fits), ++*counter: an append whose index lives on
// the device, so replays of a captured graph keep appending.
__global__ void record_dscalar_kernel(double* hist, int cap, int* counter, const double* v)
{
    const int i = *counter;
    if (i >= 0 && i < cap) hist[i] = *v;
    *counter = i + 1;
}

tigre_status record_dscalar(double* hist, int cap, int* counter, const double* v, cudaStream_t st)
{
    record_dscalar_kernel<<<1, 1, 0, st>>>(hist, cap, counter, v);
    TIGRE_LAUNCHED("record_dscalar_kernel");
    return TIGRE_OK;
}

// Storage-typed variants (BF16 / F16 / F32 storage, FP32 arithmetic, FP64 sums).
template <typename T>
__global__ void __launch_bounds__(kRedThreads) weighted_residual_t_kernel(
    const T* __restrict__ b, const T* q, const float* __restrict__ W, T* r, int64_t n,
    double* __restrict__ partials)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float d = to_f32<T>(b[i]) - to_f32<T>(q[i]);
        r[i] = from_f32<T>(W ? W[i] * d : d);
        acc = fma((double)d, (double)d, acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) diff_norm_t_kernel(const T* __restrict__ a,
                                                                  const T* __restrict__ b,
                                                                  int64_t n,
                                                                  double* __restrict__ partials)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double d = (double)to_f32<T>(a[i]) - (double)to_f32<T>(b[i]);
        acc = fma(d, d, acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

tigre_status weighted_residual_dt(tigre_dtype t, const void* b, const void* q, const float* W,
                                  void* r, int64_t n, double* partials, double* out,
                                  cudaStream_t st)
{
    TIGRE_TRY(dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        weighted_residual_t_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(
            (const T*)b, (const T*)q, W, (T*)r, n, partials);
        TIGRE_LAUNCHED("weighted_residual_t_kernel");
        return TIGRE_OK;
    }));
    return reduce_partials(partials, out, 1, st);
}

tigre_status diff_norm_dt(tigre_dtype t, const void* a, const void* b, int64_t n, double* partials,
                          double* out, cudaStream_t st)
{
    TIGRE_TRY(dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        diff_norm_t_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>((const T*)a, (const T*)b, n,
                                                                   partials);
        TIGRE_LAUNCHED("diff_norm_t_kernel");
        return TIGRE_OK;
    }));
    return reduce_partials(partials, out, 1, st);
}

static inline unsigned ew_blocks(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

tigre_status axpy_ratio(float* y, const float* x, int64_t n, const double* num, const double* den,
                        float sign, cudaStream_t st)
{
    axpy_ratio_kernel<float><<<ew_blocks(n), 256, 0, st>>>(y, x, n, num, den, sign);
    TIGRE_LAUNCHED("axpy_ratio_kernel");
    return TIGRE_OK;
}

tigre_status axpy_ratio_norm(float* y, const float* x, int64_t n, const double* num,
                             const double* den, float sign, double* partials, double* out,
                             cudaStream_t st)
{
    axpy_ratio_norm_kernel<float><<<kRedBlocks, kRedThreads, 0, st>>>(y, x, n, num, den, sign,
                                                                      partials);
    TIGRE_LAUNCHED("axpy_ratio_norm_kernel");
    return reduce_partials(partials, out, 1, st);
}

tigre_status xpay_ratio(float* y, const float* x, int64_t n, const double* num, const double* den,
                        cudaStream_t st)
{
    xpay_ratio_kernel<float><<<ew_blocks(n), 256, 0, st>>>(y, x, n, num, den);
    TIGRE_LAUNCHED("xpay_ratio_kernel");
    return TIGRE_OK;
}

tigre_status weighted_residual(const float* b, const float* q, const float* W, float* r, int64_t n,
                               double* partials, double* out, cudaStream_t st)
{
    weighted_residual_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(b, q, W, r, n, partials);
    TIGRE_LAUNCHED("weighted_residual_kernel");
    return reduce_partials(partials, out, 1, st);
}

tigre_status guarded_reciprocal(float* y, int64_t n, float floor_, cudaStream_t st)
{
    guarded_reciprocal_kernel<<<ew_blocks(n), 256, 0, st>>>(y, n, floor_);
    TIGRE_LAUNCHED("guarded_reciprocal_kernel");
    return TIGRE_OK;
}

tigre_status diff_norm(const float* a, const float* b, int64_t n, double* partials, double* out,
                       cudaStream_t st)
{
    diff_norm_partials_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(a, b, n, partials);
    TIGRE_LAUNCHED("diff_norm_partials_kernel");
    return reduce_partials(partials, out, 1, st);
}

tigre_status fill_f32(float* p, float v, int64_t n, cudaStream_t st)
{
    fill_kernel<<<ew_blocks(n), 256, 0, st>>>(p, v, n);
    TIGRE_LAUNCHED("fill_kernel");
    return TIGRE_OK;
}

tigre_status copy_dscalar(double* dst, const double* src, cudaStream_t st)
{
    copy_dscalar_kernel<<<1, 1, 0, st>>>(dst, src);
    TIGRE_LAUNCHED("copy_dscalar_kernel");
    return TIGRE_OK;
}

tigre_status combine_dscalar(double* dst, const double* src, int mode, cudaStream_t st)
{
    combine_dscalar_kernel<<<1, 1, 0, st>>>(dst, src, mode);
    TIGRE_LAUNCHED("combine_dscalar_kernel");
    return TIGRE_OK;
}

tigre_status scale_dscalar(double* dst, const double* src, double factor, cudaStream_t st)
{
    scale_dscalar_kernel<<<1, 1, 0, st>>>(dst, src, factor);
    TIGRE_LAUNCHED("scale_dscalar_kernel");
    return TIGRE_OK;
}

tigre_status dot_f64_dt(tigre_dtype t, const void* a, const void* b, int64_t n, double* d_partials,
                        double* d_out, cudaStream_t st)
{
    return dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        dot_partials_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>((const T*)a, (const T*)b, n,
                                                                   d_partials);
        TIGRE_LAUNCHED("dot_partials_kernel");
        return reduce_partials(d_partials, d_out, 0, st);
    });
}

tigre_status axpy_ratio_dt(tigre_dtype t, void* y, const void* x, int64_t n, const double* num,
                           const double* den, float sign, cudaStream_t st)
{
    return dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        axpy_ratio_kernel<T><<<ew_blocks(n), 256, 0, st>>>((T*)y, (const T*)x, n, num, den, sign);
        TIGRE_LAUNCHED("axpy_ratio_kernel");
        return TIGRE_OK;
    });
}

tigre_status axpy_ratio_norm_dt(tigre_dtype t, void* y, const void* x, int64_t n,
                                const double* num, const double* den, float sign,
                                double* partials, double* out, cudaStream_t st)
{
    return dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        axpy_ratio_norm_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(
            (T*)y, (const T*)x, n, num, den, sign, partials);
        TIGRE_LAUNCHED("axpy_ratio_norm_kernel");
        return reduce_partials(partials, out, 1, st);
    });
}

tigre_status xpay_ratio_dt(tigre_dtype t, void* y, const void* x, int64_t n, const double* num,
                           const double* den, cudaStream_t st)
{
    return dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        xpay_ratio_kernel<T><<<ew_blocks(n), 256, 0, st>>>((T*)y, (const T*)x, n, num, den);
        TIGRE_LAUNCHED("xpay_ratio_kernel");
        return TIGRE_OK;
    });
}

}  // namespace tigre
