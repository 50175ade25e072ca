// Gradient-descent total-variation minimisation (paper Sec. 2.3; the norm of
// the update is needed at every iteration).
//
// TV_eps(f) = sum_c sqrt(Dx^2 + Dy^2 + Dz^2 + eps), backward differences
// with a zero difference across the low boundary.  Voxel c enters its own
// term through +Dx, +Dy, +Dz and its forward neighbours' terms with a minus
// sign, so
//   g_c = (Dx+Dy+Dz)_c / n_c - Dx_{c+x}/n_{c+x} - Dy_{c+y}/n_{c+y} - Dz_{c+z}/n_{c+z},
// n = sqrt(D^2 + eps).  One step: x <- x - alpha g / ||g||_2 (no-op if 0).
//
// Per step: one pass computes g into an FP32 scratch volume together with
// deterministic FP64 partial sums of g^2, one block reduces them, and one
// pass applies the update.  Both passes are HBM-bound streams; the 13-point
// stencil reuse comes from L1/L2 (rows of a plane are walked in order).
#include <algorithm>
#include <cmath>

#include "vecops.cuh"

namespace tigre {

template <typename T>
__device__ __forceinline__ float ldv(const T* p)
{
    return to_f32<T>(__ldg(p));
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) tv_grad_kernel(const T* __restrict__ f,
                                                              float* __restrict__ g, int nx,
                                                              int ny, int nz, float eps,
                                                              double* __restrict__ partials,
                                                              int k_lo, int k_hi)
{
    __shared__ double sh[kRedThreads];
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t rows = (int64_t)ny * nz;
    double acc = 0.0;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = (int)(r % ny), k = (int)(r / ny);
        const T* row = f + r * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const T* c = row + i;
            const float fc = ldv(c);
            const float dx = i > 0 ? fc - ldv(c - sx) : 0.0f;
            const float dy = j > 0 ? fc - ldv(c - sy) : 0.0f;
            const float dz = k > 0 ? fc - ldv(c - sz) : 0.0f;
            float gv = (dx + dy + dz) * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps))));
            if (i + 1 < nx) {
                const float fp = ldv(c + sx);
                const float ax = fp - fc;
                const float ay = j > 0 ? fp - ldv(c + sx - sy) : 0.0f;
                const float az = k > 0 ? fp - ldv(c + sx - sz) : 0.0f;
                gv -= ax * rsqrtf(fmaf(ax, ax, fmaf(ay, ay, fmaf(az, az, eps))));
            }
            if (j + 1 < ny) {
                const float fp = ldv(c + sy);
                const float ax = i > 0 ? fp - ldv(c + sy - sx) : 0.0f;
                const float ay = fp - fc;
                const float az = k > 0 ? fp - ldv(c + sy - sz) : 0.0f;
                gv -= ay * rsqrtf(fmaf(ax, ax, fmaf(ay, ay, fmaf(az, az, eps))));
            }
            if (k + 1 < nz) {
                const float fp = ldv(c + sz);
                const float ax = i > 0 ? fp - ldv(c + sz - sx) : 0.0f;
                const float ay = j > 0 ? fp - ldv(c + sz - sy) : 0.0f;
                const float az = fp - fc;
                gv -= az * rsqrtf(fmaf(ax, ax, fmaf(ay, ay, fmaf(az, az, eps))));
            }
            g[r * nx + i] = gv;
            if (k >= k_lo && k < k_hi) acc = fma((double)gv, (double)gv, acc);
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// x <- x - (alpha * scale / ||g||) g, with ||g|| = norm[1]; no-op when ||g|| = 0.
template <typename T>
__global__ void tv_update_kernel(T* __restrict__ x, const float* __restrict__ g, int64_t n,
                                 double alpha, const double* __restrict__ scale,
                                 const double* __restrict__ norm)
{
    const double nn = norm[1];
    if (!(nn > 0.0)) return;
    const double a = alpha * (scale ? *scale : 1.0) / nn;
    const float s = isfinite(a) ? (float)a : 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        x[i] = from_f32<T>(fmaf(-s, g[i], to_f32<T>(x[i])));
}

tigre_status tv_load_kernels()
{
    cudaFuncAttributes fa;
    TIGRE_CUDA(cudaFuncGetAttributes(&fa, tv_grad_kernel<float>));
    TIGRE_CUDA(cudaFuncGetAttributes(&fa, tv_grad_kernel<__nv_bfloat16>));
    TIGRE_CUDA(cudaFuncGetAttributes(&fa, tv_grad_kernel<__half>));
    TIGRE_CUDA(cudaFuncGetAttributes(&fa, tv_update_kernel<float>));
    TIGRE_CUDA(cudaFuncGetAttributes(&fa, tv_update_kernel<__nv_bfloat16>));
    TIGRE_CUDA(cudaFuncGetAttributes(&fa, tv_update_kernel<__half>));
    return reduce_load_kernels();
}

tigre_status tv_impl(const int64_t n[3], void* vol, tigre_dtype t, int n_steps, double alpha,
                     double eps, const double* d_alpha_scale, void* scratch_g, double* d_red,
                     cudaStream_t st)
{
    return tv_impl_region(n, vol, t, n_steps, alpha, eps, d_alpha_scale, scratch_g, d_red, 0,
                          (int)n[2], st);
}

tigre_status tv_impl_region(const int64_t n[3], void* vol, tigre_dtype t, int n_steps,
                            double alpha, double eps, const double* d_alpha_scale,
                            void* scratch_g, double* d_red, int k_lo, int k_hi, cudaStream_t st)
{
    const int64_t N = n[0] * n[1] * n[2];
    double* partials = d_red;
    double* norm = d_red + kRedBlocks;
    return dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        ProfScope prof(kProfTV, st);
        for (int s = 0; s < n_steps; ++s) {
            tv_grad_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(
                (const T*)vol, (float*)scratch_g, (int)n[0], (int)n[1], (int)n[2], (float)eps,
                partials, k_lo, k_hi);
            TIGRE_LAUNCHED("tv_grad_kernel");
            TIGRE_TRY(reduce_partials(partials, norm, 1, st));
            const int64_t blocks = std::min<int64_t>((N + 255) / 256, 152 * 16);
            tv_update_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(
                (T*)vol, (const float*)scratch_g, N, alpha, d_alpha_scale, norm);
            TIGRE_LAUNCHED("tv_update_kernel");
        }
        return TIGRE_OK;
    });
}

}  // namespace tigre

using namespace tigre;

extern "C" tigre_status tigre_tv_step(const int64_t n_voxel[3], void* vol, tigre_dtype dtype,
                                      int n_steps, double alpha, double eps, void* cuda_stream)
{
    if (!n_voxel || !vol) return fail(TIGRE_ERR_INVALID_ARG, "null n_voxel or vol");
    for (int a = 0; a < 3; ++a)
        if (n_voxel[a] <= 0 || n_voxel[a] > (1 << 20))
            return fail(TIGRE_ERR_INVALID_ARG, "n_voxel out of range");
    if (!dtype_ok(dtype)) return fail(TIGRE_ERR_INVALID_ARG, "bad dtype");
    if (n_steps < 0 || !std::isfinite(alpha) || !std::isfinite(eps) || eps < 0.0)
        return fail(TIGRE_ERR_INVALID_ARG, "need n_steps >= 0, finite alpha, eps >= 0");
    if (n_steps == 0) return TIGRE_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t N = n_voxel[0] * n_voxel[1] * n_voxel[2];
    void* g = nullptr;
    void* red = nullptr;
    TIGRE_CUDA(dev_alloc(&g, sizeof(float) * (size_t)N, st));
    cudaError_t e = dev_alloc(&red, sizeof(double) * (kRedBlocks + 4), st);
    if (e != cudaSuccess) {
        dev_free(g, st);
        return cuda_fail(e, "device allocation (tv reduction)");
    }
    tigre_status s = tv_impl(n_voxel, vol, dtype, n_steps, alpha, eps, nullptr, g, (double*)red, st);
    dev_free(g, st);
    dev_free(red, st);
    return s;
}
