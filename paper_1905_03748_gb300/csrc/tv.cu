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
// deterministic partial sums of g^2, one block reduces them, and one pass
// applies the update.  Both passes are HBM streams: the gradient pass stages
// each plane in shared memory once (tv_grad_kernel), the update reads x and g
// and writes x.
#include <algorithm>
#include <cmath>

#include "vecops.cuh"

namespace tigre {

template <typename T>
__device__ __forceinline__ float ldv(const T* p)
{
    return to_f32<T>(__ldg(p));
}

// The gradient pass, as a z-march over tiles of 32 x 8 columns x 24 planes:
// a block stages the tile's planes of f (with a one-voxel halo) in shared
// memory in one batch of loads,
// computes every voxel's differences D = (Dx, Dy, Dz) and r = 1/n once, and
// takes the neighbours' terms from shared memory (x+1, y+1) and from the
// next plane's values in registers (z+1).  The gradient is
//   g_c = (Dx+Dy+Dz)_c r_c - Dx_{c+x} r_{c+x} - Dy_{c+y} r_{c+y} - Dz_{c+z} r_{c+z},
// each neighbour's term applied as one FMA.  The grid has kRedBlocks blocks
// (a fixed set of partial sums, so the norm is deterministic); block b takes
// tiles b, b + kRedBlocks, ... in x, y, z-chunk order.  g^2 over the planes
// [k_lo, k_hi) is summed in FP32 within a tile's column and in FP64 beyond.
constexpr int kTvTX = 32, kTvTY = 8, kTvKC = 24;

// D and r at the tile-local position (a, b) of a plane (a in [0, 32], b in
// [0, 8]) from the staged plane (cur) and the one below it (prev).
__device__ __forceinline__ float4 tv_dr(const float (*cur)[kTvTX + 2],
                                        const float (*prev)[kTvTX + 2], int a, int b, int gi,
                                        int gj, int p, float eps)
{
    const float fc = cur[b + 1][a + 1];
    const float dx = gi > 0 ? fc - cur[b + 1][a] : 0.0f;
    const float dy = gj > 0 ? fc - cur[b][a + 1] : 0.0f;
    const float dz = p > 0 ? fc - prev[b + 1][a + 1] : 0.0f;
    return make_float4(dx, dy, dz, rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps)))));
}

template <typename T>
__global__ void __launch_bounds__(kTvTX* kTvTY, 4) tv_grad_kernel(const T* __restrict__ f,
                                                                float* __restrict__ g, int nx,
                                                                int ny, int nz, float eps,
                                                                double* __restrict__ partials,
                                                                int k_lo, int k_hi)
{
    static_assert(kTvTX * kTvTY == kRedThreads, "one reduction slot per thread");
    constexpr int kPlane = (kTvTY + 2) * (kTvTX + 2);
    // f of planes k0 - 1 .. k0 + KC (index p - k0 + 1), staged in one batch of
    // loads per tile, so a tile waits for global memory once
    __shared__ float fs[kTvKC + 2][kTvTY + 2][kTvTX + 2];
    __shared__ float2 sx[2][kTvTY][kTvTX + 1];  // (Dx, r), x0 .. x0 + 32, plane parity
    __shared__ float2 sy[2][kTvTY + 1][kTvTX];  // (Dy, r), y0 .. y0 + 8
    __shared__ double sh[kRedThreads];
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * kTvTX + lx;
    const int ntx = (nx + kTvTX - 1) / kTvTX, nty = (ny + kTvTY - 1) / kTvTY;
    const int ntz = (nz + kTvKC - 1) / kTvKC;
    const int64_t ntiles = (int64_t)ntx * nty * ntz;
    const int64_t pstride = (int64_t)nx * ny;
    double acc = 0.0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int tx, ty, tz;
        if (ntiles < (int64_t)INT32_MAX) {  // 32-bit tile arithmetic
            const int tt = (int)t, rest = tt / ntx;
            tx = tt - rest * ntx;
            ty = rest % nty;
            tz = rest / nty;
        } else {
            const int64_t rest = t / ntx;
            tx = (int)(t - rest * ntx);
            ty = (int)(rest % nty);
            tz = (int)(rest / nty);
        }
        const int x0 = tx * kTvTX, y0 = ty * kTvTY, k0 = tz * kTvKC;
        const int k1 = min(k0 + kTvKC, nz);
        const int i = x0 + lx, j = y0 + ly;
        const bool in = i < nx && j < ny;
        __syncthreads();  // the previous tile's readers are done with the buffers
        // each thread stages one or two (row, column) slots of every plane;
        // the 18 loads of a slot are issued together
        for (int q = tid; q < kPlane; q += kRedThreads) {
            const int jj = q / (kTvTX + 2), ii = q - jj * (kTvTX + 2);
            const int gi = x0 - 1 + ii, gj = y0 - 1 + jj;
            const bool xy = (unsigned)gi < (unsigned)nx && (unsigned)gj < (unsigned)ny;
            const int64_t col = xy ? (int64_t)gj * nx + gi : 0;
#pragma unroll
            for (int pl = 0; pl < kTvKC + 2; ++pl) {
                const int p = k0 - 1 + pl;
                fs[pl][jj][ii] = xy && (unsigned)p < (unsigned)nz ? ldv(f + col + (int64_t)p * pstride)
                                                                  : 0.0f;
            }
        }
        // the halo positions: column x0 + 32 (rows 0..7) for threads 0..7,
        // row y0 + 8 (columns 0..31) for threads 8..39
        const bool halo = tid < kTvTY + kTvTX;
        const int ha = tid < kTvTY ? kTvTX : tid - kTvTY, hb = tid < kTvTY ? tid : kTvTY;
        __syncthreads();
        // D, r of plane k0: own, and the halo column / row
        float4 own = tv_dr(fs[1], fs[0], lx, ly, i, j, k0, eps);
        sx[k0 & 1][ly][lx] = make_float2(own.x, own.w);
        sy[k0 & 1][ly][lx] = make_float2(own.y, own.w);
        if (halo) {
            const float4 h = tv_dr(fs[1], fs[0], ha, hb, x0 + ha, y0 + hb, k0, eps);
            if (tid < kTvTY) sx[k0 & 1][hb][kTvTX] = make_float2(h.x, h.w);
            else sy[k0 & 1][kTvTY][ha] = make_float2(h.y, h.w);
        }
        float* gout = g + ((int64_t)k0 * ny + j) * nx + i;
        float tacc = 0.0f;
        for (int k = k0; k < k1; ++k) {
            const int cb = k & 1, nb = cb ^ 1, pc = k - k0 + 1;
            const bool up = k + 1 < nz;
            // plane k's D, r are visible; plane k - 1's are no longer read
            __syncthreads();
            float4 nxt = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
            if (up) {
                nxt = tv_dr(fs[pc + 1], fs[pc], lx, ly, i, j, k + 1, eps);
                sx[nb][ly][lx] = make_float2(nxt.x, nxt.w);
                sy[nb][ly][lx] = make_float2(nxt.y, nxt.w);
                if (halo) {
                    const float4 h = tv_dr(fs[pc + 1], fs[pc], ha, hb, x0 + ha, y0 + hb, k + 1, eps);
                    if (tid < kTvTY) sx[nb][hb][kTvTX] = make_float2(h.x, h.w);
                    else sy[nb][kTvTY][ha] = make_float2(h.y, h.w);
                }
            }
            if (in) {
                float gv = (own.x + own.y + own.z) * own.w;
                if (i + 1 < nx) {
                    const float2 e = sx[cb][ly][lx + 1];
                    gv = fmaf(-e.x, e.y, gv);
                }
                if (j + 1 < ny) {
                    const float2 e = sy[cb][ly + 1][lx];
                    gv = fmaf(-e.x, e.y, gv);
                }
                if (up) gv = fmaf(-nxt.z, nxt.w, gv);
                *gout = gv;
                if (k >= k_lo && k < k_hi) tacc = fmaf(gv, gv, tacc);
            }
            own = nxt;
            gout += pstride;
        }
        acc += (double)tacc;
    }
    sh[tid] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (tid < w) sh[tid] += sh[tid + w];
        __syncthreads();
    }
    if (tid == 0) partials[blockIdx.x] = sh[0];
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
            tv_grad_kernel<T><<<kRedBlocks, dim3(kTvTX, kTvTY), 0, st>>>(
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
