// ROF-model TV minimisation (Sec. 2.3: the second TV minimiser the paper
// uses, an image-to-image operator needing several copies of the image):
//
//   min_u  ||grad u||_(2,1) + lam/2 ||u - f||^2      (isotropic TV)
//
// by the first-order primal-dual iteration with over-relaxation 1 and step
// sizes tau = sigma = 1/sqrt(12) (||grad||^2 <= 12 for 3-D forward
// differences):
//
//   p    <- (p + sigma grad ubar) / max(1, |p + sigma grad ubar|)
//   u'   <- (u + tau div p + tau lam f) / (1 + tau lam)
//   ubar <- 2 u' - u,   u <- u'
//
// from u = ubar = f, p = 0.  grad = forward differences with zero at the last
// index of each axis; div = -grad^T.  Two kernels per iteration (the dual
// step reads ubar at +1 neighbours, the primal step reads p at -1
// neighbours); both are HBM-bound stencils: 28 algorithmic bytes per voxel
// each (dual: ubar 4 + p 12 in, p 12 out; primal: p 12 + u 4 + f 4 in, u 4 +
// ubar 4 out), neighbours served from L1/L2.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace tigre {
namespace {

struct RofDims {
    int nx, ny, nz;
    int64_t sy, sz;  // strides of y and z
};

__global__ void __launch_bounds__(256) rof_dual_kernel(const float* __restrict__ ubar,
                                                       float* __restrict__ px,
                                                       float* __restrict__ py,
                                                       float* __restrict__ pz, RofDims d,
                                                       float sigma)
{
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= d.nx || y >= d.ny) return;
    const int64_t i = z * d.sz + y * d.sy + x;
    const float c = ubar[i];
    const float gx = x + 1 < d.nx ? ubar[i + 1] - c : 0.0f;
    const float gy = y + 1 < d.ny ? ubar[i + d.sy] - c : 0.0f;
    const float gz = z + 1 < d.nz ? ubar[i + d.sz] - c : 0.0f;
    const float ax = fmaf(sigma, gx, px[i]);
    const float ay = fmaf(sigma, gy, py[i]);
    const float az = fmaf(sigma, gz, pz[i]);
    const float inv = 1.0f / fmaxf(1.0f, sqrtf(fmaf(ax, ax, fmaf(ay, ay, az * az))));
    px[i] = ax * inv;
    py[i] = ay * inv;
    pz[i] = az * inv;
}

__global__ void __launch_bounds__(256) rof_primal_kernel(const float* __restrict__ px,
                                                         const float* __restrict__ py,
                                                         const float* __restrict__ pz,
                                                         const float* __restrict__ f,
                                                         float* __restrict__ u,
                                                         float* __restrict__ ubar, RofDims d,
                                                         float tau, float tau_lam)
{
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= d.nx || y >= d.ny) return;
    const int64_t i = z * d.sz + y * d.sy + x;
    // div p = sum over axes of (p[i] if i is not last) - (p[i-1] if i is not first)
    float dv = (x + 1 < d.nx ? px[i] : 0.0f) - (x > 0 ? px[i - 1] : 0.0f);
    dv += (y + 1 < d.ny ? py[i] : 0.0f) - (y > 0 ? py[i - d.sy] : 0.0f);
    dv += (z + 1 < d.nz ? pz[i] : 0.0f) - (z > 0 ? pz[i - d.sz] : 0.0f);
    const float uo = u[i];
    const float un = fmaf(tau, dv, fmaf(tau_lam, f[i], uo)) / (1.0f + tau_lam);
    u[i] = un;
    ubar[i] = fmaf(2.0f, un, -uo);
}

}  // namespace

tigre_status rof_impl(const int64_t n[3], const float* f, float* u, double lam, int n_iter,
                      cudaStream_t st)
{
    if (!n || !f || !u) return fail(TIGRE_ERR_INVALID_ARG, "null argument");
    if (n[0] <= 0 || n[1] <= 0 || n[2] <= 0) return fail(TIGRE_ERR_INVALID_ARG, "sizes must be > 0");
    if (!(lam > 0.0) || !std::isfinite(lam)) return fail(TIGRE_ERR_INVALID_ARG, "lambda must be > 0");
    if (n_iter < 0) return fail(TIGRE_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (n[0] > INT32_MAX || n[1] > INT32_MAX || n[2] > 65535)
        return fail(TIGRE_ERR_UNSUPPORTED, "volume too large for the launch grid");
    const size_t nv = (size_t)n[0] * (size_t)n[1] * (size_t)n[2];
    const size_t bytes = nv * sizeof(float);
    // workspace: ubar, px, py, pz (and a copy of f when it aliases u)
    const bool alias = f == u;
    float* ws = nullptr;
    TIGRE_CUDA(dev_alloc((void**)&ws, bytes * (alias ? 5 : 4), st));
    float *ubar = ws, *px = ws + nv, *py = ws + 2 * nv, *pz = ws + 3 * nv;
    const float* src = f;
    tigre_status status = TIGRE_OK;
    cudaError_t e = cudaSuccess;
    if (alias) {
        float* fc = ws + 4 * nv;
        e = cudaMemcpyAsync(fc, f, bytes, cudaMemcpyDeviceToDevice, st);
        src = fc;
    } else {
        e = cudaMemcpyAsync(u, f, bytes, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(ubar, src, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(px, 0, 3 * bytes, st);
    if (e != cudaSuccess) status = cuda_fail(e, "rof setup");
    const RofDims d{(int)n[0], (int)n[1], (int)n[2], n[0], n[0] * n[1]};
    const float tau = (float)(1.0 / std::sqrt(12.0)), sigma = tau;
    const float tau_lam = (float)((double)tau * lam);
    const dim3 grid((unsigned)((n[0] + 31) / 32), (unsigned)((n[1] + 7) / 8), (unsigned)n[2]);
    if (grid.y > 65535) status = fail(TIGRE_ERR_UNSUPPORTED, "volume too large for the launch grid");
    {
        ProfScope prof(kProfTV, st);
        for (int it = 0; it < n_iter && status == TIGRE_OK; ++it) {
            rof_dual_kernel<<<grid, dim3(32, 8), 0, st>>>(ubar, px, py, pz, d, sigma);
            e = cudaGetLastError();
            count_launch();
            if (e == cudaSuccess) {
                rof_primal_kernel<<<grid, dim3(32, 8), 0, st>>>(px, py, pz, src, u, ubar, d, tau,
                                                                tau_lam);
                e = cudaGetLastError();
                count_launch();
            }
            if (e != cudaSuccess) status = cuda_fail(e, "rof kernels");
        }
    }
    dev_free(ws, st);
    return status;
}

}  // namespace tigre

extern "C" tigre_status tigre_rof_denoise(const int64_t n_voxel[3], const float* f, float* u,
                                          double lambda, int n_iter, void* cuda_stream)
{
    return tigre::rof_impl(n_voxel, f, u, lambda, n_iter, (cudaStream_t)cuda_stream);
}
