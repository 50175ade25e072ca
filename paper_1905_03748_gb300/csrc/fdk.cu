// FDK reconstruction of a circular scan (the paper's analytic reconstruction,
// used for comparison and as an initialiser; Sec. 1 and Sec. 3.2).
//
//   1. each projection pixel is weighted by DSD / sqrt(DSD^2 + u^2 + v^2);
//   2. each detector row is convolved (linear convolution, zero outside the
//      detector) with the Ram-Lak ramp kernel of the detector pitch scaled to
//      the isocentre, tau = du DSO / DSD:  h[0] = 1/(4 tau^2),
//      h[odd k] = -1/(pi k tau)^2, h[even k] = 0, times tau for the sum;
//   3. the filtered projections are backprojected voxel by voxel with the FDK
//      distance weight (DSO/(DSO-s))^2, each angle times half its angular
//      weight (half the angle between its neighbours on the circle).
//
// Step 1, 2 and the angular factor run in one kernel (one block per detector
// row, the row in shared memory); step 3 is the voxel-driven backprojector.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace tigre {
namespace {

constexpr double kPi = 3.14159265358979323846;

// One block per (row q, angle a): out[a][q][p] = wa * sum_k w(k) y[k] h(p-k).
// The kernel is even and vanishes at even non-zero offsets, so each output
// sums h0 y[p] and h[j] (y[p-j] + y[p+j]) over odd j.
template <typename TP>
__global__ void __launch_bounds__(256) fdk_filter_kernel(const TP* __restrict__ proj,
                                                         float* __restrict__ out,
                                                         const float* __restrict__ h_odd,
                                                         const float* __restrict__ ang_w, int nu,
                                                         int nv, float h0, float u0, float du,
                                                         float v0, float dv, float dsd2)
{
    extern __shared__ float row[];
    const int q = blockIdx.x, a = blockIdx.y;
    const TP* src = proj + ((int64_t)a * nv + q) * nu;
    const float v = fmaf((float)q, dv, v0);
    for (int p = threadIdx.x; p < nu; p += blockDim.x) {
        const float u = fmaf((float)p, du, u0);
        row[p] = to_f32<TP>(src[p]) * sqrtf(dsd2) * rsqrtf(dsd2 + u * u + v * v);
    }
    __syncthreads();
    const float wa = ang_w[a];
    float* dst = out + ((int64_t)a * nv + q) * nu;
    for (int p = threadIdx.x; p < nu; p += blockDim.x) {
        float acc = h0 * row[p];
        // odd offsets j = 1, 3, 5, ...; h_odd[i] holds h at j = 2 i + 1
        for (int j = 1, i = 0; j < nu; j += 2, ++i) {
            const float l = p - j >= 0 ? row[p - j] : 0.0f;
            const float r = p + j < nu ? row[p + j] : 0.0f;
            acc = fmaf(h_odd[i], l + r, acc);
        }
        dst[p] = wa * acc;
    }
}

}  // namespace

// Angular weight of each angle: half the angle between its two neighbours
// on the circle (2 pi / N for N uniform angles); the FDK factor 1/2 is
// included here.
static std::vector<float> fdk_angle_factors(const std::vector<double>& angles)
{
    const size_t n = angles.size();
    std::vector<float> out(n);
    if (n == 1) {
        out[0] = (float)kPi;  // (2 pi) / 2
        return out;
    }
    const double two_pi = 2.0 * kPi;
    std::vector<std::pair<double, size_t>> s(n);
    for (size_t i = 0; i < n; ++i) s[i] = {std::fmod(std::fmod(angles[i], two_pi) + two_pi, two_pi), i};
    std::sort(s.begin(), s.end());
    for (size_t k = 0; k < n; ++k) {
        const double prev = s[(k + n - 1) % n].first, next = s[(k + 1) % n].first;
        const double gp = std::fmod(s[k].first - prev + two_pi, two_pi);
        const double gn = std::fmod(next - s[k].first + two_pi, two_pi);
        out[s[k].second] = (float)(0.25 * (gp + gn));  // 1/2 (gap mean) x 1/2 (FDK)
    }
    return out;
}

tigre_status fdk_impl(tigre_geometry* g, const void* proj, tigre_dtype pt, void* vol,
                      tigre_dtype vt, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    if (!proj || !vol) return fail(TIGRE_ERR_INVALID_ARG, "null proj or vol pointer");
    if (!dtype_ok(pt) || !dtype_ok(vt)) return fail(TIGRE_ERR_INVALID_ARG, "bad dtype");
    const tigre_geometry_desc& d = g->desc;
    const int nu = (int)d.n_det[0], nv = (int)d.n_det[1];
    const int64_t na = (int64_t)g->angles.size();
    if ((size_t)nu * sizeof(float) > 160 * 1024)
        return fail(TIGRE_ERR_UNSUPPORTED, "detector rows longer than 40960 pixels");
    if (nv > 2147483647 || na > 65535) return fail(TIGRE_ERR_UNSUPPORTED, "too many rows or angles");
    // Ram-Lak taps at odd offsets and the angular factors (FP64 on the host).
    const double tau = d.d_det[0] * d.DSO / d.DSD;
    std::vector<float> host((size_t)(nu / 2 + 1) + (size_t)na, 0.0f);
    for (int j = 1, i = 0; j < nu; j += 2, ++i)
        host[(size_t)i] = (float)(-1.0 / (kPi * kPi * (double)j * (double)j * tau));
    const std::vector<float> aw = fdk_angle_factors(g->angles);
    std::copy(aw.begin(), aw.end(), host.begin() + (nu / 2 + 1));
    float* dtab = nullptr;
    float* filt = nullptr;
    TIGRE_CUDA(dev_alloc((void**)&dtab, sizeof(float) * host.size(), st));
    cudaError_t e = dev_alloc((void**)&filt, sizeof(float) * (size_t)(na * nv) * (size_t)nu, st);
    if (e != cudaSuccess) {
        dev_free(dtab, st);
        return cuda_fail(e, "device allocation (fdk filtered projections)");
    }
    tigre_status status = TIGRE_OK;
    e = cudaMemcpyAsync(dtab, host.data(), sizeof(float) * host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host table leaves scope after this call
    if (e != cudaSuccess) status = cuda_fail(e, "fdk table upload");
    if (status == TIGRE_OK) {
        const float u0 = (float)(-0.5 * (double)(nu - 1) * d.d_det[0] + d.off_det[0]);
        const float v0 = (float)(-0.5 * (double)(nv - 1) * d.d_det[1] + d.off_det[1]);
        const float h0 = (float)(0.25 / tau);
        const size_t smem = sizeof(float) * (size_t)nu;
        status = dispatch_dtype(pt, [&](auto tag) -> tigre_status {
            using TP = decltype(tag);
            if (smem > 48 * 1024)
                TIGRE_CUDA(cudaFuncSetAttribute(fdk_filter_kernel<TP>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem));
            fdk_filter_kernel<TP><<<dim3((unsigned)nv, (unsigned)na), 256, smem, st>>>(
                (const TP*)proj, filt, dtab, dtab + (nu / 2 + 1), nu, nv, h0, u0,
                (float)d.d_det[0], v0, (float)d.d_det[1], (float)(d.DSD * d.DSD));
            TIGRE_LAUNCHED("fdk_filter_kernel");
            return TIGRE_OK;
        });
    }
    if (status == TIGRE_OK)
        status = backward_impl(g, filt, TIGRE_F32, vol, vt, 0, na, TIGRE_BP_FDK, 0, st);
    dev_free(filt, st);
    dev_free(dtab, st);
    return status;
}

}  // namespace tigre

extern "C" tigre_status tigre_fdk(tigre_geometry_t geo, const void* proj, tigre_dtype proj_dtype,
                                  void* vol, tigre_dtype vol_dtype, void* cuda_stream)
{
    return tigre::fdk_impl(geo, proj, proj_dtype, vol, vol_dtype, (cudaStream_t)cuda_stream);
}
