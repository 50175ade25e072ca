// Ray-voxel intersection (Siddon) projector -- the paper's other projector
// (Sec. 2.1 names both; Sec. 3.1 times this one, TIGRE's default) -- and its exact
// transpose.
//
// The volume is piecewise constant: voxel (i, j, k) fills the index-space box
// [i-1/2, i+1/2] x [j-1/2, j+1/2] x [k-1/2, k+1/2].  A ray's value is
// |P - S| times the sum over the voxels the segment S->P crosses of (the
// parameter length of the crossing) x (the voxel's value).
//
// One thread per ray walks the crossed voxels in order.  Each boundary
// crossing parameter is recomputed from the index of its plane,
// t = (plane - src) / r, instead of being advanced by repeated increments, so
// crossings keep FP32 accuracy along rays thousands of voxels long.  The walk
// reads the zero-padded layout that the angle's forward projection uses (x or
// y fastest, chosen per angle), so neighbouring lanes read neighbouring
// addresses; a walk that rounds one voxel past the exit reads padding zeros
// (the padding is two voxels deep).
#include <algorithm>
#include <cmath>

#include "ray.cuh"

namespace tigre {
namespace {

// Walks the voxels of the ray to pixel (p, q), calling visit(idx, dt) with the
// element index of each voxel in the padded layout and the parameter length
// dt of the crossing.  Returns |P - S| (mm), or 0 for a ray that misses.
template <typename Visit>
__device__ __forceinline__ float siddon_walk(const FwdAngle* __restrict__ P, const FwdConst& c,
                                             int p, int q, Visit&& visit)
{
    const int layout = P->layout;
    const int n[3] = {layout ? c.ny : c.nx, layout ? c.nx : c.ny, c.nz};
    const float fp = (float)p, fq = (float)q;
    const float r[3] = {fmaf(fq, P->dq[0], fmaf(fp, P->dp[0], P->base[0])),
                        fmaf(fq, P->dq[1], fmaf(fp, P->dp[1], P->base[1])),
                        fmaf(fq, P->dq[2], fmaf(fp, P->dp[2], P->base[2]))};
    float t0 = 0.0f, t1 = 1.0f;
    float inv[3], cst[3], tn[3], pl[3], stp[3];
    int i[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = -0.5f, hi = (float)n[a] - 0.5f;
        if (r[a] != 0.0f) {
            inv[a] = 1.0f / r[a];
            const float ta = (lo - P->src[a]) * inv[a], tb = (hi - P->src[a]) * inv[a];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else {
            inv[a] = 0.0f;
            if (!(P->src[a] > lo && P->src[a] < hi)) t1 = -1.0f;
        }
    }
    if (!(t1 > t0)) return 0.0f;
    int idx = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // Voxel at the entry point (the entry face rounds into the volume).
        const int v = (int)floorf(fmaf(t0, r[a], P->src[a]) + 0.5f);
        i[a] = min(max(v, 0), n[a] - 1);
        stp[a] = r[a] > 0.0f ? 1.0f : -1.0f;
        pl[a] = (float)i[a] + 0.5f * stp[a];  // next boundary plane along the ray
        cst[a] = -P->src[a] * inv[a];
        tn[a] = r[a] != 0.0f ? fmaf(pl[a], inv[a], cst[a]) : 3.0e38f;
    }
    const int PF = n[0] + 2 * kPad, PFM = PF * (n[1] + 2 * kPad);
    idx = ((i[2] + kPad) * (n[1] + 2 * kPad) + (i[1] + kPad)) * PF + (i[0] + kPad);
    const int s0 = r[0] > 0.0f ? 1 : -1, s1 = r[1] > 0.0f ? PF : -PF, s2 = r[2] > 0.0f ? PFM : -PFM;
    const int cap = n[0] + n[1] + n[2] + 4;
    float t = t0;
    for (int it = 0; it < cap; ++it) {
        // A plane already behind t (an entry that rounded onto the wrong
        // side of it) is crossed with zero length.
        const float e = fmaxf(fminf(fminf(tn[0], tn[1]), fminf(tn[2], t1)), t);
        visit(idx, e - t);
        if (e >= t1) break;
        t = e;
        const bool a0 = tn[0] <= tn[1] && tn[0] <= tn[2];
        const bool a1 = !a0 && tn[1] <= tn[2];
        const bool a2 = !a0 && !a1;
        idx += a0 ? s0 : (a1 ? s1 : s2);
        if (a0) {
            pl[0] += stp[0];
            tn[0] = fmaf(pl[0], inv[0], cst[0]);
        } else if (a1) {
            pl[1] += stp[1];
            tn[1] = fmaf(pl[1], inv[1], cst[1]);
        } else if (a2) {
            pl[2] += stp[2];
            tn[2] = fmaf(pl[2], inv[2], cst[2]);
        }
    }
    const float u = fmaf(fp, c.du, c.u0), v = fmaf(fq, c.dv, c.v0);
    return sqrtf(c.dsd2 + u * u + v * v);
}

template <typename TV, typename TP>
__global__ void __launch_bounds__(256) siddon_fwd_kernel(const TV* __restrict__ vxy,
                                                         const TV* __restrict__ vyx,
                                                         TP* __restrict__ proj,
                                                         const FwdAngle* __restrict__ params,
                                                         FwdConst c, int a_first,
                                                         const int* __restrict__ order)
{
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int q = blockIdx.z * blockDim.y + threadIdx.y;
    const int a = order ? order[blockIdx.y] : (int)blockIdx.y;
    if (p >= c.nu || q >= c.nv) return;
    const FwdAngle* P = params + a_first + a;
    const TV* __restrict__ vol = P->layout ? vyx : vxy;
    float acc = 0.0f;
    const float seg = siddon_walk(P, c, p, q, [&](int idx, float dt) {
        acc = fmaf(dt, to_f32<TV>(__ldg(vol + idx)), acc);
    });
    proj[((int64_t)a * c.nv + q) * c.nu + p] = from_f32<TP>(acc * seg);
}

// Exact transpose: each crossing adds seg * dt * y into its voxel of the
// padded accumulator of the angle's layout.
template <typename TP>
__global__ void __launch_bounds__(256) siddon_scatter_kernel(const TP* __restrict__ proj,
                                                             float* __restrict__ acc_xy,
                                                             float* __restrict__ acc_yx,
                                                             const FwdAngle* __restrict__ params,
                                                             FwdConst c, int a_first)
{
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int q = blockIdx.z * blockDim.y + threadIdx.y;
    const int a = blockIdx.y;
    if (p >= c.nu || q >= c.nv) return;
    const float y = to_f32<TP>(proj[((int64_t)a * c.nv + q) * c.nu + p]);
    if (y == 0.0f) return;
    const FwdAngle* P = params + a_first + a;
    float* __restrict__ acc = P->layout ? acc_yx : acc_xy;
    // The length |P - S| is known only at the end of the walk's setup; it is
    // a per-ray constant, so it is computed first and folded into y.
    const float u = fmaf((float)p, c.du, c.u0), v = fmaf((float)q, c.dv, c.v0);
    const float ys = y * sqrtf(c.dsd2 + u * u + v * v);
    siddon_walk(P, c, p, q, [&](int idx, float dt) {
        if (dt > 0.0f) atomicAdd(acc + idx, dt * ys);
    });
}

}  // namespace

template <typename TV, typename TP>
tigre_status launch_siddon_forward(tigre_geometry* g, const TV* vxy, const TV* vyx, TP* proj,
                                   int64_t a0, int64_t na, const int* order, cudaStream_t st)
{
    const FwdConst c = make_fwd_const(g);
    ProfScope prof(kProfForward, st);
    for (int64_t s = 0; s < na; s += 65535) {
        const int64_t cnt = std::min<int64_t>(65535, na - s);
        dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
        siddon_fwd_kernel<TV, TP><<<grid, dim3(32, 8), 0, st>>>(
            vxy, vyx, proj + s * (int64_t)c.nu * c.nv, (const FwdAngle*)g->fwd_params.ptr, c,
            (int)(a0 + s), order);
        TIGRE_LAUNCHED("siddon_fwd_kernel");
    }
    return TIGRE_OK;
}

template <typename TP>
tigre_status launch_siddon_scatter(tigre_geometry* g, const TP* proj, float* acc_xy, float* acc_yx,
                                   int64_t a0, int64_t na, cudaStream_t st)
{
    const FwdConst c = make_fwd_const(g);
    for (int64_t s = 0; s < na; s += 65535) {
        const int64_t cnt = std::min<int64_t>(65535, na - s);
        dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
        siddon_scatter_kernel<TP><<<grid, dim3(32, 8), 0, st>>>(
            proj + s * (int64_t)c.nu * c.nv, acc_xy, acc_yx, (const FwdAngle*)g->fwd_params.ptr,
            c, (int)(a0 + s));
        TIGRE_LAUNCHED("siddon_scatter_kernel");
    }
    return TIGRE_OK;
}

#define TIGRE_SIDDON_FWD(TV, TP)                                                              \
    template tigre_status launch_siddon_forward<TV, TP>(tigre_geometry*, const TV*, const TV*, \
                                                        TP*, int64_t, int64_t, const int*,     \
                                                        cudaStream_t);
#define TIGRE_SIDDON_FWD_ALL(TV)      \
    TIGRE_SIDDON_FWD(TV, float)       \
    TIGRE_SIDDON_FWD(TV, __nv_bfloat16) \
    TIGRE_SIDDON_FWD(TV, __half)
TIGRE_SIDDON_FWD_ALL(float)
TIGRE_SIDDON_FWD_ALL(__nv_bfloat16)
TIGRE_SIDDON_FWD_ALL(__half)
template tigre_status launch_siddon_scatter<float>(tigre_geometry*, const float*, float*, float*,
                                                   int64_t, int64_t, cudaStream_t);
template tigre_status launch_siddon_scatter<__nv_bfloat16>(tigre_geometry*, const __nv_bfloat16*,
                                                           float*, float*, int64_t, int64_t,
                                                           cudaStream_t);
template tigre_status launch_siddon_scatter<__half>(tigre_geometry*, const __half*, float*, float*,
                                                    int64_t, int64_t, cudaStream_t);

}  // namespace tigre

extern "C" tigre_status tigre_geometry_set_projector(tigre_geometry_t g, int projector)
{
    if (!g || (projector != TIGRE_PROJ_INTERPOLATED && projector != TIGRE_PROJ_SIDDON))
        return tigre::fail(TIGRE_ERR_INVALID_ARG, "projector must be INTERPOLATED or SIDDON");
    g->projector = projector;
    return TIGRE_OK;
}
