// Ray setup shared by the forward projector and its exact transpose: both
// must place exactly the same samples (count K, step h, positions) on a ray.
#pragma once

#include "common.cuh"

namespace tigre {

struct FwdConst {
    int nx, ny, nz;
    int nu, nv;
    float u0, v0;    // detector coordinates (mm) of pixel (0, 0), offsets included
    float du, dv;    // pixel pitch (mm)
    float dsd2;      // DSD^2 (mm^2)
    float inv_step;  // 1 / (accuracy * min d)
    int kmax;        // more samples than the support's diagonal allows = corrupt ray
};

FwdConst make_fwd_const(const tigre_geometry_desc& d);

// Integer part and fraction of x for 0.5 <= x < 2^22 (below about 0.25 the
// sum leaves the [2^23, 2^24) binade and the split is wrong, so callers keep
// x >= 0.5).  For x exactly integral the split may be (x - 1, 1.0); linear
// interpolation is continuous there, so the interpolated value is unchanged.
__device__ __forceinline__ void split_floor(float x, int& i, float& f)
{
    const float m = __fadd_rn(x, 8388607.5f);
    i = __float_as_int(m) - 0x4B000000;
    f = __fsub_rn(x, __fsub_rn(m, 8388608.0f));
}

// Clip parameter range [t0, t1] of src + t r to (-1, n) along one axis.
__device__ __forceinline__ void clip_axis(float src, float r, int n, float& t0, float& t1)
{
    const float lo = -1.0f, hi = (float)n;
    if (r != 0.0f) {
        const float inv = 1.0f / r;
        const float ta = (lo - src) * inv, tb = (hi - src) * inv;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    } else if (!(src > lo && src < hi)) {
        t1 = -1.0f;  // parallel to the slab and outside it: empty
    }
}

// One ray in the padded index coordinates of its angle's layout.
struct Ray {
    float x0[3];  // first sample (f, m, s), padded coordinates
    float d[3];   // step between samples
    float h;      // sample weight (mm)
    int K;        // number of samples (0: the ray misses the support)
    int nf, nm, ns;
    int layout;
    bool ok;      // all samples provably inside the padded volume
};

__device__ __forceinline__ void setup_ray(const FwdAngle* __restrict__ P, const FwdConst& c,
                                          int p, int q, Ray& R)
{
    R.layout = P->layout;
    R.nf = R.layout ? c.ny : c.nx;
    R.nm = R.layout ? c.nx : c.ny;
    R.ns = c.nz;
    const float fp = (float)p, fq = (float)q;
    const float r[3] = {fmaf(fq, P->dq[0], fmaf(fp, P->dp[0], P->base[0])),
                        fmaf(fq, P->dq[1], fmaf(fp, P->dp[1], P->base[1])),
                        fmaf(fq, P->dq[2], fmaf(fp, P->dp[2], P->base[2]))};
    float t0 = 0.0f, t1 = 1.0f;
    clip_axis(P->src[0], r[0], R.nf, t0, t1);
    clip_axis(P->src[1], r[1], R.nm, t0, t1);
    clip_axis(P->src[2], r[2], R.ns, t0, t1);
    R.K = 0;
    R.ok = true;
    if (!(t1 > t0)) return;
    const float u = fmaf(fp, c.du, c.u0), v = fmaf(fq, c.dv, c.v0);
    const float len = (t1 - t0) * sqrtf(c.dsd2 + u * u + v * v);
    // K = ceil(len / step); the small guard keeps exact multiples exact.
    R.K = max(1, (int)ceilf(fmaf(len, c.inv_step, -1e-3f)));
    if (!(R.K <= c.kmax)) {
        R.ok = false;
        return;
    }
    const float invK = 1.0f / (float)R.K;
    const float dt = (t1 - t0) * invK;
    const float tm = fmaf(0.5f, dt, t0);
    R.h = len * invK;
    const int n[3] = {R.nf, R.nm, R.ns};
    const float kl = (float)(R.K - 1);
    for (int a = 0; a < 3; ++a) {
        R.x0[a] = fmaf(tm, r[a], P->src[a]) + (float)kPad;
        R.d[a] = dt * r[a];
        // Samples are affine in k: bounding both ends bounds them all.
        const float e = fmaf(kl, R.d[a], R.x0[a]);
        R.ok = R.ok && fminf(R.x0[a], e) >= 0.5f && fmaxf(R.x0[a], e) <= (float)n[a] + 2.5f;
    }
}

}  // namespace tigre
