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
    // Rays whose sample count FP32 gets wrong (see setup_ray): entries
    // [exc_start[row], exc_start[row + 1]) of exc for the detector row
    // row = angle * nv + q.
    const int* exc_start;
    const RayException* exc;
};

FwdConst make_fwd_const(const tigre_geometry* g);

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

// Bilinear interpolation of one cell of a plane, as every forward kernel
// takes it.  With taps a = (f, m), b = (f+1, m), c = (f, m+1), d = (f+1, m+1),
// the coefficients are (a, b - a, c - a, (d - c) - (b - a)) and the value at
// fractions (af, am) is a + af (b - a) + am ((c - a) + af ((d - c) - (b - a))),
// three FMAs.
__host__ __device__ __forceinline__ float4 bilinear_coefficients(float a, float b, float c, float d)
{
    const float df = b - a;
    return make_float4(a, df, c - a, (d - c) - df);
}
__device__ __forceinline__ float bilinear_value(const float4& e, float af, float am)
{
    return fmaf(am, fmaf(af, e.w, e.z), fmaf(af, e.y, e.x));
}

// The same split with the integer part left biased: b = i + 0x4B000000, the
// bit pattern of the rounded sum.  An index summed over several axes then
// removes the biases with one subtraction (modulo 2^32).
__device__ __forceinline__ void split_bits(float x, uint32_t& b, float& f)
{
    const float m = __fadd_rn(x, 8388607.5f);
    b = (uint32_t)__float_as_int(m);
    f = __fsub_rn(x, __fsub_rn(m, 8388608.0f));
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

// The FP32 set-up of ray (p, q): clip to the support (-1, n) per axis,
// chord length len (mm) and K = max(1, ceil(len / step)), 0 for a miss.
// Every operation is written with an explicit rounding (no contraction left
// to the compiler), so that each kernel that inlines it gets the same bits:
// the exception table below is built from this very computation.
__device__ __forceinline__ int ray_clip_f32(const FwdAngle* __restrict__ P, const FwdConst& c,
                                            int p, int q, const int n[3], float r[3], float& t0,
                                            float& t1, float& len)
{
    const float fp = (float)p, fq = (float)q;
    t0 = 0.0f;
    t1 = 1.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r[a] = fmaf(fq, P->dq[a], fmaf(fp, P->dp[a], P->base[a]));
        const float s = P->src[a];
        if (r[a] != 0.0f) {
            const float inv = __frcp_rn(r[a]);
            const float ta = __fmul_rn(__fsub_rn(-1.0f, s), inv);
            const float tb = __fmul_rn(__fsub_rn((float)n[a], s), inv);
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (!(s > -1.0f && s < (float)n[a])) {
            t1 = -1.0f;  // parallel to the slab and outside it: empty
        }
    }
    if (!(t1 > t0)) return 0;
    const float u = fmaf(fp, c.du, c.u0), v = fmaf(fq, c.dv, c.v0);
    len = __fmul_rn(__fsub_rn(t1, t0), __fsqrt_rn(fmaf(v, v, fmaf(u, u, c.dsd2))));
    return max(1, (int)ceilf(__fmul_rn(len, c.inv_step)));
}

// A ray of the geometry: its first sample, step, weight and sample count.
// The count is the quadrature's K = max(1, ceil(len / step - 1e-9)) with len
// from the exact chord.  FP32 carries len / step only to a few 1e-4 (more for
// rays that cross a face at a shallow angle), so for about one ray in a few
// thousand its ceil differs; those rays were found once per geometry by
// setting every ray up in FP64 as well, and their FP64 clip and count are
// looked up here.
__device__ __forceinline__ void setup_ray(const FwdAngle* __restrict__ P, const FwdConst& c,
                                          int p, int q, Ray& R)
{
    R.layout = P->layout;
    R.nf = R.layout ? c.ny : c.nx;
    R.nm = R.layout ? c.nx : c.ny;
    R.ns = c.nz;
    const int n[3] = {R.nf, R.nm, R.ns};
    float r[3], t0, t1, len;
    R.K = ray_clip_f32(P, c, p, q, n, r, t0, t1, len);
    R.h = 0.0f;
    R.ok = true;
    const int row = P->index * c.nv + q;
    for (int e = c.exc_start[row], end = c.exc_start[row + 1]; e < end; ++e) {
        const RayException x = c.exc[e];
        if (x.p == p) {
            R.K = x.K;
            t0 = x.t0;
            t1 = x.t1;
            len = x.len;
            break;
        }
    }
    if (R.K == 0) return;
    if (!(R.K <= c.kmax)) {
        R.ok = false;
        return;
    }
    const float invK = 1.0f / (float)R.K;
    const float dt = (t1 - t0) * invK;
    const float tm = fmaf(0.5f, dt, t0);
    R.h = len * invK;
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
