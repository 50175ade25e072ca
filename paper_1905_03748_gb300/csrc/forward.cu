// Interpolated ray-driven forward projector A x (paper Sec. 2.1, interpolated
// projection; one thread per detector pixel as in the paper's kernel
// organisation, Fig. 2).
//
// proj[a][q][p] = h * sum_{k<K} f~(src + t_k (P - S)/d), f~ the trilinear
// interpolant of the volume with zero outside, t_k the midpoints of K equal
// steps over the part of the ray inside the interpolant's support [-1, n],
// K = ceil(len / (accuracy * min d)), h = len / K.
//
// GB300 design:
//  * The volume is copied once per call into two zero-padded layouts (x
//    fastest, and y fastest).  Each angle reads the layout whose fastest axis
//    is closest to e_u, so the 32 rays of a warp (adjacent pixels of one
//    detector row) gather from adjacent addresses: each tap load touches 1-2
//    cache lines per warp.  The two-voxel zero border removes every bounds
//    check from the sample loop.
//  * Grid order: u-tiles fastest, then angles, then detector row bands.  The
//    blocks resident at any time belong to one row band and many angles and
//    read the same z-range of the volume.
//  * Angle pairs: when neighbouring angles are close (the rays of one pixel at
//    the two angles stay within a few voxels), a warp holds 16 pixels at two
//    angles instead of 32 pixels at one, and its gathers touch fewer cache
//    lines (3.3-3.9 % faster at 512^3 x 360 and 1024^3 x 360 / 720).
//  * floor() without conversion instructions (split_floor).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "quad.cuh"
#include "ray.cuh"

namespace tigre {

FwdConst make_fwd_const(const tigre_geometry* g)
{
    const tigre_geometry_desc& d = g->desc;
    FwdConst c;
    c.nx = (int)d.n_voxel[0];
    c.ny = (int)d.n_voxel[1];
    c.nz = (int)d.n_voxel[2];
    c.nu = (int)d.n_det[0];
    c.nv = (int)d.n_det[1];
    c.u0 = (float)(-0.5 * (double)(d.n_det[0] - 1) * d.d_det[0] + d.off_det[0]);
    c.v0 = (float)(-0.5 * (double)(d.n_det[1] - 1) * d.d_det[1] + d.off_det[1]);
    c.du = (float)d.d_det[0];
    c.dv = (float)d.d_det[1];
    c.dsd2 = (float)(d.DSD * d.DSD);
    const double dmin = std::min(d.d_voxel[0], std::min(d.d_voxel[1], d.d_voxel[2]));
    const double step = d.accuracy * dmin;
    c.inv_step = (float)(1.0 / step);
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = (double)(d.n_voxel[a] + 1) * d.d_voxel[a];
        diag2 += e * e;
    }
    c.kmax = (int)std::min(std::ceil(std::sqrt(diag2) / step) + 4.0, 1.0e8);
    c.exc_start = (const int*)g->ray_exc_start.ptr;
    c.exc = (const RayException*)g->ray_exc.ptr;
    return c;
}

// The clip of a ray to the support and its sample count in FP64, from the
// FP64 vectors of its angle: t0, t1 (rounded to FP32) and the chord length
// len (mm), K = max(1, ceil(len / step - 1e-9)) as the quadrature defines it;
// 0 when the ray misses the support.
__device__ __forceinline__ int ray_clip_f64(const FwdAngle64* __restrict__ P, int nf, int nm, int ns,
                                         int p, int q, double u0, double v0, double du, double dv,
                                         double dsd2, double inv_step, float* t0o, float* t1o,
                                         float* leno)
{
    const double fp = (double)p, fq = (double)q;
    const int n[3] = {nf, nm, ns};
    double t0 = 0.0, t1 = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double r = fma(fq, P->dq[a], fma(fp, P->dp[a], P->base[a]));
        const double s = P->src[a];
        if (r != 0.0) {
            const double ta = (-1.0 - s) / r, tb = ((double)n[a] - s) / r;
            t0 = fmax(t0, fmin(ta, tb));
            t1 = fmin(t1, fmax(ta, tb));
        } else if (!(s > -1.0 && s < (double)n[a])) {
            return 0;
        }
    }
    if (!(t1 > t0)) return 0;
    const double u = fma(fp, du, u0), v = fma(fq, dv, v0);
    const double len = (t1 - t0) * sqrt(dsd2 + u * u + v * v);
    *t0o = (float)t0;
    *t1o = (float)t1;
    *leno = (float)len;
    return max(1, (int)ceil(fma(len, inv_step, -1e-9)));
}

// FP64 constants of the detector frame for ray_clip_f64.
struct FwdConst64 {
    double u0, v0, du, dv, dsd2, inv_step;
};

// Every ray of angles [a_first, a_first + gridDim.y): set up in FP32 exactly
// as the projector kernels do and in FP64; a ray whose counts differ is an
// exception.  Pass 0 counts them per detector row, pass 1 (FILL) writes them
// into their row's slots.
template <bool FILL>
__global__ void __launch_bounds__(256) ray_exception_kernel(
    const FwdAngle* __restrict__ params, const FwdAngle64* __restrict__ p64, FwdConst c,
    FwdConst64 d, int a_first, int* __restrict__ count, const int* __restrict__ start,
    RayException* __restrict__ out)
{
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int q = blockIdx.z * blockDim.y + threadIdx.y;
    const int a = a_first + (int)blockIdx.y;
    if (p >= c.nu || q >= c.nv) return;
    const FwdAngle* P = params + a;
    const int layout = P->layout;
    const int n[3] = {layout ? c.ny : c.nx, layout ? c.nx : c.ny, c.nz};
    float r[3], t0 = 0.0f, t1 = 0.0f, len = 0.0f;
    const int K32 = ray_clip_f32(P, c, p, q, n, r, t0, t1, len);
    float t0d = 0.0f, t1d = 0.0f, lend = 0.0f;
    const int K64 = ray_clip_f64(p64 + a, n[0], n[1], n[2], p, q, d.u0, d.v0, d.du, d.dv, d.dsd2,
                                 d.inv_step, &t0d, &t1d, &lend);
    if (K64 == K32) return;
    const int row = a * c.nv + q;
    const int slot = atomicAdd(count + row, 1);
    if (FILL) out[start[row] + slot] = RayException{p, K64, t0d, t1d, lend};
}

tigre_status build_ray_exceptions(tigre_geometry* g)
{
    const tigre_geometry_desc& d = g->desc;
    const int64_t na = (int64_t)g->angles.size();
    const int64_t rows = na * d.n_det[1];
    if (rows >= (int64_t)INT32_MAX) return fail(TIGRE_ERR_UNSUPPORTED, "too many detector rows");
    TIGRE_TRY(g->ray_exc_start.ensure(sizeof(int) * (size_t)(rows + 1)));
    DeviceBuffer counts;
    TIGRE_TRY(counts.ensure(sizeof(int) * (size_t)rows));
    FwdConst c = make_fwd_const(g);
    c.exc_start = nullptr;
    c.exc = nullptr;
    const double dmin = std::min(d.d_voxel[0], std::min(d.d_voxel[1], d.d_voxel[2]));
    const FwdConst64 c64{-0.5 * (double)(d.n_det[0] - 1) * d.d_det[0] + d.off_det[0],
                         -0.5 * (double)(d.n_det[1] - 1) * d.d_det[1] + d.off_det[1],
                         d.d_det[0], d.d_det[1], d.DSD * d.DSD, 1.0 / (d.accuracy * dmin)};
    const FwdAngle* params = (const FwdAngle*)g->fwd_params.ptr;
    const FwdAngle64* p64 = (const FwdAngle64*)g->fwd_params64.ptr;
    auto pass = [&](bool fill) -> tigre_status {
        TIGRE_CUDA(cudaMemset(counts.ptr, 0, sizeof(int) * (size_t)rows));
        for (int64_t s = 0; s < na; s += 65535) {
            const int64_t cnt = std::min<int64_t>(65535, na - s);
            dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
            if (fill)
                ray_exception_kernel<true><<<grid, dim3(32, 8)>>>(
                    params, p64, c, c64, (int)s, (int*)counts.ptr, (const int*)g->ray_exc_start.ptr,
                    (RayException*)g->ray_exc.ptr);
            else
                ray_exception_kernel<false><<<grid, dim3(32, 8)>>>(params, p64, c, c64, (int)s,
                                                                    (int*)counts.ptr, nullptr,
                                                                    nullptr);
            TIGRE_LAUNCHED("ray_exception_kernel");
        }
        return TIGRE_OK;
    };
    TIGRE_TRY(pass(false));
    std::vector<int> start((size_t)rows + 1);
    TIGRE_CUDA(cudaMemcpy(start.data() + 1, counts.ptr, sizeof(int) * (size_t)rows,
                          cudaMemcpyDeviceToHost));
    start[0] = 0;
    int64_t total = 0;
    for (int64_t r = 0; r < rows; ++r) {
        total += start[(size_t)r + 1];
        if (total >= (int64_t)INT32_MAX) return fail(TIGRE_ERR_UNSUPPORTED, "too many exceptions");
        start[(size_t)r + 1] = (int)total;
    }
    TIGRE_CUDA(cudaMemcpy(g->ray_exc_start.ptr, start.data(), sizeof(int) * (size_t)(rows + 1),
                          cudaMemcpyHostToDevice));
    g->n_ray_exc = total;
    if (total > 0) {
        TIGRE_TRY(g->ray_exc.ensure(sizeof(RayException) * (size_t)total));
        TIGRE_TRY(pass(true));
    }
    TIGRE_CUDA(cudaDeviceSynchronize());
    counts.release();
    return TIGRE_OK;
}

template <typename T>
__device__ __forceinline__ float ld(const T* p)
{
    return to_f32<T>(__ldg(p));
}

// Trilinear sample k of ray R from the padded volume.
template <typename TV>
__device__ __forceinline__ float tri_sample(const TV* __restrict__ vol, const Ray& R, float kf,
                                            int PF, int PFM)
{
    int i_f, i_m, i_s;
    float af, am, as;
    split_floor(fmaf(kf, R.d[0], R.x0[0]), i_f, af);
    split_floor(fmaf(kf, R.d[1], R.x0[1]), i_m, am);
    split_floor(fmaf(kf, R.d[2], R.x0[2]), i_s, as);
    const TV* b = vol + (i_s * PFM + i_m * PF + i_f);
    const float v000 = ld(b), v100 = ld(b + 1);
    const float v010 = ld(b + PF), v110 = ld(b + PF + 1);
    const float v001 = ld(b + PFM), v101 = ld(b + PFM + 1);
    const float v011 = ld(b + PFM + PF), v111 = ld(b + PFM + PF + 1);
    const float c0 = bilinear_value(bilinear_coefficients(v000, v100, v010, v110), af, am);
    const float c1 = bilinear_value(bilinear_coefficients(v001, v101, v011, v111), af, am);
    return fmaf(as, c1 - c0, c0);
}

// One warp = 32 adjacent pixels of a detector row.  Their rays are nearly
// parallel, but each starts its samples on its own entry face of the box, so
// the k-th samples of neighbouring lanes sit at different depths and a
// warp-wide gather would touch many rows.  The warp therefore marches in
// depth order along the layout's middle axis (the main direction of the
// rays): slab j holds main-axis coordinates [Y0 + j D, Y0 + (j+1) D) with D the
// smallest per-sample advance in the warp, so each lane has at most one sample
// per slab and all lanes gather at about the same depth.  Every lane still
// adds its samples in the order k = 0..K-1, so the sums are identical to a
// per-lane loop.
template <typename TV, typename TP>
__global__ void __launch_bounds__(256) fwd_l1_kernel(const TV* __restrict__ vxy,
                                                     const TV* __restrict__ vyx,
                                                     TP* __restrict__ proj,
                                                     const FwdAngle* __restrict__ params,
                                                     FwdConst c, int a_first,
                                                     const int* __restrict__ order)
{
    const unsigned full = 0xffffffffu;
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int q = blockIdx.z * blockDim.y + threadIdx.y;
    const int a = order ? order[blockIdx.y] : (int)blockIdx.y;
    const bool inside = p < c.nu && q < c.nv;

    Ray R;
    R.K = 0;
    R.ok = true;
    if (inside) setup_ray(params + a_first + a, c, p, q, R);
    const bool active = inside && R.ok && R.K > 0;
    const unsigned act = __ballot_sync(full, active);
    const int layout = params[a_first + a].layout;  // uniform per block
    const TV* __restrict__ vol = layout ? vyx : vxy;
    const int PF = (layout ? c.ny : c.nx) + 2 * kPad;
    const int PFM = PF * ((layout ? c.nx : c.ny) + 2 * kPad);

    float acc = 0.0f;
    if (act) {
        const unsigned pos = __ballot_sync(full, active && R.d[1] > 0.0f);
        const unsigned neg = __ballot_sync(full, active && R.d[1] < 0.0f);
        int k = 0;
        float kf = 0.0f;
        if (pos == act || neg == act) {
            const float sgn = pos == act ? 1.0f : -1.0f;
            const float y0 = sgn * R.x0[1], dy = sgn * R.d[1];
            const float y1 = fmaf((float)(R.K - 1), dy, y0);
            float D = active ? dy : 3.0e38f, Y0 = active ? y0 : 3.0e38f;
            float Y1 = active ? y1 : -3.0e38f;
            int kmax = active ? R.K : 0;
            for (int o = 16; o > 0; o >>= 1) {
                D = fminf(D, __shfl_xor_sync(full, D, o));
                Y0 = fminf(Y0, __shfl_xor_sync(full, Y0, o));
                Y1 = fmaxf(Y1, __shfl_xor_sync(full, Y1, o));
                kmax = max(kmax, __shfl_xor_sync(full, kmax, o));
            }
            // A warp whose rays disagree wildly (a near-grazing ray makes D
            // tiny) skips the march; the tail loop below does the work.
            const float ns = (Y1 - Y0) / D;
            const int nslab = ns < (float)(2 * kmax + 64) ? (int)ns + 1 : 0;
            for (int j = 1; j <= nslab; ++j) {
                const float bound = fmaf((float)j, D, Y0);
                if (k < R.K && fmaf(kf, dy, y0) < bound) {
                    acc += tri_sample(vol, R, kf, PF, PFM);
                    ++k;
                    kf += 1.0f;
                }
            }
        }
        // Samples not consumed above (mixed directions, or rounding at a slab
        // edge) finish in order here.
        for (; active && k < R.K; ++k, kf += 1.0f) acc += tri_sample(vol, R, kf, PF, PFM);
    }
    if (!inside) return;
    const float out = !R.ok ? __int_as_float(0x7fc00000)  // NaN: ray failed the bounds proof
                            : acc * R.h;
    proj[((int64_t)a * c.nv + q) * c.nu + p] = from_f32<TP>(out);
}

// ----------------------------------------------------------- quad layout
// Element (s, m, f) of a quad volume holds the four taps of the cell's lower
// s-plane: (P[s][m][f], P[s][m][f+1], P[s][m+1][f], P[s][m+1][f+1]) of the
// zero-padded layout P.  A trilinear sample is then two aligned loads (planes
// s and s+1) instead of eight scalar ones (element types: quad.cuh).
//
// Elements hold the cell's bilinear coefficients (bilinear_coefficients) in
// FP32 for every storage type, formed from the taps converted to FP32 in the
// same operations the scalar kernels use, so a plane's bilinear value is three
// FMAs (bilinear_value) after one load.
__device__ __forceinline__ float4 load_fquad(const float4* p) { return load_quad(p); }

// Build the quad volume of one layout straight from the caller's volume (no
// padded copy): with P(s, m, f) the zero-bordered layout (vol[s-2][m-2][f-2]
// for layout 0, x fastest; vol[s-2][f-2][m-2] for layout 1, y fastest; zero
// outside), element (s, m, f) = (P(s,m,f), P(s,m,f+1), P(s,m+1,f),
// P(s,m+1,f+1)).  A block makes a 32 x 32 tile of one plane from a 33 x 33
// tile of P staged in shared memory, read along x (coalesced) in either
// layout; blockIdx = (f tile, m tile, s).
template <typename T>
__global__ void __launch_bounds__(256) quad_from_vol_kernel(const T* __restrict__ vol,
                                                            typename QuadOf<T>::type* __restrict__ out,
                                                            int nx, int ny, int nz, int layout)
{
    __shared__ T tile[33][33];
    const int PF = (layout ? ny : nx) + 2 * kPad, PM = (layout ? nx : ny) + 2 * kPad;
    const int f0 = blockIdx.x * 32, m0 = blockIdx.y * 32, s = blockIdx.z;
    const int z = s - kPad;
    const T zero = from_f32<T>(0.0f);
    const bool zin = (unsigned)z < (unsigned)nz;
    const T* plane = vol + (int64_t)(zin ? z : 0) * nx * ny;
    // tile[i][j] = P(s, m0 + i, f0 + j), i, j in [0, 33)
    for (int k = threadIdx.y * 32 + threadIdx.x; k < 33 * 33; k += 256) {
        int i, j;
        if (layout == 0) {  // consecutive threads: consecutive f = x
            i = k / 33;
            j = k - i * 33;
        } else {            // consecutive threads: consecutive m = x
            j = k / 33;
            i = k - j * 33;
        }
        const int m = m0 + i - kPad, f = f0 + j - kPad;
        const int x = layout ? m : f, y = layout ? f : m;
        tile[i][j] = (zin && (unsigned)x < (unsigned)nx && (unsigned)y < (unsigned)ny)
                         ? plane[(int64_t)y * nx + x]
                         : zero;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int m = m0 + i, f = f0 + threadIdx.x;
        if (m >= PM || f >= PF) continue;
        // P beyond the padded layout (f + 1 == PF or m + 1 == PM) is zero too
        const T a = tile[i][threadIdx.x], b = tile[i][threadIdx.x + 1];
        const T c = tile[i + 1][threadIdx.x], d = tile[i + 1][threadIdx.x + 1];
        typename QuadOf<T>::type* o = out + ((int64_t)s * PM + m) * PF + f;
        *o = bilinear_coefficients(to_f32<T>(a), to_f32<T>(b), to_f32<T>(c), to_f32<T>(d));
    }
}

template <typename T>
tigre_status build_quads(const tigre_geometry_desc& d, const T* vol, typename QuadOf<T>::type* out,
                         int layout, cudaStream_t st)
{
    const int nx = (int)d.n_voxel[0], ny = (int)d.n_voxel[1], nz = (int)d.n_voxel[2];
    const int PF = (layout ? ny : nx) + 2 * kPad, PM = (layout ? nx : ny) + 2 * kPad;
    if (nz + 2 * kPad > 65535) return fail(TIGRE_ERR_UNSUPPORTED, "volume too deep for one launch");
    dim3 grid((unsigned)((PF + 31) / 32), (unsigned)((PM + 31) / 32), (unsigned)(nz + 2 * kPad));
    quad_from_vol_kernel<T><<<grid, dim3(32, 8), 0, st>>>(vol, out, nx, ny, nz, layout);
    TIGRE_LAUNCHED("quad_from_vol_kernel");
    return TIGRE_OK;
}

// Bias of a quad element index built from split_bits parts: the three
// splits' 0x4B000000 and the slab's first plane, modulo 2^32.
__host__ __device__ __forceinline__ uint32_t quad_index_bias(int PF, int PFM, int s_off)
{
    return 0x4B000000u * (uint32_t)(PFM + PF + 1) + (uint32_t)s_off * (uint32_t)PFM;
}

// Trilinear sample kf of a ray from the quad volume qv; ym = x0[1] + kf d[1]
// (the march's depth coordinate, which the caller has already formed).
template <typename TV>
__device__ __forceinline__ float tri_sample_quad(const typename QuadOf<TV>::type* __restrict__ qv,
                                                 const Ray& R, float kf, float ym, int PF, int PFM,
                                                 uint32_t bias)
{
    uint32_t b_f, b_m, b_s;
    float af, am, as;
    split_bits(fmaf(kf, R.d[0], R.x0[0]), b_f, af);
    split_bits(ym, b_m, am);
    split_bits(fmaf(kf, R.d[2], R.x0[2]), b_s, as);
    const uint32_t e = b_s * (uint32_t)PFM + b_m * (uint32_t)PF + b_f - bias;
    const typename QuadOf<TV>::type* b = qv + e;
    const float c0 = bilinear_value(load_fquad(b), af, am);        // plane s
    const float c1 = bilinear_value(load_fquad(b + PFM), af, am);  // plane s+1
    return fmaf(as, c1 - c0, c0);
}

// Samples k and k + 1 of a ray (kf = k, depth coordinates ym0 and ym1), added
// to acc in that order when t0 (resp. t1) holds.  Both samples' loads are
// issued before either interpolation, so four gathers are in flight per
// thread; a sample not taken reads the volume's first element and adds
// nothing, so the sum is bitwise the one-sample-at-a-time sum.
template <typename TV>
__device__ __forceinline__ void tri_pair_quad(const typename QuadOf<TV>::type* __restrict__ qv,
                                              const Ray& R, float kf, float ym0, float ym1, int PF,
                                              int PFM, uint32_t bias, bool t0, bool t1, float& acc)
{
    using Q = typename QuadOf<TV>::type;
    uint32_t f0, m0, z0, f1, m1, z1;
    float af0, am0, as0, af1, am1, as1;
    const float kf1 = kf + 1.0f;
    split_bits(fmaf(kf, R.d[0], R.x0[0]), f0, af0);
    split_bits(ym0, m0, am0);
    split_bits(fmaf(kf, R.d[2], R.x0[2]), z0, as0);
    split_bits(fmaf(kf1, R.d[0], R.x0[0]), f1, af1);
    split_bits(ym1, m1, am1);
    split_bits(fmaf(kf1, R.d[2], R.x0[2]), z1, as1);
    const Q* b0 = t0 ? qv + (z0 * (uint32_t)PFM + m0 * (uint32_t)PF + f0 - bias) : qv;
    const Q* b1 = t1 ? qv + (z1 * (uint32_t)PFM + m1 * (uint32_t)PF + f1 - bias) : qv;
    const float4 lo0 = load_fquad(b0);
    const float4 hi0 = load_fquad(b0 + PFM);
    const float4 lo1 = load_fquad(b1);
    const float4 hi1 = load_fquad(b1 + PFM);
    {
        const float c0 = bilinear_value(lo0, af0, am0), c1 = bilinear_value(hi0, af0, am0);
        if (t0) acc += fmaf(as0, c1 - c0, c0);
    }
    {
        const float c0 = bilinear_value(lo1, af1, am1), c1 = bilinear_value(hi1, af1, am1);
        if (t1) acc += fmaf(as1, c1 - c0, c0);
    }
}

// Restriction of a projection to one axial slab (out-of-core mode): only the
// samples whose z cell (padded index) lies in [cell_lo, cell_hi) count, the
// volume buffer's plane 0 is padded plane plane0, results add into the
// output, and the launch covers detector rows from q0 (the rows the slab can
// reach).
struct SlabRange {
    int cell_lo, cell_hi, plane0, q0;
    // x-y brick of the slab (padded cell ranges; +-1000000 = unbounded) and,
    // when not null, the detector columns [x, y] per angle whose rays can
    // reach the brick (blocks wholly outside return at once).
    int bx_lo, bx_hi, by_lo, by_hi;
    const int2* prange;
};

// Members of a batched launch: blockIdx.z = member * tiles + row tile; member
// i's quad volumes start vol_stride quads and its projections proj_stride
// elements after member 0's.  The default is a single member.
struct FwdBatch {
    int tiles = 1 << 30;
    int64_t vol_stride = 0, proj_stride = 0;
};

// First k in [0, K] whose z cell satisfies pred (pred monotone along the ray).
template <typename P>
__device__ __forceinline__ int first_k(int K, P pred)
{
    int lo = 0, hi = K;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pred(mid))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int axis_cell(const Ray& R, int ax, int k)
{
    int i;
    float f;
    split_floor(fmaf((float)k, R.d[ax], R.x0[ax]), i, f);
    return i;
}

// Narrow [kb, ke) to the samples whose cell along axis ax lies in [lo, hi)
// (monotone along the ray, so the samples in range form one interval).
__device__ __forceinline__ void cut_axis(const Ray& R, int ax, int lo, int hi, int& kb, int& ke)
{
    if (lo <= -1000000 && hi >= 1000000) return;
    const float dd = R.d[ax];
    if (dd > 0.0f) {
        kb = max(kb, first_k(R.K, [&](int k) { return axis_cell(R, ax, k) >= lo; }));
        ke = min(ke, first_k(R.K, [&](int k) { return axis_cell(R, ax, k) >= hi; }));
    } else if (dd < 0.0f) {
        kb = max(kb, first_k(R.K, [&](int k) { return axis_cell(R, ax, k) < hi; }));
        ke = min(ke, first_k(R.K, [&](int k) { return axis_cell(R, ax, k) < lo; }));
    } else {
        const int c0 = axis_cell(R, ax, 0);
        if (!(c0 >= lo && c0 < hi)) ke = kb;
    }
}

// The L1 kernel's depth-ordered march, gathering from quad volumes.  With
// SLAB, each ray processes only its samples [kb, ke) inside the slab (and
// brick).  With PAIR, the march advances two depth steps at a time and each
// lane takes up to two samples per step (tri_pair_quad).  With AG > 1 a warp
// holds 32 / AG pixels of one detector row at AG neighbouring angles (order
// is then the angle-group table, blockIdx.y the group; not with PAIR); each
// ray is marched exactly as with AG = 1.
// Occupancy: 6 blocks per SM (40 registers).  With angle pairs: 130.3 ms per
// 512^3 x 360 projection against 136.7 at 5 blocks and 143.2 at 7 or 8.  One
// angle per warp in core: 308.0 ms per 1024^3 x 90 against 312.6 at 7 (32
// registers, spilling in the march loop).
// With a Batch, several volumes of the same geometry are projected in one
// launch (blockIdx.z runs over member 0's row tiles, then member 1's, ...).
template <typename TV, typename TP, bool SLAB = false, bool PAIR = false, int AG = 1,
          bool BATCH = false>
__global__ void __launch_bounds__(256, 6) fwd_quad_kernel(
    const typename QuadOf<TV>::type* __restrict__ qxy,
    const typename QuadOf<TV>::type* __restrict__ qyx, TP* __restrict__ proj,
    const FwdAngle* __restrict__ params, FwdConst c, int a_first, const int* __restrict__ order,
    SlabRange sr, FwdBatch bt = FwdBatch{})
{
    static_assert(AG == 1 || !PAIR, "angle groups: single-sample march only");
    using Q = typename QuadOf<TV>::type;
    constexpr int CW = 32 / AG;  // detector columns per warp
    const unsigned full = 0xffffffffu;
    // (batched launches only: single launches keep the member arithmetic and
    // its registers out of the kernel)
    const int member = BATCH ? (int)blockIdx.z / bt.tiles : 0;
    const int tile = (int)blockIdx.z - member * bt.tiles;
    if (BATCH) {
        qxy += member * bt.vol_stride;
        qyx += member * bt.vol_stride;
        proj += member * bt.proj_stride;
    }
    // Each 16-lane half of a warp holds 8 pixels of two neighbouring angles
    // (pairs: lane = 2 * pixel + angle; groups of 4: lanes 8j..8j+7 hold angle
    // j).  A 128-bit warp load is served a half-warp at a time, and 8 pixels of
    // two neighbouring angles touch fewer 128-byte lines than 16 pixels of one
    // angle do.
    const int lane_p = AG == 2 ? (int)threadIdx.x >> 1 : (int)threadIdx.x % CW;
    const int lane_a = AG == 2 ? (int)threadIdx.x & 1 : (int)threadIdx.x / CW;
    const int p = blockIdx.x * CW + (AG == 1 ? (int)threadIdx.x : lane_p);
    const int q = (SLAB ? sr.q0 : 0) + tile * (int)blockDim.y + (int)threadIdx.y;
    const int a = AG > 1  ? order[blockIdx.y * AG + lane_a]
                  : order ? order[blockIdx.y]
                          : (int)blockIdx.y;
    if (SLAB && sr.prange) {  // uniform per block: all its rays miss the brick
        const int p0 = (int)blockIdx.x * CW;
        bool hit = false;
        for (int j = 0; j < AG; ++j) {
            const int aj = AG > 1 ? order[blockIdx.y * AG + j] : a;
            if (aj < 0) continue;
            const int2 pr = sr.prange[a_first + aj];
            hit = hit || !(p0 + CW - 1 < pr.x || p0 > pr.y);
        }
        if (!hit) return;
    }
    const bool inside = p < c.nu && q < c.nv && (AG == 1 || a >= 0);

    Ray R;
    R.K = 0;
    R.ok = true;
    if (inside) setup_ray(params + a_first + a, c, p, q, R);
    int kb = 0, ke = R.K;
    if (SLAB && inside && R.ok && R.K > 0) {
        cut_axis(R, 2, sr.cell_lo, sr.cell_hi, kb, ke);
        // the brick's x-y ranges, on the layout's (f, m) axes
        cut_axis(R, 0, R.layout ? sr.by_lo : sr.bx_lo, R.layout ? sr.by_hi : sr.bx_hi, kb, ke);
        cut_axis(R, 1, R.layout ? sr.bx_lo : sr.by_lo, R.layout ? sr.bx_hi : sr.by_hi, kb, ke);
    }
    const bool active = inside && R.ok && ke > kb;
    const unsigned act = __ballot_sync(full, active);
    // uniform per block (a group's first slot always holds an angle)
    const int layout = params[a_first + (AG > 1 ? order[blockIdx.y * AG] : a)].layout;
    const Q* __restrict__ vol = layout ? qyx : qxy;
    const int PF = (layout ? c.ny : c.nx) + 2 * kPad;
    const int PFM = PF * ((layout ? c.nx : c.ny) + 2 * kPad);
    const int s_off = SLAB ? sr.plane0 : 0;

    float acc = 0.0f;
    if (act) {
        const unsigned pos = __ballot_sync(full, active && R.d[1] > 0.0f);
        const unsigned neg = __ballot_sync(full, active && R.d[1] < 0.0f);
        const uint32_t bias = quad_index_bias(PF, PFM, s_off);
        // sample counters in float (exact: K < 2^24)
        const float kef = (float)ke;
        float kf = (float)kb;
        if (pos == act || neg == act) {
            const float sgn = pos == act ? 1.0f : -1.0f;
            const float y0 = sgn * R.x0[1], dy = sgn * R.d[1];
            const float ys = fmaf((float)kb, dy, y0);
            const float y1 = fmaf((float)(ke - 1), dy, y0);
            float D = active ? dy : 3.0e38f, Y0 = active ? ys : 3.0e38f;
            float Y1 = active ? y1 : -3.0e38f;
            int kmax = active ? ke - kb : 0;
            for (int o = 16; o > 0; o >>= 1) {
                D = fminf(D, __shfl_xor_sync(full, D, o));
                Y0 = fminf(Y0, __shfl_xor_sync(full, Y0, o));
                Y1 = fmaxf(Y1, __shfl_xor_sync(full, Y1, o));
                kmax = max(kmax, __shfl_xor_sync(full, kmax, o));
            }
            const float ns = (Y1 - Y0) / D;
            const int nslab = ns < (float)(2 * kmax + 64) ? (int)ns + 1 : 0;
            // sgn * ym is the depth coordinate fmaf(kf, dy, y0) (the sign
            // flip is exact), and ym feeds the sample's m split
            if (PAIR) {
                const float D2 = 2.0f * D;
                const float nj = (float)((nslab + 1) / 2);
                for (float jf = 1.0f; jf <= nj; jf += 1.0f) {
                    const float bound = fmaf(jf, D2, Y0);
                    const float ym0 = fmaf(kf, R.d[1], R.x0[1]);
                    const float ym1 = fmaf(kf + 1.0f, R.d[1], R.x0[1]);
                    const bool t0 = kf < kef && sgn * ym0 < bound;
                    const bool t1 = t0 && kf + 1.0f < kef && sgn * ym1 < bound;
                    if (__any_sync(full, t0))
                        tri_pair_quad<TV>(vol, R, kf, ym0, ym1, PF, PFM, bias, t0, t1, acc);
                    kf += (float)((int)t0 + (int)t1);
                }
            } else {
                // one loop per march direction: for sgn = -1 the test
                // -ym < bound is ym > -bound, with -bound = fmaf(jf, -D, -Y0)
                // exactly
                const float nj = (float)nslab;
                auto march = [&](auto neg) {
                    constexpr bool NEG = decltype(neg)::value;
                    const float Ds = NEG ? -D : D, Ys = NEG ? -Y0 : Y0;
                    for (float jf = 1.0f; jf <= nj; jf += 1.0f) {
                        const float bound = fmaf(jf, Ds, Ys);
                        const float ym = fmaf(kf, R.d[1], R.x0[1]);
                        if (kf < kef && (NEG ? ym > bound : ym < bound)) {
                            acc += tri_sample_quad<TV>(vol, R, kf, ym, PF, PFM, bias);
                            kf += 1.0f;
                        }
                    }
                };
                if (sgn > 0.0f)
                    march(std::false_type{});
                else
                    march(std::true_type{});
            }
        }
        for (; active && kf < kef; kf += 1.0f)
            acc += tri_sample_quad<TV>(vol, R, kf, fmaf(kf, R.d[1], R.x0[1]), PF, PFM, bias);
    }
    if (!inside) return;
    TP* o = proj + ((int64_t)a * c.nv + q) * c.nu + p;
    if (!R.ok) {
        *o = from_f32<TP>(__int_as_float(0x7fc00000));
    } else if (SLAB) {
        if (active) *o = from_f32<TP>(to_f32<TP>(*o) + acc * R.h);
    } else {
        *o = from_f32<TP>(acc * R.h);
    }
}

// out (padded, x fastest): out[z+P][y+P][x+P] = vol[z][y][x].
template <typename T>
__global__ void pad_xy_kernel(const T* __restrict__ vol, T* __restrict__ out, int nx, int ny,
                              int nz)
{
    const int y = blockIdx.y, z = blockIdx.z;
    const int PF = nx + 2 * kPad, PM = ny + 2 * kPad;
    const T* src = vol + ((int64_t)z * ny + y) * nx;
    T* dst = out + ((int64_t)(z + kPad) * PM + (y + kPad)) * PF + kPad;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x)
        dst[x] = src[x];
}

// out (padded, y fastest): out[z+P][x+P][y+P] = vol[z][y][x], 32x32 tiles.
template <typename T>
__global__ void pad_yx_kernel(const T* __restrict__ vol, T* __restrict__ out, int nx, int ny,
                              int nz)
{
    __shared__ T tile[32][33];
    const int z = blockIdx.z;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const T* src = vol + (int64_t)z * ny * nx;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + j;
        if (x < nx && y < ny) tile[j][threadIdx.x] = src[(int64_t)y * nx + x];
    }
    __syncthreads();
    const int PF = ny + 2 * kPad, PM = nx + 2 * kPad;
    T* dst = out + (int64_t)(z + kPad) * PM * PF;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + i;
        if (x < nx && y < ny) dst[(int64_t)(x + kPad) * PF + (y + kPad)] = tile[threadIdx.x][i];
    }
}

size_t padded_elems(const tigre_geometry_desc& d)
{
    return (size_t)(d.n_voxel[0] + 2 * kPad) * (size_t)(d.n_voxel[1] + 2 * kPad) *
           (size_t)(d.n_voxel[2] + 2 * kPad);
}

// Tag identifying a zero-bordered padded layout (element size, dims, layout).
static uint64_t layout_tag(const tigre_geometry_desc& d, size_t elem, int layout)
{
    return 1ull + (uint64_t)elem + 16ull * (uint64_t)layout +
           64ull * ((uint64_t)d.n_voxel[0] + 1048583ull * ((uint64_t)d.n_voxel[1] +
                                                           1048583ull * (uint64_t)d.n_voxel[2]));
}

// Size `buf` for a padded layout and zero it (border included) whenever the
// layout it holds changes; the interior is overwritten by every call.
tigre_status ensure_padded(DeviceBuffer& buf, const tigre_geometry_desc& d, size_t elem,
                           int layout, cudaStream_t st)
{
    const size_t bytes = padded_elems(d) * elem;
    const uint64_t tag = layout_tag(d, elem, layout);
    if (buf.bytes < bytes || buf.tag != tag) {
        TIGRE_TRY(buf.ensure(bytes));
        TIGRE_CUDA(cudaMemsetAsync(buf.ptr, 0, bytes, st));
        buf.tag = tag;
    }
    return TIGRE_OK;
}

template <typename TV>
tigre_status fill_padded(const tigre_geometry_desc& d, const TV* vol, TV* out, int layout,
                         cudaStream_t st)
{
    const int nx = (int)d.n_voxel[0], ny = (int)d.n_voxel[1], nz = (int)d.n_voxel[2];
    if (layout == 0) {
        dim3 grid((unsigned)((nx + 255) / 256), (unsigned)ny, (unsigned)nz);
        pad_xy_kernel<TV><<<grid, 256, 0, st>>>(vol, out, nx, ny, nz);
        TIGRE_LAUNCHED("pad_xy_kernel");
    } else {
        dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 31) / 32), (unsigned)nz);
        pad_yx_kernel<TV><<<grid, dim3(32, 8), 0, st>>>(vol, out, nx, ny, nz);
        TIGRE_LAUNCHED("pad_yx_kernel");
    }
    return TIGRE_OK;
}

tigre_status build_quads_f32(const tigre_geometry_desc& d, const float* vol, float4* out, int layout,
                             cudaStream_t st)
{
    return build_quads<float>(d, vol, out, layout, st);
}


// The angle-group table (groups of 2 or 4 angles: gi = 0 or 1) of the
// partial range [a0, a0 + na), indices relative to a0; built on the host and
// uploaded on first use, then kept by the handle.
static tigre_status range_group_table(tigre_geometry* g, int gi, int64_t a0, int64_t na,
                                      const int** table, int64_t* ngroups)
{
    const std::pair<int64_t, int64_t> key(a0, na);
    auto it = g->range_groups[gi].find(key);
    if (it == g->range_groups[gi].end()) {
        const AngleGroups ag = build_angle_groups(g->desc, g->angles.data() + a0, na);
        const std::vector<int>& tab = ag.table[gi];
        DeviceBuffer buf;
        TIGRE_TRY(buf.ensure(sizeof(int) * std::max<size_t>(tab.size(), 1)));
        if (!tab.empty()) {
            const cudaError_t e = cudaMemcpy(buf.ptr, tab.data(), sizeof(int) * tab.size(),
                                             cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                buf.release();
                return cuda_fail(e, "angle-group table upload");
            }
        }
        it = g->range_groups[gi].emplace(key, buf).first;
        g->range_n_groups[gi][key] = (int64_t)(tab.size() / (gi ? 4 : 2));
    }
    *table = (const int*)it->second.ptr;
    *ngroups = g->range_n_groups[gi][key];
    return TIGRE_OK;
}

// Layouts the angles [a0, a0 + na) read.
static void needed_layouts(const tigre_geometry* g, int64_t a0, int64_t na, bool need[2])
{
    need[0] = need[1] = false;
    for (int64_t a = a0; a < a0 + na; ++a) need[g->layout[(size_t)a]] = true;
}

static tigre_status brick_pixel_ranges(tigre_geometry* g, const int2** out);

// Whether an in-core projection marches x-y bricks: the automatic path, F32
// volume, projector interpolated, and a volume wider than one brick.  Its
// rays then read one brick's planes at a time, which stay in L2 (1024^3 x
// 720: 1790 vs 2012 ms of kernels); a 512^2 plane is one brick.
static bool in_core_bricks(const tigre_geometry* g, tigre_dtype vt)
{
    const tigre_geometry_desc& d = g->desc;
    const int64_t e = g->brick;
    return g->fwd_path == 0 && vt == TIGRE_F32 && g->projector == TIGRE_PROJ_INTERPOLATED &&
           e > 0 && (d.n_voxel[0] > e || d.n_voxel[1] > e);
}

tigre_status forward_workspace(tigre_geometry* g, tigre_dtype vt, int64_t a0, int64_t na,
                               cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (!dtype_ok(vt)) return fail(TIGRE_ERR_INVALID_ARG, "bad dtype");
    const tigre_geometry_desc& d = g->desc;
    if (padded_elems(d) >= (size_t)INT32_MAX) return TIGRE_OK;  // refused by the projection
    bool need[2];
    needed_layouts(g, a0, na, need);
    const bool siddon = g->projector == TIGRE_PROJ_SIDDON;
    if (!siddon && g->fwd_path == 2) {
        if (!g->err_flag.ptr) {
            TIGRE_TRY(g->err_flag.ensure(sizeof(int)));
            TIGRE_CUDA(cudaMemsetAsync(g->err_flag.ptr, 0, sizeof(int), st));
        }
        return tma_workspace(g, dtype_size(vt), need);
    }
    const bool use_quad = !siddon && (g->fwd_path == 0 || g->fwd_path >= 3);
    if (in_core_bricks(g, vt)) {  // the bricks' pixel ranges, before any capture
        const int2* pr = nullptr;
        TIGRE_TRY(brick_pixel_ranges(g, &pr));
    }
    DeviceBuffer* bufs[2] = {&g->vol_xy, &g->vol_yx};
    DeviceBuffer* qbufs[2] = {&g->vol_qxy, &g->vol_qyx};
    for (int l = 0; l < 2; ++l) {
        if (!need[l]) continue;
        // the quad paths build their quads from the volume itself; the
        // scalar and Siddon paths read the zero-bordered layouts
        if (use_quad)
            TIGRE_TRY(qbufs[l]->ensure(padded_elems(d) * sizeof(float4)));  // 4 FP32 coefficients
        else
            TIGRE_TRY(ensure_padded(*bufs[l], d, dtype_size(vt), l, st));
    }
    return TIGRE_OK;
}

tigre_status forward_impl(tigre_geometry* g, const void* vol, tigre_dtype vt, void* proj,
                          tigre_dtype pt, int64_t a0, int64_t na, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (!vol || !proj) return fail(TIGRE_ERR_INVALID_ARG, "null vol or proj pointer");
    if (!dtype_ok(vt) || !dtype_ok(pt)) return fail(TIGRE_ERR_INVALID_ARG, "bad dtype");
    const tigre_geometry_desc& d = g->desc;
    if (padded_elems(d) >= (size_t)INT32_MAX)
        return fail(TIGRE_ERR_UNSUPPORTED,
                    "in-core forward projection needs (nx+4)(ny+4)(nz+4) < 2^31; use out-of-core");
    if (d.n_det[1] > 65535 * 8)
        return fail(TIGRE_ERR_UNSUPPORTED, "detector too large for one launch");
    const FwdConst c = make_fwd_const(g);
    TIGRE_TRY(forward_workspace(g, vt, a0, na, st));
    bool need[2];
    needed_layouts(g, a0, na, need);
    const bool siddon = g->projector == TIGRE_PROJ_SIDDON;
    const bool use_tma = !siddon && g->fwd_path == 2;
    const bool use_quad = !siddon && (g->fwd_path == 0 || g->fwd_path >= 3);
    const bool pair = g->fwd_path == 4;
    // Full-range launches visit the angles grouped by memory layout, so the
    // blocks resident at one time read one layout's z-slab (half the L2
    // working set of an interleaved order).
    const int* order = (a0 == 0 && na == (int64_t)g->angles.size() && na <= 65535)
                           ? (const int*)g->angle_order.ptr
                           : nullptr;
    if (use_tma) {
        return dispatch_dtype(vt, [&](auto vtag) -> tigre_status {
            using TV = decltype(vtag);
            return dispatch_dtype(pt, [&](auto ptag) -> tigre_status {
                using TP = decltype(ptag);
                return launch_forward_tma<TV, TP>(g, (const TV*)vol, (TP*)proj, a0, na, need,
                                                  (int*)g->err_flag.ptr, st);
            });
        });
    }

    return dispatch_dtype(vt, [&](auto vtag) -> tigre_status {
        using TV = decltype(vtag);
        using Q = typename QuadOf<TV>::type;
        DeviceBuffer* bufs[2] = {&g->vol_xy, &g->vol_yx};
        DeviceBuffer* qbufs[2] = {&g->vol_qxy, &g->vol_qyx};
        static_assert(sizeof(Q) == 4 * sizeof(float), "a quad is four FP32 coefficients");
        for (int l = 0; l < 2; ++l) {
            if (!need[l]) continue;
            if (use_quad)
                TIGRE_TRY(build_quads<TV>(d, (const TV*)vol, (Q*)qbufs[l]->ptr, l, st));
            else
                TIGRE_TRY(fill_padded<TV>(d, (const TV*)vol, (TV*)bufs[l]->ptr, l, st));
        }
        return dispatch_dtype(pt, [&](auto ptag) -> tigre_status {
            using TP = decltype(ptag);
            if (siddon)
                return launch_siddon_forward<TV, TP>(g, (const TV*)g->vol_xy.ptr,
                                                     (const TV*)g->vol_yx.ptr, (TP*)proj, a0, na,
                                                     order, st);
            if constexpr (std::is_same<TV, float>::value && std::is_same<TP, float>::value) {
                if (in_core_bricks(g, vt) && pt == TIGRE_F32) {
                    // the whole volume as one slab, marched brick by brick;
                    // the bricks' partial sums add into zeroed projections
                    TIGRE_CUDA(cudaMemsetAsync(proj, 0, sizeof(float) * (size_t)na * c.nu * c.nv, st));
                    float4* const quads[2] = {(float4*)g->vol_qxy.ptr, (float4*)g->vol_qyx.ptr};
                    return forward_slab_impl(g, d, quads, (float*)proj, a0, na, -1000000, 1000000,
                                             0, st);
                }
            }
            ProfScope prof(kProfForward, st);
            const int ag = g->fwd_path == 5   ? 2
                           : g->fwd_path == 6 ? 4
                           : g->fwd_path == 0 ? g->auto_angle_group
                                              : 1;
            if (use_quad && ag > 1 && (order || na <= 65535 * (int64_t)ag)) {
                const int gi = ag == 4 ? 1 : 0;
                const int* table = nullptr;
                int64_t ngroups = 0;
                if (order) {  // the full range
                    table = (const int*)g->angle_groups[gi].ptr;
                    ngroups = g->n_groups[gi];
                } else {
                    TIGRE_TRY(range_group_table(g, gi, a0, na, &table, &ngroups));
                }
                if (ngroups <= 65535) {
                    dim3 grid((unsigned)((c.nu + 32 / ag - 1) / (32 / ag)), (unsigned)ngroups,
                              (unsigned)((c.nv + 7) / 8));
                    auto kern = ag == 4 ? fwd_quad_kernel<TV, TP, false, false, 4>
                                        : fwd_quad_kernel<TV, TP, false, false, 2>;
                    kern<<<grid, dim3(32, 8), 0, st>>>(
                        (const Q*)g->vol_qxy.ptr, (const Q*)g->vol_qyx.ptr, (TP*)proj,
                        (const FwdAngle*)g->fwd_params.ptr, c, order ? 0 : (int)a0, table,
                        SlabRange{0, 0, 0, 0, 0, 0, 0, 0, nullptr}, FwdBatch{});
                    TIGRE_LAUNCHED("fwd_quad_kernel");
                    return TIGRE_OK;
                }
            }
            if (use_quad) {
                for (int64_t s = 0; s < na; s += 65535) {
                    const int64_t cnt = std::min<int64_t>(65535, na - s);
                    dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt,
                              (unsigned)((c.nv + 7) / 8));
                    auto kern = pair ? fwd_quad_kernel<TV, TP, false, true>
                                     : fwd_quad_kernel<TV, TP, false, false>;
                    kern<<<grid, dim3(32, 8), 0, st>>>(
                        (const Q*)g->vol_qxy.ptr, (const Q*)g->vol_qyx.ptr,
                        (TP*)proj + s * (int64_t)c.nu * c.nv, (const FwdAngle*)g->fwd_params.ptr,
                        c, (int)(a0 + s), order, SlabRange{0, 0, 0, 0, 0, 0, 0, 0, nullptr}, FwdBatch{});
                    TIGRE_LAUNCHED("fwd_quad_kernel");
                }
                return TIGRE_OK;
            }
            const int64_t step = 65535;
            for (int64_t s = 0; s < na; s += step) {
                const int64_t cnt = std::min(step, na - s);
                dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
                fwd_l1_kernel<TV, TP><<<grid, dim3(32, 8), 0, st>>>(
                    (const TV*)g->vol_xy.ptr, (const TV*)g->vol_yx.ptr,
                    (TP*)proj + s * (int64_t)c.nu * c.nv, (const FwdAngle*)g->fwd_params.ptr, c,
                    (int)(a0 + s), order);
                TIGRE_LAUNCHED("fwd_l1_kernel");
            }
            return TIGRE_OK;
        });
    });
}

tigre_status forward_batch_impl(tigre_geometry* g, const void* vols, void* projs, int batch,
                                 tigre_dtype dt, void* const quad[2], cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    const tigre_geometry_desc& d = g->desc;
    const int64_t na = (int64_t)g->angles.size();
    if (g->projector != TIGRE_PROJ_INTERPOLATED || g->fwd_path != 0)
        return fail(TIGRE_ERR_UNSUPPORTED, "batched projection: interpolated projector, automatic path");
    if (padded_elems(d) >= (size_t)INT32_MAX || na > 65535)
        return fail(TIGRE_ERR_UNSUPPORTED, "batched projection: volume or angle count too large");
    const FwdConst c = make_fwd_const(g);
    const int tiles = (c.nv + 7) / 8;
    if ((int64_t)tiles * batch > 65535) return fail(TIGRE_ERR_UNSUPPORTED, "batch too large");
    bool need[2];
    needed_layouts(g, 0, na, need);
    const int64_t nvox = d.n_voxel[0] * d.n_voxel[1] * d.n_voxel[2];
    const int64_t pe = (int64_t)padded_elems(d);
    return dispatch_dtype(dt, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        using Q = typename QuadOf<T>::type;
        for (int i = 0; i < batch; ++i)
            for (int l = 0; l < 2; ++l)
                if (need[l])
                    TIGRE_TRY(build_quads<T>(d, (const T*)vols + i * nvox, (Q*)quad[l] + i * pe, l,
                                             st));
        FwdBatch bt;
        bt.tiles = tiles;
        bt.vol_stride = pe;
        bt.proj_stride = na * c.nu * c.nv;
        ProfScope prof(kProfForward, st);
        // the automatic path of forward_impl for a full-range projection
        if (g->auto_angle_group == 2) {
            dim3 grid((unsigned)((c.nu + 15) / 16), (unsigned)g->n_groups[0], (unsigned)(tiles * batch));
            fwd_quad_kernel<T, T, false, false, 2, true><<<grid, dim3(32, 8), 0, st>>>(
                (const Q*)quad[0], (const Q*)quad[1], (T*)projs, (const FwdAngle*)g->fwd_params.ptr,
                c, 0, (const int*)g->angle_groups[0].ptr, SlabRange{0, 0, 0, 0, 0, 0, 0, 0, nullptr},
                bt);
        } else {
            dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)na, (unsigned)(tiles * batch));
            fwd_quad_kernel<T, T, false, false, 1, true><<<grid, dim3(32, 8), 0, st>>>(
                (const Q*)quad[0], (const Q*)quad[1], (T*)projs, (const FwdAngle*)g->fwd_params.ptr,
                c, 0, (const int*)g->angle_order.ptr, SlabRange{0, 0, 0, 0, 0, 0, 0, 0, nullptr}, bt);
        }
        TIGRE_LAUNCHED("fwd_quad_kernel(batch)");
        return TIGRE_OK;
    });
}

// Detector columns [lo, hi] per (brick, angle) whose rays can reach the x-y
// brick (its voxels extended by 1.5 voxels, the interpolation support),
// from the perspective image of the brick's corners on the detector, with
// two columns of margin; computed in FP64 once per geometry and kept on the
// device.  A brick the source could be inside of gets the whole detector.
static tigre_status brick_pixel_ranges(tigre_geometry* g, const int2** out)
{
    const tigre_geometry_desc& d = g->desc;
    const int64_t edge = g->brick;
    const int64_t nbx = (d.n_voxel[0] + edge - 1) / edge;
    const int64_t nby = (d.n_voxel[1] + edge - 1) / edge;
    const int64_t na = (int64_t)g->angles.size();
    const size_t bytes = sizeof(int2) * (size_t)(nbx * nby * na);
    const uint64_t tag = 1 + (uint64_t)edge;
    if (g->brick_prange.tag != tag || g->brick_prange.bytes < bytes) {
        const int nu = (int)d.n_det[0];
        const double u0 = -0.5 * (double)(nu - 1) * d.d_det[0] + d.off_det[0];
        std::vector<int2> h((size_t)(nbx * nby * na));
        auto world = [&](int ax, double idx) {
            return (idx - 0.5 * (double)(d.n_voxel[ax] - 1)) * d.d_voxel[ax] + d.off_origin[ax];
        };
        for (int64_t by = 0; by < nby; ++by)
            for (int64_t bx = 0; bx < nbx; ++bx) {
                const double xs[2] = {world(0, (double)(bx * edge) - 1.5),
                                      world(0, (double)std::min<int64_t>((bx + 1) * edge, d.n_voxel[0]) - 1.0 + 1.5)};
                const double ys[2] = {world(1, (double)(by * edge) - 1.5),
                                      world(1, (double)std::min<int64_t>((by + 1) * edge, d.n_voxel[1]) - 1.0 + 1.5)};
                for (int64_t a = 0; a < na; ++a) {
                    const double cs = std::cos(g->angles[(size_t)a]), sn = std::sin(g->angles[(size_t)a]);
                    double lo = 1e300, hi = -1e300;
                    bool ok = true;
                    for (double X : xs)
                        for (double Y : ys) {
                            const double depth = d.DSO - (X * cs + Y * sn);
                            if (!(depth > 0.0)) ok = false;
                            const double u = (-X * sn + Y * cs) * d.DSD / depth;
                            lo = std::min(lo, u);
                            hi = std::max(hi, u);
                        }
                    int plo = 0, phi = nu - 1;
                    if (ok) {
                        plo = (int)std::max(0.0, std::floor((lo - u0) / d.d_det[0]) - 2.0);
                        phi = (int)std::min((double)(nu - 1), std::ceil((hi - u0) / d.d_det[0]) + 2.0);
                    }
                    h[(size_t)((by * nbx + bx) * na + a)] = make_int2(plo, phi);
                }
            }
        TIGRE_TRY(g->brick_prange.ensure(bytes));
        TIGRE_CUDA(cudaMemcpy(g->brick_prange.ptr, h.data(), bytes, cudaMemcpyHostToDevice));
        g->brick_prange.tag = tag;
    }
    *out = (const int2*)g->brick_prange.ptr;
    return TIGRE_OK;
}

// One axial slab of an out-of-core projection: pad[l] hold the slab's
// zero-padded F32 layouts (planes of padded index plane0 .. for the
// sub-volume description sd), quad[l] receive their quad volumes, and the
// samples with z cells in [cell_lo, cell_hi) add into proj.
tigre_status forward_slab_impl(tigre_geometry* g, const tigre_geometry_desc& sd,
                               float4* const quad[2], float* proj, int64_t a0, int64_t na,
                               int cell_lo, int cell_hi, int plane0, cudaStream_t st)
{
    (void)sd;
    const tigre_geometry_desc& d = g->desc;
    if (g->projector != TIGRE_PROJ_INTERPOLATED)
        return fail(TIGRE_ERR_UNSUPPORTED, "out-of-core projection is interpolated only");
    const FwdConst c = make_fwd_const(g);
    // Rows whose rays can have samples in the slab's cells: z (unpadded
    // index) in [cell_lo - P, cell_hi - P), within the support [-1, nz].
    int q_lo = 0, q_hi = c.nv;
    {
        const double za = std::max((double)(cell_lo - kPad), -1.5);
        const double zb = std::min((double)(cell_hi - kPad), (double)d.n_voxel[2] + 0.5);
        double lo, hi;
        if (detector_row_range(d, za, zb, &lo, &hi)) {
            q_lo = (int)std::max(0.0, std::floor(lo) - 2.0);
            q_hi = (int)std::min((double)c.nv, std::ceil(hi) + 3.0);
        }
    }
    if (q_hi <= q_lo) return TIGRE_OK;
    // x-y bricks of at most brick^2 voxels: the rays resident at one time
    // then read one brick's planes, which stay in L2 (a quad plane of a
    // 3072^2 slab alone is larger than L2).
    const int64_t edge = g->brick;
    const int64_t nbx = (d.n_voxel[0] + edge - 1) / edge;
    const int64_t nby = (d.n_voxel[1] + edge - 1) / edge;
    const int2* pr = nullptr;
    if (nbx * nby > 1) TIGRE_TRY(brick_pixel_ranges(g, &pr));
    const int64_t na_all = (int64_t)g->angles.size();
    auto kern = g->fwd_path == 4 ? fwd_quad_kernel<float, float, true, true>
                                 : fwd_quad_kernel<float, float, true, false>;
    // Angle pairs where the in-core projection takes them (the automatic
    // choice or the pair path): group table of the full range (absolute
    // indices) or of [a0, a0 + na) (indices relative to a0).
    const int* table = nullptr;
    int64_t ngroups = 0;
    int pair_first = 0;
    if (g->fwd_path == 5 || (g->fwd_path == 0 && g->auto_angle_group == 2)) {
        if (a0 == 0 && na == na_all) {
            table = (const int*)g->angle_groups[0].ptr;
            ngroups = g->n_groups[0];
        } else {
            TIGRE_TRY(range_group_table(g, 0, a0, na, &table, &ngroups));
            pair_first = (int)a0;
        }
        if (ngroups > 65535) table = nullptr;
    }
    ProfScope prof(kProfForward, st);
    for (int64_t by = 0; by < nby; ++by)
        for (int64_t bx = 0; bx < nbx; ++bx) {
            // first / last bricks own the cells of the zero border too
            const int bx_lo = bx == 0 ? -1000000 : (int)(bx * edge + kPad);
            const int bx_hi = bx == nbx - 1 ? 1000000 : (int)((bx + 1) * edge + kPad);
            const int by_lo = by == 0 ? -1000000 : (int)(by * edge + kPad);
            const int by_hi = by == nby - 1 ? 1000000 : (int)((by + 1) * edge + kPad);
            const int2* brick_pr = pr ? pr + (by * nbx + bx) * na_all : nullptr;
            const SlabRange sr{cell_lo, cell_hi, plane0, q_lo, bx_lo, bx_hi, by_lo, by_hi, brick_pr};
            if (table) {
                dim3 grid((unsigned)((c.nu + 15) / 16), (unsigned)ngroups,
                          (unsigned)((q_hi - q_lo + 7) / 8));
                fwd_quad_kernel<float, float, true, false, 2><<<grid, dim3(32, 8), 0, st>>>(
                    quad[0], quad[1], proj, (const FwdAngle*)g->fwd_params.ptr, c, pair_first,
                    table, sr, FwdBatch{});
                TIGRE_LAUNCHED("fwd_quad_kernel(slab, pairs)");
                continue;
            }
            for (int64_t s = 0; s < na; s += 65535) {
                const int64_t cnt = std::min<int64_t>(65535, na - s);
                dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt,
                          (unsigned)((q_hi - q_lo + 7) / 8));
                kern<<<grid, dim3(32, 8), 0, st>>>(
                    quad[0], quad[1], proj + s * (int64_t)c.nu * c.nv,
                    (const FwdAngle*)g->fwd_params.ptr, c, (int)(a0 + s), nullptr, sr, FwdBatch{});
                TIGRE_LAUNCHED("fwd_quad_kernel(slab)");
            }
        }
    return TIGRE_OK;
}

// Sum of K over the rays of a launch-sized block of angles (ray setup only).
__global__ void __launch_bounds__(256) sample_count_kernel(const FwdAngle* __restrict__ params,
                                                           FwdConst c, int a_first,
                                                           unsigned long long* total)
{
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int q = blockIdx.z * blockDim.y + threadIdx.y;
    const int a = blockIdx.y;
    int K = 0;
    if (p < c.nu && q < c.nv) {
        Ray R;
        setup_ray(params + a_first + a, c, p, q, R);
        K = R.ok ? R.K : 0;
    }
    for (int o = 16; o > 0; o >>= 1) K += __shfl_down_sync(0xffffffffu, K, o);
    if ((threadIdx.x & 31) == 0 && K) atomicAdd(total, (unsigned long long)K);
}

}  // namespace tigre

extern "C" tigre_status tigre_geometry_set_brick(tigre_geometry_t g, int64_t edge)
{
    if (!g || edge < 0) return tigre::fail(TIGRE_ERR_INVALID_ARG, "brick edge must be >= 0");
    g->brick = edge == 0 ? tigre::kBrickDefault : edge;
    return TIGRE_OK;
}

extern "C" tigre_status tigre_geometry_set_forward_path(tigre_geometry_t g, int path)
{
    if (!g || path < 0 || path > 6) return tigre::fail(TIGRE_ERR_INVALID_ARG, "path must be 0..6");
    g->fwd_path = path;
    return TIGRE_OK;
}

extern "C" tigre_status tigre_geometry_error_flags(tigre_geometry_t g, int* flags, int clear)
{
    if (!g || !flags) return tigre::fail(TIGRE_ERR_INVALID_ARG, "null argument");
    *flags = 0;
    if (!g->err_flag.ptr) return TIGRE_OK;
    TIGRE_CUDA(cudaMemcpy(flags, g->err_flag.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear) TIGRE_CUDA(cudaMemset(g->err_flag.ptr, 0, sizeof(int)));
    return TIGRE_OK;
}

extern "C" tigre_status tigre_forward_samples(tigre_geometry_t g, int64_t angle_begin,
                                              int64_t angle_count, int64_t* samples)
{
    using namespace tigre;
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, angle_begin, angle_count));
    if (!samples) return fail(TIGRE_ERR_INVALID_ARG, "null output");
    const FwdConst c = make_fwd_const(g);
    unsigned long long* d = nullptr;
    TIGRE_CUDA(dev_alloc_sync((void**)&d, sizeof(unsigned long long)));
    tigre_status st = TIGRE_OK;
    cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
    for (int64_t s = 0; e == cudaSuccess && s < angle_count; s += 65535) {
        const int64_t cnt = std::min<int64_t>(65535, angle_count - s);
        dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
        sample_count_kernel<<<grid, dim3(32, 8)>>>((const FwdAngle*)g->fwd_params.ptr, c,
                                                   (int)(angle_begin + s), d);
        count_launch();
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_fail(e, "tigre_forward_samples");
    dev_free_sync(d);
    *samples = (int64_t)h;
    return st;
}

extern "C" tigre_status tigre_forward(tigre_geometry_t geo, const void* vol, tigre_dtype vol_dtype,
                                      void* proj, tigre_dtype proj_dtype, int64_t angle_begin,
                                      int64_t angle_count, void* cuda_stream)
{
    return tigre::forward_impl(geo, vol, vol_dtype, proj, proj_dtype, angle_begin, angle_count,
                               (cudaStream_t)cuda_stream);
}
