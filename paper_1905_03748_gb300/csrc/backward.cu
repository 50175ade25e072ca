// Backprojection A^T y (paper Sec. 2.2).
//
// Voxel-driven (FDK or pseudo-matched weights): each thread owns one (x, y)
// column and NZ consecutive voxels of it, as in the paper's organisation
// (Fig. 4: each thread updates N_z voxels), and loops over all angles of the
// call.  Per angle the detector column coordinate u and the FDK weight are
// the same for the whole z-column; only the row coordinate v moves, linearly
// in z.  Per voxel and angle:
//   s = X.(cos t, sin t, 0), mag = DSD/(DSO - s),
//   (u, v) = ((X.e_u) mag, X_z mag) -> bilinear tap of the projection,
//   FDK:     w = (DSO/(DSO - s))^2
//   matched: w = (dx dy dz)/(du dv) * |X - S| * DSD^2/(DSO - s)^3.
//
// GB300 layout: the projections are first copied into a buffer with zero
// columns (two) and rows around the detector: in v, as many rows as the
// volume's shadow can reach beyond the detector for this geometry (bounded
// on the host), so the per-voxel loop has neither clamps nor branches; u is
// clamped once per column and angle.  In-core launches use a quad buffer:
// element (r, c) holds the four FP32 bilinear coefficients of the cell
// (c, c+1) x (r, r+1) for every storage type, so a voxel-angle pair costs one
// aligned 16-byte load and three FMAs instead of four scalar loads, their
// addresses and three lerps (the kernel is bound by instruction issue).  Out-of-core slab launches read a
// band of rows per slab, which spans the cone's spread (hundreds of rows at
// 3072^3): they build quads of a quarter of the angles at a time, in the
// bytes a plain band of all angles takes.
// Grid order: x-tiles fastest, z-chunks slowest, so resident blocks share one
// band of detector rows per angle in L2.
//
// Exact adjoint: the transpose of the forward projector, each ray scattering
// h * trilinear weight * y into the 8 corner voxels of each of its samples
// (FP32 atomics into padded accumulators in the same two layouts as the
// forward projector, so a warp's atomics hit adjacent addresses).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "quad.cuh"
#include "ray.cuh"

namespace tigre {

constexpr int kBpNZ = 16;  // voxels per thread along z

struct BpConst {
    int nx, ny, nz, nu, nv;
    int PU, PV;        // padded buffer row length and rows per angle
    int pv_lo;         // zero rows above the detector
    int z_first, z_end;  // voxel planes computed by this launch
    int z_out0;          // plane of the output buffer's first plane
    float x0, y0, z0;  // world position (mm) of voxel (0, 0, 0)
    float dx, dy, dz;
    float DSO, DSD;
    float inv_du, inv_dv;
    float pu_off, pv_off;  // pixel index = coordinate / pitch + offset
    float wscale;          // (dx dy dz)/(du dv) * DSD^2
};

// 1/sqrt(x) straight from the special-function unit (PTX rsqrt.approx, inputs
// below the smallest normal flushed to zero).  Used where x = (w l)^2, the
// squared matched weight times source-voxel distance: w l is about
// (dx dy dz)/(du dv) times the squared magnification (at least 1), so x stays
// far inside the normal range for any voxel volume per pixel area above
// 1e-18 mm, and there it returns what rsqrtf does without rsqrtf's denormal
// handling.
__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}


// The bilinear coefficients (bilinear_coefficients: u along columns, v along
// rows) of the cell (c, c+1) x (r, r+1) at `cell`, from the plain (QUADP
// false) or the quad (true) zero-bordered projection buffer.  Quads store the
// coefficients; the plain buffer holds taps, whose coefficients are formed
// after the load in the same FP32 operations.
template <typename TP, bool QUADP> struct ProjTaps;
template <typename TP> struct ProjTaps<TP, false> {
    using E = TP;
    static __device__ __forceinline__ float4 load(const E* cell, int PU)
    {
        return bilinear_coefficients(to_f32<TP>(__ldg(cell)), to_f32<TP>(__ldg(cell + 1)),
                                     to_f32<TP>(__ldg(cell + PU)),
                                     to_f32<TP>(__ldg(cell + PU + 1)));
    }
};
template <typename TP> struct ProjTaps<TP, true> {
    using E = typename QuadOf<TP>::type;
    static __device__ __forceinline__ float4 load(const E* cell, int) { return load_quad(cell); }
};

// SART == true: also accumulate the backprojection of the all-ones
// projections (the normaliser V^-1 = A_w^T 1, from the same weights and
// interpolation) and finish with vol += lambda * num / den (den > 1e-12),
// clamped at zero when nonneg.
// Shape (512^3 x 360, one launch).  Plain buffer, 16 voxels per thread at 5
// blocks per SM (48 registers): matched 51.2 ms, FDK 46.5 ms.  Quad buffer
// (bilinear coefficients), matched: 16 voxels at 3 blocks 37.4 ms (16 at 4:
// 37.9; 12 at 6: 41.2; 12 at 5: 40.7; 10 at 6: 39.7; 14 at 5: 44.3; 1024^3 x
// 180: 142 at 16 / 3 or 4 against 155 at 12 / 6); FDK: 16 voxels at 3 blocks
// 34.3 ms (16 at 4: 36.5; 12 at 5: 58.0; 8 at 6: 48.5).  SART form (twice the
// accumulators): plain 16 at 3 blocks 74.2 ms per SIRT pass over 360 angles
// and 88.1 per OS-SART sweep of 20-angle subsets; quads with 12 voxels at 4
// blocks 56.4 and 58.9 ms (8 at 6: 58.0 and 61.0; 16 at 3: 57.6 and 61.7).
template <int MODE, bool SART, bool QUADP>
constexpr int bp_blocks_per_sm()
{
    return !QUADP ? (SART ? 3 : 5) : SART ? 4 : 3;
}
template <int MODE, bool SART, bool QUADP>
constexpr int bp_voxels_per_thread()
{
    return !QUADP ? 16 : SART ? 12 : 16;
}
static_assert(bp_voxels_per_thread<TIGRE_BP_FDK, false, false>() <= kBpNZ &&
                  bp_voxels_per_thread<TIGRE_BP_MATCHED, false, true>() <= kBpNZ &&
                  bp_voxels_per_thread<TIGRE_BP_FDK, false, true>() <= kBpNZ,
              "the row-band bounds assume chunks of at most kBpNZ planes");

// Members of a batched launch: blockIdx.z = member * chunks + z chunk; member
// i reads projections proj_stride elements and writes the volume vol_stride
// voxels after member 0's.  The default is a single member.
struct BpBatch {
    int chunks = 1 << 30;
    int64_t proj_stride = 0, vol_stride = 0;
};

template <typename TP, typename TV, int NZ, int MODE, bool SART, bool QUADP, bool BATCH = false>
__global__ void __launch_bounds__(256, (bp_blocks_per_sm<MODE, SART, QUADP>())) bp_voxel_kernel(
                                                       const typename ProjTaps<TP, QUADP>::E* __restrict__ pp,
                                                       TV* __restrict__ vol,
                                                       const BpAngle* __restrict__ params,
                                                       BpConst c, int a_first, int na,
                                                       int accumulate, float lambda = 0.0f,
                                                       int nonneg = 0,
                                                       BpBatch bt = BpBatch{})
{
    // (instances with BATCH only: the others keep the member arithmetic and
    // its registers out of the kernel)
    const int member = BATCH ? (int)blockIdx.z / bt.chunks : 0;
    if (BATCH) {
        pp += member * bt.proj_stride;
        vol += member * bt.vol_stride;
    }
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int zb = c.z_first + ((int)blockIdx.z - member * bt.chunks) * NZ;
    if (x >= c.nx || y >= c.ny) return;
    const float X = fmaf((float)x, c.dx, c.x0);
    const float Y = fmaf((float)y, c.dy, c.y0);
    const float Zb = fmaf((float)zb, c.dz, c.z0);
    const int PU = c.PU;
    const int64_t PA = (int64_t)PU * c.PV;
    const float pu_hi = (float)c.nu + 0.5f;
    const float pv_off = c.pv_off + (float)c.pv_lo;
    // a row's element offset from split_bits parts: (b - 0x4B000000) PU, one
    // multiply-add modulo 2^32
    const uint32_t row_bias = 0x4B000000u * (uint32_t)PU;

    float acc[NZ];
    float nrm[SART ? NZ : 1];
#pragma unroll
    for (int k = 0; k < NZ; ++k) acc[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < (SART ? NZ : 1); ++k) nrm[k] = 0.0f;

    for (int a = 0; a < na; ++a) {
        const BpAngle A = params[a_first + a];
        const float s = fmaf(X, A.c, Y * A.s);
        const float inv_den = 1.0f / (c.DSO - s);
        const float mag = c.DSD * inv_den;
        const float u = fmaf(Y, A.c, -X * A.s) * mag;
        // Clamp far outside the detector onto the zero border, then pad.
        const float pu = fminf(fmaxf(fmaf(u, c.inv_du, c.pu_off), -1.5f), pu_hi) + (float)kPad;
        int ip;
        float fu;
        split_floor(pu, ip, fu);
        const typename ProjTaps<TP, QUADP>::E* col = pp + (int64_t)a * PA + ip;
        // Padded row coordinate of voxel k: within [2, PV - 2) by the
        // host-side bound on the volume's shadow.
        const float pv0 = fmaf(Zb * mag, c.inv_dv, pv_off);
        const float dpv = c.dz * mag * c.inv_dv;
        float tu = 0.0f;  // bilinear weight of the all-ones image along u
        if (SART)
            tu = ((unsigned)(ip - kPad) < (unsigned)c.nu ? 1.0f - fu : 0.0f) +
                 ((unsigned)(ip - kPad + 1) < (unsigned)c.nu ? fu : 0.0f);
        // matched: voxel k's weight w |source - voxel| is taken as
        // sqrt(u) = u rsqrt(u) with u = (w Z)^2 + w^2 |(ex, ey)|^2, one
        // multiply fewer per voxel than w (l2 rsqrt(l2))
        float w, w2lxy = 0.0f, wdz = 0.0f, wZb = 0.0f;
        if (MODE == TIGRE_BP_FDK) {
            const float t = c.DSO * inv_den;
            w = t * t;
        } else {
            const float ex = X - A.srcx, ey = Y - A.srcy;
            w = c.wscale * inv_den * inv_den * inv_den;
            w2lxy = (w * w) * fmaf(ex, ex, ey * ey);
            wdz = w * c.dz;
            wZb = w * Zb;
        }
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
            uint32_t bq;
            float fv;
            split_bits(fmaf((float)k, dpv, pv0), bq, fv);
            // the cell of columns ip, ip + 1 and rows iq, iq + 1 (iq = bq - 0x4B000000)
            const auto* cell = col + (bq * (uint32_t)PU - row_bias);
            const float val = bilinear_value(ProjTaps<TP, QUADP>::load(cell, PU), fu, fv);
            float wk = w;
            if (MODE != TIGRE_BP_FDK) {
                const float Zw = fmaf((float)k, wdz, wZb);
                const float u2 = fmaf(Zw, Zw, w2lxy);
                wk = u2 * rsqrt_sfu(u2);
            }
            acc[k] = fmaf(wk, val, acc[k]);
            if (SART) {
                const uint32_t qq = bq - (0x4B000000u + (uint32_t)c.pv_lo);
                const float tv = (qq < (unsigned)c.nv ? 1.0f - fv : 0.0f) +
                                 (qq + 1u < (unsigned)c.nv ? fv : 0.0f);
                nrm[k] = fmaf(wk, tu * tv, nrm[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
        const int z = zb + k;
        if (z < c.z_end) {
            TV* o = vol + ((int64_t)(z - c.z_out0) * c.ny + y) * c.nx + x;
            if (SART) {
                const float den = nrm[k];
                float v = to_f32<TV>(*o);
                if (den > 1e-12f) v = fmaf(lambda, acc[k] / den, v);
                if (nonneg) v = fmaxf(v, 0.0f);
                *o = from_f32<TV>(v);
            } else {
                const float prev = accumulate ? to_f32<TV>(*o) : 0.0f;
                *o = from_f32<TV>(prev + acc[k]);
            }
        }
    }
}

template <typename TP>
__device__ __forceinline__ TP pix_or_zero(const TP* row, int p, int nu)
{
    return (unsigned)p < (unsigned)nu ? row[p] : from_f32<TP>(0.0f);
}

// Write the whole zero-bordered buffer of one angle range: with
// Z(r, c) = y[a][r - pv_lo][c - 2] (zero outside the detector), the plain
// buffer holds out[a][r][c] = Z(r, c), the quad buffer the FP32 bilinear
// coefficients of the cell (Z(r, c), Z(r, c+1), Z(r+1, c), Z(r+1, c+1)).
template <typename TP, bool QUADP>
__global__ void pad_proj_kernel(const TP* __restrict__ in,
                                typename ProjTaps<TP, QUADP>::E* __restrict__ out, int nu, int nv,
                                int PU, int PV, int pv_lo)
{
    const int r = blockIdx.y, a = blockIdx.z;
    const int q = r - pv_lo;
    typename ProjTaps<TP, QUADP>::E* dst = out + ((int64_t)a * PV + r) * PU;
    const TP* row0 = in + ((int64_t)a * nv + q) * nu;
    const TP* row1 = row0 + nu;
    const bool in0 = (unsigned)q < (unsigned)nv, in1 = (unsigned)(q + 1) < (unsigned)nv;
    const TP z = from_f32<TP>(0.0f);
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < PU; col += gridDim.x * blockDim.x) {
        const int p = col - kPad;
        const TP a00 = in0 ? pix_or_zero(row0, p, nu) : z;
        if constexpr (!QUADP) {
            dst[col] = a00;
        } else {
            const TP a01 = in0 ? pix_or_zero(row0, p + 1, nu) : z;
            const TP a10 = in1 ? pix_or_zero(row1, p, nu) : z;
            const TP a11 = in1 ? pix_or_zero(row1, p + 1, nu) : z;
            dst[col] = bilinear_coefficients(to_f32<TP>(a00), to_f32<TP>(a01), to_f32<TP>(a10),
                                             to_f32<TP>(a11));
        }
    }
}

// Exact adjoint: scatter every sample of each ray.
template <typename TP>
__global__ void __launch_bounds__(256) adj_scatter_kernel(const TP* __restrict__ proj,
                                                          float* __restrict__ acc_xy,
                                                          float* __restrict__ acc_yx,
                                                          const FwdAngle* __restrict__ params,
                                                          FwdConst c, int a_first)
{
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int q = blockIdx.z * blockDim.y + threadIdx.y;
    const int a = blockIdx.y;
    if (p >= c.nu || q >= c.nv) return;
    const float yv = to_f32<TP>(proj[((int64_t)a * c.nv + q) * c.nu + p]);
    if (yv == 0.0f) return;
    Ray R;
    setup_ray(params + a_first + a, c, p, q, R);
    if (!R.ok || R.K == 0) return;
    float* __restrict__ acc = R.layout ? acc_yx : acc_xy;
    const int PF = R.nf + 2 * kPad;
    const int PFM = PF * (R.nm + 2 * kPad);
    const float hy = R.h * yv;
    float kf = 0.0f;
    for (int k = 0; k < R.K; ++k, kf += 1.0f) {
        int i_f, i_m, i_s;
        float af, am, as;
        split_floor(fmaf(kf, R.d[0], R.x0[0]), i_f, af);
        split_floor(fmaf(kf, R.d[1], R.x0[1]), i_m, am);
        split_floor(fmaf(kf, R.d[2], R.x0[2]), i_s, as);
        float* b = acc + (i_s * PFM + i_m * PF + i_f);
        const float s0 = hy * (1.0f - as), s1 = hy * as;
        const float m00 = s0 * (1.0f - am), m01 = s0 * am, m10 = s1 * (1.0f - am), m11 = s1 * am;
        atomicAdd(b, m00 * (1.0f - af));
        atomicAdd(b + 1, m00 * af);
        atomicAdd(b + PF, m01 * (1.0f - af));
        atomicAdd(b + PF + 1, m01 * af);
        atomicAdd(b + PFM, m10 * (1.0f - af));
        atomicAdd(b + PFM + 1, m10 * af);
        atomicAdd(b + PFM + PF, m11 * (1.0f - af));
        atomicAdd(b + PFM + PF + 1, m11 * af);
    }
}

// vol[z][y][x] (+)= acc_xy[z+P][y+P][x+P] + acc_yx[z+P][x+P][y+P].
template <typename TV>
__global__ void adj_finish_kernel(const float* __restrict__ acc_xy,
                                  const float* __restrict__ acc_yx, TV* __restrict__ vol, int nx,
                                  int ny, int nz, int accumulate)
{
    __shared__ float tile[32][33];
    const int z = blockIdx.z;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int64_t zp = z + kPad;
    if (acc_yx) {
        const int PF = ny + 2 * kPad, PM = nx + 2 * kPad;
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            const int y = y0 + threadIdx.x, x = x0 + i;
            tile[i][threadIdx.x] =
                (x < nx && y < ny) ? acc_yx[(zp * PM + x + kPad) * PF + y + kPad] : 0.0f;
        }
    }
    __syncthreads();
    const int PF = nx + 2 * kPad, PM = ny + 2 * kPad;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + j;
        if (x >= nx || y >= ny) continue;
        float v = acc_xy ? acc_xy[(zp * PM + y + kPad) * PF + x + kPad] : 0.0f;
        if (acc_yx) v += tile[threadIdx.x][j];
        TV* o = vol + ((int64_t)z * ny + y) * nx + x;
        if (accumulate) v += to_f32<TV>(*o);
        *o = from_f32<TV>(v);
    }
}

// Bound, over every voxel a launch can touch (z-chunks rounded up to NZ) and
// every angle, of the detector row coordinate a voxel projects to; the padded
// buffer gets enough zero rows that all of them land inside it.
static BpConst make_bp_const(const tigre_geometry_desc& d)
{
    BpConst c;
    c.nx = (int)d.n_voxel[0];
    c.ny = (int)d.n_voxel[1];
    c.nz = (int)d.n_voxel[2];
    c.nu = (int)d.n_det[0];
    c.nv = (int)d.n_det[1];
    const double x0 = -0.5 * (double)(d.n_voxel[0] - 1) * d.d_voxel[0] + d.off_origin[0];
    const double y0 = -0.5 * (double)(d.n_voxel[1] - 1) * d.d_voxel[1] + d.off_origin[1];
    const double z0 = -0.5 * (double)(d.n_voxel[2] - 1) * d.d_voxel[2] + d.off_origin[2];
    c.x0 = (float)x0;
    c.y0 = (float)y0;
    c.z0 = (float)z0;
    c.dx = (float)d.d_voxel[0];
    c.dy = (float)d.d_voxel[1];
    c.dz = (float)d.d_voxel[2];
    c.DSO = (float)d.DSO;
    c.DSD = (float)d.DSD;
    c.inv_du = (float)(1.0 / d.d_det[0]);
    c.inv_dv = (float)(1.0 / d.d_det[1]);
    c.pu_off = (float)(0.5 * (double)(d.n_det[0] - 1) - d.off_det[0] / d.d_det[0]);
    c.pv_off = (float)(0.5 * (double)(d.n_det[1] - 1) - d.off_det[1] / d.d_det[1]);
    c.wscale = (float)(d.d_voxel[0] * d.d_voxel[1] * d.d_voxel[2] / (d.d_det[0] * d.d_det[1]) *
                       d.DSD * d.DSD);
    const double x1 = x0 + (double)(d.n_voxel[0] - 1) * d.d_voxel[0];
    const double y1 = y0 + (double)(d.n_voxel[1] - 1) * d.d_voxel[1];
    // Launches may start at any plane (z-slabs), so the last chunk of NZ
    // planes can reach up to nz + NZ - 2: bound that far.
    const int64_t nzc = d.n_voxel[2] + kBpNZ;
    const double z1 = z0 + (double)(nzc - 1) * d.d_voxel[2];
    const double R = std::sqrt(std::max(x0 * x0, x1 * x1) + std::max(y0 * y0, y1 * y1));
    const double mags[2] = {d.DSD / (d.DSO + R), d.DSD / (d.DSO - R)};
    double vmin = 1e300, vmax = -1e300;
    for (double Z : {z0, z1})
        for (double m : mags) {
            const double pv = Z * m / d.d_det[1] + (double)c.pv_off;
            vmin = std::min(vmin, pv);
            vmax = std::max(vmax, pv);
        }
    c.pv_lo = (int)std::max(2.0, std::ceil(-vmin) + 2.0);
    const int pv_hi = (int)std::max(2.0, std::ceil(vmax - (double)(c.nv - 1)) + 2.0);
    c.PV = c.nv + c.pv_lo + pv_hi;
    c.PU = c.nu + 2 * kPad;
    c.z_first = 0;
    c.z_end = c.nz;
    c.z_out0 = 0;
    return c;
}

// A launch over planes [z_first, z_end) pads only the detector rows those
// planes reach, with two rows of margin on either side for FP32 rounding.
// Its last chunk of NZ planes may run past z_end (those voxels are computed,
// and read rows, but not written): for any NZ <= kBpNZ it ends before
// z_end + kBpNZ - 1, the bound taken here.
static void bp_slab_band(BpConst& c, const tigre_geometry_desc& d, int z_first, int z_end)
{
    const int64_t z_last = (int64_t)z_end + kBpNZ - 2;
    double lo, hi;
    if (!detector_row_range(d, (double)z_first, (double)z_last, &lo, &hi)) return;
    const int r_lo = (int)std::floor(lo) - 2;
    const int r_hi = (int)std::ceil(hi) + 3;
    c.pv_lo = -r_lo;
    c.PV = r_hi - r_lo + 1;
}

size_t bp_slab_pad_bytes(const tigre_geometry_desc& d, int64_t slab, int64_t na)
{
    size_t most = 0;
    const int64_t nz = d.n_voxel[2];
    for (int64_t z0 = 0; z0 < nz; z0 += slab) {
        BpConst c = make_bp_const(d);
        bp_slab_band(c, d, (int)z0, (int)std::min(nz, z0 + slab));
        most = std::max(most, (size_t)na * (size_t)c.PU * (size_t)c.PV * sizeof(float));
    }
    return most;
}

// Whether a backprojection with weight w reads quad projections (both
// voxel-driven weights do, the in-core SART update included; out-of-core
// slab launches build them a quarter of the angles at a time).
static bool bp_reads_quads(tigre_bp_weight w)
{
    return w == TIGRE_BP_MATCHED || w == TIGRE_BP_FDK;
}

tigre_status backward_workspace(tigre_geometry* g, tigre_dtype pt, tigre_bp_weight w, int64_t a0,
                                int64_t na)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (!dtype_ok(pt)) return fail(TIGRE_ERR_INVALID_ARG, "bad dtype");
    const tigre_geometry_desc& d = g->desc;
    if (w == TIGRE_BP_EXACT_ADJOINT) {
        if (padded_elems(d) >= (size_t)INT32_MAX) return TIGRE_OK;  // refused by the operator
        bool need[2] = {false, false};
        for (int64_t a = a0; a < a0 + na; ++a) need[g->layout[(size_t)a]] = true;
        DeviceBuffer* bufs[2] = {&g->adj_xy, &g->adj_yx};
        for (int l = 0; l < 2; ++l)
            if (need[l]) TIGRE_TRY(bufs[l]->ensure(padded_elems(d) * sizeof(float)));
        return TIGRE_OK;
    }
    const BpConst c = make_bp_const(d);
    const size_t elem = bp_reads_quads(w) ? sizeof(float4) : dtype_size(pt);
    return g->proj_pad.ensure((size_t)na * (size_t)c.PU * (size_t)c.PV * elem);
}

// The launch of a voxel-driven backprojection over the planes c describes.
template <typename TP, typename TV, bool QUADP>
static tigre_status run_voxel_bp(tigre_geometry* g, const BpConst& c, const TP* proj, TV* vol,
                                 int64_t a0, int64_t na, tigre_bp_weight w, int accumulate,
                                 cudaStream_t st, bool sart, float lambda, int nonneg,
                                 int batch = 1, void* ws = nullptr)
{
    using Q = typename ProjTaps<TP, QUADP>::E;
    static_assert(sizeof(Q) == (QUADP ? 4 * sizeof(float) : sizeof(TP)),
                  "a quad is four FP32 coefficients");
    const size_t pelems = (size_t)na * (size_t)c.PU * (size_t)c.PV;
    Q* pp = (Q*)ws;
    if (!pp) {
        TIGRE_TRY(g->proj_pad.ensure(pelems * sizeof(Q)));
        g->proj_pad.tag = 0;
        pp = (Q*)g->proj_pad.ptr;
    }
    // a batch's projections are consecutive angle blocks of one long buffer
    for (int64_t s = 0; s < na * batch; s += 65535) {
        const int64_t cnt = std::min<int64_t>(65535, na * batch - s);
        dim3 grid((unsigned)((c.PU + 255) / 256), (unsigned)c.PV, (unsigned)cnt);
        pad_proj_kernel<TP, QUADP><<<grid, 256, 0, st>>>(proj + s * (int64_t)c.nu * c.nv,
                                                   pp + s * (int64_t)c.PU * c.PV, c.nu, c.nv,
                                                   c.PU, c.PV, c.pv_lo);
        TIGRE_LAUNCHED("pad_proj_kernel");
    }
    const BpAngle* params = (const BpAngle*)g->bp_params.ptr;
    const dim3 block(32, 8);
    ProfScope prof(kProfBackproject, st);
    // One kernel instance: MODE and SART fixed, NZ voxels per thread.
    auto launch = [&](auto mode, auto sart_tag) -> tigre_status {
        constexpr int M = decltype(mode)::value;
        constexpr bool S = decltype(sart_tag)::value;
        constexpr int NZ = bp_voxels_per_thread<M, S, QUADP>();
        const int chunks = (c.z_end - c.z_first + NZ - 1) / NZ;
        dim3 grid((unsigned)((c.nx + 31) / 32), (unsigned)((c.ny + 7) / 8),
                  (unsigned)((int64_t)chunks * batch));
        if (grid.y > 65535 || (int64_t)chunks * batch > 65535)
            return fail(TIGRE_ERR_UNSUPPORTED, "volume too large");
        BpBatch bt;
        if (batch > 1) {
            bt.chunks = chunks;
            bt.proj_stride = (int64_t)pelems;
            bt.vol_stride = (int64_t)c.nx * c.ny * c.nz;
        }
        // Single launches take the instance without member offsets (512^3 x
        // 360: FDK 36.3 vs 41.6 ms, matched 40.8 vs 41.2), except the SART
        // update, whose instance with them compiles to a faster kernel (SIRT
        // pass 58.0 vs 59.0 ms); with one member the offsets are zero.
        constexpr bool kSingle = !S;  // SART: the instance with offsets only
        if (!kSingle || batch > 1)
            bp_voxel_kernel<TP, TV, NZ, M, S, QUADP, true><<<grid, block, 0, st>>>(
                pp, vol, params, c, (int)a0, (int)na, S ? 0 : accumulate, lambda, nonneg, bt);
        else if constexpr (kSingle)
            bp_voxel_kernel<TP, TV, NZ, M, S, QUADP><<<grid, block, 0, st>>>(
                pp, vol, params, c, (int)a0, (int)na, accumulate, lambda, nonneg, bt);
        return TIGRE_OK;
    };
    using Fdk = std::integral_constant<int, TIGRE_BP_FDK>;
    using Matched = std::integral_constant<int, TIGRE_BP_MATCHED>;
    tigre_status ls;
    if (sart)
        ls = w == TIGRE_BP_FDK ? launch(Fdk{}, std::true_type{}) : launch(Matched{}, std::true_type{});
    else
        ls = w == TIGRE_BP_FDK ? launch(Fdk{}, std::false_type{})
                               : launch(Matched{}, std::false_type{});
    TIGRE_TRY(ls);
    TIGRE_LAUNCHED("bp_voxel_kernel");
    return TIGRE_OK;
}

// Voxel planes [z_first, z_end) into an output buffer whose first plane is
// z_out0 (in-core: 0, nz, 0; out-of-core slabs: the slab's planes).
template <typename TP, typename TV>
tigre_status launch_voxel_bp(tigre_geometry* g, const TP* proj, TV* vol, int64_t a0, int64_t na,
                             tigre_bp_weight w, int accumulate, cudaStream_t st, bool sart = false,
                             float lambda = 0.0f, int nonneg = 0, int z_first = 0, int z_end = -1,
                             int z_out0 = 0)
{
    const tigre_geometry_desc& d = g->desc;
    BpConst c = make_bp_const(d);
    if (z_end >= 0) {
        if (z_first < 0 || z_end > c.nz || z_first >= z_end || z_out0 > z_first)
            return fail(TIGRE_ERR_INVALID_ARG, "bad z range");
        c.z_first = z_first;
        c.z_end = z_end;
        c.z_out0 = z_out0;
        bp_slab_band(c, d, z_first, z_end);
    }
    if (!bp_reads_quads(w))
        return run_voxel_bp<TP, TV, false>(g, c, proj, vol, a0, na, w, accumulate, st, sart,
                                           lambda, nonneg);
    if (z_end < 0)
        return run_voxel_bp<TP, TV, true>(g, c, proj, vol, a0, na, w, accumulate, st, sart, lambda,
                                          nonneg);
    // A slab's band of quads for all angles would take four times the plain
    // band, so slab launches take their angles a quarter at a time (the
    // later quarters adding into the slab): the band of one quarter fits in
    // the bytes of the plain band.
    if (sart || na < 4)
        return run_voxel_bp<TP, TV, false>(g, c, proj, vol, a0, na, w, accumulate, st, sart,
                                           lambda, nonneg);
    const int64_t chunk = na / 4;
    for (int64_t c0 = 0; c0 < na; c0 += chunk) {
        const int64_t cnt = std::min(chunk, na - c0);
        TIGRE_TRY((run_voxel_bp<TP, TV, true>(g, c, proj + c0 * (int64_t)c.nu * c.nv, vol, a0 + c0,
                                              cnt, w, c0 > 0 ? 1 : accumulate, st, false, 0.0f,
                                              0)));
    }
    return TIGRE_OK;
}


size_t backward_batch_workspace_bytes(const tigre_geometry* g, tigre_dtype dt)
{
    const BpConst c = make_bp_const(g->desc);
    (void)dt;  // quads hold FP32 coefficients for every storage type
    return (size_t)g->angles.size() * (size_t)c.PU * (size_t)c.PV * sizeof(float4);
}

tigre_status backward_batch_impl(tigre_geometry* g, const void* projs, void* vols, int batch,
                                 tigre_dtype dt, tigre_bp_weight w, void* ws, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    if (!bp_reads_quads(w))
        return fail(TIGRE_ERR_UNSUPPORTED, "batched backprojection: matched or FDK weights");
    const BpConst c = make_bp_const(g->desc);
    const int64_t na = (int64_t)g->angles.size();
    return dispatch_dtype(dt, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        return run_voxel_bp<T, T, true>(g, c, (const T*)projs, (T*)vols, 0, na, w, 0, st, false,
                                        0.0f, 0, batch, ws);
    });
}

tigre_status backward_slab_impl(tigre_geometry* g, const float* proj, float* vol_slab, int64_t a0,
                                int64_t na, tigre_bp_weight w, int accumulate, int z_first,
                                int z_end, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (w == TIGRE_BP_EXACT_ADJOINT)
        return fail(TIGRE_ERR_UNSUPPORTED, "out-of-core backprojection is voxel-driven");
    return launch_voxel_bp<float, float>(g, proj, vol_slab, a0, na, w, accumulate, st, false, 0.0f,
                                         0, z_first, z_end, z_first);
}

tigre_status sart_update_dt(tigre_geometry* g, tigre_dtype t, const void* r, void* x, int64_t a0,
                            int64_t na, tigre_bp_weight w, float lambda, int nonneg,
                            cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (w == TIGRE_BP_EXACT_ADJOINT)
        return fail(TIGRE_ERR_UNSUPPORTED, "SIRT/OS-SART use the voxel-driven backprojector");
    return dispatch_dtype(t, [&](auto tag) -> tigre_status {
        using T = decltype(tag);
        return launch_voxel_bp<T, T>(g, (const T*)r, (T*)x, a0, na, w, 0, st, true, lambda,
                                     nonneg);
    });
}

tigre_status sart_update_impl(tigre_geometry* g, const float* r, float* x, int64_t a0, int64_t na,
                              tigre_bp_weight w, float lambda, int nonneg, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (w == TIGRE_BP_EXACT_ADJOINT)
        return fail(TIGRE_ERR_UNSUPPORTED, "SIRT/OS-SART use the voxel-driven backprojector");
    return launch_voxel_bp<float, float>(g, r, x, a0, na, w, 0, st, true, lambda, nonneg);
}

template <typename TP, typename TV>
static tigre_status launch_adjoint(tigre_geometry* g, const TP* proj, TV* vol, int64_t a0,
                                   int64_t na, int accumulate, cudaStream_t st)
{
    const tigre_geometry_desc& d = g->desc;
    if (padded_elems(d) >= (size_t)INT32_MAX)
        return fail(TIGRE_ERR_UNSUPPORTED, "exact adjoint needs (nx+4)(ny+4)(nz+4) < 2^31");
    const FwdConst c = make_fwd_const(g);
    bool need[2] = {false, false};
    for (int64_t a = a0; a < a0 + na; ++a) need[g->layout[(size_t)a]] = true;
    DeviceBuffer* bufs[2] = {&g->adj_xy, &g->adj_yx};
    const size_t bytes = padded_elems(d) * sizeof(float);
    for (int l = 0; l < 2; ++l) {
        if (!need[l]) continue;
        TIGRE_TRY(bufs[l]->ensure(bytes));
        bufs[l]->tag = 0;  // contents are accumulator data, not a zero-bordered layout
        TIGRE_CUDA(cudaMemsetAsync(bufs[l]->ptr, 0, bytes, st));
    }
    float* axy = need[0] ? (float*)g->adj_xy.ptr : nullptr;
    float* ayx = need[1] ? (float*)g->adj_yx.ptr : nullptr;
    ProfScope prof(kProfAdjoint, st);
    if (g->projector == TIGRE_PROJ_SIDDON) {
        TIGRE_TRY(launch_siddon_scatter<TP>(g, proj, axy, ayx, a0, na, st));
    } else {
        for (int64_t s = 0; s < na; s += 65535) {
            const int64_t cnt = std::min<int64_t>(65535, na - s);
            dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
            adj_scatter_kernel<TP><<<grid, dim3(32, 8), 0, st>>>(
                proj + s * (int64_t)c.nu * c.nv, axy, ayx, (const FwdAngle*)g->fwd_params.ptr, c,
                (int)(a0 + s));
            TIGRE_LAUNCHED("adj_scatter_kernel");
        }
    }
    dim3 grid((unsigned)((c.nx + 31) / 32), (unsigned)((c.ny + 31) / 32), (unsigned)c.nz);
    adj_finish_kernel<TV><<<grid, dim3(32, 8), 0, st>>>(axy, ayx, vol, c.nx, c.ny, c.nz,
                                                        accumulate);
    TIGRE_LAUNCHED("adj_finish_kernel");
    return TIGRE_OK;
}

tigre_status backward_impl(tigre_geometry* g, const void* proj, tigre_dtype pt, void* vol,
                           tigre_dtype vt, int64_t a0, int64_t na, tigre_bp_weight w,
                           int accumulate, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (!vol || !proj) return fail(TIGRE_ERR_INVALID_ARG, "null vol or proj pointer");
    if (!dtype_ok(vt) || !dtype_ok(pt)) return fail(TIGRE_ERR_INVALID_ARG, "bad dtype");
    if (w != TIGRE_BP_MATCHED && w != TIGRE_BP_FDK && w != TIGRE_BP_EXACT_ADJOINT)
        return fail(TIGRE_ERR_INVALID_ARG, "bad backprojection weight");
    return dispatch_dtype(pt, [&](auto ptag) -> tigre_status {
        using TP = decltype(ptag);
        return dispatch_dtype(vt, [&](auto vtag) -> tigre_status {
            using TV = decltype(vtag);
            if (w == TIGRE_BP_EXACT_ADJOINT)
                return launch_adjoint<TP, TV>(g, (const TP*)proj, (TV*)vol, a0, na, accumulate, st);
            return launch_voxel_bp<TP, TV>(g, (const TP*)proj, (TV*)vol, a0, na, w, accumulate, st);
        });
    });
}

}  // namespace tigre

extern "C" tigre_status tigre_backward(tigre_geometry_t geo, const void* proj,
                                       tigre_dtype proj_dtype, void* vol, tigre_dtype vol_dtype,
                                       int64_t angle_begin, int64_t angle_count,
                                       tigre_bp_weight weight, void* cuda_stream)
{
    return tigre::backward_impl(geo, proj, proj_dtype, vol, vol_dtype, angle_begin, angle_count,
                                weight, 0, (cudaStream_t)cuda_stream);
}
