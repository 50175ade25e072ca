// Forward projector, shared-memory slab path (TMA + mbarrier double buffer).
//
// Same definition as the L1 path (forward.cu, paper Sec. 2.1): each ray's
// K midpoint samples of the trilinear interpolant, summed in order k = 0..K-1
// and scaled by h.  Only where the taps come from differs.
//
// A block owns 32 x 8 adjacent pixels of one angle (8 warps = 8 detector
// rows).  Their rays cross the volume roughly along the layout's middle
// axis m.  The block walks m in slabs of TS cell layers; for each slab it
// computes the exact tap range of all samples that fall in it (a block
// min/max of the first and last sample of each ray), and one thread issues a
// 3-D TMA box load of FB x (TS+1) x SB voxels (f, m, s) into shared memory.
// Coordinates outside the volume read zeros (TMA out-of-bounds fill), which
// are exactly the interpolant's virtual zero voxels.  Two stages alternate:
// the load of slab i+2 is in flight while slab i is being sampled.  Taps are
// shared-memory loads with compile-time offsets (+1, +FB, +(TS+1)FB), so the
// per-sample cost is ~40 instructions and no L1 tag lookups.
//
// Waits on an mbarrier are bounded; a timeout, a tile that would not hold a
// slab's taps, or rays that do not all run the same way along m set an error
// bit and NaN the affected rays (the host chooses this path only when a
// conservative bound says none of these can happen).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "ray.cuh"

namespace tigre {

constexpr int kTmaFB = 96;  // box width along f (voxels)
constexpr int kTmaSB = 16;  // box height along s
constexpr int kTmaTS = 5;   // cell layers per slab along m (box depth TS + 1)

template <typename TV>
struct TileCfg {
    static constexpr int FB = kTmaFB, SB = kTmaSB, TS = kTmaTS, MP = kTmaTS + 1;
    static constexpr int SP = MP * FB;    // elements per s-plane of the box
    static constexpr int STAGE = SB * SP; // elements per stage
    static constexpr uint32_t STAGE_BYTES = (uint32_t)(STAGE * sizeof(TV));
    static constexpr int ALIGN = 16 / (int)sizeof(TV);  // TMA x granularity (elements)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false if the phase did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ int cell_of(float x)
{
    int i;
    float f;
    split_floor(x, i, f);
    return i;
}

__device__ __forceinline__ int floor_div(int a, int b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Error bits written to the flag word.
constexpr int kErrTimeout = 1, kErrTile = 2, kErrDirection = 4;

template <typename TV, typename TP>
__global__ void __launch_bounds__(256) fwd_tma_kernel(const __grid_constant__ CUtensorMap map0,
                                                      const __grid_constant__ CUtensorMap map1,
                                                      TP* __restrict__ proj,
                                                      const FwdAngle* __restrict__ params,
                                                      FwdConst c, int a_first,
                                                      int* __restrict__ err)
{
    using C = TileCfg<TV>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned: round the base up (the
    // launch allocates 128 spare bytes).
    const uint32_t raw = smem_u32(smem_raw);
    TV* tiles = reinterpret_cast<TV*>(smem_raw + ((128u - (raw & 127u)) & 127u));
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int red[8][4];
    __shared__ int st_base[2], st_ok[2];
    __shared__ int blk[3];  // C0, nslab, ascending

    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
    const int p = blockIdx.x * 32 + lane;
    const int q = blockIdx.z * 8 + warp;
    const int a = blockIdx.y;
    const bool inside = p < c.nu && q < c.nv;
    const FwdAngle* P = params + a_first + a;
    const CUtensorMap* map = P->layout ? &map1 : &map0;

    Ray R;
    R.K = 0;
    R.ok = true;
    if (inside) setup_ray(P, c, p, q, R);
    const bool active = inside && R.ok && R.K > 0;
    const int any = __syncthreads_or(active);
    const int all_pos = __syncthreads_and(!active || R.d[1] > 0.0f);
    const int all_neg = __syncthreads_and(!active || R.d[1] < 0.0f);
    bool bad = inside && !R.ok;
    float acc = 0.0f;

    if (any && (all_pos || all_neg)) {
        const bool asc = all_pos != 0;
        // Cells along m of the first and last sample of this ray.
        const int cf = active ? cell_of(R.x0[1]) : 0;
        const int cl = active ? cell_of(fmaf((float)(R.K - 1), R.d[1], R.x0[1])) : 0;
        {
            int v0 = active ? (asc ? cf : -cf) : INT32_MAX;  // min of oriented first cell
            int v1 = active ? (asc ? cl : -cl) : INT32_MIN;  // max of oriented last cell
            for (int o = 16; o > 0; o >>= 1) {
                v0 = min(v0, __shfl_xor_sync(full, v0, o));
                v1 = max(v1, __shfl_xor_sync(full, v1, o));
            }
            if (lane == 0) {
                red[warp][0] = v0;
                red[warp][1] = v1;
            }
            if (tid == 0) {
                mbar_init(smem_u32(&bars[0]), 1);
                mbar_init(smem_u32(&bars[1]), 1);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            __syncthreads();
            if (tid == 0) {
                int m0 = INT32_MAX, m1 = INT32_MIN;
                for (int w = 0; w < 8; ++w) {
                    m0 = min(m0, red[w][0]);
                    m1 = max(m1, red[w][1]);
                }
                blk[0] = asc ? m0 : -m0;  // first cell layer visited
                blk[1] = (m1 - m0) / C::TS + 1;
                blk[2] = asc;
            }
            __syncthreads();
        }
        const int C0 = blk[0], nslab = blk[1];

        // Sample range of slab s: cells [lo, lo + TS), lo = C0 + s TS going
        // up, C0 - (s + 1) TS + 1 going down; returns the first sample index
        // past the slab, starting from kstart.
        auto slab_lo = [&](int s) { return asc ? C0 + s * C::TS : C0 - (s + 1) * C::TS + 1; };
        auto slab_end = [&](int s, int kstart) -> int {
            if (!active) return kstart;
            const int lo = slab_lo(s), hi = lo + C::TS;
            const float bound = asc ? (float)hi : (float)lo;
            int kn = (int)ceilf((bound - R.x0[1]) / R.d[1]);
            kn = min(max(kn, kstart), R.K);
            auto beyond = [&](int k) {
                const int cm = cell_of(fmaf((float)k, R.d[1], R.x0[1]));
                return asc ? cm >= hi : cm < lo;
            };
            // Exact membership (cells are monotone in k): the estimate is off
            // by at most one sample, but the loops are bounded by K, not trust.
            while (kn < R.K && !beyond(kn)) ++kn;
            while (kn > kstart && beyond(kn - 1)) --kn;
            return kn;
        };

        // Reduce the tap range of slab s over the block and issue its load.
        auto issue = [&](int s, int k_begin, int k_end) {
            int v[4] = {INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN};
            if (k_end > k_begin) {
                const int f0 = cell_of(fmaf((float)k_begin, R.d[0], R.x0[0]));
                const int f1 = cell_of(fmaf((float)(k_end - 1), R.d[0], R.x0[0]));
                const int s0 = cell_of(fmaf((float)k_begin, R.d[2], R.x0[2]));
                const int s1 = cell_of(fmaf((float)(k_end - 1), R.d[2], R.x0[2]));
                v[0] = min(f0, f1);
                v[1] = max(f0, f1) + 1;
                v[2] = min(s0, s1);
                v[3] = max(s0, s1) + 1;
            }
            for (int o = 16; o > 0; o >>= 1) {
                v[0] = min(v[0], __shfl_xor_sync(full, v[0], o));
                v[1] = max(v[1], __shfl_xor_sync(full, v[1], o));
                v[2] = min(v[2], __shfl_xor_sync(full, v[2], o));
                v[3] = max(v[3], __shfl_xor_sync(full, v[3], o));
            }
            if (lane == 0)
                for (int j = 0; j < 4; ++j) red[warp][j] = v[j];
            __syncthreads();
            if (tid == 0) {
                int fmin = INT32_MAX, fmax = INT32_MIN, smin = INT32_MAX, smax = INT32_MIN;
                for (int w = 0; w < 8; ++w) {
                    fmin = min(fmin, red[w][0]);
                    fmax = max(fmax, red[w][1]);
                    smin = min(smin, red[w][2]);
                    smax = max(smax, red[w][3]);
                }
                const int stage = s & 1;
                const int lo = slab_lo(s);
                int F0 = 0, S0 = 0, ok = 1;
                if (fmin <= fmax) {
                    F0 = floor_div(fmin - kPad, C::ALIGN) * C::ALIGN;  // unpadded, aligned
                    S0 = smin - kPad;
                    ok = (fmax - kPad < F0 + C::FB) && (smax - kPad < S0 + C::SB);
                }
                st_ok[stage] = ok;
                // smem index of padded cell (cs, cm, cf) = cs SP + cm FB + cf - base
                st_base[stage] = (S0 + kPad) * C::SP + lo * C::FB + (F0 + kPad);
                const uint32_t bar = smem_u32(&bars[stage]);
                mbar_expect_tx(bar, C::STAGE_BYTES);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load_3d(smem_u32(tiles + stage * C::STAGE), map, F0, lo - kPad, S0, bar);
            }
            __syncthreads();
        };

        int k0 = 0;
        int k1 = slab_end(0, 0);
        issue(0, 0, k1);
        int k2 = k1;
        if (nslab > 1) {
            k2 = slab_end(1, k1);
            issue(1, k1, k2);
        }
        bool timed_out = false;
        int waited = 0;  // slabs whose load has completed
        for (int s = 0; s < nslab; ++s) {
            const int stage = s & 1;
            const bool landed = mbar_wait_bounded(smem_u32(&bars[stage]), (uint32_t)((s >> 1) & 1));
            if (__syncthreads_or(!landed)) {  // block-uniform decision
                timed_out = true;
                break;
            }
            waited = s + 1;
            const TV* tile = tiles + stage * C::STAGE;
            const int base = st_base[stage];
            const bool ok = st_ok[stage] != 0;
            int n = k1 - k0;
            int nmax = n;
            for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(full, nmax, o));
            if (!ok && n > 0) bad = true;
            if (!ok && tid == 0) atomicOr(err, kErrTile);
            float kf = (float)k0;
            for (int j = 0; j < nmax; ++j, kf += 1.0f) {
                if (ok && j < n) {
                    int i_f, i_m, i_s;
                    float af, am, as;
                    split_floor(fmaf(kf, R.d[0], R.x0[0]), i_f, af);
                    split_floor(fmaf(kf, R.d[1], R.x0[1]), i_m, am);
                    split_floor(fmaf(kf, R.d[2], R.x0[2]), i_s, as);
                    const TV* b = tile + (i_s * C::SP + i_m * C::FB + i_f - base);
                    const float v000 = to_f32<TV>(b[0]), v100 = to_f32<TV>(b[1]);
                    const float v010 = to_f32<TV>(b[C::FB]), v110 = to_f32<TV>(b[C::FB + 1]);
                    const float v001 = to_f32<TV>(b[C::SP]), v101 = to_f32<TV>(b[C::SP + 1]);
                    const float v011 = to_f32<TV>(b[C::SP + C::FB]);
                    const float v111 = to_f32<TV>(b[C::SP + C::FB + 1]);
                    const float c0 =
                        bilinear_value(bilinear_coefficients(v000, v100, v010, v110), af, am);
                    const float c1 =
                        bilinear_value(bilinear_coefficients(v001, v101, v011, v111), af, am);
                    acc += fmaf(as, c1 - c0, c0);
                }
            }
            __syncthreads();  // every warp is done with this stage
            int k3 = k2;
            if (s + 2 < nslab) {
                k3 = slab_end(s + 2, k2);
                issue(s + 2, k2, k3);
            }
            k0 = k1;
            k1 = k2;
            k2 = k3;
        }
        if (timed_out) {
            // Give loads still in flight a bounded chance to land before exit.
            for (int s = waited; s < min(nslab, waited + 2); ++s)
                mbar_wait_bounded(smem_u32(&bars[s & 1]), (uint32_t)((s >> 1) & 1));
            if (tid == 0) atomicOr(err, kErrTimeout);
            bad = bad || active;
        }
    } else if (any) {
        if (tid == 0) atomicOr(err, kErrDirection);
        bad = bad || active;
    }
    if (!inside) return;
    const float out = bad ? __int_as_float(0x7fc00000) : acc * R.h;
    proj[((int64_t)a * c.nv + q) * c.nu + p] = from_f32<TP>(out);
}

// ------------------------------------------------------------------- host

// out[z][x][y] = vol[z][y][x] with row pitch `pitch` (elements), 32x32 tiles.
template <typename T>
__global__ void transpose_yx_kernel(const T* __restrict__ vol, T* __restrict__ out, int nx, int ny,
                                    int pitch)
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
    T* dst = out + (int64_t)z * nx * pitch;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + i;
        if (x < nx && y < ny) dst[(int64_t)x * pitch + y] = tile[threadIdx.x][i];
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

template <typename TV>
static CUtensorMapDataType tma_dtype();
template <> CUtensorMapDataType tma_dtype<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tma_dtype<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> CUtensorMapDataType tma_dtype<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

template <typename TV>
static tigre_status encode_map(CUtensorMap* map, const void* base, int nf, int nm, int ns,
                               int pitch)
{
    using C = TileCfg<TV>;
    auto fn = encode_fn();
    if (!fn) return fail(TIGRE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[3] = {(cuuint64_t)nf, (cuuint64_t)nm, (cuuint64_t)ns};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(TV),
                                   (cuuint64_t)pitch * (cuuint64_t)nm * sizeof(TV)};
    const cuuint32_t box[3] = {(cuuint32_t)C::FB, (cuuint32_t)C::MP, (cuuint32_t)C::SB};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, tma_dtype<TV>(), 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TIGRE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return TIGRE_OK;
}

// Conservative host bound: can every block-slab of this geometry be staged in
// one box, and do all rays of a block run the same way along m?
bool tma_forward_fits(const tigre_geometry_desc& d, size_t elem)
{
    const double rx = 0.5 * (double)(d.n_voxel[0] + 1) * d.d_voxel[0] + std::fabs(d.off_origin[0]);
    const double ry = 0.5 * (double)(d.n_voxel[1] + 1) * d.d_voxel[1] + std::fabs(d.off_origin[1]);
    const double rz = 0.5 * (double)(d.n_voxel[2] + 1) * d.d_voxel[2] + std::fabs(d.off_origin[2]);
    const double R = std::sqrt(rx * rx + ry * ry);
    if (!(R < d.DSO)) return false;
    const double phi = std::asin(R / d.DSO);
    const double kDeg = M_PI / 180.0;
    if (45.0 * kDeg + phi > 75.0 * kDeg) return false;
    const double tan_max = std::tan(45.0 * kDeg + phi);
    const double Lmax = std::sqrt((d.DSO + R) * (d.DSO + R) + rz * rz);
    const double dfm = std::min(d.d_voxel[0], d.d_voxel[1]);  // f axis is x or y
    const double dmM = std::max(d.d_voxel[0], d.d_voxel[1]);  // m axis is the other
    const int align = 16 / (int)elem;
    // 32 pixels span 32 du L/DSD perpendicular to the rays; a ray at angle
    // a to the m axis crosses a plane m = const 1/cos(a) times as far apart.
    const double lat_f = 32.0 * d.d_det[0] * Lmax / d.DSD / dfm / std::cos(45.0 * kDeg + phi);
    const double need_f = lat_f + kTmaTS * (dmM / dfm) * tan_max + 2.0 + 1.0 + (align - 1);
    const double vmax = 0.5 * (double)d.n_det[1] * d.d_det[1] + std::fabs(d.off_det[1]);
    const double slope = vmax / (d.DSD * std::cos(45.0 * kDeg + phi));
    const double lat_s = 8.0 * d.d_det[1] * Lmax / d.DSD / d.d_voxel[2];
    // A row's rays cross a plane m = const at depths that differ by up to the
    // f-extent, and z = v depth / DSD moves with depth: rows far from the
    // mid-plane need that much more height.
    const double couple = (vmax / d.DSD) * need_f * dfm / d.d_voxel[2];
    const double need_s = lat_s + couple + kTmaTS * (dmM / d.d_voxel[2]) * slope + 2.0 + 1.0;
    return need_f <= (double)kTmaFB && need_s <= (double)kTmaSB;
}

tigre_status tma_workspace(tigre_geometry* g, size_t elem, const bool need[2])
{
    const tigre_geometry_desc& d = g->desc;
    const size_t nx = (size_t)d.n_voxel[0], ny = (size_t)d.n_voxel[1], nz = (size_t)d.n_voxel[2];
    const size_t align = 16 / elem;  // TileCfg<TV>::ALIGN
    if (need[0]) {
        const size_t pitch = (nx + align - 1) / align * align;
        TIGRE_TRY(g->vol_xy.ensure(pitch * ny * nz * elem));
    }
    if (need[1]) {
        const size_t pitch = (ny + align - 1) / align * align;
        TIGRE_TRY(g->vol_yx.ensure(pitch * nx * nz * elem));
    }
    return TIGRE_OK;
}

template <typename TV, typename TP>
tigre_status launch_forward_tma(tigre_geometry* g, const TV* vol, TP* proj, int64_t a0, int64_t na,
                                const bool need[2], int* d_err, cudaStream_t st)
{
    using C = TileCfg<TV>;
    const tigre_geometry_desc& d = g->desc;
    const int nx = (int)d.n_voxel[0], ny = (int)d.n_voxel[1], nz = (int)d.n_voxel[2];
    const int align = C::ALIGN;
    CUtensorMap maps[2];
    std::memset(maps, 0, sizeof(maps));
    if (need[0]) {
        const bool direct = (nx % align == 0) && ((uintptr_t)vol % 16 == 0);
        const int pitch = (nx + align - 1) / align * align;
        const void* src = vol;
        if (!direct) {
            TIGRE_TRY(g->vol_xy.ensure((size_t)pitch * ny * nz * sizeof(TV)));
            g->vol_xy.tag = 0;
            TIGRE_CUDA(cudaMemcpy2DAsync(g->vol_xy.ptr, (size_t)pitch * sizeof(TV), vol,
                                         (size_t)nx * sizeof(TV), (size_t)nx * sizeof(TV),
                                         (size_t)ny * nz, cudaMemcpyDeviceToDevice, st));
            src = g->vol_xy.ptr;
        }
        TIGRE_TRY(encode_map<TV>(&maps[0], src, nx, ny, nz, pitch));
    }
    if (need[1]) {
        const int pitch = (ny + align - 1) / align * align;
        TIGRE_TRY(g->vol_yx.ensure((size_t)pitch * nx * nz * sizeof(TV)));
        g->vol_yx.tag = 0;
        dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 31) / 32), (unsigned)nz);
        transpose_yx_kernel<TV><<<grid, dim3(32, 8), 0, st>>>(vol, (TV*)g->vol_yx.ptr, nx, ny, pitch);
        TIGRE_LAUNCHED("transpose_yx_kernel");
        TIGRE_TRY(encode_map<TV>(&maps[1], g->vol_yx.ptr, ny, nx, nz, pitch));
    }
    const size_t smem = 2 * (size_t)C::STAGE_BYTES + 128;
    static_assert(C::STAGE_BYTES % 128 == 0, "stages must keep 128-byte alignment");
    static bool attr_set[3][3] = {};
    bool& set = attr_set[sizeof(TV) == 4 ? 0 : (std::is_same<TV, __half>::value ? 2 : 1)]
                        [sizeof(TP) == 4 ? 0 : (std::is_same<TP, __half>::value ? 2 : 1)];
    if (!set) {
        TIGRE_CUDA(cudaFuncSetAttribute(fwd_tma_kernel<TV, TP>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        set = true;
    }
    const FwdConst c = make_fwd_const(g);
    ProfScope prof(kProfForward, st);
    for (int64_t s = 0; s < na; s += 65535) {
        const int64_t cnt = std::min<int64_t>(65535, na - s);
        dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
        fwd_tma_kernel<TV, TP><<<grid, dim3(32, 8), smem, st>>>(
            maps[0], maps[1], proj + s * (int64_t)c.nu * c.nv, (const FwdAngle*)g->fwd_params.ptr,
            c, (int)(a0 + s), d_err);
        TIGRE_LAUNCHED("fwd_tma_kernel");
    }
    return TIGRE_OK;
}

#define TIGRE_INST(TV, TP)                                                                       \
    template tigre_status launch_forward_tma<TV, TP>(tigre_geometry*, const TV*, TP*, int64_t,   \
                                                     int64_t, const bool[2], int*, cudaStream_t);
TIGRE_INST(float, float)
TIGRE_INST(float, __nv_bfloat16)
TIGRE_INST(float, __half)
TIGRE_INST(__nv_bfloat16, float)
TIGRE_INST(__nv_bfloat16, __nv_bfloat16)
TIGRE_INST(__nv_bfloat16, __half)
TIGRE_INST(__half, float)
TIGRE_INST(__half, __nv_bfloat16)
TIGRE_INST(__half, __half)
#undef TIGRE_INST

}  // namespace tigre
