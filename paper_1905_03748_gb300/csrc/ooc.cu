// Out-of-core operators: the paper's splitting (Alg. 1 for the projection,
// Alg. 2 for the backprojection, Sec. 2.1-2.2) recast for one GPU whose
// volume lives in host memory.
//
// Forward (Alg. 1): the volume is cut into axial slabs (z ranges).  Slab s
// is copied to the device on a copy stream while slab s-1 is projected, then
// zero-padded and projected, and its partial sums are added into the
// projections, which stay on the device for all slabs.  A sample belongs to
// the slab that holds its lower z tap (cells [z0, z1)); the slab buffer holds
// planes z0..z1 (one halo plane), so every sample finds both z taps and the
// slab sums add up to the in-core projection (up to FP32 summation order).
// The paper accumulates partial projections with a separate kernel (Sec. 2.1:
// about 0.01 % of a projection launch); here the slab kernel adds into the
// output directly.
//
// Backward (Alg. 2): each z-slab of the volume is backprojected from all
// angles into a device slab buffer and copied out while the next slab is
// computed (two slab buffers).  Projections are either device-resident or
// streamed from host memory in angle chunks through two buffers, as in
// Alg. 2.
//
// Host volumes and host projections are F32.  Pageable host memory is
// page-locked for the duration of the call (cudaHostRegister), the paper's
// page-locking step (Alg. 1/2, "page-lock image memory").
#include <algorithm>
#include <cmath>

#include "ray.cuh"

namespace tigre {

namespace {

__device__ __forceinline__ int cell_at(const Ray& R, int axis, int k)
{
    int i;
    float f;
    split_floor(fmaf((float)k, R.d[axis], R.x0[axis]), i, f);
    return i;
}

// First k in [0, K] with pred(k) true, for pred monotone false -> true.
template <typename P>
__device__ __forceinline__ int first_true(int K, P pred)
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

// Adds to proj the samples whose z cell (padded) lies in [cell_lo, cell_hi),
// reading a padded slab layout whose plane 0 is full padded plane plane0.
__global__ void __launch_bounds__(256) fwd_slab_kernel(const float* __restrict__ vxy,
                                                       const float* __restrict__ vyx,
                                                       float* __restrict__ proj,
                                                       const FwdAngle* __restrict__ params,
                                                       FwdConst c, int a_first, int cell_lo,
                                                       int cell_hi, int plane0)
{
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int q = blockIdx.z * blockDim.y + threadIdx.y;
    const int a = blockIdx.y;
    if (p >= c.nu || q >= c.nv) return;
    Ray R;
    setup_ray(params + a_first + a, c, p, q, R);
    float* out = proj + ((int64_t)a * c.nv + q) * c.nu + p;
    if (!R.ok) {
        *out = __int_as_float(0x7fc00000);
        return;
    }
    if (R.K == 0) return;
    int kb, ke;
    if (R.d[2] > 0.0f) {
        kb = first_true(R.K, [&](int k) { return cell_at(R, 2, k) >= cell_lo; });
        ke = first_true(R.K, [&](int k) { return cell_at(R, 2, k) >= cell_hi; });
    } else if (R.d[2] < 0.0f) {
        kb = first_true(R.K, [&](int k) { return cell_at(R, 2, k) < cell_hi; });
        ke = first_true(R.K, [&](int k) { return cell_at(R, 2, k) < cell_lo; });
    } else {
        const int cz = cell_at(R, 2, 0);
        const bool in = cz >= cell_lo && cz < cell_hi;
        kb = 0;
        ke = in ? R.K : 0;
    }
    if (ke <= kb) return;
    const float* __restrict__ vol = R.layout ? vyx : vxy;
    const int PF = R.nf + 2 * kPad;
    const int PFM = PF * (R.nm + 2 * kPad);
    float acc = 0.0f;
    float kf = (float)kb;
    for (int k = kb; k < ke; ++k, kf += 1.0f) {
        int i_f, i_m, i_s;
        float af, am, as;
        split_floor(fmaf(kf, R.d[0], R.x0[0]), i_f, af);
        split_floor(fmaf(kf, R.d[1], R.x0[1]), i_m, am);
        split_floor(fmaf(kf, R.d[2], R.x0[2]), i_s, as);
        const float* b = vol + ((i_s - plane0) * PFM + i_m * PF + i_f);
        const float v000 = __ldg(b), v100 = __ldg(b + 1);
        const float v010 = __ldg(b + PF), v110 = __ldg(b + PF + 1);
        const float v001 = __ldg(b + PFM), v101 = __ldg(b + PFM + 1);
        const float v011 = __ldg(b + PFM + PF), v111 = __ldg(b + PFM + PF + 1);
        const float c00 = fmaf(af, v100 - v000, v000);
        const float c10 = fmaf(af, v110 - v010, v010);
        const float c01 = fmaf(af, v101 - v001, v001);
        const float c11 = fmaf(af, v111 - v011, v011);
        const float c0 = fmaf(am, c10 - c00, c00);
        const float c1 = fmaf(am, c11 - c01, c01);
        acc += fmaf(as, c1 - c0, c0);
    }
    *out += acc * R.h;
}

// Page-locks a host range for the lifetime of the object unless it already is.
struct HostPin {
    void* ptr = nullptr;
    bool registered = false;
    tigre_status pin(const void* p, size_t bytes)
    {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost)
            return TIGRE_OK;  // already pinned
        cudaGetLastError();
        cudaError_t e = cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();  // keep going pageable: copies become synchronous
            return TIGRE_OK;
        }
        ptr = const_cast<void*>(p);
        registered = true;
        return TIGRE_OK;
    }
    ~HostPin()
    {
        if (registered) cudaHostUnregister(ptr);
    }
};

struct Streams {
    cudaStream_t copy = nullptr;
    cudaEvent_t ev[8] = {};
    ~Streams()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (copy) cudaStreamDestroy(copy);
    }
    tigre_status init()
    {
        TIGRE_CUDA(cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking));
        for (cudaEvent_t& e : ev) TIGRE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return TIGRE_OK;
    }
};

// Device buffers owned for one call.
struct Bufs {
    std::vector<void*> p;
    ~Bufs()
    {
        for (void* x : p) cudaFree(x);
    }
    template <typename T>
    tigre_status alloc(T** out, size_t count)
    {
        void* x = nullptr;
        cudaError_t e = cudaMalloc(&x, sizeof(T) * std::max<size_t>(count, 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(e, "cudaMalloc(out-of-core buffer)");
        }
        p.push_back(x);
        *out = (T*)x;
        return TIGRE_OK;
    }
};

int64_t auto_slab_planes(const tigre_geometry_desc& d, int64_t per_plane_bytes)
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 16;
    }
    const int64_t budget = (int64_t)(free_b / 2);
    const int64_t s = std::max<int64_t>(1, budget / std::max<int64_t>(per_plane_bytes, 1) - 6);
    return std::min<int64_t>(s, d.n_voxel[2]);
}

}  // namespace

tigre_status forward_ooc_impl(tigre_geometry* g, const float* vol_host, float* proj, int64_t a0,
                              int64_t na, int64_t slab, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (!vol_host || !proj) return fail(TIGRE_ERR_INVALID_ARG, "null vol or proj pointer");
    const tigre_geometry_desc& d = g->desc;
    const int64_t nx = d.n_voxel[0], ny = d.n_voxel[1], nz = d.n_voxel[2];
    const int64_t plane = nx * ny;
    if (slab <= 0) slab = auto_slab_planes(d, 4 * (2 * plane + 2 * (nx + 4) * (ny + 4)));
    slab = std::min(slab, nz);
    tigre_geometry_desc sd = d;
    sd.n_voxel[2] = slab + 1;
    if (padded_elems(sd) >= (size_t)INT32_MAX)
        return fail(TIGRE_ERR_UNSUPPORTED, "slab too large for 32-bit indexing; use thinner slabs");
    const FwdConst c = make_fwd_const(d);
    bool need[2] = {false, false};
    for (int64_t a = a0; a < a0 + na; ++a) need[g->layout[(size_t)a]] = true;

    HostPin pin;
    TIGRE_TRY(pin.pin(vol_host, sizeof(float) * (size_t)(plane * nz)));
    Streams S;
    TIGRE_TRY(S.init());
    Bufs B;
    float* raw[2];
    float* pad[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; ++i) TIGRE_TRY(B.alloc(&raw[i], (size_t)(plane * (slab + 1))));
    for (int l = 0; l < 2; ++l)
        if (need[l]) TIGRE_TRY(B.alloc(&pad[l], padded_elems(sd)));
    TIGRE_CUDA(cudaMemsetAsync(proj, 0, sizeof(float) * (size_t)(na * c.nu * c.nv), st));
    for (int l = 0; l < 2; ++l)
        if (pad[l]) TIGRE_CUDA(cudaMemsetAsync(pad[l], 0, sizeof(float) * padded_elems(sd), st));
    cudaEvent_t* copied = S.ev;       // [2]
    cudaEvent_t* consumed = S.ev + 2; // [2]
    TIGRE_CUDA(cudaEventRecord(consumed[0], st));
    TIGRE_CUDA(cudaEventRecord(consumed[1], st));
    const int64_t nslab = (nz + slab - 1) / slab;
    for (int64_t s = 0; s < nslab; ++s) {
        const int b = (int)(s & 1);
        const int64_t z0 = s * slab, z1 = std::min(nz, z0 + slab);
        const int64_t planes = std::min(z1 + 1, nz) - z0;  // with the halo plane
        TIGRE_CUDA(cudaStreamWaitEvent(S.copy, consumed[b], 0));
        TIGRE_CUDA(cudaMemcpyAsync(raw[b], vol_host + z0 * plane, sizeof(float) * (size_t)(planes * plane),
                                   cudaMemcpyHostToDevice, S.copy));
        TIGRE_CUDA(cudaEventRecord(copied[b], S.copy));
        TIGRE_CUDA(cudaStreamWaitEvent(st, copied[b], 0));
        tigre_geometry_desc pd = d;
        pd.n_voxel[2] = planes;
        for (int l = 0; l < 2; ++l)
            if (pad[l]) TIGRE_TRY(fill_padded_f32(pd, raw[b], pad[l], l, st));
        if (planes < slab + 1)  // a shorter last slab: clear the stale planes above it
            for (int l = 0; l < 2; ++l)
                if (pad[l]) {
                    const int64_t pp = (l ? ny : nx) + 2 * kPad, pm = (l ? nx : ny) + 2 * kPad;
                    const int64_t from = (planes + kPad) * pp * pm;
                    TIGRE_CUDA(cudaMemsetAsync(pad[l] + from, 0,
                                               sizeof(float) * (size_t)(padded_elems(sd) - from), st));
                }
        TIGRE_CUDA(cudaEventRecord(consumed[b], st));
        // Cells of this slab in padded z: [z0+P, z1+P); the first slab also owns
        // the cells below plane 0, the last the cells above plane nz-1.
        const int cell_lo = s == 0 ? -1000000 : (int)(z0 + kPad);
        const int cell_hi = s == nslab - 1 ? 1000000 : (int)(z1 + kPad);
        ProfScope prof(kProfForward, st);
        for (int64_t a = 0; a < na; a += 65535) {
            const int64_t cnt = std::min<int64_t>(65535, na - a);
            dim3 grid((unsigned)((c.nu + 31) / 32), (unsigned)cnt, (unsigned)((c.nv + 7) / 8));
            fwd_slab_kernel<<<grid, dim3(32, 8), 0, st>>>(pad[0], pad[1],
                                                          proj + a * (int64_t)c.nu * c.nv,
                                                          (const FwdAngle*)g->fwd_params.ptr, c,
                                                          (int)(a0 + a), cell_lo, cell_hi, (int)z0);
            TIGRE_LAUNCHED("fwd_slab_kernel");
        }
    }
    TIGRE_CUDA(cudaStreamSynchronize(st));
    return TIGRE_OK;
}

tigre_status backward_ooc_impl(tigre_geometry* g, const float* proj, int proj_on_host,
                               float* vol_host, int64_t a0, int64_t na, tigre_bp_weight w,
                               int64_t slab, int64_t chunk, cudaStream_t st)
{
    TIGRE_TRY(check_geometry(g));
    TIGRE_TRY(check_range(g, a0, na));
    if (!vol_host || !proj) return fail(TIGRE_ERR_INVALID_ARG, "null vol or proj pointer");
    if (w == TIGRE_BP_EXACT_ADJOINT)
        return fail(TIGRE_ERR_UNSUPPORTED, "out-of-core backprojection is voxel-driven");
    const tigre_geometry_desc& d = g->desc;
    const int64_t nx = d.n_voxel[0], ny = d.n_voxel[1], nz = d.n_voxel[2];
    const int64_t plane = nx * ny;
    const int64_t pix = d.n_det[0] * d.n_det[1];
    if (slab <= 0) slab = auto_slab_planes(d, 4 * 2 * plane);
    slab = std::min(slab, nz);
    if (chunk <= 0) chunk = std::min<int64_t>(na, 32);
    chunk = std::min(chunk, na);

    HostPin pin_v, pin_p;
    TIGRE_TRY(pin_v.pin(vol_host, sizeof(float) * (size_t)(plane * nz)));
    if (proj_on_host) TIGRE_TRY(pin_p.pin(proj, sizeof(float) * (size_t)(pix * na)));
    Streams S;
    TIGRE_TRY(S.init());
    Bufs B;
    float* out[2];
    float* pbuf[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; ++i) TIGRE_TRY(B.alloc(&out[i], (size_t)(plane * slab)));
    if (proj_on_host)
        for (int i = 0; i < 2; ++i) TIGRE_TRY(B.alloc(&pbuf[i], (size_t)(pix * chunk)));
    cudaEvent_t* out_free = S.ev;       // [2] slab buffer copied out
    cudaEvent_t* out_ready = S.ev + 2;  // [2] slab buffer computed
    cudaEvent_t* p_ready = S.ev + 4;    // [2] projection chunk landed
    cudaEvent_t* p_free = S.ev + 6;     // [2] projection chunk consumed
    for (int i = 0; i < 2; ++i) {
        TIGRE_CUDA(cudaEventRecord(out_free[i], st));
        TIGRE_CUDA(cudaEventRecord(p_free[i], st));
    }
    const int64_t nslab = (nz + slab - 1) / slab;
    int64_t chunk_counter = 0;
    for (int64_t s = 0; s < nslab; ++s) {
        const int b = (int)(s & 1);
        const int z0 = (int)(s * slab), z1 = (int)std::min(nz, (int64_t)z0 + slab);
        float* dst = out[b];  // plane z lands at out[b][z - z0]
        TIGRE_CUDA(cudaStreamWaitEvent(st, out_free[b], 0));
        if (!proj_on_host) {
            TIGRE_TRY(backward_slab_impl(g, proj, dst, a0, na, w, 0, z0, z1, st));
        } else {
            for (int64_t c0 = 0; c0 < na; c0 += chunk, ++chunk_counter) {
                const int pb = (int)(chunk_counter & 1);
                const int64_t cnt = std::min(chunk, na - c0);
                TIGRE_CUDA(cudaStreamWaitEvent(S.copy, p_free[pb], 0));
                TIGRE_CUDA(cudaMemcpyAsync(pbuf[pb], proj + c0 * pix, sizeof(float) * (size_t)(cnt * pix),
                                           cudaMemcpyHostToDevice, S.copy));
                TIGRE_CUDA(cudaEventRecord(p_ready[pb], S.copy));
                TIGRE_CUDA(cudaStreamWaitEvent(st, p_ready[pb], 0));
                TIGRE_TRY(backward_slab_impl(g, pbuf[pb], dst, a0 + c0, cnt, w, c0 > 0 ? 1 : 0, z0,
                                             z1, st));
                TIGRE_CUDA(cudaEventRecord(p_free[pb], st));
            }
        }
        TIGRE_CUDA(cudaEventRecord(out_ready[b], st));
        TIGRE_CUDA(cudaStreamWaitEvent(S.copy, out_ready[b], 0));
        TIGRE_CUDA(cudaMemcpyAsync(vol_host + (int64_t)z0 * plane, out[b],
                                   sizeof(float) * (size_t)((z1 - z0) * plane),
                                   cudaMemcpyDeviceToHost, S.copy));
        TIGRE_CUDA(cudaEventRecord(out_free[b], S.copy));
    }
    TIGRE_CUDA(cudaStreamSynchronize(S.copy));
    TIGRE_CUDA(cudaStreamSynchronize(st));
    return TIGRE_OK;
}

}  // namespace tigre

extern "C" tigre_status tigre_forward_ooc(tigre_geometry_t geo, const float* vol_host, float* proj,
                                          int64_t angle_begin, int64_t angle_count,
                                          int64_t slab_planes, void* cuda_stream)
{
    return tigre::forward_ooc_impl(geo, vol_host, proj, angle_begin, angle_count, slab_planes,
                                   (cudaStream_t)cuda_stream);
}

extern "C" tigre_status tigre_backward_ooc(tigre_geometry_t geo, const float* proj,
                                           int proj_on_host, float* vol_host, int64_t angle_begin,
                                           int64_t angle_count, tigre_bp_weight weight,
                                           int64_t slab_planes, int64_t angle_chunk,
                                           void* cuda_stream)
{
    return tigre::backward_ooc_impl(geo, proj, proj_on_host, vol_host, angle_begin, angle_count,
                                    weight, slab_planes, angle_chunk, (cudaStream_t)cuda_stream);
}
