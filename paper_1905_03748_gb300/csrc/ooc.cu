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
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "ray.cuh"
#include "vecops.cuh"

namespace tigre {

namespace {

// Page-locks a host range for the lifetime of the object unless it already is.
struct HostPin {
    void* ptr = nullptr;
    bool registered = false;
    bool pinned = false;  // page-locked, by this object or already
    tigre_status pin(const void* p, size_t bytes)
    {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost) {
            pinned = true;  // already page-locked
            return TIGRE_OK;
        }
        cudaGetLastError();
        cudaError_t e = cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();  // keep going pageable: copies become synchronous
            return TIGRE_OK;
        }
        ptr = const_cast<void*>(p);
        registered = true;
        pinned = true;
        return TIGRE_OK;
    }
    ~HostPin()
    {
        if (registered) cudaHostUnregister(ptr);
    }
};

struct Streams {
    cudaStream_t copy = nullptr;
    cudaEvent_t ev[12] = {};
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
        for (void* x : p) dev_free_sync(x);
    }
    template <typename T>
    tigre_status alloc(T** out, size_t count)
    {
        void* x = nullptr;
        cudaError_t e = dev_alloc_sync(&x, sizeof(T) * std::max<size_t>(count, 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(e, "device allocation (out-of-core buffer)");
        }
        p.push_back(x);
        *out = (T*)x;
        return TIGRE_OK;
    }
};

// Thickest slab whose zero-padded buffers (slab + 1 planes) index in 32 bits.
int64_t max_slab_planes(const tigre_geometry_desc& d)
{
    const int64_t per = (d.n_voxel[0] + 2 * kPad) * (d.n_voxel[1] + 2 * kPad);
    return std::max<int64_t>(1, ((int64_t)INT32_MAX - 1) / per - 2 - 2 * kPad);
}

int64_t auto_slab_planes(const tigre_geometry_desc& d, int64_t per_plane_bytes)
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 16;
    }
    const int64_t budget = (int64_t)(free_b / 2);
    const int64_t s = std::max<int64_t>(1, budget / std::max<int64_t>(per_plane_bytes, 1) - 6);
    return std::min<int64_t>(std::min<int64_t>(s, d.n_voxel[2]), max_slab_planes(d));
}

// The forward projection of a volume cut into z-slabs of `slab` planes: quad
// buffers for slab + 1 planes (the halo plane) and their zero borders, in
// the layouts the angles use, built straight from each raw slab.
struct FwdSlabs {
    tigre_geometry* g = nullptr;
    tigre_geometry_desc sd{};
    int64_t slab = 0, nslab = 0;
    float4* quad[2] = {nullptr, nullptr};

    static size_t bytes(const tigre_geometry_desc& d, int64_t slab, const bool need[2])
    {
        tigre_geometry_desc t = d;
        t.n_voxel[2] = slab + 1;
        return (size_t)((need[0] ? 1 : 0) + (need[1] ? 1 : 0)) * padded_elems(t) * sizeof(float4);
    }

    tigre_status init(tigre_geometry* g_, int64_t slab_, const bool need[2], Bufs& B,
                      cudaStream_t st)
    {
        g = g_;
        const int64_t nz = g->desc.n_voxel[2];
        slab = std::min(slab_, nz);
        nslab = (nz + slab - 1) / slab;
        sd = g->desc;
        sd.n_voxel[2] = slab + 1;
        if (padded_elems(sd) >= (size_t)INT32_MAX)
            return fail(TIGRE_ERR_UNSUPPORTED, "slab too large for 32-bit indexing; use thinner slabs");
        (void)st;
        for (int l = 0; l < 2; ++l)
            if (need[l]) TIGRE_TRY(B.alloc(&quad[l], padded_elems(sd)));
        return TIGRE_OK;
    }

    // Adds the partial projections of slab s into proj.  src (device) holds
    // the slab's planes z0 .. z0 + planes - 1, the halo plane included; after
    // the quads are built from it, `filled` (if any) is recorded on st.  The
    // quads of the slab's planes and their borders (planes + 4 quad planes)
    // are all its samples read: a slab's own cells and the plane above them,
    // and at the volume's ends the samples the rays' in-bounds proof allows
    // (down to padded plane 0, up to padded plane nz + 3).
    tigre_status project(int64_t s, const float* src, float* proj, int64_t a0, int64_t na,
                         cudaStream_t st, cudaEvent_t filled = nullptr)
    {
        const tigre_geometry_desc& d = g->desc;
        const int64_t nz = d.n_voxel[2];
        const int64_t z0 = s * slab, z1 = std::min(nz, z0 + slab);
        const int64_t planes = std::min(z1 + 1, nz) - z0;  // with the halo plane
        tigre_geometry_desc pd = d;
        pd.n_voxel[2] = planes;
        for (int l = 0; l < 2; ++l)
            if (quad[l]) TIGRE_TRY(build_quads_f32(pd, src, quad[l], l, st));
        if (filled) TIGRE_CUDA(cudaEventRecord(filled, st));
        // Cells of this slab in padded z: [z0+P, z1+P); the first slab also owns
        // the cells below plane 0, the last the cells above plane nz-1.
        const int cell_lo = s == 0 ? -1000000 : (int)(z0 + kPad);
        const int cell_hi = s == nslab - 1 ? 1000000 : (int)(z1 + kPad);
        return forward_slab_impl(g, sd, quad, proj, a0, na, cell_lo, cell_hi, (int)z0, st);
    }
};

void layouts_used(const tigre_geometry* g, int64_t a0, int64_t na, bool need[2])
{
    need[0] = need[1] = false;
    for (int64_t a = a0; a < a0 + na; ++a) need[g->layout[(size_t)a]] = true;
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
    if (slab <= 0) slab = auto_slab_planes(d, 4 * 2 * plane + 16 * 2 * (nx + 4) * (ny + 4));
    slab = std::min(slab, nz);
    bool need[2];
    layouts_used(g, a0, na, need);

    HostPin pin;
    TIGRE_TRY(pin.pin(vol_host, sizeof(float) * (size_t)(plane * nz)));
    Streams S;
    TIGRE_TRY(S.init());
    Bufs B;
    float* raw[2];
    for (int i = 0; i < 2; ++i) TIGRE_TRY(B.alloc(&raw[i], (size_t)(plane * (slab + 1))));
    FwdSlabs F;
    TIGRE_TRY(F.init(g, slab, need, B, st));
    TIGRE_CUDA(cudaMemsetAsync(proj, 0, sizeof(float) * (size_t)(na * n_pix(g)), st));
    cudaEvent_t* copied = S.ev;       // [2]
    cudaEvent_t* consumed = S.ev + 2; // [2]
    TIGRE_CUDA(cudaEventRecord(consumed[0], st));
    TIGRE_CUDA(cudaEventRecord(consumed[1], st));
    for (int64_t s = 0; s < F.nslab; ++s) {
        const int b = (int)(s & 1);
        const int64_t z0 = s * slab, z1 = std::min(nz, z0 + slab);
        const int64_t planes = std::min(z1 + 1, nz) - z0;  // with the halo plane
        TIGRE_CUDA(cudaStreamWaitEvent(S.copy, consumed[b], 0));
        TIGRE_CUDA(cudaMemcpyAsync(raw[b], vol_host + z0 * plane, sizeof(float) * (size_t)(planes * plane),
                                   cudaMemcpyHostToDevice, S.copy));
        TIGRE_CUDA(cudaEventRecord(copied[b], S.copy));
        TIGRE_CUDA(cudaStreamWaitEvent(st, copied[b], 0));
        TIGRE_TRY(F.project(s, raw[b], proj, a0, na, st, consumed[b]));
    }
    TIGRE_CUDA(cudaStreamSynchronize(st));
    return TIGRE_OK;
}

// With slab_dots (device, one double per slab), slab_dots[s] = ||slab s||^2 of
// the backprojection, summed on the device before the slab is copied out.
tigre_status backward_ooc_impl(tigre_geometry* g, const float* proj, int proj_on_host,
                               float* vol_host, int64_t a0, int64_t na, tigre_bp_weight w,
                               int64_t slab, int64_t chunk, cudaStream_t st,
                               double* slab_dots = nullptr)
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
    double* dot_partials = nullptr;
    if (slab_dots) TIGRE_TRY(B.alloc(&dot_partials, (size_t)kRedBlocks));
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
        if (slab_dots)
            TIGRE_TRY(dot_f64(dst, dst, (int64_t)(z1 - z0) * plane, dot_partials, slab_dots + s, st));
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

// ------------------------------------------------------- out-of-core CGLS
//
// CGLS (same iteration as tigre_cgls) when its six vectors do not fit on the
// device.  Two placements, chosen from the device budget:
//
// Placement 1 ("host vectors"): the volume-sized vectors x, p, s live in
// pinned host memory and are streamed through the GPU in z-slabs; the
// projection-sized b, r, q stay on the device.  ||s||^2 is summed slab by
// slab on the device as the backprojection produces s; x += alpha p and
// p = s + beta p run in one pass over the x, p and s slabs.  Device memory:
// three projection sets plus slab buffers.
//
// Placement 2 ("streamed direction"): x, r, q stay on the device; only the
// search direction p lives in host memory (in the caller's x buffer, which
// is free while x is on the device), streamed through in z-slabs.  s = A^T r
// is never stored: one pass backprojects slab by slab for ||s||^2 only, and
// a second pass recomputes each slab of s (bitwise the same), updates
// x += alpha p and p = s + beta p there, copies the new p slab out, and
// projects it into q = A p for the next iteration (the slab's halo plane is
// the first plane of the next slab, so a slab is projected once its
// successor's p is known).  Device memory: one volume, two projection sets
// and slab buffers; host memory: none beyond the caller's b and x.  An
// iteration costs one projection and two backprojections instead of one of
// each; the last iteration only streams p for x += alpha p.

namespace tigre {
namespace {

// The placement-1 direction update on one slab, in the in-core CGLS's FP32
// fused multiply-adds: x += alpha p, then p = s + beta p.
__global__ void __launch_bounds__(256) cgls_slab_axpy_kernel(float* __restrict__ x,
                                                             const float* __restrict__ p,
                                                             int64_t n, float alpha)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fmaf(alpha, p[i], x[i]);
}

__global__ void __launch_bounds__(256) cgls_slab_xpay_kernel(float* __restrict__ p,
                                                             const float* __restrict__ s,
                                                             int64_t n, float beta)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fmaf(beta, p[i], s[i]);
}

// Placement 1's direction update folded into the next projection's slab
// stream: per slab, p and s (each with the halo plane) and x come in; x +=
// alpha p on the slab's own planes and p = s + beta p on all of them run on
// the device (the fused multiply-adds of the separate update pass, so the
// same bits); x and the new p go back to host memory on a stream of their
// own while the new p is projected into q.  A slab's halo plane is read from
// host memory before the next slab writes its own update of that plane back:
// the copies in run in slab order on one stream, and a slab's copies out wait
// for its update, which waits for its copies in.
tigre_status forward_ooc_update(tigre_geometry* g, float* p_host, const float* s_host,
                                float* x_host, float alpha, float beta, float* proj, int64_t slab,
                                cudaStream_t st)
{
    const tigre_geometry_desc& d = g->desc;
    const int64_t nz = d.n_voxel[2], plane = d.n_voxel[0] * d.n_voxel[1];
    const int64_t na = (int64_t)g->angles.size();
    slab = std::max<int64_t>(1, std::min(slab, nz));
    bool need[2];
    layouts_used(g, 0, na, need);
    Streams in, out;
    TIGRE_TRY(in.init());
    TIGRE_TRY(out.init());
    Bufs B;
    float *rp[2], *rs[2], *rx[2];
    for (int i = 0; i < 2; ++i) {
        TIGRE_TRY(B.alloc(&rp[i], (size_t)(plane * (slab + 1))));
        TIGRE_TRY(B.alloc(&rs[i], (size_t)(plane * (slab + 1))));
        TIGRE_TRY(B.alloc(&rx[i], (size_t)(plane * slab)));
    }
    FwdSlabs F;
    TIGRE_TRY(F.init(g, slab, need, B, st));
    TIGRE_CUDA(cudaMemsetAsync(proj, 0, sizeof(float) * (size_t)(na * n_pix(g)), st));
    cudaEvent_t* copied = in.ev;       // [2] copies in done
    cudaEvent_t* updated = in.ev + 2;  // [2] x and p updated
    cudaEvent_t* filled = in.ev + 4;   // [2] p copied into the padded layouts
    cudaEvent_t* written = in.ev + 6;  // [2] x and p back in host memory
    for (int b = 0; b < 2; ++b) {
        TIGRE_CUDA(cudaEventRecord(filled[b], st));
        TIGRE_CUDA(cudaEventRecord(written[b], st));
    }
    const dim3 grid(4 * 152), block(256);
    for (int64_t s = 0; s < F.nslab; ++s) {
        const int b = (int)(s & 1);
        const int64_t z0 = s * slab, z1 = std::min(nz, z0 + slab);
        const int64_t planes = std::min(z1 + 1, nz) - z0;  // with the halo plane
        const int64_t own = (z1 - z0) * plane, all = planes * plane, off = z0 * plane;
        TIGRE_CUDA(cudaStreamWaitEvent(in.copy, filled[b], 0));
        TIGRE_CUDA(cudaStreamWaitEvent(in.copy, written[b], 0));
        TIGRE_CUDA(cudaMemcpyAsync(rp[b], p_host + off, sizeof(float) * (size_t)all,
                                   cudaMemcpyHostToDevice, in.copy));
        TIGRE_CUDA(cudaMemcpyAsync(rs[b], s_host + off, sizeof(float) * (size_t)all,
                                   cudaMemcpyHostToDevice, in.copy));
        TIGRE_CUDA(cudaMemcpyAsync(rx[b], x_host + off, sizeof(float) * (size_t)own,
                                   cudaMemcpyHostToDevice, in.copy));
        TIGRE_CUDA(cudaEventRecord(copied[b], in.copy));
        TIGRE_CUDA(cudaStreamWaitEvent(st, copied[b], 0));
        cgls_slab_axpy_kernel<<<grid, block, 0, st>>>(rx[b], rp[b], own, alpha);
        TIGRE_LAUNCHED("cgls_slab_axpy_kernel");
        cgls_slab_xpay_kernel<<<grid, block, 0, st>>>(rp[b], rs[b], all, beta);
        TIGRE_LAUNCHED("cgls_slab_xpay_kernel");
        TIGRE_CUDA(cudaEventRecord(updated[b], st));
        TIGRE_CUDA(cudaStreamWaitEvent(out.copy, updated[b], 0));
        TIGRE_CUDA(cudaMemcpyAsync(x_host + off, rx[b], sizeof(float) * (size_t)own,
                                   cudaMemcpyDeviceToHost, out.copy));
        TIGRE_CUDA(cudaMemcpyAsync(p_host + off, rp[b], sizeof(float) * (size_t)own,
                                   cudaMemcpyDeviceToHost, out.copy));
        TIGRE_CUDA(cudaEventRecord(written[b], out.copy));
        TIGRE_TRY(F.project(s, rp[b], proj, 0, na, st, filled[b]));
    }
    for (int b = 0; b < 2; ++b) TIGRE_CUDA(cudaStreamWaitEvent(st, written[b], 0));
    TIGRE_CUDA(cudaStreamSynchronize(st));
    return TIGRE_OK;
}

// Sum of the per-slab values in slab order (host FP64 combine of nslab scalars).
tigre_status sum_slab_dots(const double* d_dots, int64_t nslab, double* out)
{
    std::vector<double> h((size_t)nslab);
    TIGRE_CUDA(cudaMemcpy(h.data(), d_dots, sizeof(double) * (size_t)nslab, cudaMemcpyDeviceToHost));
    double t = 0.0;
    for (double v : h) t += v;
    *out = t;
    return TIGRE_OK;
}

__global__ void set_dscalar_kernel(double* dst, double v) { *dst = v; }

tigre_status set_dscalar(double* dst, double v, cudaStream_t st)
{
    set_dscalar_kernel<<<1, 1, 0, st>>>(dst, v);
    TIGRE_LAUNCHED("set_dscalar_kernel");
    return TIGRE_OK;
}

// Progress lines on stderr (pass, slab count, seconds since the call began)
// when the environment variable TIGRE_PROGRESS is set; for runs long enough
// that a caller wants to see where time goes before they finish.
struct Progress {
    bool on = std::getenv("TIGRE_PROGRESS") != nullptr;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    void flag(const char* what, bool v)
    {
        if (!on) return;
        std::fprintf(stderr, "tigre cgls(out-of-core): %s: %s\n", what, v ? "yes" : "no");
        std::fflush(stderr);
    }
    void note(const char* what, int it)
    {
        if (!on) return;
        const double s =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        std::fprintf(stderr, "tigre cgls(out-of-core): %s iteration %d done at %.1f s\n", what, it, s);
        std::fflush(stderr);
    }
};

constexpr int64_t kMaxSlabPlanes = 256;
constexpr int kScalarSlots = 16;

struct OocPlan {
    int placement = 0;  // 1 host vectors, 2 streamed direction
    int64_t slab = 0;   // z planes per slab
};

// Device bytes of placement 2 besides x, r, q: three direction slabs with
// their halo plane, one s slab, the forward slab buffers, the
// backprojector's padded projection band and the per-slab inner products.
size_t placement2_workspace(const tigre_geometry* g, int64_t slab, const bool need[2])
{
    const tigre_geometry_desc& d = g->desc;
    const int64_t plane = d.n_voxel[0] * d.n_voxel[1];
    const int64_t nslab = (d.n_voxel[2] + slab - 1) / slab;
    return sizeof(float) * (size_t)(plane * (3 * (slab + 1) + slab)) +
           FwdSlabs::bytes(d, slab, need) +
           bp_slab_pad_bytes(d, slab, (int64_t)g->angles.size()) +
           sizeof(double) * (size_t)(nslab + kRedBlocks + kScalarSlots);
}

// Placement 1: the larger of the projection's slab buffers (the update folded
// into it: p and s with the halo plane, x, two of each) and the
// backprojection's or the last update pass's (they run one after the other),
// plus the backprojector's projection band, which the handle keeps.
size_t placement1_workspace(const tigre_geometry* g, int64_t slab, const bool need[2])
{
    const tigre_geometry_desc& d = g->desc;
    const int64_t plane = d.n_voxel[0] * d.n_voxel[1];
    const int64_t nslab = (d.n_voxel[2] + slab - 1) / slab;
    const size_t fwd = sizeof(float) * (size_t)(4 * plane * (slab + 1) + 2 * plane * slab) +
                       FwdSlabs::bytes(d, slab, need);
    const size_t bwd = sizeof(float) * (size_t)(4 * plane * slab);
    return std::max(fwd, bwd) + bp_slab_pad_bytes(d, slab, (int64_t)g->angles.size()) +
           sizeof(double) * (size_t)(nslab + 2 * kRedBlocks + kScalarSlots);
}

// Slab thicknesses the backprojector fills without waste: it computes z in
// chunks of 16 voxels per thread, so a slab of 100 planes costs 112.  Thin
// slabs (under 16 planes) and the whole volume are always allowed.
bool whole_chunks(int64_t slab, int64_t nz)
{
    constexpr int64_t kChunk = 16;
    return slab < kChunk || slab % kChunk == 0 || slab >= nz;
}

// The placement and slab thickness for a device budget (0: the free device
// memory less 1 GiB): placement 2 with the thickest slab (at most
// kMaxSlabPlanes) that fits, else placement 1 likewise, else OOM.
tigre_status plan_ooc(const tigre_geometry* g, int64_t budget, OocPlan* out)
{
    if (budget <= 0) {
        size_t free_b = 0, total_b = 0;
        TIGRE_CUDA(cudaMemGetInfo(&free_b, &total_b));
        budget = std::max<int64_t>(0, (int64_t)free_b - ((int64_t)1 << 30));
    }
    const int64_t nvox = n_vox(g), m = n_pix(g) * (int64_t)g->angles.size();
    const int64_t nz = g->desc.n_voxel[2];
    bool need[2];
    layouts_used(g, 0, (int64_t)g->angles.size(), need);
    const int64_t top = std::min(std::min(nz, kMaxSlabPlanes), max_slab_planes(g->desc));
    const int64_t base2 = (int64_t)sizeof(float) * (nvox + 2 * m);
    for (int64_t slab = top; slab >= 1; --slab)
        if (whole_chunks(slab, nz) && base2 + (int64_t)placement2_workspace(g, slab, need) <= budget) {
            *out = OocPlan{2, slab};
            return TIGRE_OK;
        }
    const int64_t base1 = (int64_t)sizeof(float) * 3 * m;
    for (int64_t slab = top; slab >= 1; --slab)
        if (whole_chunks(slab, nz) && base1 + (int64_t)placement1_workspace(g, slab, need) <= budget) {
            *out = OocPlan{1, slab};
            return TIGRE_OK;
        }
    return fail(TIGRE_ERR_OOM, "device budget below three projection sets plus one-plane slabs");
}

}  // namespace

// Placement 1 (host vectors).
static tigre_status cgls_host_vectors(tigre_geometry* g, const float* b_host, float* x_host,
                                      const tigre_solver_opts* o, double* h_hist, int64_t slab)
{
    cudaStream_t st = (cudaStream_t)o->cuda_stream;
    const tigre_geometry_desc& d = g->desc;
    const int64_t nvox = n_vox(g), na = (int64_t)g->angles.size(), m = n_pix(g) * na;
    const int64_t nz = d.n_voxel[2], plane = d.n_voxel[0] * d.n_voxel[1];
    slab = std::max<int64_t>(1, std::min(slab, nz));
    const int64_t nslab = (nz + slab - 1) / slab;
    Progress prog;
    HostPin pin_x;
    TIGRE_TRY(pin_x.pin(x_host, sizeof(float) * (size_t)nvox));
    float *hp = nullptr, *hs = nullptr;
    TIGRE_CUDA(cudaHostAlloc((void**)&hp, sizeof(float) * (size_t)nvox, cudaHostAllocDefault));
    struct HostFree {
        float* p;
        ~HostFree() { if (p) cudaFreeHost(p); }
    } free_p{hp};
    TIGRE_CUDA(cudaHostAlloc((void**)&hs, sizeof(float) * (size_t)nvox, cudaHostAllocDefault));
    HostFree free_s{hs};
    Bufs B;
    float *b, *r, *q;
    double *sc, *sdots;
    TIGRE_TRY(B.alloc(&b, (size_t)m));
    TIGRE_TRY(B.alloc(&r, (size_t)m));
    TIGRE_TRY(B.alloc(&q, (size_t)m));
    TIGRE_TRY(B.alloc(&sc, (size_t)(kRedBlocks + kScalarSlots)));
    TIGRE_TRY(B.alloc(&sdots, (size_t)nslab));
    double* partials = sc;
    double* qq = sc + kRedBlocks;       // [2]
    double* rr = sc + kRedBlocks + 2;   // [2]
    double* gam = sc + kRedBlocks + 4;  // gamma (host-set)
    // x += alpha p and p = s + beta p, slab by slab through the device: p and
    // x in, x out; then s in where x was, p out.  Consecutive slabs alternate
    // between two streams, each with its own pair of slab buffers (they exist
    // only for the pass), so one slab's host copies overlap the other's
    // copies and kernels; the two copy directions run on separate engines.
    auto update = [&](float alpha, float beta) -> tigre_status {
        Bufs U;
        Streams side[2];
        float *up[2], *uv[2];
        for (int k = 0; k < 2; ++k) {
            TIGRE_TRY(side[k].init());
            TIGRE_TRY(U.alloc(&up[k], (size_t)(plane * slab)));
            TIGRE_TRY(U.alloc(&uv[k], (size_t)(plane * slab)));
        }
        // both start after the work queued on st (which wrote s, p and x)
        TIGRE_CUDA(cudaEventRecord(side[0].ev[0], st));
        for (int k = 0; k < 2; ++k) TIGRE_CUDA(cudaStreamWaitEvent(side[k].copy, side[0].ev[0], 0));
        const dim3 grid(4 * 152), block(256);
        int64_t i = 0;
        for (int64_t z0 = 0; z0 < nz; z0 += slab, ++i) {
            const int64_t n = plane * std::min(slab, nz - z0), off = plane * z0;
            const size_t bytes = sizeof(float) * (size_t)n;
            cudaStream_t ss = side[i & 1].copy;
            float* P = up[i & 1];
            float* V = uv[i & 1];
            TIGRE_CUDA(cudaMemcpyAsync(P, hp + off, bytes, cudaMemcpyHostToDevice, ss));
            TIGRE_CUDA(cudaMemcpyAsync(V, x_host + off, bytes, cudaMemcpyHostToDevice, ss));
            cgls_slab_axpy_kernel<<<grid, block, 0, ss>>>(V, P, n, alpha);
            TIGRE_LAUNCHED("cgls_slab_axpy_kernel");
            TIGRE_CUDA(cudaMemcpyAsync(x_host + off, V, bytes, cudaMemcpyDeviceToHost, ss));
            TIGRE_CUDA(cudaMemcpyAsync(V, hs + off, bytes, cudaMemcpyHostToDevice, ss));
            cgls_slab_xpay_kernel<<<grid, block, 0, ss>>>(P, V, n, beta);
            TIGRE_LAUNCHED("cgls_slab_xpay_kernel");
            TIGRE_CUDA(cudaMemcpyAsync(hp + off, P, bytes, cudaMemcpyDeviceToHost, ss));
        }
        // st continues after both; the next projection reads p from host memory
        for (int k = 0; k < 2; ++k) {
            TIGRE_CUDA(cudaEventRecord(side[k].ev[1], side[k].copy));
            TIGRE_CUDA(cudaStreamWaitEvent(st, side[k].ev[1], 0));
        }
        TIGRE_CUDA(cudaStreamSynchronize(st));
        return TIGRE_OK;
    };
    prog.flag("volume buffer page-locked", pin_x.pinned);
    prog.note("setup (host p and s page-locked)", -1);
    TIGRE_CUDA(cudaMemcpyAsync(b, b_host, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, st));
    // r = b - A x0; p = A^T r; gamma = ||p||^2
    TIGRE_TRY(forward_ooc_impl(g, x_host, q, 0, na, slab, st));
    TIGRE_TRY(weighted_residual(b, q, nullptr, r, m, partials, rr, st));
    TIGRE_TRY(backward_ooc_impl(g, r, 0, hp, 0, na, o->bp_weight, slab, 0, st, sdots));
    double gamma = 0.0;
    TIGRE_TRY(sum_slab_dots(sdots, nslab, &gamma));
    prog.note("first direction (A x0, A^T r)", -1);
    // The direction update of iteration it - 1 runs inside iteration it's
    // projection of the new p; the last one is a pass of its own.
    bool pending = false;
    float pend_alpha = 0.0f, pend_beta = 0.0f;
    for (int it = 0; it < o->n_iter; ++it) {
        if (pending)
            TIGRE_TRY(forward_ooc_update(g, hp, hs, x_host, pend_alpha, pend_beta, q, slab, st));
        else
            TIGRE_TRY(forward_ooc_impl(g, hp, q, 0, na, slab, st));
        TIGRE_TRY(dot_f64(q, q, m, partials, qq, st));
        double hqq = 0.0;
        TIGRE_CUDA(cudaMemcpyAsync(&hqq, qq, sizeof(double), cudaMemcpyDeviceToHost, st));
        TIGRE_CUDA(cudaStreamSynchronize(st));
        const double alpha = hqq != 0.0 ? gamma / hqq : 0.0;
        // r -= alpha q on the device (alpha = gamma / qq from device slots)
        TIGRE_TRY(set_dscalar(gam, gamma, st));
        TIGRE_TRY(axpy_ratio_norm(r, q, m, gam, qq, -1.0f, partials, rr, st));
        if (h_hist) {
            double rn[2];
            TIGRE_CUDA(cudaMemcpyAsync(rn, rr, sizeof(rn), cudaMemcpyDeviceToHost, st));
            TIGRE_CUDA(cudaStreamSynchronize(st));
            h_hist[it] = rn[1];
        }
        // s = A^T r with ||s||^2 per slab; then x += alpha p, p = s + beta p
        prog.note(it ? "previous update and projection (x, p; A p)" : "projection (A p)", it);
        TIGRE_TRY(backward_ooc_impl(g, r, 0, hs, 0, na, o->bp_weight, slab, 0, st, sdots));
        double gamma_new = 0.0;
        TIGRE_TRY(sum_slab_dots(sdots, nslab, &gamma_new));
        prog.note("backprojection (A^T r)", it);
        pending = true;
        pend_alpha = (float)alpha;
        pend_beta = (float)(gamma != 0.0 ? gamma_new / gamma : 0.0);
        gamma = gamma_new;
    }
    if (pending) {
        TIGRE_TRY(update(pend_alpha, pend_beta));
        prog.note("last update pass (x += alpha p)", o->n_iter - 1);
    }
    TIGRE_CUDA(cudaStreamSynchronize(st));
    return TIGRE_OK;
}

// Placement 2 (streamed direction).
static tigre_status cgls_streamed_direction(tigre_geometry* g, const float* b_host, float* x_host,
                                            const tigre_solver_opts* o, double* h_hist,
                                            int64_t slab)
{
    cudaStream_t st = (cudaStream_t)o->cuda_stream;
    const tigre_geometry_desc& d = g->desc;
    const int64_t nvox = n_vox(g), na = (int64_t)g->angles.size(), m = n_pix(g) * na;
    const int64_t nz = d.n_voxel[2], plane = d.n_voxel[0] * d.n_voxel[1];
    bool need[2];
    layouts_used(g, 0, na, need);
    HostPin pin_x, pin_b;
    TIGRE_TRY(pin_x.pin(x_host, sizeof(float) * (size_t)nvox));
    TIGRE_TRY(pin_b.pin(b_host, sizeof(float) * (size_t)m));
    Streams S;
    TIGRE_TRY(S.init());
    Bufs B;
    float *xd, *r, *q, *Sb, *P[3];
    double *sc, *dots;
    TIGRE_TRY(B.alloc(&xd, (size_t)nvox));
    TIGRE_TRY(B.alloc(&r, (size_t)m));
    TIGRE_TRY(B.alloc(&q, (size_t)m));
    FwdSlabs F;
    TIGRE_TRY(F.init(g, slab, need, B, st));
    slab = F.slab;
    const int64_t nslab = F.nslab;
    for (int i = 0; i < 3; ++i) TIGRE_TRY(B.alloc(&P[i], (size_t)(plane * (slab + 1))));
    TIGRE_TRY(B.alloc(&Sb, (size_t)(plane * slab)));
    TIGRE_TRY(B.alloc(&sc, (size_t)(kRedBlocks + kScalarSlots)));
    TIGRE_TRY(B.alloc(&dots, (size_t)nslab));
    TIGRE_TRY(g->proj_pad.ensure(bp_slab_pad_bytes(d, slab, na)));
    double* partials = sc;
    double* qq = sc + kRedBlocks;        // ||q||^2
    double* rr = sc + kRedBlocks + 2;    // [2] ||r||^2, ||r||
    double* gam = sc + kRedBlocks + 4;   // gamma
    double* gnew = sc + kRedBlocks + 5;  // gamma of the next direction
    double* xx = sc + kRedBlocks + 6;    // ||x0||^2

    TIGRE_CUDA(cudaMemcpyAsync(xd, x_host, sizeof(float) * (size_t)nvox, cudaMemcpyHostToDevice, st));
    TIGRE_CUDA(cudaMemcpyAsync(r, b_host, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, st));
    // r = b - A x0, skipped for x0 = 0 (then r = b exactly, as A 0 = 0).
    TIGRE_TRY(dot_f64(xd, xd, nvox, partials, xx, st));
    double hxx = 0.0;
    TIGRE_CUDA(cudaMemcpyAsync(&hxx, xx, sizeof(double), cudaMemcpyDeviceToHost, st));
    TIGRE_CUDA(cudaStreamSynchronize(st));
    if (hxx != 0.0) {
        TIGRE_CUDA(cudaMemsetAsync(q, 0, sizeof(float) * (size_t)m, st));
        for (int64_t s = 0; s < nslab; ++s) TIGRE_TRY(F.project(s, xd + s * slab * plane, q, 0, na, st));
        TIGRE_TRY(weighted_residual(r, q, nullptr, q, m, partials, rr, st));  // q = b - A x0
        std::swap(r, q);
    }

    enum Pass { kInit, kNorm, kUpdate, kXOnly };
    cudaEvent_t* h2d = S.ev;      // [3] direction slab landed in P[i]
    cudaEvent_t* upd = S.ev + 3;  // [3] new direction slab ready in P[i]
    cudaEvent_t* fwd = S.ev + 6;  // [3] P[i] no longer read by the device
    cudaEvent_t* d2h = S.ev + 9;  // [3] P[i] copied out
    auto planes_of = [&](int64_t s) { return std::min(nz, (s + 1) * slab) - s * slab; };
    auto fetch = [&](int64_t s) -> tigre_status {  // old direction slab s into P[s % 3]
        const int i = (int)(s % 3);
        TIGRE_CUDA(cudaStreamWaitEvent(S.copy, fwd[i], 0));
        TIGRE_CUDA(cudaMemcpyAsync(P[i], x_host + s * slab * plane,
                                   sizeof(float) * (size_t)(planes_of(s) * plane),
                                   cudaMemcpyHostToDevice, S.copy));
        TIGRE_CUDA(cudaEventRecord(h2d[i], S.copy));
        return TIGRE_OK;
    };
    // Project slab s of the new direction; `next` is the first plane of slab
    // s + 1 (its halo plane), null for the last slab.
    auto project = [&](int64_t s, const float* next) -> tigre_status {
        const int i = (int)(s % 3);
        if (next)
            TIGRE_CUDA(cudaMemcpyAsync(P[i] + slab * plane, next, sizeof(float) * (size_t)plane,
                                       cudaMemcpyDeviceToDevice, st));
        TIGRE_TRY(F.project(s, P[i], q, 0, na, st));
        TIGRE_CUDA(cudaEventRecord(fwd[i], st));
        return TIGRE_OK;
    };
    auto sweep = [&](Pass pass, double* gamma_out) -> tigre_status {
        for (int i = 0; i < 3; ++i) {
            TIGRE_CUDA(cudaEventRecord(fwd[i], st));
            TIGRE_CUDA(cudaEventRecord(d2h[i], S.copy));
        }
        const bool streams_p = pass == kUpdate || pass == kXOnly;
        if (streams_p) TIGRE_TRY(fetch(0));
        for (int64_t s = 0; s < nslab; ++s) {
            const int i = (int)(s % 3);
            const int64_t z0 = s * slab, n = planes_of(s) * plane;
            if (streams_p && s + 1 < nslab) TIGRE_TRY(fetch(s + 1));  // overlaps this slab
            if (streams_p) {
                TIGRE_CUDA(cudaStreamWaitEvent(st, h2d[i], 0));
                TIGRE_TRY(axpy_ratio(xd + z0 * plane, P[i], n, gam, qq, 1.0f, st));  // x += alpha p
                if (pass == kXOnly) {
                    TIGRE_CUDA(cudaEventRecord(fwd[i], st));
                    continue;
                }
            }
            if (pass == kInit) TIGRE_CUDA(cudaStreamWaitEvent(st, d2h[i], 0));
            float* sl = pass == kInit ? P[i] : Sb;  // s = A^T r on this slab
            TIGRE_TRY(backward_slab_impl(g, r, sl, 0, na, o->bp_weight, 0, (int)z0,
                                         (int)(z0 + planes_of(s)), st));
            if (pass != kUpdate) TIGRE_TRY(dot_f64(sl, sl, n, partials, dots + s, st));
            if (pass == kNorm) continue;
            if (pass == kUpdate) TIGRE_TRY(xpay_ratio(P[i], Sb, n, gnew, gam, st));  // p = s + beta p
            TIGRE_CUDA(cudaEventRecord(upd[i], st));
            TIGRE_CUDA(cudaStreamWaitEvent(S.copy, upd[i], 0));
            TIGRE_CUDA(cudaMemcpyAsync(x_host + z0 * plane, P[i], sizeof(float) * (size_t)n,
                                       cudaMemcpyDeviceToHost, S.copy));
            TIGRE_CUDA(cudaEventRecord(d2h[i], S.copy));
            if (s > 0) TIGRE_TRY(project(s - 1, P[i]));
        }
        if (pass == kInit || pass == kUpdate) TIGRE_TRY(project(nslab - 1, nullptr));
        TIGRE_CUDA(cudaStreamSynchronize(S.copy));
        TIGRE_CUDA(cudaStreamSynchronize(st));
        if (gamma_out) {
            std::vector<double> h((size_t)nslab);
            TIGRE_CUDA(cudaMemcpy(h.data(), dots, sizeof(double) * (size_t)nslab, cudaMemcpyDeviceToHost));
            double t = 0.0;
            for (double v : h) t += v;
            *gamma_out = t;
        }
        return TIGRE_OK;
    };

    // p = A^T r (into the host buffer), gamma = ||p||^2, q = A p
    Progress prog;
    prog.flag("volume buffer page-locked", pin_x.pinned);
    prog.flag("projection buffer page-locked", pin_b.pinned);
    prog.note("setup", -1);
    TIGRE_CUDA(cudaMemsetAsync(q, 0, sizeof(float) * (size_t)m, st));
    double gamma = 0.0;
    TIGRE_TRY(sweep(kInit, &gamma));
    prog.note("first direction (A^T r, A p)", -1);
    TIGRE_TRY(set_dscalar(gam, gamma, st));
    for (int it = 0; it < o->n_iter; ++it) {
        // alpha = gamma / ||q||^2: r -= alpha q here, x += alpha p in the sweep
        TIGRE_TRY(dot_f64(q, q, m, partials, qq, st));
        TIGRE_TRY(axpy_ratio_norm(r, q, m, gam, qq, -1.0f, partials, rr, st));
        if (h_hist) {
            TIGRE_CUDA(cudaMemcpyAsync(h_hist + it, rr + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
            TIGRE_CUDA(cudaStreamSynchronize(st));
        }
        if (it == o->n_iter - 1) {
            TIGRE_TRY(sweep(kXOnly, nullptr));
            prog.note("x update", it);
            break;
        }
        double gamma_new = 0.0;
        TIGRE_TRY(sweep(kNorm, &gamma_new));
        prog.note("norm pass (A^T r)", it);
        TIGRE_TRY(set_dscalar(gnew, gamma_new, st));
        TIGRE_CUDA(cudaMemsetAsync(q, 0, sizeof(float) * (size_t)m, st));
        TIGRE_TRY(sweep(kUpdate, nullptr));
        prog.note("update pass (A^T r, x, p, A p)", it);
        TIGRE_TRY(set_dscalar(gam, gamma_new, st));
    }
    TIGRE_CUDA(cudaMemcpyAsync(x_host, xd, sizeof(float) * (size_t)nvox, cudaMemcpyDeviceToHost, st));
    TIGRE_CUDA(cudaStreamSynchronize(st));
    return TIGRE_OK;
}

tigre_status cgls_ooc_impl(tigre_geometry* g, const float* b_host, float* x_host,
                           const tigre_solver_opts* o, double* h_hist)
{
    TIGRE_TRY(check_geometry(g));
    OocPlan plan;
    TIGRE_TRY(plan_ooc(g, o->device_budget_bytes, &plan));
    if (plan.placement == 2) return cgls_streamed_direction(g, b_host, x_host, o, h_hist, plan.slab);
    return cgls_host_vectors(g, b_host, x_host, o, h_hist, plan.slab);
}

}  // namespace tigre

extern "C" tigre_status tigre_cgls_ooc_plan(tigre_geometry_t geo, int64_t device_budget_bytes,
                                            int* placement, int64_t* slab_planes)
{
    using namespace tigre;
    if (!placement || !slab_planes) return fail(TIGRE_ERR_INVALID_ARG, "null output");
    TIGRE_TRY(check_geometry(geo));
    OocPlan plan;
    TIGRE_TRY(plan_ooc(geo, device_budget_bytes, &plan));
    *placement = plan.placement;
    *slab_planes = plan.slab;
    return TIGRE_OK;
}

extern "C" tigre_status tigre_cgls_ooc_plan_desc(const tigre_geometry_desc* desc,
                                                 const double* angles, int64_t n_angles,
                                                 int64_t device_budget_bytes, int* placement,
                                                 int64_t* slab_planes)
{
    using namespace tigre;
    if (!placement || !slab_planes) return fail(TIGRE_ERR_INVALID_ARG, "null output");
    if (device_budget_bytes <= 0)
        return fail(TIGRE_ERR_INVALID_ARG, "planning without a device needs an explicit budget");
    TIGRE_TRY(validate_desc(desc, angles, n_angles));
    // A host-only geometry: the planner reads the description, the number of
    // angles and the memory layouts they use; no device state is made.
    tigre_geometry g;
    g.desc = *desc;
    g.angles.assign(angles, angles + n_angles);
    g.layout.resize((size_t)n_angles);
    for (int64_t a = 0; a < n_angles; ++a) g.layout[(size_t)a] = angle_layout(angles[a]);
    OocPlan plan;
    TIGRE_TRY(plan_ooc(&g, device_budget_bytes, &plan));
    *placement = plan.placement;
    *slab_planes = plan.slab;
    return TIGRE_OK;
}

// ------------------------------------------------ out-of-core TV (halo buffers)
//
// The paper's splitting of a regulariser (Sec. 2.3) on one GPU whose volume
// lives in host memory: in rounds of k = min(depth, steps left) steps, each
// z-slab is copied to the device with k planes of buffer on each side (the
// previous round's values: the slab below has already been written back,
// so its old top planes are kept aside first), takes its k steps on its own,
// and writes its own planes back.  A buffer as deep as the number of
// independent steps keeps the slab's interior exact; the norm of the update
// is approximated from the slab's own voxels as if uniformly distributed over
// the volume, ||g|| ~ ||g_slab|| sqrt(N / N_slab).

namespace tigre {

tigre_status tv_ooc_impl(const int64_t n[3], float* vol_host, int n_steps, double alpha,
                         double eps, int64_t slab, int64_t depth, cudaStream_t st)
{
    if (!n || !vol_host) return fail(TIGRE_ERR_INVALID_ARG, "null n_voxel or vol");
    for (int a = 0; a < 3; ++a)
        if (n[a] <= 0 || n[a] > (1 << 20)) return fail(TIGRE_ERR_INVALID_ARG, "n_voxel out of range");
    if (n_steps < 0 || !std::isfinite(alpha) || !std::isfinite(eps) || eps < 0.0)
        return fail(TIGRE_ERR_INVALID_ARG, "need n_steps >= 0, finite alpha, eps >= 0");
    if (depth < 1) return fail(TIGRE_ERR_INVALID_ARG, "halo depth must be >= 1");
    const int64_t nz = n[2], plane = n[0] * n[1], N = plane * nz;
    if (slab <= 0) slab = nz;
    slab = std::min(slab, nz);
    if (depth > slab && slab < nz)
        return fail(TIGRE_ERR_INVALID_ARG, "halo depth must not exceed the slab thickness");
    if (n_steps == 0) return TIGRE_OK;
    const int64_t sub_planes = std::min(nz, slab + 2 * depth);
    if (plane * sub_planes > INT32_MAX) return fail(TIGRE_ERR_UNSUPPORTED, "slab too large");
    HostPin pin;
    TIGRE_TRY(pin.pin(vol_host, sizeof(float) * (size_t)N));
    Bufs B;
    float *dsub, *dg;
    double* dred;
    TIGRE_TRY(B.alloc(&dsub, (size_t)(plane * sub_planes)));
    TIGRE_TRY(B.alloc(&dg, (size_t)(plane * sub_planes)));
    TIGRE_TRY(B.alloc(&dred, (size_t)(kRedBlocks + 4)));
    std::vector<float> saved((size_t)(plane * std::min(depth, nz)));
    const size_t pb = sizeof(float) * (size_t)plane;
    for (int done = 0; done < n_steps;) {
        const int k = (int)std::min<int64_t>(depth, n_steps - done);
        for (int64_t z0 = 0; z0 < nz; z0 += slab) {
            const int64_t z1 = std::min(nz, z0 + slab);
            const int64_t lo = std::min<int64_t>(k, z0), hi = std::min<int64_t>(k, nz - z1);
            const int64_t own = z1 - z0, planes = lo + own + hi;
            // buffer below: the previous slab's top planes as they were before
            // its write-back; the slab and the buffer above are still old
            if (lo > 0)
                TIGRE_CUDA(cudaMemcpyAsync(dsub, saved.data() + (size_t)((k - lo) * plane), pb * lo,
                                           cudaMemcpyHostToDevice, st));
            TIGRE_CUDA(cudaMemcpyAsync(dsub + lo * plane, vol_host + z0 * plane, pb * (own + hi),
                                       cudaMemcpyHostToDevice, st));
            TIGRE_CUDA(cudaStreamSynchronize(st));
            if (z1 < nz)  // keep this slab's old top k planes for the next slab
                std::copy(vol_host + (z1 - k) * plane, vol_host + z1 * plane, saved.begin());
            const int64_t sn[3] = {n[0], n[1], planes};
            const double a = alpha * std::sqrt((double)(own * plane) / (double)N);
            TIGRE_TRY(tv_impl_region(sn, dsub, TIGRE_F32, k, a, eps, nullptr, dg, dred, (int)lo,
                                     (int)(lo + own), st));
            TIGRE_CUDA(cudaMemcpyAsync(vol_host + z0 * plane, dsub + lo * plane, pb * own,
                                       cudaMemcpyDeviceToHost, st));
            TIGRE_CUDA(cudaStreamSynchronize(st));
        }
        done += k;
    }
    return TIGRE_OK;
}

}  // namespace tigre

extern "C" tigre_status tigre_tv_step_ooc(const int64_t n_voxel[3], float* vol_host, int n_steps,
                                          double alpha, double eps, int64_t slab_planes,
                                          int64_t halo_depth, void* cuda_stream)
{
    return tigre::tv_ooc_impl(n_voxel, vol_host, n_steps, alpha, eps, slab_planes, halo_depth,
                              (cudaStream_t)cuda_stream);
}
