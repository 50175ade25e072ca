// Geometry handle, parameter upload, workspaces and error reporting.
//
// The per-angle parameters are computed on the host in FP64 from the
// circular cone-beam frame (source S = DSO (cos t, sin t, 0), detector centre
// D = -(DSD - DSO)(cos t, sin t, 0), e_u = (-sin t, cos t, 0), e_v = z) and
// rounded once to FP32 for the kernels.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"

namespace tigre {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

tigre_status fail(tigre_status st, const std::string& msg)
{
    set_error(msg);
    return st;
}

tigre_status cuda_fail(cudaError_t err, const char* what)
{
    set_error(std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) +
              ")");
    return err == cudaErrorMemoryAllocation ? TIGRE_ERR_OOM : TIGRE_ERR_CUDA;
}

// ------------------------------------------------------ workspace allocator
// Every device workspace the library allocates goes through dev_alloc /
// dev_free (stream-ordered) or dev_alloc_sync / dev_free_sync (buffers not
// tied to one stream).  By default they are cudaMallocAsync / cudaFreeAsync
// and cudaMalloc / cudaFree; tigre_set_allocator installs a caller's pair
// instead.  The pair may only change while no geometry handle or CGLS state
// is alive, so every pointer is freed by the allocator that made it.
static std::mutex g_alloc_mu;
static tigre_alloc_fn g_alloc = nullptr;
static tigre_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::atomic<int64_t> g_live_handles{0};

void handle_created() { g_live_handles.fetch_add(1); }
void handle_destroyed() { g_live_handles.fetch_sub(1); }

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) bytes = 1;
    if (g_alloc) {
        *p = g_alloc(bytes, (void*)st, g_alloc_ctx);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

void dev_free(void* p, cudaStream_t st)
{
    if (!p) return;
    if (g_free)
        g_free(p, (void*)st, g_alloc_ctx);
    else
        cudaFreeAsync(p, st);
}

cudaError_t dev_alloc_sync(void** p, size_t bytes)
{
    if (bytes == 0) bytes = 1;
    if (g_alloc) {
        *p = g_alloc(bytes, nullptr, g_alloc_ctx);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void dev_free_sync(void* p)
{
    if (!p) return;
    if (g_free) {
        // the buffer may be in use on any stream: let all work finish first
        // (cudaFree does the same implicitly)
        cudaDeviceSynchronize();
        g_free(p, nullptr, g_alloc_ctx);
    } else {
        cudaFree(p);
    }
}

tigre_status DeviceBuffer::ensure(size_t need)
{
    if (need <= bytes && ptr) return TIGRE_OK;
    release();
    if (need == 0) return TIGRE_OK;
    cudaError_t e = dev_alloc_sync(&ptr, need);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        cudaGetLastError();
        return cuda_fail(e, "device allocation (workspace)");
    }
    bytes = need;
    return TIGRE_OK;
}

void DeviceBuffer::release()
{
    if (ptr) dev_free_sync(ptr);
    ptr = nullptr;
    bytes = 0;
    tag = 0;
}

std::vector<uint64_t> workspace_signature(const tigre_geometry* g)
{
    std::vector<uint64_t> sig;
    for (const DeviceBuffer* b : {&g->vol_xy, &g->vol_yx, &g->vol_qxy, &g->vol_qyx, &g->proj_pad,
                                  &g->adj_xy, &g->adj_yx, &g->err_flag, &g->brick_prange}) {
        sig.push_back((uint64_t)(uintptr_t)b->ptr);
        sig.push_back(b->tag);
    }
    sig.push_back((uint64_t)g->fwd_path);
    sig.push_back((uint64_t)g->projector);
    return sig;
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

tigre_status validate_desc(const tigre_geometry_desc* d, const double* angles, int64_t na)
{
    if (!d || !angles) return fail(TIGRE_ERR_INVALID_ARG, "null geometry or angles");
    if (na <= 0) return fail(TIGRE_ERR_INVALID_ARG, "n_angles must be > 0");
    if (!finite_pos(d->DSO) || !finite_pos(d->DSD) || !(d->DSD > d->DSO))
        return fail(TIGRE_ERR_INVALID_ARG, "need 0 < DSO < DSD (finite)");
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (d->n_voxel[a] <= 0 || d->n_voxel[a] > (1 << 20))
            return fail(TIGRE_ERR_INVALID_ARG, "n_voxel out of range");
        if (!finite_pos(d->d_voxel[a])) return fail(TIGRE_ERR_INVALID_ARG, "d_voxel must be > 0");
        if (!std::isfinite(d->off_origin[a]))
            return fail(TIGRE_ERR_INVALID_ARG, "off_origin must be finite");
        double half = 0.5 * (double)(d->n_voxel[a] + 1) * d->d_voxel[a] + std::fabs(d->off_origin[a]);
        if (a < 2) r2 += half * half;
    }
    if (!(std::sqrt(r2) < d->DSO))
        return fail(TIGRE_ERR_INVALID_ARG, "source orbit intersects the volume (DSO too small)");
    for (int a = 0; a < 2; ++a) {
        if (d->n_det[a] <= 0 || d->n_det[a] > (1 << 20))
            return fail(TIGRE_ERR_INVALID_ARG, "n_det out of range");
        if (!finite_pos(d->d_det[a])) return fail(TIGRE_ERR_INVALID_ARG, "d_det must be > 0");
        if (!std::isfinite(d->off_det[a])) return fail(TIGRE_ERR_INVALID_ARG, "off_det must be finite");
    }
    if (!(std::isfinite(d->accuracy) && d->accuracy >= 1e-3 && d->accuracy <= 4.0))
        return fail(TIGRE_ERR_INVALID_ARG, "accuracy must be in [1e-3, 4] voxels");
    for (int64_t i = 0; i < na; ++i)
        if (!std::isfinite(angles[i])) return fail(TIGRE_ERR_INVALID_ARG, "angles must be finite");
    return TIGRE_OK;
}

tigre_status check_geometry(tigre_geometry* g)
{
    if (!g) return fail(TIGRE_ERR_INVALID_ARG, "null geometry handle");
    int dev = -1;
    TIGRE_CUDA(cudaGetDevice(&dev));
    if (g->device < 0) g->device = dev;
    if (dev != g->device)
        return fail(TIGRE_ERR_INVALID_ARG, "geometry handle used on another device");
    if (!g->uploaded) TIGRE_TRY(upload_params(g));
    return TIGRE_OK;
}

tigre_status check_range(const tigre_geometry* g, int64_t begin, int64_t count)
{
    if (begin < 0 || count <= 0 || begin + count > (int64_t)g->angles.size())
        return fail(TIGRE_ERR_INVALID_ARG, "angle range outside the geometry's angles");
    return TIGRE_OK;
}

bool detector_row_range(const tigre_geometry_desc& d, double za, double zb, double* lo, double* hi)
{
    // Farthest distance from the rotation axis of the support box (voxel
    // centres -1 .. n along x and y, offsets included).
    double r2 = 0.0;
    for (int k = 0; k < 2; ++k) {
        const double h = 0.5 * (double)(d.n_voxel[k] + 1) * d.d_voxel[k];
        const double e = std::max(std::fabs(d.off_origin[k] - h), std::fabs(d.off_origin[k] + h));
        r2 += e * e;
    }
    const double R = std::sqrt(r2);
    if (!(R < d.DSO)) return false;
    // A point at depth L = DSO - X.(cos, sin) in [DSO - R, DSO + R] and height
    // z lies on the ray of detector height v = z DSD / L (the source is at z = 0).
    const double mags[2] = {d.DSD / (d.DSO + R), d.DSD / (d.DSO - R)};
    const double zc = 0.5 * (double)(d.n_voxel[2] - 1);
    const double pv_off = 0.5 * (double)(d.n_det[1] - 1) - d.off_det[1] / d.d_det[1];
    double vlo = 1e300, vhi = -1e300;
    for (double zi : {za, zb}) {
        const double Z = (zi - zc) * d.d_voxel[2] + d.off_origin[2];
        for (double m : mags) {
            const double q = Z * m / d.d_det[1] + pv_off;
            vlo = std::min(vlo, q);
            vhi = std::max(vhi, q);
        }
    }
    *lo = vlo;
    *hi = vhi;
    return true;
}

// Memory layout an angle's forward projection reads: rays of one detector
// row spread along e_u = (-sin, cos, 0), so the layout whose fastest axis is
// the one e_u is closest to (1: y fastest, when |cos| > |sin|).
int angle_layout(double t) { return std::fabs(std::cos(t)) > std::fabs(std::sin(t)) ? 1 : 0; }

// Angle groups for the angle-interleaved forward kernel.  Rays through one
// pixel at neighbouring angles pass within a few voxels of each other, so a
// warp of (32 / size) pixels x size angles gathers from fewer cache lines
// than 32 pixels of one angle.  A group holds angles of one layout and one
// march direction (the sign of the ray along the layout's depth axis),
// neighbours in angle; -1 fills a short group.
AngleGroups build_angle_groups(const tigre_geometry_desc& d, const double* angles, int64_t na)
{
    AngleGroups out;
    std::vector<int> cls[4];
    const double pi = std::acos(-1.0);
    const double centre[4] = {1.5 * pi, 0.5 * pi, pi, 0.0};
    for (int64_t a = 0; a < na; ++a) {
        const double t = angles[a];
        const int l = angle_layout(t);
        const double main = l ? std::cos(t) : std::sin(t);
        cls[l * 2 + (main > 0.0 ? 1 : 0)].push_back((int)a);
    }
    for (int k = 0; k < 4; ++k)
        std::stable_sort(cls[k].begin(), cls[k].end(), [&](int i, int j) {
            return std::remainder(angles[i] - centre[k], 2.0 * pi) <
                   std::remainder(angles[j] - centre[k], 2.0 * pi);
        });
    // Median angular gap inside pairs x the largest distance of a voxel from
    // the rotation axis = how far apart (in voxels) the rays of one pixel at
    // paired angles get.  Pairs paid at 6.3 voxels (512^3 x 360: 3.8 %,
    // 1024^3 x 720: 3.9 %) and 12.6 (1024^3 x 360: 3.3 %); groups of four
    // lost 9 % at 50 (1024^3 x 90).
    std::vector<double> gaps;
    for (const std::vector<int>& v : cls)
        for (size_t i = 0; i + 1 < v.size(); i += 2)
            gaps.push_back(std::fabs(std::remainder(angles[v[i + 1]] - angles[v[i]], 2.0 * pi)));
    if (!gaps.empty()) {
        std::nth_element(gaps.begin(), gaps.begin() + gaps.size() / 2, gaps.end());
        const double wx = 0.5 * (double)d.n_voxel[0] * d.d_voxel[0] + std::fabs(d.off_origin[0]);
        const double wy = 0.5 * (double)d.n_voxel[1] * d.d_voxel[1] + std::fabs(d.off_origin[1]);
        out.drift = gaps[gaps.size() / 2] * std::sqrt(wx * wx + wy * wy) /
                    std::min(d.d_voxel[0], d.d_voxel[1]);
        out.auto_pairs = out.drift <= kPairDriftVoxels;
    }
    for (int gi = 0; gi < 2; ++gi) {
        const size_t size = gi ? 4 : 2;
        for (const std::vector<int>& v : cls)
            for (size_t i = 0; i < v.size(); i += size)
                for (size_t j = 0; j < size; ++j)
                    out.table[gi].push_back(i + j < v.size() ? v[i + j] : -1);
    }
    return out;
}

tigre_status upload_params(tigre_geometry* g)
{
    const tigre_geometry_desc& d = g->desc;
    const int64_t na = (int64_t)g->angles.size();
    std::vector<FwdAngle> fwd((size_t)na);
    std::vector<FwdAngle64> fwd64((size_t)na);
    std::vector<BpAngle> bp((size_t)na);
    g->layout.assign((size_t)na, 0);
    const double nu = (double)d.n_det[0], nv = (double)d.n_det[1];
    const double u0 = -0.5 * (nu - 1.0) * d.d_det[0] + d.off_det[0];
    const double v0 = -0.5 * (nv - 1.0) * d.d_det[1] + d.off_det[1];
    for (int64_t a = 0; a < na; ++a) {
        const double t = g->angles[(size_t)a];
        const double c = std::cos(t), s = std::sin(t);
        const double S[3] = {d.DSO * c, d.DSO * s, 0.0};
        const double D[3] = {-(d.DSD - d.DSO) * c, -(d.DSD - d.DSO) * s, 0.0};
        const double eu[3] = {-s, c, 0.0};
        const double ev[3] = {0.0, 0.0, 1.0};
        double src[3], base[3], dp[3], dq[3];
        for (int k = 0; k < 3; ++k) {
            src[k] = (S[k] - d.off_origin[k]) / d.d_voxel[k] + 0.5 * (double)(d.n_voxel[k] - 1);
            base[k] = (D[k] - S[k] + u0 * eu[k] + v0 * ev[k]) / d.d_voxel[k];
            dp[k] = d.d_det[0] * eu[k] / d.d_voxel[k];
            dq[k] = d.d_det[1] * ev[k] / d.d_voxel[k];
        }
        // Rays of one detector row spread along e_u: choose the memory layout
        // whose fastest axis is the one e_u is closest to.
        const int layout = angle_layout(t);
        const int perm[3] = {layout ? 1 : 0, layout ? 0 : 1, 2};
        FwdAngle& f = fwd[(size_t)a];
        FwdAngle64& f64 = fwd64[(size_t)a];
        std::memset(&f, 0, sizeof(f));
        for (int k = 0; k < 3; ++k) {
            f64.src[k] = src[perm[k]];
            f64.base[k] = base[perm[k]];
            f64.dp[k] = dp[perm[k]];
            f64.dq[k] = dq[perm[k]];
            f.src[k] = (float)src[perm[k]];
            f.base[k] = (float)base[perm[k]];
            f.dp[k] = (float)dp[perm[k]];
            f.dq[k] = (float)dq[perm[k]];
        }
        f.layout = layout;
        f.index = (int)a;
        g->layout[(size_t)a] = layout;
        bp[(size_t)a] = BpAngle{(float)c, (float)s, (float)S[0], (float)S[1]};
    }
    // Angle indices grouped by layout (stable), for full-range projections.
    std::vector<int> order;
    order.reserve((size_t)na);
    for (int l = 0; l < 2; ++l)
        for (int64_t a = 0; a < na; ++a)
            if (g->layout[(size_t)a] == l) order.push_back((int)a);
    TIGRE_TRY(g->angle_order.ensure(sizeof(int) * (size_t)na));
    TIGRE_CUDA(cudaMemcpy(g->angle_order.ptr, order.data(), sizeof(int) * (size_t)na,
                          cudaMemcpyHostToDevice));
    {
        const AngleGroups ag = build_angle_groups(d, g->angles.data(), na);
        g->auto_angle_group = ag.auto_pairs ? 2 : 1;
        for (int gi = 0; gi < 2; ++gi) {
            const std::vector<int>& tab = ag.table[gi];
            g->n_groups[gi] = (int64_t)(tab.size() / (gi ? 4 : 2));
            TIGRE_TRY(g->angle_groups[gi].ensure(sizeof(int) * std::max<size_t>(tab.size(), 1)));
            if (!tab.empty())
                TIGRE_CUDA(cudaMemcpy(g->angle_groups[gi].ptr, tab.data(), sizeof(int) * tab.size(),
                                      cudaMemcpyHostToDevice));
        }
    }
    TIGRE_TRY(g->fwd_params.ensure(sizeof(FwdAngle) * (size_t)na));
    TIGRE_TRY(g->bp_params.ensure(sizeof(BpAngle) * (size_t)na));
    TIGRE_TRY(g->fwd_params64.ensure(sizeof(FwdAngle64) * (size_t)na));
    TIGRE_CUDA(cudaMemcpy(g->fwd_params.ptr, fwd.data(), sizeof(FwdAngle) * (size_t)na,
                          cudaMemcpyHostToDevice));
    TIGRE_CUDA(cudaMemcpy(g->fwd_params64.ptr, fwd64.data(), sizeof(FwdAngle64) * (size_t)na,
                          cudaMemcpyHostToDevice));
    TIGRE_TRY(build_ray_exceptions(g));
    TIGRE_CUDA(cudaMemcpy(g->bp_params.ptr, bp.data(), sizeof(BpAngle) * (size_t)na,
                          cudaMemcpyHostToDevice));
    g->uploaded = true;
    return TIGRE_OK;
}

}  // namespace tigre

using namespace tigre;

extern "C" {

const char* tigre_last_error(void) { return g_last_error.c_str(); }

tigre_status tigre_geometry_create(const tigre_geometry_desc* desc, const double* angles,
                                   int64_t n_angles, tigre_geometry_t* out)
{
    if (!out) return fail(TIGRE_ERR_INVALID_ARG, "null output handle pointer");
    *out = nullptr;
    TIGRE_TRY(validate_desc(desc, angles, n_angles));
    tigre_geometry* g = new (std::nothrow) tigre_geometry();
    if (!g) return fail(TIGRE_ERR_OOM, "host allocation failed");
    handle_created();
    g->desc = *desc;
    g->angles.assign(angles, angles + n_angles);
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        tigre_geometry_destroy(g);
        return cuda_fail(e, "cudaGetDevice");
    }
    tigre_status st = upload_params(g);
    if (st != TIGRE_OK) {
        tigre_geometry_destroy(g);
        return st;
    }
    *out = g;
    set_error("");
    return TIGRE_OK;
}

tigre_status tigre_geometry_destroy(tigre_geometry_t g)
{
    if (!g) return TIGRE_OK;
    g->fwd_params.release();
    g->fwd_params64.release();
    g->ray_exc_start.release();
    g->ray_exc.release();
    g->bp_params.release();
    g->angle_order.release();
    g->angle_groups[0].release();
    g->angle_groups[1].release();
    for (int gi = 0; gi < 2; ++gi)
        for (auto& kv : g->range_groups[gi]) kv.second.release();
    g->vol_xy.release();
    g->vol_yx.release();
    g->vol_qxy.release();
    g->vol_qyx.release();
    g->proj_pad.release();
    g->adj_xy.release();
    g->adj_yx.release();
    g->err_flag.release();
    g->brick_prange.release();
    g->scratch_vol.release();
    g->scratch_red.release();
    delete g;
    handle_destroyed();
    return TIGRE_OK;
}

tigre_status tigre_set_allocator(tigre_alloc_fn alloc, tigre_free_fn free_fn, void* ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(TIGRE_ERR_INVALID_ARG, "give both alloc and free, or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_live_handles.load() != 0)
        return fail(TIGRE_ERR_INVALID_ARG,
                    "the allocator can only change while no geometry or CGLS handle is alive");
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = alloc ? ctx : nullptr;
    return TIGRE_OK;
}

tigre_status tigre_solver_opts_default(tigre_solver_opts* o)
{
    if (!o) return fail(TIGRE_ERR_INVALID_ARG, "null opts");
    std::memset(o, 0, sizeof(*o));
    o->n_iter = 10;
    o->lambda = 1.0;
    o->subset_size = 20;
    o->tv_steps = 0;
    o->tv_alpha = 0.002;
    o->tv_eps = 1e-8;
    o->bp_weight = TIGRE_BP_MATCHED;
    o->nonneg = 0;
    o->storage = TIGRE_F32;
    o->device_budget_bytes = 0;
    o->timeout_ms = 0;
    o->flags = 0;
    o->cuda_stream = nullptr;
    return TIGRE_OK;
}

}  // extern "C"

extern "C" tigre_status tigre_forward_angle_groups(const tigre_geometry_desc* desc,
                                                   const double* angles, int64_t n_angles,
                                                   int size, int* table, int64_t capacity,
                                                   int64_t* n_groups, double* drift,
                                                   int* auto_pairs)
{
    using namespace tigre;
    if (!desc || !angles || n_angles <= 0 || !n_groups || !drift || !auto_pairs)
        return fail(TIGRE_ERR_INVALID_ARG, "null argument or no angles");
    if (size != 2 && size != 4) return fail(TIGRE_ERR_INVALID_ARG, "group size must be 2 or 4");
    for (int k = 0; k < 3; ++k)
        if (desc->n_voxel[k] <= 0 || !(desc->d_voxel[k] > 0.0) || !std::isfinite(desc->d_voxel[k]) ||
            !std::isfinite(desc->off_origin[k]))
            return fail(TIGRE_ERR_INVALID_ARG, "voxel counts and sizes must be > 0 and finite");
    for (int64_t a = 0; a < n_angles; ++a)
        if (!std::isfinite(angles[a])) return fail(TIGRE_ERR_INVALID_ARG, "angles must be finite");
    const AngleGroups ag = build_angle_groups(*desc, angles, n_angles);
    const std::vector<int>& tab = ag.table[size == 4 ? 1 : 0];
    *n_groups = (int64_t)(tab.size() / (size_t)size);
    *drift = ag.drift;
    *auto_pairs = ag.auto_pairs ? 1 : 0;
    if (table) {
        if (capacity < (int64_t)tab.size())
            return fail(TIGRE_ERR_INVALID_ARG, "table capacity below n_groups * size");
        std::copy(tab.begin(), tab.end(), table);
    }
    return TIGRE_OK;
}

