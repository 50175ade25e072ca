// Internal declarations shared by the translation units of libtigre103.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/tigre103.h"

namespace tigre {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);
tigre_status fail(tigre_status st, const std::string& msg);
tigre_status cuda_fail(cudaError_t err, const char* what);

#define TIGRE_CUDA(call)                                             \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::tigre::cuda_fail(e_, #call); \
    } while (0)

#define TIGRE_TRY(call)                            \
    do {                                           \
        tigre_status s_ = (call);                  \
        if (s_ != TIGRE_OK) return s_;             \
    } while (0)

// Count a kernel launch and check for a launch error right after it.
void count_launch();
#define TIGRE_LAUNCHED(name)                                           \
    do {                                                               \
        ::tigre::count_launch();                                       \
        cudaError_t e_ = cudaGetLastError();                           \
        if (e_ != cudaSuccess) return ::tigre::cuda_fail(e_, name);    \
    } while (0)

// Kernel classes timed by tigre_profile_read.
enum ProfKind { kProfForward = 0, kProfBackproject = 1, kProfAdjoint = 2, kProfTV = 3, kProfKinds = 4 };
bool profiling();
// Records CUDA events around a scope on `st` while profiling is enabled.
class ProfScope {
public:
    ProfScope(int kind, cudaStream_t st);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

private:
    int kind_;
    cudaStream_t st_;
    cudaEvent_t a_{}, b_{};
    bool active_ = false;
};

inline size_t dtype_size(tigre_dtype t) { return t == TIGRE_F32 ? 4 : 2; }
inline bool dtype_ok(tigre_dtype t) { return t == TIGRE_F32 || t == TIGRE_BF16 || t == TIGRE_F16; }

// ------------------------------------------------------------- conversions

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// Dispatch a functor templated on the storage type of one buffer.
template <typename F>
tigre_status dispatch_dtype(tigre_dtype t, F&& f)
{
    switch (t) {
    case TIGRE_F32: return f(float{});
    case TIGRE_BF16: return f(__nv_bfloat16{});
    case TIGRE_F16: return f(__half{});
    }
    return fail(TIGRE_ERR_INVALID_ARG, "unknown dtype");
}

// ---------------------------------------------------------- device buffers

// Device workspace allocation (see tigre_set_allocator): stream-ordered
// pairs, and pairs for buffers not tied to one stream.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
cudaError_t dev_alloc_sync(void** p, size_t bytes);
void dev_free_sync(void* p);
// Live geometry handles and CGLS states (the allocator may change only at 0).
void handle_created();
void handle_destroyed();

// A grow-only device buffer owned by a geometry handle.
struct DeviceBuffer {
    void* ptr = nullptr;
    size_t bytes = 0;
    uint64_t tag = 0;  // what the buffer's zero border was laid out for (0 = nothing)
    tigre_status ensure(size_t need);
    void release();
};

constexpr int64_t kBrickDefault = 512;  // x-y brick edge of out-of-core slab projections
constexpr double kPairDriftVoxels = 16.0;  // automatic 2-angle warps up to this ray drift

// Host-side angle groups of the forward projector (sizes 2 and 4).
struct AngleGroups {
    std::vector<int> table[2];  // group size 2, 4: angle indices, -1 filling short groups
    double drift = 0.0;         // voxels between the rays of one pixel at paired angles
    bool auto_pairs = false;    // the automatic path uses 2-angle warps
};
int angle_layout(double t);
// Groups of `size` neighbouring angles of one layout and march direction
// among angles[0 .. na), as indices into that array (-1 fills a short group).
AngleGroups build_angle_groups(const tigre_geometry_desc& d, const double* angles, int64_t na);
// Checks of a geometry description and its angles (host only).
tigre_status validate_desc(const tigre_geometry_desc* d, const double* angles, int64_t na);

// Per-angle parameters of the forward projector, expressed in the index
// coordinates of the padded volume layout the angle uses.  "f", "m", "s" are
// the fastest, middle and slowest memory axes of that layout.
struct FwdAngle {
    float src[3];   // source position (f, m, s), unpadded index units
    float base[3];  // (P - S)/d for pixel (0, 0)
    float dp[3];    // change of (P - S)/d per pixel along u
    float dq[3];    // change of (P - S)/d per pixel along v
    int layout;     // 0: x fastest (vol as given), 1: y fastest (transposed)
    int index;      // the angle's index (its FwdAngle64 entry)
    int pad_[2];
};
static_assert(sizeof(FwdAngle) == 64, "FwdAngle must stay 64 bytes");

// The same vectors in FP64 (not rounded to FP32), for the once-per-geometry
// search of rays whose FP32 sample count is wrong.
struct FwdAngle64 {
    double src[3], base[3], dp[3], dq[3];
};

// A ray whose FP32 set-up gets its sample count wrong: its pixel column and
// its FP64 clip (rounded to FP32) and count.
struct RayException {
    int p;         // detector column
    int K;         // samples (0: the ray misses the support)
    float t0, t1;  // clip of src + t (P - S)
    float len;     // chord length (mm)
};

// Per-angle parameters of the voxel-driven backprojector.
struct BpAngle {
    float c, s;       // cos, sin of the angle
    float srcx, srcy; // source position (mm)
};

}  // namespace tigre

// The opaque handle of the C ABI.
struct tigre_geometry {
    tigre_geometry_desc desc;
    std::vector<double> angles;
    int device = -1;
    bool uploaded = false;
    tigre::DeviceBuffer fwd_params;   // FwdAngle[n_angles]
    tigre::DeviceBuffer fwd_params64; // FwdAngle64[n_angles]
    tigre::DeviceBuffer ray_exc_start; // int[n_angles * nv + 1]: rows' first exception
    tigre::DeviceBuffer ray_exc;       // RayException[n_ray_exc], grouped by detector row
    int64_t n_ray_exc = 0;
    tigre::DeviceBuffer bp_params;    // BpAngle[n_angles]
    tigre::DeviceBuffer angle_order;  // int[n_angles]: angle indices grouped by layout
    // Angle groups of 2 and 4 (index 0, 1) for the angle-interleaved forward
    // kernel: int[n_groups * size], -1 filling a short group.
    tigre::DeviceBuffer angle_groups[2];
    int64_t n_groups[2] = {0, 0};
    // The same tables for partial angle ranges (begin, count), indices relative
    // to the range's first angle; built on first use (OS-SART's subsets).
    std::map<std::pair<int64_t, int64_t>, tigre::DeviceBuffer> range_groups[2];
    std::map<std::pair<int64_t, int64_t>, int64_t> range_n_groups[2];
    // Angles per warp of the automatic forward path (1 or 2): 2 when rays of
    // one pixel at grouped angles stay within a few voxels of each other.
    int auto_angle_group = 1;
    tigre::DeviceBuffer vol_xy;       // padded volume, x fastest
    tigre::DeviceBuffer vol_yx;       // padded volume, y fastest
    tigre::DeviceBuffer vol_qxy;      // quad volumes of the two padded layouts
    tigre::DeviceBuffer vol_qyx;
    tigre::DeviceBuffer proj_pad;     // zero-bordered projections for the backprojector
    tigre::DeviceBuffer adj_xy;       // FP32 padded accumulators of the exact adjoint
    tigre::DeviceBuffer adj_yx;
    tigre::DeviceBuffer scratch_vol;  // FP32 volume-sized scratch
    tigre::DeviceBuffer scratch_red;  // reduction partials / device scalars
    std::vector<int> layout;          // forward-projector layout per angle (host copy)
    // 0 auto, 1 L1 scalar, 2 TMA slab, 3 quad, 4 quad pairs, 5 / 6 quad with
    // 2 / 4 angles per warp
    int fwd_path = 0;
    int projector = 0;                // TIGRE_PROJ_INTERPOLATED or TIGRE_PROJ_SIDDON
    tigre::DeviceBuffer err_flag;     // int: error bits set by kernels (bounds, timeouts)
    tigre::DeviceBuffer brick_prange; // int2 per (x-y brick, angle): detector columns reaching it
    int64_t brick = tigre::kBrickDefault;  // x-y brick edge (voxels) of slab projections
};

namespace tigre {

constexpr int kPad = 2;  // zero voxels around the volume in the padded layouts

tigre_status upload_params(tigre_geometry* g);
// Sets every ray of the geometry up in FP32 (as the projector kernels do) and
// in FP64, and keeps the rays whose sample counts differ (forward.cu).
tigre_status build_ray_exceptions(tigre_geometry* g);
// Detector row coordinates [lo, hi] (row index units, continuous) that any
// point of the support with z in [za, zb] (voxel index units) projects to,
// over all angles; false when the source can be inside the support (no bound).
bool detector_row_range(const tigre_geometry_desc& d, double za, double zb, double* lo, double* hi);
size_t padded_elems(const tigre_geometry_desc& d);
// Out-of-core building blocks: the quad volume of a layout of the
// (sub-)volume described by d, built straight from it (its zero borders
// included); the projection of one slab's quads; and the voxel-driven
// backprojection of planes [z_first, z_end) into a slab buffer whose first
// plane is z_first.
tigre_status build_quads_f32(const tigre_geometry_desc& d, const float* vol, float4* out, int layout,
                             cudaStream_t st);
tigre_status forward_slab_impl(tigre_geometry* g, const tigre_geometry_desc& sd,
                               float4* const quad[2], float* proj, int64_t a0, int64_t na,
                               int cell_lo, int cell_hi, int plane0, cudaStream_t st);
// Bytes of the zero-bordered F32 quad projection buffer that slab launches of
// `slab` planes over na angles need at most (the largest row band).
size_t bp_slab_pad_bytes(const tigre_geometry_desc& d, int64_t slab, int64_t na);
tigre_status backward_slab_impl(tigre_geometry* g, const float* proj, float* vol_slab, int64_t a0,
                                int64_t na, tigre_bp_weight w, int accumulate, int z_first,
                                int z_end, cudaStream_t st);

// CGLS with host-resident volume vectors (ooc.cu).
tigre_status cgls_ooc_impl(tigre_geometry* g, const float* b_host, float* x_host,
                           const tigre_solver_opts* o, double* h_hist);

// Siddon projector and its transpose (siddon.cu); volumes in the padded
// layouts, accumulators as for the exact adjoint.
template <typename TV, typename TP>
tigre_status launch_siddon_forward(tigre_geometry* g, const TV* vxy, const TV* vyx, TP* proj,
                                   int64_t a0, int64_t na, const int* order, cudaStream_t st);
template <typename TP>
tigre_status launch_siddon_scatter(tigre_geometry* g, const TP* proj, float* acc_xy, float* acc_yx,
                                   int64_t a0, int64_t na, cudaStream_t st);

// Shared-memory slab forward projector (forward_tma.cu).
bool tma_forward_fits(const tigre_geometry_desc& d, size_t elem);
template <typename TV, typename TP>
tigre_status launch_forward_tma(tigre_geometry* g, const TV* vol, TP* proj, int64_t a0, int64_t na,
                                const bool need[2], int* d_err, cudaStream_t st);
// Pitched volume copies the TMA path reads (elem: bytes per element).
tigre_status tma_workspace(tigre_geometry* g, size_t elem, const bool need[2]);
// Every cached workspace of the geometry handle that a forward projection
// (volume stored as vt) or a backprojection (projections stored as pt) of
// the angles [a0, a0 + na) uses, allocated and zero-bordered ahead of the
// call.  The operators allocate only through these, and nothing once they
// have run with the same arguments; a stream capture (where allocation is
// refused) therefore runs them first.
tigre_status forward_workspace(tigre_geometry* g, tigre_dtype vt, int64_t a0, int64_t na,
                               cudaStream_t st);
tigre_status backward_workspace(tigre_geometry* g, tigre_dtype pt, tigre_bp_weight w, int64_t a0,
                                int64_t na);
// Identity of the cached workspaces (addresses and layout tags); a captured
// graph that holds these addresses replays only while it is unchanged.
std::vector<uint64_t> workspace_signature(const tigre_geometry* g);
// Several reconstructions of one geometry in one launch each (the batched
// CGLS): `batch` volumes (contiguous, storage dt) projected over all angles
// into `batch` consecutive projection sets, through the caller's quad
// workspaces (batch x padded_elems quads of dt per layout the angles use);
// and the voxel-driven backprojection
// of `batch` projection sets into `batch` volumes through a workspace of
// batch x backward_batch_workspace_bytes.  Each member's numbers are the
// single-volume operators' bit for bit.
tigre_status forward_batch_impl(tigre_geometry* g, const void* vols, void* projs, int batch,
                                 tigre_dtype dt, void* const quad[2], cudaStream_t st);
size_t backward_batch_workspace_bytes(const tigre_geometry* g, tigre_dtype dt);
tigre_status backward_batch_impl(tigre_geometry* g, const void* projs, void* vols, int batch,
                                 tigre_dtype dt, tigre_bp_weight w, void* ws, cudaStream_t st);
tigre_status ensure_padded(DeviceBuffer& buf, const tigre_geometry_desc& d, size_t elem, int layout,
                           cudaStream_t st);
tigre_status check_geometry(tigre_geometry* g);
tigre_status check_range(const tigre_geometry* g, int64_t begin, int64_t count);

inline int64_t n_vox(const tigre_geometry* g)
{
    return g->desc.n_voxel[0] * g->desc.n_voxel[1] * g->desc.n_voxel[2];
}
inline int64_t n_pix(const tigre_geometry* g) { return g->desc.n_det[0] * g->desc.n_det[1]; }

// ------------------------------------------------------ internal operators

// Forward projection with FP32 accumulation (see tigre_forward).
tigre_status forward_impl(tigre_geometry* g, const void* vol, tigre_dtype vt, void* proj,
                          tigre_dtype pt, int64_t a0, int64_t na, cudaStream_t st);
// Backprojection; accumulate != 0 adds into vol instead of overwriting.
tigre_status backward_impl(tigre_geometry* g, const void* proj, tigre_dtype pt, void* vol,
                           tigre_dtype vt, int64_t a0, int64_t na, tigre_bp_weight w,
                           int accumulate, cudaStream_t st);
tigre_status tv_impl(const int64_t n[3], void* vol, tigre_dtype t, int n_steps, double alpha,
                     double eps, const double* d_alpha_scale, void* scratch_g,
                     double* d_red, cudaStream_t st);
// Same, with ||g|| summed over the planes [k_lo, k_hi) only (all planes are
// updated): the out-of-core split's per-slab norm.
tigre_status tv_impl_region(const int64_t n[3], void* vol, tigre_dtype t, int n_steps,
                            double alpha, double eps, const double* d_alpha_scale,
                            void* scratch_g, double* d_red, int k_lo, int k_hi, cudaStream_t st);

// ------------------------------------------------------------ vector ops
// All reductions are deterministic: a fixed grid writes per-block FP64
// partial sums, then one block adds them in a fixed order.

constexpr int kRedBlocks = 608;      // 152 SMs x 4
constexpr int kRedThreads = 256;

// out[0] = sum_i a_i * b_i (FP64) over n elements of float arrays.
tigre_status dot_f64(const float* a, const float* b, int64_t n, double* d_partials, double* d_out,
                     cudaStream_t st);

// SART-type update fused into the voxel-driven backprojector:
// x += lambda * (sum_a w_a bil_a(r)) / (sum_a w_a bil_a(1)) over the angle
// range (no update where the denominator is <= 1e-12), then x = max(x, 0) if
// nonneg.  r: device F32 (na, nv, nu); x: device F32 volume.
tigre_status sart_update_impl(tigre_geometry* g, const float* r, float* x, int64_t a0, int64_t na,
                              tigre_bp_weight w, float lambda, int nonneg, cudaStream_t st);
// Same with r and x stored in dtype t (FP32 arithmetic).
tigre_status sart_update_dt(tigre_geometry* g, tigre_dtype t, const void* r, void* x, int64_t a0,
                            int64_t na, tigre_bp_weight w, float lambda, int nonneg,
                            cudaStream_t st);

}  // namespace tigre
