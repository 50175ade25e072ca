/*
 * tigre103.h -- C ABI of the GB300 (sm_103a) cone-beam CT library.
 *
 * The operators of iterative cone-beam CT (paper Eq. 1: A x = b + e, with A
 * the ray/element intersection operator; every iterative method applies A
 * and A^T at least once per iteration, Sec. 2):
 *
 *   tigre_forward   interpolated ray-driven forward projection  A x  (Sec. 2.1)
 *   tigre_backward  voxel-driven weighted backprojection A^T y (Sec. 2.2),
 *                   FDK or pseudo-matched weights, or the exact transpose of
 *                   tigre_forward
 *   tigre_tv_step   gradient-descent total-variation steps (Sec. 2.3)
 *   tigre_sirt / tigre_sart / tigre_cgls
 *                   SIRT, OS-SART (+TV), CGLS drivers (Sec. 3.2 uses CGLS
 *                   and OS-SART) with every iterate resident on the device
 *
 * Conventions (all lengths mm, angles rad):
 *   volume  vol[k][j][i], shape (nz, ny, nx), x fastest, contiguous;
 *           voxel centre X = ((i-(nx-1)/2) dx, (j-(ny-1)/2) dy,
 *                             (k-(nz-1)/2) dz) + off_origin
 *   orbit   source S = DSO (cos t, sin t, 0), detector centre
 *           D = -(DSD-DSO)(cos t, sin t, 0), e_u = (-sin t, cos t, 0),
 *           e_v = (0, 0, 1); pixel (p, q) centre
 *           D + ((p-(nu-1)/2) du + off_u) e_u + ((q-(nv-1)/2) dv + off_v) e_v
 *   projections proj[a][q][p], shape (n_angles, nv, nu), u fastest.
 *
 * Forward projection: the trilinear interpolant of the volume (zero outside,
 * i.e. virtual zero voxels at index -1 and n) is integrated along the ray
 * source -> pixel centre by the midpoint rule: the ray is clipped to the
 * support [-1, n] per axis, K = max(1, ceil(len / (accuracy * min d) - 1e-9))
 * samples of step h = len / K at the midpoints (K as computed in FP64 for every
 * ray: rays whose FP32 set-up would round K differently are found once, when
 * the handle is created); proj = h * sum f(sample), mm x density.
 *
 * Backprojection (voxel-driven): for each voxel centre X and angle, s =
 * X.(cos t, sin t, 0); the line source->X meets the detector at
 * (u, v) = (X.e_u, X_z) * DSD/(DSO - s); the projection is interpolated
 * bilinearly there (zero outside the detector) and weighted by
 *   TIGRE_BP_FDK:      (DSO/(DSO - s))^2
 *   TIGRE_BP_MATCHED:  (dx dy dz)/(du dv) * |X - S| * DSD^2 / (DSO - s)^3
 *                      (voxel volume over the ray tube cross-section of one
 *                      pixel at X: approximates the transpose of A)
 *   TIGRE_BP_EXACT_ADJOINT: the exact transpose of tigre_forward (each
 *                      sample scatters h * trilinear weight * y).
 *
 * Memory: the caller owns every volume / projection buffer.  Unless a
 * function says otherwise they are DEVICE pointers (e.g. PyTorch tensors),
 * contiguous, in the stated dtype.  The library owns only workspaces, which
 * it caches inside the geometry handle and frees in tigre_geometry_destroy.
 * A geometry handle is used by one host thread / one stream at a time.
 *
 * Errors: every function returns a tigre_status and never throws or aborts.
 * On failure tigre_last_error() returns a message for the calling thread.
 */
#ifndef TIGRE103_H
#define TIGRE103_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TIGRE_API __attribute__((visibility("default")))
#else
#define TIGRE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TIGRE_OK = 0,
    TIGRE_ERR_INVALID_ARG = 1, /* bad pointer, size, dtype or geometry */
    TIGRE_ERR_OOM = 2,         /* device or pinned allocation failed / over budget */
    TIGRE_ERR_CUDA = 3,        /* CUDA runtime error; see tigre_last_error() */
    TIGRE_ERR_TIMEOUT = 4,     /* a host wait exceeded opts.timeout_ms */
    TIGRE_ERR_UNSUPPORTED = 5  /* valid request the library does not implement */
} tigre_status;

/* Storage type of a volume / projection buffer.  Arithmetic is FP32 along
 * every ray and voxel sum whatever the storage type; solver scalars FP64. */
typedef enum { TIGRE_F32 = 0, TIGRE_BF16 = 1, TIGRE_F16 = 2 } tigre_dtype;

typedef enum {
    TIGRE_BP_MATCHED = 0,
    TIGRE_BP_FDK = 1,
    TIGRE_BP_EXACT_ADJOINT = 2
} tigre_bp_weight;

/* Circular cone-beam geometry (Sec. 3.1 experiments: N^3 voxels, N^2 pixels,
 * N angles).  accuracy = forward-projection ray step in voxels (0.5 typical). */
typedef struct {
    double DSO, DSD;       /* source-origin and source-detector distance */
    int64_t n_voxel[3];    /* nx, ny, nz */
    double d_voxel[3];     /* dx, dy, dz */
    double off_origin[3];  /* volume centre offset */
    int64_t n_det[2];      /* nu, nv */
    double d_det[2];       /* du, dv */
    double off_det[2];     /* detector offset along e_u, e_v */
    double accuracy;
} tigre_geometry_desc;

typedef struct tigre_geometry* tigre_geometry_t;

/* The circular cone-beam geometry of the paper's experiments (Sec. 3.1:
 * DSO, DSD, voxel and detector grids, projection angles).  Validate the
 * description and copy the angles (host array of n_angles
 * doubles).  Requires DSO > 0, DSD > DSO, all sizes > 0, finite values, and a
 * source orbit outside the volume.  Invalid arguments are rejected before any
 * CUDA call; a valid geometry is bound to the current device and its
 * per-angle parameters are uploaded synchronously (so create handles before
 * any stream capture).  *out must be released by tigre_geometry_destroy. */
TIGRE_API tigre_status tigre_geometry_create(const tigre_geometry_desc* desc, const double* angles,
                                   int64_t n_angles, tigre_geometry_t* out);
TIGRE_API tigre_status tigre_geometry_destroy(tigre_geometry_t geo);

/* Sec. 2.1, the interpolated ray-driven projection:
 * proj[0 .. angle_count) = A vol for angles angle_begin .. +angle_count.
 * vol: device (nz, ny, nx) in vol_dtype; proj: device (angle_count, nv, nu) in
 * proj_dtype, overwritten.  Asynchronous on cuda_stream (a cudaStream_t; NULL
 * = legacy default stream). */
TIGRE_API tigre_status tigre_forward(tigre_geometry_t geo, const void* vol, tigre_dtype vol_dtype,
                           void* proj, tigre_dtype proj_dtype, int64_t angle_begin,
                           int64_t angle_count, void* cuda_stream);

/* Sec. 2.2, the voxel-driven backprojection (FDK or pseudo-matched weights,
 * or the exact transpose of tigre_forward):
 * vol = sum over angles angle_begin .. +angle_count of the weighted
 * backprojection of proj (device (angle_count, nv, nu), proj_dtype).  vol:
 * device (nz, ny, nx) in vol_dtype, overwritten.  Asynchronous. */
TIGRE_API tigre_status tigre_backward(tigre_geometry_t geo, const void* proj, tigre_dtype proj_dtype,
                            void* vol, tigre_dtype vol_dtype, int64_t angle_begin,
                            int64_t angle_count, tigre_bp_weight weight, void* cuda_stream);

/* Sec. 2.3, TV minimisation by gradient descent:
 * n_steps of x <- x - alpha g / ||g||_2, g the gradient of
 * TV_eps(x) = sum sqrt(Dx^2 + Dy^2 + Dz^2 + eps) with backward differences
 * (zero across the low boundary); a step with ||g|| = 0 leaves x unchanged.
 * vol: device (nz, ny, nx), updated in place.  ||g|| is reduced in FP64.
 * Uses a scratch volume (FP32) allocated per call.  Asynchronous. */
TIGRE_API tigre_status tigre_tv_step(const int64_t n_voxel[3], void* vol, tigre_dtype dtype, int n_steps,
                           double alpha, double eps, void* cuda_stream);

/* tigre_tv_step without any device allocation (the paper has no counterpart:
 * this is a service for callers that cannot allocate device memory while they
 * run, such as a real-time loop that reserved all GPU memory at start-up
 * because cudaMalloc/cudaFree can synchronise the device and take unbounded
 * time, or a process whose memory another allocator already holds).  Same
 * arguments and results as tigre_tv_step; the gradient and the FP64 reduction
 * live in one fixed scratch array compiled into the library (16 MiB + 5 KiB,
 * held on every GPU that loads the library until the process exits).
 * Volumes of more than 4,194,304 voxels are rejected with
 * TIGRE_ERR_INVALID_ARG.  The first call on a device (n_steps = 0 is
 * enough) is its set-up: with that device current it looks up the scratch
 * address (cudaGetSymbolAddress) and loads the TV kernels, and CUDA's lazy
 * module loading takes device memory for that code then.  Make that call at
 * start-up, before reserving the device memory and before any stream capture;
 * later calls allocate nothing.  All calls share the scratch: calls that
 * overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  No state carries over between calls. */
TIGRE_API tigre_status tigre_tv_step_noalloc(const int64_t n_voxel[3], void* vol, tigre_dtype dtype,
                                             int n_steps, double alpha, double eps,
                                             void* cuda_stream);

/* The placement (1 or 2, see TIGRE_OUT_OF_CORE) and the slab thickness in
 * z planes that an out-of-core tigre_cgls on this geometry uses under
 * device_budget_bytes (0 = free device memory less 1 GiB).  Sec. 2 sizes the
 * paper's splits from the memory each GPU has; this is that decision for one
 * GPU.  TIGRE_ERR_OOM when the budget is below three projection sets plus
 * one-plane slabs.  Queries free memory only; allocates nothing. */
TIGRE_API tigre_status tigre_cgls_ooc_plan(tigre_geometry_t geo, int64_t device_budget_bytes,
                                           int* placement, int64_t* slab_planes);
/* The same decision from a geometry description and its angles, on the host
 * alone (no device, no handle): device_budget_bytes must be > 0.  Errors as
 * tigre_geometry_create for the description, TIGRE_ERR_OOM as above. */
TIGRE_API tigre_status tigre_cgls_ooc_plan_desc(const tigre_geometry_desc* desc,
                                                const double* angles, int64_t n_angles,
                                                int64_t device_budget_bytes, int* placement,
                                                int64_t* slab_planes);

/* Out-of-core forward projection (paper Alg. 1 on one GPU): vol_host is a
 * HOST pointer (F32, (nz, ny, nx)), streamed to the device in axial slabs of
 * slab_planes planes (0 = sized from free device memory) on a copy stream,
 * overlapped with the projection of the previous slab; partial projections
 * accumulate into proj (DEVICE, F32, (angle_count, nv, nu), overwritten).
 * Pageable host memory is page-locked for the call.  Synchronous. */
TIGRE_API tigre_status tigre_forward_ooc(tigre_geometry_t geo, const float* vol_host, float* proj,
                                         int64_t angle_begin, int64_t angle_count,
                                         int64_t slab_planes, void* cuda_stream);

/* Out-of-core voxel-driven backprojection (paper Alg. 2 on one GPU): each
 * axial slab of vol_host (HOST, F32, overwritten) is backprojected from all
 * angles on the device and copied out while the next slab is computed.
 * proj (F32) is a device pointer, or with proj_on_host != 0 a host pointer
 * streamed in chunks of angle_chunk angles through two device buffers.
 * weight: MATCHED or FDK.  Synchronous. */
TIGRE_API tigre_status tigre_backward_ooc(tigre_geometry_t geo, const float* proj,
                                          int proj_on_host, float* vol_host, int64_t angle_begin,
                                          int64_t angle_count, tigre_bp_weight weight,
                                          int64_t slab_planes, int64_t angle_chunk,
                                          void* cuda_stream);

/* Solver flags. */
#define TIGRE_HOST_RESIDENT 0x1u /* proj / vol are host pointers (out-of-core mode) */
#define TIGRE_GRAPH 0x2u         /* stepwise CGLS: replay captured iteration pairs (CUDA graphs) */
/* tigre_cgls only: proj and vol are HOST pointers (F32) and CGLS runs with
 * part of its state in host memory, the volume streamed through the device in
 * axial slabs (paper Alg. 1 and 2 on one GPU).  device_budget_bytes (0 = free
 * device memory less 1 GiB) bounds ALL device memory the call uses and picks
 * the placement (see tigre_cgls_ooc_plan):
 *   2, when x and two projection sets fit: x, r, q on the device, only the
 *      search direction in host memory -- inside the caller's vol buffer,
 *      which holds x again on return -- and s = A^T r recomputed instead of
 *      stored (two backprojections per iteration); no host allocation;
 *   1, otherwise: x, p, s in host memory (two volumes of pinned host memory
 *      allocated for the call), b, r, q on the device.
 * Both give the in-core iterates up to FP32 summation order. */
#define TIGRE_OUT_OF_CORE 0x4u
/* The initial guess is zero, so vol is not read: the library zeroes it on the
 * device (a host-resident vol is not copied in), and CGLS starts from r = b
 * as the method's initialisation states, without projecting x0 (the same
 * bits as projecting a zero x0).  Not with TIGRE_OUT_OF_CORE. */
#define TIGRE_X0_ZERO 0x8u

typedef struct {
    int n_iter;                 /* iterations (default 10) */
    double lambda;              /* SIRT / OS-SART relaxation (default 1) */
    int subset_size;            /* OS-SART angles per subset (default 20) */
    int tv_steps;               /* OS-SART: TV steps after each iteration (0 = off) */
    double tv_alpha;            /* TV step = tv_alpha * ||x_after - x_before|| */
    double tv_eps;              /* TV smoothing (default 1e-8) */
    tigre_bp_weight bp_weight;  /* backprojector (default MATCHED) */
    int nonneg;                 /* clamp x >= 0 after each update (SIRT/OS-SART) */
    tigre_dtype storage;        /* storage type of the iterates (default F32) */
    int64_t device_budget_bytes;/* 0 = free device memory; used by out-of-core */
    int64_t timeout_ms;         /* SIRT / OS-SART / in-core CGLS: the final wait for
                                   the queued iterations is bounded by this many ms
                                   (default 0 = none).  On expiry TIGRE_ERR_TIMEOUT:
                                   the work completes on its stream (device buffers
                                   become valid once it drains), resid_hist is not
                                   filled and host-resident vol is not copied back. */
    uint32_t flags;             /* TIGRE_HOST_RESIDENT, TIGRE_GRAPH, TIGRE_OUT_OF_CORE,
                                   TIGRE_X0_ZERO */
    void* cuda_stream;          /* stream for all work (NULL = default) */
} tigre_solver_opts;

/* Device workspace allocator.  alloc(bytes, cuda_stream, ctx) returns device
 * memory usable on cuda_stream (NULL on failure: the call then returns
 * TIGRE_ERR_OOM); free_fn(ptr, cuda_stream, ctx) releases it once the work
 * already queued on cuda_stream is done.  cuda_stream is NULL for buffers
 * cached in a geometry handle, which the library frees only after a device
 * synchronisation.  Every workspace the library allocates afterwards goes
 * through the pair (e.g. a framework's caching allocator); both NULL restores
 * cudaMallocAsync / cudaFreeAsync (cudaMalloc / cudaFree for cached buffers).
 * Process-wide; TIGRE_ERR_INVALID_ARG while any geometry handle or CGLS state
 * is alive, so each buffer is freed by the allocator that made it.  The
 * paper's implementation allocates its outputs on every call (Sec. 4 names
 * this as a cost); here outputs are the caller's and only workspaces remain. */
typedef void* (*tigre_alloc_fn)(size_t bytes, void* cuda_stream, void* ctx);
typedef void (*tigre_free_fn)(void* ptr, void* cuda_stream, void* ctx);
TIGRE_API tigre_status tigre_set_allocator(tigre_alloc_fn alloc, tigre_free_fn free_fn, void* ctx);

/* Fill *opts with the defaults listed above (no counterpart in the paper). */
TIGRE_API tigre_status tigre_solver_opts_default(tigre_solver_opts* opts);

/* SIRT, one of the iterative methods that apply A and A^T every iteration
 * (Sec. 2): (x <- x + lambda V A_w^T W (b - A x), W = 1/(A 1), V = 1/(A_w^T 1),
 * reciprocals of values <= 1e-12 set to 0).  proj: b (n_angles, nv, nu) F32;
 * vol: (nz, ny, nx) F32 initial guess in, result out.  resid_hist (host,
 * n_iter doubles, may be NULL) receives ||b - A x_k|| before update k. */
TIGRE_API tigre_status tigre_sirt(tigre_geometry_t geo, const void* proj, void* vol,
                        const tigre_solver_opts* opts, double* resid_hist);

/* OS-SART (Sec. 3.2 reconstructs the Ichthyosaur with it, subsets of 200
 * angles): the SIRT update applied per subset of subset_size consecutive
 * angles, subsets in order; with tv_steps > 0, tigre_tv_step after each full
 * iteration with alpha = tv_alpha * ||x - x_prev||.  resid_hist[k] =
 * sqrt(sum over subsets of ||b_s - A_s x||^2) during iteration k. */
TIGRE_API tigre_status tigre_sart(tigre_geometry_t geo, const void* proj, void* vol,
                        const tigre_solver_opts* opts, double* resid_hist);

/* CGLS (Sec. 3.2 reconstructs the coffee bean with it) with FP64 inner
 * products computed on the device; x0 = vol on entry
 * (r0 = b - A x0).  resid_hist[k] = ||r|| after iteration k.  proj, vol and
 * the iterates are stored in opts->storage (F32, BF16 or F16): every ray and
 * voxel sum and every vector update is computed in FP32 and rounded once to
 * the storage type; inner products, norms and step lengths stay FP64 on the
 * device.  Out-of-core (TIGRE_OUT_OF_CORE) stores F32 only.  F16 storage
 * has a narrow range: A^T r and A p grow to ~||A||^2 ||b|| (about 1e6 for
 * mm-unit ray sums of a 64^3 head), so the caller scales b (CGLS is linear
 * in b) to keep them below 65504; BF16 has FP32's range. */
TIGRE_API tigre_status tigre_cgls(tigre_geometry_t geo, const void* proj, void* vol,
                        const tigre_solver_opts* opts, double* resid_hist);

/* Stepwise CGLS (no counterpart in the paper; the same iteration as
 * tigre_cgls) for callers that
 * interleave several reconstructions or time single iterations.
 * begin: device proj (b) and vol (x0, updated in place) must stay valid until
 *        end; computes r = b - A x0, p = A^T r, gamma = ||p||^2 and allocates
 *        the workspace (2 projection- and 2 volume-sized FP32 buffers) stream-
 *        ordered on opts->cuda_stream.  TIGRE_HOST_RESIDENT is not accepted.
 * iterate: enqueues n_iter iterations on that stream (no host sync).
 * history: copies the first n residual norms (n <= iterations done) to the
 *        host, synchronising the stream.
 * end:   releases the workspace (stream-ordered) and the handle. */
typedef struct tigre_cgls_state* tigre_cgls_t;
TIGRE_API tigre_status tigre_cgls_begin(tigre_geometry_t geo, const void* proj, void* vol,
                                        const tigre_solver_opts* opts, tigre_cgls_t* out);
TIGRE_API tigre_status tigre_cgls_iterate(tigre_cgls_t state, int n_iter);
TIGRE_API tigre_status tigre_cgls_history(tigre_cgls_t state, double* resid_hist, int n);
TIGRE_API tigre_status tigre_cgls_end(tigre_cgls_t state);

/* Batched CGLS (no counterpart in the paper, which reconstructs one volume at
 * a time with the Sec. 3.2 CGLS; a service for reconstruction servers): batch
 * problems that share the geometry handle and opts->storage, iterated
 * together.  Each iteration projects the batch's search directions in ONE
 * forward-projector launch and backprojects its residuals in ONE voxel-driven
 * backprojector launch (the member index runs over the grid); inner
 * products, norms, step lengths and vector updates are each member's own.
 * Every member's x and residual history are bitwise those of tigre_cgls on
 * that problem alone.
 * begin: projs[i] (b) and vols[i] (x0, updated in place) are DEVICE buffers
 *        in opts->storage, valid until end.  Flags: TIGRE_GRAPH (replay
 *        captured iteration pairs; needs a non-default stream) and
 *        TIGRE_X0_ZERO (x_i zeroed, r_i = b_i).  The handle must use the
 *        interpolated projector and the automatic forward path; bp_weight
 *        MATCHED or FDK.  Workspaces (owned by the batch, stream-ordered on
 *        opts->cuda_stream): per member 4 iterate vectors, a quad copy of the
 *        zero-bordered volume per layout and one of the padded projections
 *        (16 bytes of FP32 coefficients per padded voxel or pixel).  Otherwise as tigre_cgls_begin; TIGRE_ERR_UNSUPPORTED for
 *        other flags, projectors or weights.
 * iterate: enqueues n_iter iterations of every member (no host sync).
 * history: the first n residual norms of member member_index (synchronises).
 * end:   releases the workspaces (stream-ordered) and the handle. */
typedef struct tigre_cgls_batch* tigre_cgls_batch_t;
TIGRE_API tigre_status tigre_cgls_batch_begin(tigre_geometry_t geo, int batch,
                                              const void* const* projs, void* const* vols,
                                              const tigre_solver_opts* opts,
                                              tigre_cgls_batch_t* out);
TIGRE_API tigre_status tigre_cgls_batch_iterate(tigre_cgls_batch_t state, int n_iter);
TIGRE_API tigre_status tigre_cgls_batch_history(tigre_cgls_batch_t state, int member_index,
                                                double* resid_hist, int n);
TIGRE_API tigre_status tigre_cgls_batch_end(tigre_cgls_batch_t state);

/* Checkpoint / resume of a stepwise CGLS (no counterpart in the paper; lets a
 * long reconstruction stop and continue, e.g. across job limits or when a
 * server preempts it).  save: copies the state's residual r (n_angles x nv x
 * nu) and search direction p (nz x ny x nx), in the state's storage type, to
 * HOST buffers of r_bytes and p_bytes (TIGRE_ERR_INVALID_ARG, nothing copied,
 * when either is smaller than its vector), and returns gamma = ||A^T r||^2
 * and the iterations done; synchronises the stream.  With the caller's x at
 * that point these are the whole state.  resume: a stepwise state from such
 * a checkpoint -- proj is b, vol holds the checkpoint's x (DEVICE,
 * opts->storage), r_host / p_host (r_bytes / p_bytes, checked as for save) /
 * gamma as saved -- that skips the initial A x0 and A^T r; its iterations
 * continue bitwise as the saved state's would have.  Its history covers the
 * iterations run after resuming. */
TIGRE_API tigre_status tigre_cgls_save(tigre_cgls_t state, void* r_host, size_t r_bytes,
                                       void* p_host, size_t p_bytes, double* gamma,
                                       int* iterations);
TIGRE_API tigre_status tigre_cgls_resume(tigre_geometry_t geo, const void* proj, void* vol,
                                         const void* r_host, size_t r_bytes, const void* p_host,
                                         size_t p_bytes, double gamma,
                                         const tigre_solver_opts* opts, tigre_cgls_t* out);

/* Out-of-core gradient-descent TV (Sec. 2.3's splitting of a regulariser,
 * on one GPU): vol_host is a HOST F32 volume (nz, ny, nx), updated in place.
 * In rounds of k = min(halo_depth, steps left) steps, each axial slab of
 * slab_planes planes (0 = the whole volume) is copied to the device with k
 * planes of buffer on each side holding the previous round's values, takes k
 * steps x <- x - alpha g/||g|| on its own, and writes its own planes back.
 * The buffer keeps each slab's interior exact for the k steps; ||g|| is
 * approximated from the slab's own voxels as if uniformly distributed over
 * the volume, ||g_slab|| sqrt(N / N_slab), as the paper does instead of a
 * synchronisation per step.  With one slab this is tigre_tv_step.  Needs
 * 1 <= halo_depth <= slab_planes (unless one slab).  Pageable memory is
 * page-locked for the call.  Synchronous. */
TIGRE_API tigre_status tigre_tv_step_ooc(const int64_t n_voxel[3], float* vol_host, int n_steps,
                                         double alpha, double eps, int64_t slab_planes,
                                         int64_t halo_depth, void* cuda_stream);

/* ROF-model TV minimisation (Sec. 2.3, the second TV minimiser the paper
 * uses): u = argmin ||grad u||_(2,1) + lambda/2 ||u - f||^2 (isotropic TV,
 * forward differences, zero at the last index of each axis), by n_iter steps
 * of the first-order primal-dual iteration (over-relaxation 1, step sizes
 * 1/sqrt(12)) from u = f and zero dual.  f, u: DEVICE F32 (nz, ny, nx); u is
 * overwritten and may be f itself.  lambda > 0.  Allocates four (five when u
 * is f) volumes of workspace stream-ordered for the call; asynchronous on
 * cuda_stream.  No counterpart of the voxel order's halo splitting is needed
 * on one device. */
TIGRE_API tigre_status tigre_rof_denoise(const int64_t n_voxel[3], const float* f, float* u,
                                         double lambda, int n_iter, void* cuda_stream);

/* FDK reconstruction of a circular scan over all the handle's angles (the
 * paper's analytic reconstruction, Sec. 1 and Sec. 3.2, for comparison and as
 * an initialiser): each projection is weighted by DSD/sqrt(DSD^2+u^2+v^2),
 * each detector row convolved (linearly, zero outside) with the Ram-Lak
 * kernel of pitch tau = du DSO/DSD (h0 = 1/(4 tau^2), h at odd k =
 * -1/(pi k tau)^2, even k zero; times tau for the sum), and the result
 * backprojected with the FDK weight (DSO/(DSO-s))^2, each angle times half
 * its angular weight (half the angle between its neighbours on the circle).
 * proj: DEVICE (n_angles, nv, nu) in proj_dtype; vol: DEVICE (nz, ny, nx) in
 * vol_dtype, overwritten.  Allocates the filtered projections (F32)
 * stream-ordered for the call.  Asynchronous on cuda_stream except for one
 * small table upload. */
TIGRE_API tigre_status tigre_fdk(tigre_geometry_t geo, const void* proj, tigre_dtype proj_dtype,
                                 void* vol, tigre_dtype vol_dtype, void* cuda_stream);

/* Projector of this handle (Sec. 2.1 offers both; Sec. 3.1 times SIDDON, which
 * is TIGRE's default): INTERPOLATED (default here) samples the trilinear interpolant at the
 * midpoints of K equal steps; SIDDON integrates the piecewise-constant volume
 * exactly, voxel (i,j,k) filling [i-1/2, i+1/2] x ... in index space, as the
 * sum of its intersection lengths (mm) with the ray times the voxel values.
 * The choice applies to tigre_forward, to TIGRE_BP_EXACT_ADJOINT (the
 * transpose of the chosen projector) and to the solvers; the voxel-driven
 * MATCHED and FDK backprojectors are the same for both.  Out-of-core
 * projection supports INTERPOLATED only (TIGRE_ERR_UNSUPPORTED otherwise). */
typedef enum { TIGRE_PROJ_INTERPOLATED = 0, TIGRE_PROJ_SIDDON = 1 } tigre_projector;
TIGRE_API tigre_status tigre_geometry_set_projector(tigre_geometry_t geo, int projector);

/* Alg. 1 on one GPU: edge (voxels) of the x-y bricks into which out-of-core
 * projections cut
 * each z-slab (0 = default 512).  Rays resident on the GPU at one time then
 * read one brick's planes, which stay in L2; at 3072^2 a single quad plane
 * of the slab is larger than L2.  In-core projections on the automatic path
 * (forward path 0, F32 volume and projections) march the same bricks when
 * the volume is wider than one brick (1024^3 x 720: 11 % faster).  Only the
 * partial sums' order changes. */
TIGRE_API tigre_status tigre_geometry_set_brick(tigre_geometry_t geo, int64_t edge);

/* Kernel choice for this handle's Sec. 2.1 projector (no counterpart in the
 * paper): 0 = automatic (the quad
 * gather kernel; with 2 angles per warp when the rays of one pixel at paired
 * angles stay within 16 voxels of each other, e.g. 512^3 x 360), 1 = scalar
 * L1 gather kernel, 2 = shared-memory slab kernel (TMA-staged; only for
 * geometries whose ray bundles fit its staging box, otherwise it reports
 * error bit 2 and NaN), 3 = quad gather kernel (two 16-byte loads per sample
 * from a layout holding each cell plane's four bilinear coefficients in FP32,
 * whatever the volume's storage type; 16 bytes per padded voxel and memory
 * layout in workspace), 4 = quad gather kernel taking a
 * ray's samples two at a time (both samples' loads issued together), 5 / 6 =
 * quad gather kernel whose warps hold 16 pixels x 2 / 8 pixels x 4 angles
 * (neighbouring angles of one memory layout and march direction, so a warp's
 * gathers share cache lines; a partial angle range groups its own angles).
 * All compute the same sums in the same order and give identical results.
 * Out-of-core slab projections use the quad kernel: two samples at a time for
 * path 4, warps of 2 angles for path 5 and for path 0 when it pairs angles,
 * one angle per warp otherwise. */
TIGRE_API tigre_status tigre_geometry_set_forward_path(tigre_geometry_t geo, int path);

/* Scheduling of the Sec. 2.1 projector's threads (no counterpart in the
 * paper, whose kernel gives each thread one pixel of one angle): the angle
 * groups the forward projector's paths 5 / 6 (and path 0 when it pairs
 * angles) read, computed on the host (no device needed): size (2 or 4)
 * angle indices per group, each group of one memory layout (|cos| > |sin| or
 * not) and one march direction, neighbours in angle, -1 filling a short
 * group; n_groups groups.  drift = the median angle gap inside pairs times
 * the largest distance of a voxel from the rotation axis, in voxels;
 * auto_pairs = 1 when the automatic path pairs angles (drift <= 16).  table
 * may be NULL (sizes only); otherwise it holds capacity ints, at least
 * n_groups * size, or the call fails with INVALID_ARG. */
TIGRE_API tigre_status tigre_forward_angle_groups(const tigre_geometry_desc* desc,
                                                  const double* angles, int64_t n_angles,
                                                  int size, int* table, int64_t capacity,
                                                  int64_t* n_groups, double* drift,
                                                  int* auto_pairs);

/* (No counterpart in the paper.)  Error bits raised by kernels of this
 * handle (1 = a bounded wait timed out,
 * 2 = a slab did not fit its staging box, 4 = rays of one block ran opposite
 * ways; the affected outputs are NaN).  Synchronous; clear != 0 resets. */
TIGRE_API tigre_status tigre_geometry_error_flags(tigre_geometry_t geo, int* flags, int clear);

/* The work of one Sec. 2.1 forward projection: total quadrature samples
 * (sum of K over rays) of tigre_forward for the
 * angle range: the algorithmic work of one forward projection.  Runs a
 * ray-setup kernel on the current device and synchronises. */
TIGRE_API tigre_status tigre_forward_samples(tigre_geometry_t geo, int64_t angle_begin,
                                             int64_t angle_count, int64_t* samples);

/* Profiling (no counterpart in the paper; Sec. 3.1 reports kernel and
 * transfer times apart): tigre_profile_enable(1) resets the counters and
 * starts timing
 * the main kernel of each operator call with CUDA events on its stream;
 * tigre_profile_read(kind, ...) waits for the recorded events and returns the
 * number of timed calls and their total device time.  kind: 0 forward
 * projection, 1 voxel-driven backprojection, 2 exact-adjoint scatter, 3 TV
 * step.  tigre_launch_count() is the number of kernels the library launched
 * since the last tigre_profile_enable. */
TIGRE_API tigre_status tigre_profile_enable(int on);
TIGRE_API tigre_status tigre_profile_read(int kind, int64_t* calls, double* total_ms);
TIGRE_API int64_t tigre_launch_count(void);

/* Message describing the last failure on the calling thread ("" if none;
 * no counterpart in the paper). */
TIGRE_API const char* tigre_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TIGRE103_H */
