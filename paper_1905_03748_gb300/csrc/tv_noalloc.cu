// tigre_tv_step_noalloc: the TV steps of tigre_tv_step without any device
// allocation.
//
// Who needs it: callers that cannot allocate device memory while they run.
// A real-time reconstruction loop (for example in image-guided radiotherapy)
// typically reserves all the GPU memory it will ever use at start-up and then
// must not call the allocator, because cudaMalloc / cudaFree can synchronise
// the whole device and take an unbounded time.  A process whose device memory
// is owned by another allocator (a framework's caching allocator that already
// holds the free memory) may see a library's own cudaMalloc fail, or fragment
// that pool.  tigre_tv_step allocates a volume-sized gradient and a reduction
// area on every call; this entry point instead uses one fixed scratch array
// compiled into the library.
//
// The scratch array below is a device symbol: a GPU holds it (16 MiB + 5 KiB)
// from the moment this library's code is loaded on it until the process
// exits.  In host code its name is only a stand-in for the symbol, not a
// device address, so the address is looked up once per device with
// cudaGetSymbolAddress and cached.  That look-up, and the loading of the TV
// kernels (CUDA loads a module's code lazily, on first use, and loading takes
// device memory), happen in the first call made with a device current --
// also when that call has n_steps = 0.  A caller that reserves its device
// memory at start-up therefore makes one call per device first (n_steps = 0
// is enough), before the reservation and before any stream capture.
#include <cmath>
#include <mutex>

#include "vecops.cuh"

namespace tigre {

// Largest volume the fixed scratch serves: 4,194,304 voxels (160^3 is 4,096,000).
constexpr int64_t kNoAllocMaxVoxels = int64_t(1) << 22;
// FP32 gradient, then the FP64 reduction area (partials + norm slots).
constexpr int64_t kNoAllocRedDoubles = kRedBlocks + 4;
constexpr int64_t kNoAllocFloats = kNoAllocMaxVoxels + 2 * kNoAllocRedDoubles;

static __device__ __align__(256) float g_tv_noalloc_scratch[kNoAllocFloats];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
tigre_status scratch_address(float** out)
{
    int dev = -1;
    TIGRE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(TIGRE_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_tv_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                             "cudaGetSymbolAddress(TV scratch)");
        }
        TIGRE_TRY(tv_load_kernels());
        g_scratch_addr[dev] = p;
    }
    *out = (float*)g_scratch_addr[dev];
    return TIGRE_OK;
}
}  // namespace

}  // namespace tigre

using namespace tigre;

extern "C" tigre_status tigre_tv_step_noalloc(const int64_t n_voxel[3], void* vol,
                                              tigre_dtype dtype, int n_steps, double alpha,
                                              double eps, void* cuda_stream)
{
    if (!n_voxel || !vol) return fail(TIGRE_ERR_INVALID_ARG, "null n_voxel or vol");
    for (int a = 0; a < 3; ++a)
        if (n_voxel[a] <= 0 || n_voxel[a] > (1 << 20))
            return fail(TIGRE_ERR_INVALID_ARG, "n_voxel out of range");
    if (!dtype_ok(dtype)) return fail(TIGRE_ERR_INVALID_ARG, "bad dtype");
    if (n_steps < 0 || !std::isfinite(alpha) || !std::isfinite(eps) || eps < 0.0)
        return fail(TIGRE_ERR_INVALID_ARG, "need n_steps >= 0, finite alpha, eps >= 0");
    const int64_t N = n_voxel[0] * n_voxel[1] * n_voxel[2];
    if (N > kNoAllocMaxVoxels)
        return fail(TIGRE_ERR_INVALID_ARG,
                    "tigre_tv_step_noalloc: the volume has " + std::to_string(N) +
                        " voxels, more than its fixed scratch holds (4194304); use tigre_tv_step");
    float* scratch = nullptr;
    TIGRE_TRY(scratch_address(&scratch));  // first call on a device: the set-up
    if (n_steps == 0) return TIGRE_OK;
    // Every kernel writes the gradient and the reduction partials in full
    // before reading them, so nothing left by an earlier call is used.
    double* red = reinterpret_cast<double*>(scratch + kNoAllocMaxVoxels);
    return tv_impl(n_voxel, vol, dtype, n_steps, alpha, eps, nullptr, scratch, red,
                   (cudaStream_t)cuda_stream);
}
