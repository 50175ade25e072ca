// Launch counting and per-kernel-class event timing.
//
// Every kernel launch of the library goes through TIGRE_LAUNCHED, which
// counts it.  When profiling is on, the operator entry points also bracket
// their main kernels with CUDA events on the launching stream; the elapsed
// times are summed when read.  (Events are recorded only while enabled, so
// the default path costs one relaxed atomic increment per launch.)
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "../../include/tigre103.h"

namespace tigre {

static std::atomic<int64_t> g_launches{0};
static std::atomic<int> g_profiling{0};
static std::mutex g_mu;

struct EventPair {
    cudaEvent_t a, b;
    int kind;
};
static std::vector<EventPair> g_pairs;
static double g_ms[kProfKinds];
static int64_t g_count[kProfKinds];

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool profiling() { return g_profiling.load(std::memory_order_relaxed) != 0; }

ProfScope::ProfScope(int kind, cudaStream_t st) : kind_(kind), st_(st)
{
    if (!profiling()) return;
    // Work captured into a graph does not run now: nothing to time.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st_, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(a_, st_);
    active_ = true;
}

ProfScope::~ProfScope()
{
    if (!active_) return;
    cudaEventRecord(b_, st_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pairs.push_back(EventPair{a_, b_, kind_});
}

// Fold recorded event pairs into the totals (synchronises on each event).
static void drain()
{
    for (EventPair& p : g_pairs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.kind] += ms;
            g_count[p.kind] += 1;
        }
        cudaGetLastError();
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pairs.clear();
}

}  // namespace tigre

using namespace tigre;

extern "C" {

tigre_status tigre_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    for (int k = 0; k < kProfKinds; ++k) {
        g_ms[k] = 0.0;
        g_count[k] = 0;
    }
    g_launches.store(0);
    g_profiling.store(on ? 1 : 0);
    return TIGRE_OK;
}

tigre_status tigre_profile_read(int kind, int64_t* calls, double* total_ms)
{
    if (kind < 0 || kind >= kProfKinds || !calls || !total_ms)
        return fail(TIGRE_ERR_INVALID_ARG, "bad profile kind or null output");
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    *calls = g_count[kind];
    *total_ms = g_ms[kind];
    return TIGRE_OK;
}

int64_t tigre_launch_count(void) { return g_launches.load(); }

}  // extern "C"
