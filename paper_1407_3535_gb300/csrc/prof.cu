// Launch accounting and optional per-kernel CUDA-event timing.
//
// Every launcher in the library wraps its kernel launch in a LaunchScope.
// The scope always counts the launch; when timing is enabled it records a
// CUDA event pair on the launching stream so that per-kernel device time can
// be read back after the work completes (opta_dbg_profile_*).
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "opta_debug.h"

namespace opta {

namespace {

struct Rec {
    const char *name;
    cudaEvent_t a, b;
};

std::mutex g_mu;
unsigned long long g_launches = 0;
bool g_timing = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

LaunchScope::LaunchScope(const char *name, cudaStream_t s) : name_(name), s_(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_launches;
    if (g_timing) {
        a_ = take_event();
        cudaEventRecord(static_cast<cudaEvent_t>(a_), s_);
    }
}

LaunchScope::~LaunchScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s_);
    g_recs.push_back({name_, static_cast<cudaEvent_t>(a_), b});
}

cudaError_t ensure_smem(const void *func, size_t bytes) {
    // the attribute applies to the device current when it is set, so the
    // limit already raised is remembered per (kernel, device)
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = set[std::make_pair(func, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

}  // namespace opta

using namespace opta;

extern "C" {

void opta_dbg_scan1_wait(uint64_t wait_ns, int32_t stall) { set_scan1_wait(wait_ns, stall); }

uint64_t opta_dbg_launch_count(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_launches;
}

void opta_dbg_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing = on != 0;
}

int32_t opta_dbg_profile_read(char *names, int32_t name_stride, double *total_ms,
                              int64_t *launches, int32_t capacity) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<std::string> keys;
    std::vector<double> tot;
    std::vector<int64_t> cnt;
    for (const Rec &r : g_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        size_t k = 0;
        for (; k < keys.size(); ++k) if (keys[k] == r.name) break;
        if (k == keys.size()) { keys.emplace_back(r.name); tot.push_back(0.0); cnt.push_back(0); }
        tot[k] += ms;
        cnt[k] += 1;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    const int n = (int)keys.size();
    for (int i = 0; i < n && i < capacity; ++i) {
        if (names && name_stride > 0) {
            std::strncpy(names + (size_t)i * name_stride, keys[i].c_str(), name_stride - 1);
            names[(size_t)i * name_stride + name_stride - 1] = 0;
        }
        if (total_ms) total_ms[i] = tot[i];
        if (launches) launches[i] = cnt[i];
    }
    return n;
}

}  // extern "C"
