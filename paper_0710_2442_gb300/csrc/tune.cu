// tune.cu -- the launch-configuration autotuner.
//
// A launch is identified by a key (kernel, precisions, link format, flags,
// lattice extents).  The first time a key is seen the candidates are timed
// on the caller's stream with CUDA events (per candidate: a warm-up launch,
// one timed launch, then two timed bursts of four back-to-back launches
// unless the single launch took longer than 300 us; the best time per launch
// counts), and the fastest is kept: a later candidate must be faster by more
// than a margin (1 %; the batch's tile size asks 5 %) to replace an earlier one.  Tuning synchronises the stream, so the
// first call for a new key is slower; it is skipped while the stream is being
// captured into a graph (the fallback is used and the key is not stored).
// A decision from the cache file that is not among the current candidates
// (written by another build) is ignored and the key is tuned again.
//
// Environment:
//   WILSON_TUNE=0            never time candidates (use the fallback)
//   WILSON_TUNE_CACHE=path   load decisions from / append them to a file
//   WILSON_TUNE_VERBOSE=1    report decisions on stderr
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

#include "internal.h"

namespace wl {

namespace {

struct Entry {
    LaunchConfig cfg;
    float us;
};

std::mutex g_mutex;
std::map<std::string, Entry>* g_cache = nullptr;
bool g_loaded = false;

bool env_flag(const char* name, bool dflt) {
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    return !(v[0] == '0' && v[1] == 0);
}

// "sm<major><minor>-<SM count>" of the current device, looked up once per
// device ordinal (every hop launch asks for it).
std::string device_tag() {
    static std::mutex m;
    static std::string tags[64];
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cacheable = dev >= 0 && dev < 64;
    if (cacheable) {
        std::lock_guard<std::mutex> lk(m);
        if (!tags[dev].empty()) return tags[dev];
    }
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return "dev?";
    }
    char buf[64];
    snprintf(buf, sizeof(buf), "sm%d%d-%d", major, minor, sms);
    if (cacheable) {
        std::lock_guard<std::mutex> lk(m);
        tags[dev] = buf;
    }
    return buf;
}

void load_file() {
    g_loaded = true;
    const char* path = std::getenv("WILSON_TUNE_CACHE");
    if (!path || !*path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string key;
        Entry e;
        if (is >> key >> e.cfg.block >> e.cfg.variant >> e.us) (*g_cache)[key] = e;
    }
}

void append_file(const std::string& key, const Entry& e) {
    const char* path = std::getenv("WILSON_TUNE_CACHE");
    if (!path || !*path) return;
    std::ofstream f(path, std::ios::app);
    f << key << ' ' << e.cfg.block << ' ' << e.cfg.variant << ' ' << e.us << '\n';
}

}  // namespace

const std::vector<LaunchConfig>& hop_candidates() {
    static const std::vector<LaunchConfig> c = [] {
        std::vector<LaunchConfig> v;
        for (int block : {64, 128, 256})
            for (int var = 0; var < 6; var++) v.push_back(LaunchConfig{block, var});
        return v;
    }();
    return c;
}

namespace {

// The cached decision for the device-tagged key, if it is among the current
// candidates.
bool cached(const std::string& key, const std::vector<LaunchConfig>& candidates, LaunchConfig& out) {
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!g_cache) g_cache = new std::map<std::string, Entry>();
    if (!g_loaded) load_file();
    auto it = g_cache->find(key);
    if (it == g_cache->end()) return false;
    bool known = candidates.empty();
    for (const LaunchConfig& c : candidates)
        known = known || (c.block == it->second.cfg.block && c.variant == it->second.cfg.variant);
    if (known) out = it->second.cfg;
    return known;
}

}  // namespace

LaunchConfig tune_lookup(const std::string& key0, const std::vector<LaunchConfig>& candidates,
                         const LaunchConfig& fallback) {
    LaunchConfig c;
    return cached(device_tag() + "|" + key0, candidates, c) ? c : fallback;
}

LaunchConfig tune_launch(const std::string& key0, const std::vector<LaunchConfig>& candidates,
                         const LaunchConfig& fallback, cudaStream_t st,
                         const std::function<void(const LaunchConfig&)>& run, double margin) {
    const std::string key = device_tag() + "|" + key0;
    {
        LaunchConfig c;
        if (cached(key, candidates, c)) return c;
    }
    if (!env_flag("WILSON_TUNE", true) || candidates.empty()) return fallback;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    WL_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return fallback;

    NvtxRange nvtx_tune("wilson autotune");
    cudaEvent_t e0, e1;
    WL_CUDA(cudaEventCreate(&e0));
    WL_CUDA(cudaEventCreate(&e1));
    // Each candidate is timed once alone and then, unless that launch took
    // longer than 300 us (its launch gap is then negligible and bursts would
    // make tuning slow), twice as a burst of kBurst back-to-back launches, the
    // way operators run; the best time per launch counts.  A later candidate
    // replaces the best one only when it is faster by more than the margin,
    // so candidates within timing noise of each other resolve to the same
    // (earlier) choice in every process.
    constexpr int kBurst = 4;
    Entry best{fallback, 1e30f};
    for (const LaunchConfig& c : candidates) {
        run(c);  // warm-up
        if (cudaGetLastError() != cudaSuccess) continue;  // candidate not launchable here
        float ms_best = 1e30f;
        int burst = 1;
        for (int rep = 0; rep < 3; rep++) {
            WL_CUDA(cudaEventRecord(e0, st));
            for (int b = 0; b < burst; b++) run(c);
            WL_CUDA(cudaEventRecord(e1, st));
            WL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            WL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            ms /= burst;
            if (ms < ms_best) ms_best = ms;
            if (rep == 0 && ms < 0.3f) burst = kBurst;
        }
        if (cudaGetLastError() != cudaSuccess) continue;
        const float us = ms_best * 1e3f;
        if (env_flag("WILSON_TUNE_VERBOSE", false))
            fprintf(stderr, "[wilson tune]   %s block %d variant %d: %.2f us\n", key.c_str(), c.block, c.variant, us);
        if (us < (float)(1.0 - margin) * best.us) best = Entry{c, us};
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (env_flag("WILSON_TUNE_VERBOSE", false))
        fprintf(stderr, "[wilson tune] %s -> block %d variant %d (%.2f us)\n", key.c_str(), best.cfg.block,
                best.cfg.variant, best.us);
    std::lock_guard<std::mutex> lk(g_mutex);
    (*g_cache)[key] = best;
    append_file(key, best);
    return best.cfg;
}

}  // namespace wl
