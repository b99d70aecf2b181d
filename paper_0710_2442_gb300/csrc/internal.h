// internal.h -- host-side declarations shared by the translation units of
// libwilson_gb300 (not part of the C ABI).
#pragma once

#include <functional>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/wilson.h"
#include "common.cuh"
#include "reduce.cuh"

namespace wl {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define WL_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw ::wl::Error(e_ == cudaErrorMemoryAllocation ? 3 : 2,                         \
                              std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

#define WL_LAUNCH_CHECK() WL_CUDA(cudaGetLastError())

#define WL_REQUIRE(cond, msg)                                      \
    do {                                                           \
        if (!(cond)) throw ::wl::Error(1, std::string(msg));       \
    } while (0)

// Launch of a kernel that begins with pdl_wait() (common.cuh), with the
// programmatic-serialization attribute: its blocks may be scheduled while the
// previous kernel on the stream drains, which hides the launch gap and the
// last wave's tail.  Launches into a stream that is being captured stay plain:
// measured, the attribute made the captured CG iterations slower (the graph
// already removes the launch gaps).  WILSON_PDL=0 launches every one plainly.
bool pdl_enabled();
template <typename... KArgs, typename... Args>
void launch_dep_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     const Args&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    cfg.numAttrs = pdl_enabled() && cs == cudaStreamCaptureStatusNone ? 1 : 0;
    WL_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}
template <typename... KArgs, typename... Args>
void launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, const Args&... args) {
    launch_dep_smem(kernel, grid, block, 0, st, args...);
}

// ---------------------------------------------------------------------------
// device memory owned by the library
// ---------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    explicit DevBuf(size_t n) { alloc(n); }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    void alloc(size_t n) {
        release();
        if (n) WL_CUDA(cudaMalloc(&p, n));
        bytes = n;
    }
    void ensure(size_t n) { if (n > bytes) alloc(n); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------------------
// autotuner (tune.cu)
// ---------------------------------------------------------------------------
struct LaunchConfig {
    int block = 128;
    int variant = 0;
};

// The launch configuration for `key`.  On the first request (and when tuning
// is enabled, WILSON_TUNE != 0, and the stream is not being captured) every
// candidate is timed by running `run` on the stream with CUDA events, and the
// fastest is cached (in memory, and in the file named by WILSON_TUNE_CACHE if
// set).  `run` must be idempotent: it is executed several times.
// margin: a later candidate replaces the best one so far only when it is
// faster by more than this fraction (so that near-ties resolve to the
// earlier candidate).
LaunchConfig tune_launch(const std::string& key, const std::vector<LaunchConfig>& candidates,
                         const LaunchConfig& fallback, cudaStream_t st,
                         const std::function<void(const LaunchConfig&)>& run, double margin = 0.01);
// The decision for `key` if one is cached (in memory or in the cache file)
// and among `candidates`, else `fallback`; never times anything and never
// synchronises.
LaunchConfig tune_lookup(const std::string& key, const std::vector<LaunchConfig>& candidates,
                         const LaunchConfig& fallback);
const std::vector<LaunchConfig>& hop_candidates();

// Geometry from dims and phases; stride rounded up to 64 sites.
Geom make_geom(const int dims[4], const double ph[4][2]);

inline int spinor_chunk_rows(Prec p) { return p == P_F64 ? 12 : p == P_F32 ? 6 : 3; }
long long spinor_field_bytes(Prec p, int stride);          // one parity, one rhs
long long gauge_bytes(Prec p, int recon, int stride);      // both parities, 4 directions
long long gauge_block_bytes(Prec p, int recon, int stride);

// A prepared spinor field: nrhs x (1 or 2 parities) SoA blocks.
struct SpinorField {
    Prec prec = P_F32;
    int subset = 0;      // 0 even, 1 odd, 2 full
    int nrhs = 1;
    Geom g{};
    DevBuf buf;
    long long pbytes = 0;   // bytes of one parity block of one rhs
    int nparity() const { return subset == 2 ? 2 : 1; }
    // pointer to parity block p (absolute parity 0/1) of rhs k
    void* block(int p, int k = 0) const {
        int slot = subset == 2 ? p : 0;
        return static_cast<char*>(buf.p) + (size_t)(k * nparity() + slot) * pbytes;
    }
    // bytes from one right-hand side's blocks to the next one's
    long long rstep() const { return (long long)nparity() * pbytes; }
    void alloc(Prec p, int sub, int nr, const Geom& geom);
};

struct GaugeField {
    Prec prec = P_F32;
    int recon = 12;
    Geom g{};
    DevBuf buf;
};

// Per-device scratch: reduction partials and counters.
struct Reduction {
    DevBuf partials;   // doubles
    DevBuf counters;   // unsigned ints, zeroed
    DevBuf results;    // doubles
    int capacity = 0;
    void init(int cap, int ncounters, cudaStream_t st);
    // Slots counter_slot .. counter_slot + nrhs - 1 (one per right-hand side).
    RedArgs args(int counter_slot, int op, double* result, CGScalars* sc) const {
        RedArgs r;
        r.partials = partials.as<double>() + (size_t)counter_slot * capacity;
        r.counter = counters.as<unsigned int>() + counter_slot;
        r.result = result;
        r.sc = sc;
        r.op = op;
        r.slot_cap = capacity;
        return r;
    }
};

// ---------------------------------------------------------------------------
// kernel launchers
// ---------------------------------------------------------------------------
struct HopLaunch {
    void* out;             // output parity block (parity out_parity), or parity-0 block if full
    const void* in;        // input block of parity 1 - out_parity, or parity-0 block if full
    const void* x;         // xpay block, parity out_parity (or parity-0 block if full); may be null
    long long out_pstep;   // full launches: byte offset of the parity-1 block from the parity-0 block
    long long in_pstep;
    long long x_pstep;
    int nrhs;              // right-hand sides in one launch (0 or 1: one)
    long long out_rstep;   // byte offset between consecutive right-hand sides
    long long in_rstep;
    long long x_rstep;
    int skip_stride;       // ints between the per-rhs skip flags
    const GaugeField* gauge;
    Prec sprec;
    int out_parity;        // single-parity launches
    int full;              // 1: both output parities in one launch
    int dagger;            // 1: projectors swapped (the hop of g5 D g5)
    int xpay;              // out = x + a * D in   (else out = a * D in)
    double a;
    const RedArgs* red;    // |out|^2 into a reducer, or null
    const int* skip;       // device flags (one per rhs): nonzero -> that rhs does nothing
    int block;             // threads per block (0 = autotuned)
    int variant;           // kernel register-budget variant when block > 0
    int grid_cap;          // max blocks of a reducing launch (0 = no cap)
    int tune_only;         // 1: tune the launch configuration if it is not known yet, launch nothing else
    int no_tune;           // 1: take a cached decision or the default configuration, never time candidates
};
void launch_hop(const HopLaunch& L, cudaStream_t st);
int hop_grid_blocks(const Geom& g, int block, int grid_cap);

// canonical <-> SoA
void pack_spinor(const SpinorField& f, int rhs, const double* canon, cudaStream_t st);
void unpack_spinor(const SpinorField& f, int rhs, double* canon, cudaStream_t st);
void pack_gauge(GaugeField& gf, const double* canon, cudaStream_t st);

int device_sm_count();

// NVTX range for profilers (nsys/ncu timelines); no cost without a tool.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Set the calling thread's message returned by wilson_last_error().
void record_error(const std::string& msg);

// Argument checks shared by the entry points (api.cu), so that every entry
// point validates the same way.
Geom checked_geom(const wilson_lattice* L);      // extents, phases, volume; WILSON_ERR_ARG
void check_ptr(const void* p, const char* what);  // non-null and 16-byte aligned; WILSON_ERR_ARG
void check_device();                              // a CUDA device exists; WILSON_ERR_CUDA
bool is_device_ptr(const void* p);                // device or managed memory

// DevBuf objects that borrow memory the library does not own through them
// (a fixed array, a stream-ordered pool): the guard detaches them before
// their destructors run, so those never free it.
struct BorrowGuard {
    DevBuf* bufs[8];
    int n = 0;
    void borrow(DevBuf& b, void* p, size_t bytes) {
        b.p = p;
        b.bytes = bytes;
        bufs[n++] = &b;
    }
    ~BorrowGuard() {
        for (int i = 0; i < n; i++) {
            bufs[i]->p = nullptr;
            bufs[i]->bytes = 0;
        }
    }
};

}  // namespace wl

// The opaque handles of the C ABI (wilson.h).
struct wilson_gauge_s {
    wl::GaugeField f;
    mutable std::mutex m;
    mutable wl::SpinorField tmp;  // intermediate field of the Schur operator
};
struct wilson_spinor_s {
    wl::SpinorField f;
    wl::Geom g;
};
