// noalloc.cu -- wilson_dslash_eo_noalloc: the even-odd hopping term and the
// Schur operator on canonical FP64 device fields, with no device allocation.
//
// Why it exists.  wilson_dslash_eo packs its canonical inputs into the
// kernels' SoA layout in memory it takes from a device memory pool.  Some
// callers cannot let a library allocate device memory at all: hosts whose
// memory manager owns the whole device (a framework's caching allocator, a
// fixed arena sized to the card), and latency-critical loops that must never
// block in the allocator or grow a pool behind the caller's back.  This entry
// point runs the same kernels with the packed fields placed in one file-scope
// device array of fixed size instead.
//
// The scratch array.  WILSON_NOALLOC_SCRATCH_BYTES (32 MiB) of device memory
// declared below; every GPU that loads the library holds it until the
// process exits.  It holds the packed FP64 links (1152 B per half-lattice
// site) and up to three packed FP64 half fields (192 B per site each), so
// lattices with V/2 up to about 19,000 sites fit (8^4, 12^4, 12^3 x 22, ...).
// Larger lattices are rejected with WILSON_ERR_ARG before anything runs.
//
// Host code cannot use the array's name as a device address: in host code
// the name denotes a host-side stand-in.  The first call in each CUDA
// context (with that context's device current) resolves the real address
// with cudaGetSymbolAddress and caches it under the context's unique ID, so
// a context torn down and created again (cudaDeviceReset) resolves it anew.
//
// No tuning, no synchronisation.  The call never times launch
// configurations: it takes the one an earlier wilson_dslash_eo call on the
// same lattice chose (or the WILSON_TUNE_CACHE file holds), else a fixed
// default.  It neither allocates nor synchronises.
//
// Sharing.  All calls on a device use the same array, and it keeps whatever
// the previous call left there.  Nothing here needs it cleared: every byte a
// kernel reads is written earlier in the same call.  Calls are asynchronous
// on the given stream; two calls whose work overlaps on the GPU (different
// streams, or host threads) race on the array and must be serialised by the
// caller.
#include <cuda.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>

#include "../../include/wilson.h"
#include "internal.h"

using namespace wl;

static __device__ __align__(256) unsigned char g_noalloc_scratch[WILSON_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mutex;

// Unique ID of the current CUDA context (never reused within a process), or
// 0 where the driver does not provide one.  Driver entry points are taken
// through the runtime, so the library does not link the driver library.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f1);
            get_id = reinterpret_cast<GetId>(f2);
        }
        cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current context (resolved once
// per context; resolved on every call where the driver gives no context ID).
void* scratch_address() {
    // The runtime calls before this one (pointer attributes) made the device's
    // primary context current; without a current context the ID is 0 and the
    // address is resolved afresh.
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    static std::map<unsigned long long, void*> addr;
    const unsigned long long ctx = current_context_id();
    if (ctx != 0) {
        auto it = addr.find(ctx);
        if (it != addr.end()) return it->second;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        throw Error(WILSON_ERR_CUDA,
                    std::string("cudaGetSymbolAddress(no-allocation scratch): ") + cudaGetErrorString(e));
    if (ctx != 0) addr[ctx] = p;
    return p;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace

extern "C" int wilson_dslash_eo_noalloc(double* out, const double* gauge, const double* in,
                                        const wilson_lattice* L, int out_parity, double kappa, int op,
                                        void* stream) {
    try {
        const Geom g = checked_geom(L);
        check_ptr(out, "out");
        check_ptr(gauge, "gauge");
        check_ptr(in, "in");
        WL_REQUIRE(out_parity == 0 || out_parity == 1, "out_parity must be 0 or 1");
        WL_REQUIRE(op == WILSON_OP_HOP || op == WILSON_OP_SCHUR || op == WILSON_OP_SCHUR_DAG,
                   "op must be HOP, SCHUR or SCHUR_DAG");
        WL_REQUIRE(std::isfinite(kappa), "kappa must be finite");
        WL_REQUIRE(out != in, "out must not alias in");

        // scratch layout: links | in | out | tmp
        const size_t gbytes = align256((size_t)gauge_bytes(P_F64, 18, g.stride));
        const size_t pbytes = align256((size_t)spinor_field_bytes(P_F64, g.stride));
        const size_t need = gbytes + 3 * pbytes;
        if (need > (size_t)WILSON_NOALLOC_SCRATCH_BYTES)
            throw Error(WILSON_ERR_ARG, "lattice too large for the no-allocation scratch: needs " +
                                            std::to_string(need) + " bytes, the array holds " +
                                            std::to_string((size_t)WILSON_NOALLOC_SCRATCH_BYTES));
        check_device();
        WL_REQUIRE(is_device_ptr(out) && is_device_ptr(in) && is_device_ptr(gauge),
                   "wilson_dslash_eo_noalloc takes device pointers");
        char* base = static_cast<char*>(scratch_address());
        cudaStream_t st = static_cast<cudaStream_t>(stream);

        const int pin = op == WILSON_OP_HOP ? 1 - out_parity : out_parity;
        GaugeField gf;
        SpinorField a, b, t;
        BorrowGuard guard;  // the views never free the array
        gf.prec = P_F64;
        gf.recon = 18;
        gf.g = g;
        guard.borrow(gf.buf, base, gbytes);
        auto view = [&](SpinorField& f, int subset, size_t off) {
            f.prec = P_F64;
            f.subset = subset;
            f.nrhs = 1;
            f.g = g;
            f.pbytes = (long long)pbytes;
            guard.borrow(f.buf, base + off, pbytes);
        };
        view(a, pin, gbytes);
        view(b, out_parity, gbytes + pbytes);
        view(t, 1 - out_parity, gbytes + 2 * pbytes);

        pack_gauge(gf, gauge, st);
        pack_spinor(a, 0, in, st);
        if (op == WILSON_OP_HOP) {
            HopLaunch h{};
            h.out = b.block(out_parity);
            h.in = a.block(pin);
            h.gauge = &gf;
            h.sprec = P_F64;
            h.no_tune = 1;
            h.out_parity = out_parity;
            h.a = 1.0;
            launch_hop(h, st);
        } else {
            const int dag = op == WILSON_OP_SCHUR_DAG;
            HopLaunch h1{};
            h1.out = t.block(1 - out_parity);
            h1.in = a.block(pin);
            h1.gauge = &gf;
            h1.sprec = P_F64;
            h1.no_tune = 1;
            h1.out_parity = 1 - out_parity;
            h1.dagger = dag;
            h1.a = 1.0;
            launch_hop(h1, st);
            HopLaunch h2{};
            h2.out = b.block(out_parity);
            h2.in = t.block(1 - out_parity);
            h2.x = a.block(pin);
            h2.xpay = 1;
            h2.a = -kappa * kappa;
            h2.gauge = &gf;
            h2.sprec = P_F64;
            h2.no_tune = 1;
            h2.out_parity = out_parity;
            h2.dagger = dag;
            launch_hop(h2, st);
        }
        unpack_spinor(b, 0, out, st);
        record_error("");
        return WILSON_OK;
    } catch (const Error& e) {
        record_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        record_error(e.what());
        return WILSON_ERR_CUDA;
    } catch (...) {
        record_error("unknown exception");
        return WILSON_ERR_CUDA;
    }
}
