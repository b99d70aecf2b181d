// noalloc.cu -- wilson_dslash_eo_noalloc: the even-odd hopping term and the
// Schur operator on canonical FP64 device fields, with no device allocation.
//
// Why it exists.  wilson_dslash_eo packs its canonical inputs into the
// kernels' SoA layout in memory it allocates per call.  Some callers cannot
// let a library call cudaMalloc: code issuing work while a stream is being
// captured into a CUDA graph (allocation is not permitted there), hosts whose
// memory manager owns the whole device (a framework caching allocator or a
// fixed arena), and latency-critical loops that must never block on the
// allocator or trigger an implicit device synchronisation in cudaFree.  This
// entry point runs the same kernels with the packed fields placed in one
// file-scope device array of fixed size instead.
//
// The scratch array.  WILSON_NOALLOC_SCRATCH_BYTES (32 MiB) of device memory
// declared below; every GPU that loads the library holds it until the
// process exits.  It holds the packed FP64 links (1152 B per half-lattice
// site) and up to three packed FP64 half fields (192 B per site each), so
// lattices with V/2 up to about 19,000 sites fit (8^4, 12^4, 8^3 x 32, ...).
// Larger lattices are rejected with WILSON_ERR_ARG before anything runs.
//
// Host code cannot use the array's name as a device address: in host code
// the name denotes a host-side stand-in.  The first call on each device (with
// that device current) resolves the real address with cudaGetSymbolAddress
// and caches it; make that first call before any stream capture begins.
//
// Sharing.  All calls on a device use the same array, and it keeps whatever
// the previous call left there.  Nothing here needs it cleared: every byte a
// kernel reads is written earlier in the same call.  Calls are asynchronous
// on the given stream; two calls whose work overlaps on the GPU (different
// streams, or host threads) race on the array and must be serialised by the
// caller.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/wilson.h"
#include "internal.h"

using namespace wl;

static __device__ __align__(256) unsigned char g_noalloc_scratch[WILSON_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (resolved once
// per device).
void* scratch_address() {
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            throw Error(WILSON_ERR_CUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                                             cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// Non-owning views into the scratch array; the guard detaches them before
// the views' destructors run, so nothing is ever freed.
struct ViewGuard {
    DevBuf* bufs[4];
    int n = 0;
    ~ViewGuard() {
        for (int i = 0; i < n; i++) {
            bufs[i]->p = nullptr;
            bufs[i]->bytes = 0;
        }
    }
};

}  // namespace

extern "C" int wilson_dslash_eo_noalloc(double* out, const double* gauge, const double* in,
                                        const wilson_lattice* L, int out_parity, double kappa, int op,
                                        void* stream) {
    try {
        WL_REQUIRE(L != nullptr, "lattice descriptor is NULL");
        long long V = 1;
        for (int mu = 0; mu < 4; mu++) {
            const int d = L->dims[mu];
            WL_REQUIRE(d >= 2 && (d % 2) == 0, "every lattice extent must be even and >= 2");
            V *= d;
            const double re = L->bc_phase[mu][0], im = L->bc_phase[mu][1];
            WL_REQUIRE(std::isfinite(re) && std::isfinite(im) && std::fabs(re * re + im * im - 1.0) <= 1e-12,
                       "boundary phases must have unit modulus");
        }
        WL_REQUIRE(V < (1LL << 31), "lattice volume must be below 2^31 sites");
        for (const void* p : {(const void*)out, (const void*)gauge, (const void*)in}) {
            WL_REQUIRE(p != nullptr, "a field pointer is NULL");
            WL_REQUIRE((reinterpret_cast<uintptr_t>(p) & 15) == 0, "field pointers must be 16-byte aligned");
        }
        WL_REQUIRE(out_parity == 0 || out_parity == 1, "out_parity must be 0 or 1");
        WL_REQUIRE(op == WILSON_OP_HOP || op == WILSON_OP_SCHUR || op == WILSON_OP_SCHUR_DAG,
                   "op must be HOP, SCHUR or SCHUR_DAG");
        WL_REQUIRE(std::isfinite(kappa), "kappa must be finite");
        WL_REQUIRE(out != in, "out must not alias in");
        const Geom g = make_geom(L->dims, L->bc_phase);

        // scratch layout: links | in | out | tmp
        const size_t gbytes = align256((size_t)gauge_bytes(P_F64, 18, g.stride));
        const size_t pbytes = align256((size_t)spinor_field_bytes(P_F64, g.stride));
        const size_t need = gbytes + 3 * pbytes;
        if (need > (size_t)WILSON_NOALLOC_SCRATCH_BYTES)
            throw Error(WILSON_ERR_ARG, "lattice too large for the no-allocation scratch: needs " +
                                            std::to_string(need) + " bytes, the array holds " +
                                            std::to_string((size_t)WILSON_NOALLOC_SCRATCH_BYTES));
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            throw Error(WILSON_ERR_CUDA, "no CUDA device available");
        }
        WL_REQUIRE(on_device(out) && on_device(in) && on_device(gauge),
                   "wilson_dslash_eo_noalloc takes device pointers");
        char* base = static_cast<char*>(scratch_address());
        cudaStream_t st = static_cast<cudaStream_t>(stream);

        const int pin = op == WILSON_OP_HOP ? 1 - out_parity : out_parity;
        GaugeField gf;
        SpinorField a, b, t;
        ViewGuard guard;
        guard.bufs[guard.n++] = &gf.buf;
        guard.bufs[guard.n++] = &a.buf;
        guard.bufs[guard.n++] = &b.buf;
        guard.bufs[guard.n++] = &t.buf;
        gf.prec = P_F64;
        gf.recon = 18;
        gf.g = g;
        gf.buf.p = base;
        gf.buf.bytes = gbytes;
        auto view = [&](SpinorField& f, int subset, size_t off) {
            f.prec = P_F64;
            f.subset = subset;
            f.nrhs = 1;
            f.g = g;
            f.pbytes = (long long)pbytes;
            f.buf.p = base + off;
            f.buf.bytes = pbytes;
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
