// api.cu -- the extern "C" entry points declared in include/wilson.h.
//
// Every entry point validates its arguments on the host, catches every C++
// exception, records a thread-local message and returns a wilson_status.
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wilson.h"
#include "solver.h"

using namespace wl;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

template <class F>
int guarded(F&& f) {
    try {
        f();
        g_last_error.clear();
        return WILSON_OK;
    } catch (const Error& e) {
        return fail(e.code, e.what());
    } catch (const std::bad_alloc&) {
        return fail(WILSON_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(WILSON_ERR_CUDA, e.what());
    } catch (...) {
        return fail(WILSON_ERR_CUDA, "unknown exception");
    }
}

Prec to_prec(int p) {
    WL_REQUIRE(p >= WILSON_F64 && p <= WILSON_BF16, "unknown precision");
    return static_cast<Prec>(p);
}

// Library-owned staging for host-side canonical fields.
struct Staging {
    std::mutex m;
    DevBuf buf;
};
Staging& staging() {
    static Staging s;
    return s;
}

// Staging for page-locked host memory, with its own copy streams, so that
// the copies of one call overlap the kernels of another: an import's
// host-to-device copy runs on copy_in while the caller's stream still
// computes, and only the pack kernel waits for it; an export unpacks into
// one of two buffers, copies out on copy_out, and orders the caller's stream
// after the copy.  Events guard the buffers' reuse; nothing waits on the host.
struct AsyncStaging {
    std::mutex m;
    int device = -1;
    DevBuf in, out[2];
    int next_out = 0;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    cudaEvent_t in_free = nullptr, in_ready = nullptr, out_ready = nullptr, out_free[2] = {nullptr, nullptr};
    // Set up on the current device the first time; false if another device
    // owns it (the caller then takes the synchronous path).
    bool bind() {
        int dev = 0;
        WL_CUDA(cudaGetDevice(&dev));
        if (device >= 0) return device == dev;
        WL_CUDA(cudaStreamCreateWithFlags(&copy_in, cudaStreamNonBlocking));
        WL_CUDA(cudaStreamCreateWithFlags(&copy_out, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&in_free, &in_ready, &out_ready, &out_free[0], &out_free[1]})
            WL_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        // the "free" events start out complete
        for (cudaEvent_t e : {in_free, out_free[0], out_free[1]}) WL_CUDA(cudaEventRecord(e, copy_in));
        device = dev;
        return true;
    }
};
AsyncStaging& async_staging() {
    static AsyncStaging s;
    return s;
}

bool is_pinned_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Copy a canonical field to the device if it lives in host memory; returns a
// device pointer valid until the next staging call on the stream.
const double* device_view(const double* p, size_t bytes, DevBuf& tmp, cudaStream_t st) {
    if (is_device_ptr(p)) return p;
    tmp.ensure(bytes);
    WL_CUDA(cudaMemcpyAsync(tmp.p, p, bytes, cudaMemcpyHostToDevice, st));
    return tmp.as<const double>();
}

// Internal stream used by the solver for graph capture (the caller's stream
// may be the legacy default stream, which cannot be captured).
struct SolveStream {
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};
SolveStream& solve_stream() {
    static thread_local SolveStream ss;
    if (!ss.s) {
        WL_CUDA(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
        WL_CUDA(cudaEventCreateWithFlags(&ss.e0, cudaEventDisableTiming));
        WL_CUDA(cudaEventCreateWithFlags(&ss.e1, cudaEventDisableTiming));
    }
    return ss;
}


// Workspace of the stateless operator calls: one memory pool per device that
// keeps its memory after release (release threshold: unlimited).  A call
// takes its packed fields from the pool with cudaMallocFromPoolAsync and
// returns them with cudaFreeAsync, both ordered on the caller's stream, so
// the call never synchronises: the pool reuses the memory once the stream
// has passed the release (a later call on another stream gets other memory
// or an ordering dependency the pool inserts).  Only the first call of a new
// size grows the pool.
cudaMemPool_t stateless_pool() {
    static std::mutex m;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(m);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        WL_CUDA(cudaMemPoolCreate(&pool, &props));
        unsigned long long keep = ~0ULL;
        WL_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        pools[dev] = pool;
    }
    return pools[dev];
}

// Stream-ordered allocations of one call, released on the stream when the
// call's scope ends (also when it throws).
struct StreamAllocs {
    cudaStream_t st;
    void* p[4] = {nullptr, nullptr, nullptr, nullptr};
    int n = 0;
    explicit StreamAllocs(cudaStream_t s) : st(s) {}
    void* get(size_t bytes) {
        void* q = nullptr;
        WL_CUDA(cudaMallocFromPoolAsync(&q, bytes, stateless_pool(), st));
        p[n++] = q;
        return q;
    }
    ~StreamAllocs() {
        for (int i = 0; i < n; i++) cudaFreeAsync(p[i], st);
    }
};

// A packed FP64 field of one parity subset (0, 1 or 2 = both) in pool memory.
void borrow_spinor(SpinorField& f, int subset, const Geom& g, StreamAllocs& a, BorrowGuard& guard) {
    f.prec = P_F64;
    f.subset = subset;
    f.nrhs = 1;
    f.g = g;
    f.pbytes = spinor_field_bytes(P_F64, g.stride);
    const size_t bytes = (size_t)f.pbytes * f.nparity();
    guard.borrow(f.buf, a.get(bytes), bytes);
}
void borrow_gauge(GaugeField& gf, const Geom& g, StreamAllocs& a, BorrowGuard& guard) {
    gf.prec = P_F64;
    gf.recon = 18;
    gf.g = g;
    const size_t bytes = (size_t)gauge_bytes(P_F64, 18, g.stride);
    guard.borrow(gf.buf, a.get(bytes), bytes);
}

}  // namespace

void wl::record_error(const std::string& msg) { g_last_error = msg; }

// Checks shared by all entry points (declared in internal.h).
Geom wl::checked_geom(const wilson_lattice* L) {
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
    return make_geom(L->dims, L->bc_phase);
}

void wl::check_ptr(const void* p, const char* what) {
    WL_REQUIRE(p != nullptr, std::string(what) + " is NULL");
    WL_REQUIRE((reinterpret_cast<uintptr_t>(p) & 15) == 0, std::string(what) + " is not 16-byte aligned");
}

void wl::check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        throw Error(WILSON_ERR_CUDA, "no CUDA device available");
    }
}

bool wl::is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
extern "C" {

const char* wilson_last_error(void) { return g_last_error.c_str(); }

int wilson_version(void) { return 100; }

wilson_solver_params wilson_solver_defaults(int inner) {
    wilson_solver_params p;
    p.inner = inner;
    p.recon = inner == WILSON_F64 ? 18 : 12;
    p.tol = 1e-10;
    p.maxiter = 100000;
    p.max_restarts = 1000;
    p.delta = 0.0;
    p.use_initial_guess = 0;
    p.reliable = 1;
    p.block_cg = 0;
    return p;
}

int wilson_dslash(double* out, const double* gauge, const double* in, const wilson_lattice* L, double kappa,
                  int op, void* stream) {
    return guarded([&] {
        const Geom g = checked_geom(L);
        check_ptr(out, "out");
        check_ptr(gauge, "gauge");
        check_ptr(in, "in");
        WL_REQUIRE(op == WILSON_OP_HOP || op == WILSON_OP_M, "wilson_dslash: op must be HOP or M");
        WL_REQUIRE(std::isfinite(kappa), "kappa must be finite");
        WL_REQUIRE(out != in, "out must not alias in");
        check_device();
        WL_REQUIRE(is_device_ptr(out) && is_device_ptr(in) && is_device_ptr(gauge),
                   "wilson_dslash takes device pointers");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        StreamAllocs mem(st);
        GaugeField gf;
        SpinorField a, b;
        BorrowGuard guard;  // declared last: detaches the views first, and mem releases the memory last
        borrow_gauge(gf, g, mem, guard);
        borrow_spinor(a, 2, g, mem, guard);
        borrow_spinor(b, 2, g, mem, guard);
        pack_gauge(gf, gauge, st);
        pack_spinor(a, 0, in, st);
        HopLaunch h{};
        h.out = b.block(0);
        h.in = a.block(0);
        h.x = a.block(0);
        h.out_pstep = b.pbytes;
        h.in_pstep = a.pbytes;
        h.x_pstep = a.pbytes;
        h.full = 1;
        h.gauge = &gf;
        h.sprec = P_F64;
        h.xpay = op == WILSON_OP_M;
        h.a = op == WILSON_OP_M ? -kappa : 1.0;
        launch_hop(h, st);
        unpack_spinor(b, 0, out, st);
    });
}

int wilson_dslash_eo(double* out, const double* gauge, const double* in, const wilson_lattice* L,
                     int out_parity, double kappa, int op, void* stream) {
    return guarded([&] {
        const Geom g = checked_geom(L);
        check_ptr(out, "out");
        check_ptr(gauge, "gauge");
        check_ptr(in, "in");
        WL_REQUIRE(out_parity == 0 || out_parity == 1, "out_parity must be 0 or 1");
        WL_REQUIRE(op == WILSON_OP_HOP || op == WILSON_OP_SCHUR || op == WILSON_OP_SCHUR_DAG,
                   "wilson_dslash_eo: op must be HOP, SCHUR or SCHUR_DAG");
        WL_REQUIRE(std::isfinite(kappa), "kappa must be finite");
        WL_REQUIRE(out != in, "out must not alias in");
        check_device();
        WL_REQUIRE(is_device_ptr(out) && is_device_ptr(in) && is_device_ptr(gauge),
                   "wilson_dslash_eo takes device pointers");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        StreamAllocs mem(st);
        const int pin = op == WILSON_OP_HOP ? 1 - out_parity : out_parity;
        GaugeField gf;
        SpinorField a, b, t;
        BorrowGuard guard;  // declared last: detaches the views first, and mem releases the memory last
        borrow_gauge(gf, g, mem, guard);
        borrow_spinor(a, pin, g, mem, guard);
        borrow_spinor(b, out_parity, g, mem, guard);
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
            // Mhat_p = 1 - kappa^2 D_{p,1-p} D_{1-p,p}
            borrow_spinor(t, 1 - out_parity, g, mem, guard);
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
    });
}

static SolveParams checked_params(const wilson_solver_params* p, double kappa) {
    WL_REQUIRE(p != nullptr, "solver parameters are NULL");
    WL_REQUIRE(std::isfinite(kappa), "kappa must be finite");
    WL_REQUIRE(p->tol > 0 && std::isfinite(p->tol), "tol must be positive");
    WL_REQUIRE(p->maxiter > 0, "maxiter must be positive");
    WL_REQUIRE(p->recon == 12 || p->recon == 18, "recon must be 12 or 18");
    SolveParams prm;
    prm.inner = to_prec(p->inner);
    prm.recon = p->recon;
    prm.tol = p->tol;
    prm.maxiter = p->maxiter;
    prm.max_restarts = p->max_restarts > 0 ? p->max_restarts : 1000;
    prm.delta = p->delta;
    prm.use_initial_guess = p->use_initial_guess;
    prm.reliable = p->reliable;
    prm.block_cg = p->block_cg;
    return prm;
}

static void copy_stats(wilson_solve_stats* o, const SolveStats& s, int rc) {
    o->status = rc;
    o->outer_iters = s.outer_iters;
    o->inner_iters = s.inner_iters;
    o->hop_applications = s.hop_applications;
    o->true_rel_resid = s.true_rel_resid;
    o->seconds = s.seconds;
    o->inner_seconds = s.inner_seconds;
    o->outer_f32 = s.outer_f32;
}

int wilson_cg_solve(double* x, const double* gauge, const double* b, const wilson_lattice* L, double kappa,
                    const wilson_solver_params* p, wilson_solve_stats* st_out, void* stream) {
    SolveStats stats;
    int rc = guarded([&] {
        const Geom g = checked_geom(L);
        check_ptr(x, "x");
        check_ptr(gauge, "gauge");
        check_ptr(b, "b");
        WL_REQUIRE(x != b, "x must not alias b");
        const SolveParams prm = checked_params(p, kappa);
        check_device();
        WL_REQUIRE(is_device_ptr(x) && is_device_ptr(b) && is_device_ptr(gauge),
                   "wilson_cg_solve takes device pointers");
        cudaStream_t caller = static_cast<cudaStream_t>(stream);
        SolveStream& ss = solve_stream();
        WL_CUDA(cudaEventRecord(ss.e0, caller));
        WL_CUDA(cudaStreamWaitEvent(ss.s, ss.e0, 0));
        stats = cg_solve(x, gauge, b, 1, g, kappa, prm, ss.s)[0];
        WL_CUDA(cudaEventRecord(ss.e1, ss.s));
        WL_CUDA(cudaStreamWaitEvent(caller, ss.e1, 0));
        WL_CUDA(cudaStreamSynchronize(caller));
        if (stats.status != 0)
            throw Error(stats.status, stats.status == WILSON_ERR_NOCONV ? "solve did not converge"
                                                                        : "NaN or Inf in the solve");
    });
    if (st_out) copy_stats(st_out, stats, rc);
    return rc;
}

int wilson_cg_solve_multi(double* x, const double* gauge, const double* b, int nrhs, const wilson_lattice* L,
                          double kappa, const wilson_solver_params* p, wilson_solve_stats* st_out, void* stream) {
    std::vector<SolveStats> stats;
    int rc = guarded([&] {
        const Geom g = checked_geom(L);
        check_ptr(x, "x");
        check_ptr(gauge, "gauge");
        check_ptr(b, "b");
        WL_REQUIRE(nrhs >= 1 && nrhs <= 64, "nrhs must be in 1..64");
        WL_REQUIRE(x != b, "x must not alias b");
        const SolveParams prm = checked_params(p, kappa);
        WL_REQUIRE(!prm.block_cg || nrhs <= 16, "block CG takes at most 16 right-hand sides");
        check_device();
        WL_REQUIRE(is_device_ptr(x) && is_device_ptr(b) && is_device_ptr(gauge),
                   "wilson_cg_solve_multi takes device pointers");
        cudaStream_t caller = static_cast<cudaStream_t>(stream);
        SolveStream& ss = solve_stream();
        WL_CUDA(cudaEventRecord(ss.e0, caller));
        WL_CUDA(cudaStreamWaitEvent(ss.s, ss.e0, 0));
        stats = cg_solve(x, gauge, b, nrhs, g, kappa, prm, ss.s);
        WL_CUDA(cudaEventRecord(ss.e1, ss.s));
        WL_CUDA(cudaStreamWaitEvent(caller, ss.e1, 0));
        WL_CUDA(cudaStreamSynchronize(caller));
        int worst = 0;
        for (const SolveStats& s : stats)
            if (s.status != 0 && (worst == 0 || s.status == WILSON_ERR_NUMERIC)) worst = s.status;
        if (worst != 0)
            throw Error(worst, worst == WILSON_ERR_NOCONV ? "a right-hand side did not converge"
                                                          : "NaN or Inf in a right-hand side's solve");
    });
    if (st_out)
        for (int k = 0; k < (int)stats.size(); k++) copy_stats(st_out + k, stats[k], stats[k].status);
    return rc;
}

int wilson_batch_solve(int n, const wilson_problem* probs, const wilson_solver_params* p, wilson_solve_stats* st_out,
                       wilson_batch_info* info, void* stream) {
    return guarded([&] {
        WL_REQUIRE(n >= 1 && n <= 4096, "n must be in 1..4096");
        WL_REQUIRE(probs != nullptr && st_out != nullptr, "problems or stats array is NULL");
        SolveParams prm = checked_params(p, 0.0);
        WL_REQUIRE(prm.inner == P_F32 || prm.inner == P_F16 || prm.inner == P_BF16,
                   "batched solves run an F32, F16 or BF16 inner CG");
        WL_REQUIRE(p->recon == 12, "batched solves store the inner links with 12 reals");
        long long sites = 0;
        for (int i = 0; i < n; i++) {
            const wilson_problem& q = probs[i];
            const Geom g = checked_geom(&q.L);
            sites += 2LL * g.Vh;
            check_ptr(q.gauge, "problem gauge");
            check_ptr(q.b, "problem b");
            check_ptr(q.x, "problem x");
            WL_REQUIRE(std::isfinite(q.kappa), "kappa must be finite");
            WL_REQUIRE((const void*)q.x != (const void*)q.b, "x must not alias b");
        }
        WL_REQUIRE(sites < (1LL << 31), "total sites must be below 2^31");
        check_device();
        for (int i = 0; i < n; i++)
            WL_REQUIRE(is_device_ptr(probs[i].x) && is_device_ptr(probs[i].b) && is_device_ptr(probs[i].gauge),
                       "wilson_batch_solve takes device pointers");
        cudaStream_t caller = static_cast<cudaStream_t>(stream);
        SolveStream& ss = solve_stream();
        WL_CUDA(cudaEventRecord(ss.e0, caller));
        WL_CUDA(cudaStreamWaitEvent(ss.s, ss.e0, 0));
        batch_solve(n, probs, prm, st_out, info, ss.s);
        WL_CUDA(cudaEventRecord(ss.e1, ss.s));
        WL_CUDA(cudaStreamWaitEvent(caller, ss.e1, 0));
        WL_CUDA(cudaStreamSynchronize(caller));
        int worst = 0;
        for (int i = 0; i < n; i++)
            if (st_out[i].status != 0 && (worst == 0 || st_out[i].status == WILSON_ERR_NUMERIC)) worst = st_out[i].status;
        if (worst) throw Error(worst, "a problem of the batch did not converge");
    });
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
int wilson_gauge_create(wilson_gauge** out, const double* canon, const wilson_lattice* L, int prec, int recon,
                        void* stream) {
    return guarded([&] {
        WL_REQUIRE(out != nullptr, "handle pointer is NULL");
        *out = nullptr;
        const Geom g = checked_geom(L);
        check_ptr(canon, "gauge");
        const Prec p = to_prec(prec);
        WL_REQUIRE(recon == 12 || recon == 18, "recon must be 12 or 18");
        check_device();
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        std::unique_ptr<wilson_gauge_s> h(new wilson_gauge_s);
        h->f.prec = p;
        h->f.recon = recon;
        h->f.g = g;
        h->f.buf.alloc(gauge_bytes(p, recon, g.stride));
        DevBuf tmp;
        const double* d = device_view(canon, sizeof(double) * 72 * 2 * (size_t)g.Vh, tmp, st);
        pack_gauge(h->f, d, st);
        WL_CUDA(cudaStreamSynchronize(st));
        *out = h.release();
    });
}

int wilson_gauge_destroy(wilson_gauge* g) {
    return guarded([&] { delete g; });
}

int wilson_spinor_create(wilson_spinor** out, const wilson_lattice* L, int subset, int nrhs, int prec) {
    return guarded([&] {
        WL_REQUIRE(out != nullptr, "handle pointer is NULL");
        *out = nullptr;
        const Geom g = checked_geom(L);
        WL_REQUIRE(subset >= 0 && subset <= 2, "subset must be EVEN, ODD or FULL");
        WL_REQUIRE(nrhs >= 1 && nrhs <= 64, "nrhs must be in 1..64");
        const Prec p = to_prec(prec);
        check_device();
        std::unique_ptr<wilson_spinor_s> h(new wilson_spinor_s);
        h->g = g;
        h->f.alloc(p, subset, nrhs, g);
        WL_CUDA(cudaMemset(h->f.buf.p, 0, h->f.buf.bytes));
        *out = h.release();
    });
}

int wilson_spinor_destroy(wilson_spinor* s) {
    return guarded([&] { delete s; });
}

long long wilson_spinor_bytes(const wilson_spinor* s) { return s ? (long long)s->f.buf.bytes : 0; }

int wilson_spinor_import(wilson_spinor* s, const double* canon, void* stream) {
    return guarded([&] {
        WL_REQUIRE(s != nullptr, "spinor handle is NULL");
        check_ptr(canon, "canonical field");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const size_t per = sizeof(double) * 24 * (size_t)s->g.Vh * (s->f.subset == 2 ? 2 : 1);
        if (is_device_ptr(canon)) {
            for (int k = 0; k < s->f.nrhs; k++) pack_spinor(s->f, k, canon + (per / sizeof(double)) * k, st);
            return;
        }
        AsyncStaging& as = async_staging();
        std::unique_lock<std::mutex> lk(as.m);
        if (is_pinned_host(canon) && as.bind()) {
            const size_t bytes = per * s->f.nrhs;
            as.in.ensure(bytes);
            WL_CUDA(cudaStreamWaitEvent(as.copy_in, as.in_free, 0));  // the last pack is done with the buffer
            WL_CUDA(cudaMemcpyAsync(as.in.p, canon, bytes, cudaMemcpyHostToDevice, as.copy_in));
            WL_CUDA(cudaEventRecord(as.in_ready, as.copy_in));
            WL_CUDA(cudaStreamWaitEvent(st, as.in_ready, 0));
            for (int k = 0; k < s->f.nrhs; k++)
                pack_spinor(s->f, k, as.in.as<const double>() + (per / sizeof(double)) * k, st);
            WL_CUDA(cudaEventRecord(as.in_free, st));
            return;
        }
        lk.unlock();
        {
            Staging& sg = staging();
            std::lock_guard<std::mutex> lk(sg.m);
            sg.buf.ensure(per * s->f.nrhs);
            WL_CUDA(cudaMemcpyAsync(sg.buf.p, canon, per * s->f.nrhs, cudaMemcpyHostToDevice, st));
            for (int k = 0; k < s->f.nrhs; k++)
                pack_spinor(s->f, k, sg.buf.as<const double>() + (per / sizeof(double)) * k, st);
            // the staging buffer is reused by the next call: finish with it first
            WL_CUDA(cudaStreamSynchronize(st));
        }
    });
}

int wilson_spinor_export(const wilson_spinor* s, double* canon, void* stream) {
    return guarded([&] {
        WL_REQUIRE(s != nullptr, "spinor handle is NULL");
        check_ptr(canon, "canonical field");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const size_t per = sizeof(double) * 24 * (size_t)s->g.Vh * (s->f.subset == 2 ? 2 : 1);
        if (is_device_ptr(canon)) {
            for (int k = 0; k < s->f.nrhs; k++) unpack_spinor(s->f, k, canon + (per / sizeof(double)) * k, st);
            return;
        }
        AsyncStaging& as = async_staging();
        std::unique_lock<std::mutex> lk(as.m);
        if (is_pinned_host(canon) && as.bind()) {
            const size_t bytes = per * s->f.nrhs;
            const int i = as.next_out;
            as.next_out ^= 1;
            DevBuf& ob = as.out[i];
            if (ob.bytes < bytes) {
                WL_CUDA(cudaEventSynchronize(as.out_free[i]));  // the buffer is about to be replaced
                ob.ensure(bytes);
            }
            WL_CUDA(cudaStreamWaitEvent(st, as.out_free[i], 0));  // its last copy-out is done
            for (int k = 0; k < s->f.nrhs; k++)
                unpack_spinor(s->f, k, ob.as<double>() + (per / sizeof(double)) * k, st);
            WL_CUDA(cudaEventRecord(as.out_ready, st));
            WL_CUDA(cudaStreamWaitEvent(as.copy_out, as.out_ready, 0));
            WL_CUDA(cudaMemcpyAsync(canon, ob.p, bytes, cudaMemcpyDeviceToHost, as.copy_out));
            WL_CUDA(cudaEventRecord(as.out_free[i], as.copy_out));
            WL_CUDA(cudaStreamWaitEvent(st, as.out_free[i], 0));  // the caller's stream is ordered after the copy
            return;
        }
        lk.unlock();
        {
            Staging& sg = staging();
            std::lock_guard<std::mutex> lk(sg.m);
            sg.buf.ensure(per * s->f.nrhs);
            for (int k = 0; k < s->f.nrhs; k++)
                unpack_spinor(s->f, k, sg.buf.as<double>() + (per / sizeof(double)) * k, st);
            WL_CUDA(cudaMemcpyAsync(canon, sg.buf.p, per * s->f.nrhs, cudaMemcpyDeviceToHost, st));
            WL_CUDA(cudaStreamSynchronize(st));
        }
    });
}

int wilson_dslash_h(wilson_spinor* out, const wilson_gauge* gh, const wilson_spinor* in, double kappa, int op,
                    void* stream) {
    return guarded([&] {
        WL_REQUIRE(out && gh && in, "NULL handle");
        WL_REQUIRE(out != in, "out must not be in");
        WL_REQUIRE(std::isfinite(kappa), "kappa must be finite");
        const GaugeField& gf = gh->f;
        const SpinorField& a = in->f;
        SpinorField& b = out->f;
        for (int mu = 0; mu < 4; mu++)
            WL_REQUIRE(a.g.L[mu] == gf.g.L[mu] && b.g.L[mu] == gf.g.L[mu], "lattice mismatch");
        WL_REQUIRE(a.prec == b.prec, "in and out precision differ");
        WL_REQUIRE(a.nrhs == b.nrhs, "in and out nrhs differ");
        WL_REQUIRE(gf.prec == a.prec, "gauge and spinor precision differ");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        HopLaunch h{};
        h.gauge = &gf;
        h.sprec = a.prec;
        h.nrhs = a.nrhs;
        h.out_rstep = b.rstep();
        h.in_rstep = a.rstep();
        h.x_rstep = a.rstep();
        h.a = 1.0;
        if (op == WILSON_OP_HOP || op == WILSON_OP_M) {
            if (a.subset == 2) {
                WL_REQUIRE(b.subset == 2, "full input needs a full output");
                h.out = b.block(0);
                h.in = a.block(0);
                h.x = a.block(0);
                h.out_pstep = b.pbytes;
                h.in_pstep = a.pbytes;
                h.x_pstep = a.pbytes;
                h.full = 1;
                h.xpay = op == WILSON_OP_M;
                h.a = op == WILSON_OP_M ? -kappa : 1.0;
            } else {
                WL_REQUIRE(op == WILSON_OP_HOP, "M needs full fields");
                WL_REQUIRE(b.subset == 1 - a.subset, "HOP maps parity 1-p to parity p");
                h.out = b.block(b.subset);
                h.in = a.block(a.subset);
                h.out_parity = b.subset;
            }
            launch_hop(h, st);
        } else if (op == WILSON_OP_SCHUR || op == WILSON_OP_SCHUR_DAG) {
            WL_REQUIRE(a.subset != 2 && b.subset == a.subset, "SCHUR maps parity p to parity p");
            // the intermediate field of the other parity lives with the gauge handle
            std::lock_guard<std::mutex> lk(gh->m);
            SpinorField& t = gh->tmp;
            if (!t.buf.p || t.prec != a.prec || t.nrhs < a.nrhs || t.subset != 1 - a.subset)
                t.alloc(a.prec, 1 - a.subset, a.nrhs, a.g);
            const int dag = op == WILSON_OP_SCHUR_DAG;
            HopLaunch h1 = h;
            h1.out = t.block(1 - a.subset);
            h1.in = a.block(a.subset);
            h1.out_rstep = t.rstep();
            h1.out_parity = 1 - a.subset;
            h1.dagger = dag;
            launch_hop(h1, st);
            HopLaunch h2 = h;
            h2.out = b.block(b.subset);
            h2.in = t.block(1 - a.subset);
            h2.in_rstep = t.rstep();
            h2.x = a.block(a.subset);
            h2.xpay = 1;
            h2.a = -kappa * kappa;
            h2.out_parity = b.subset;
            h2.dagger = dag;
            launch_hop(h2, st);
        } else {
            throw Error(WILSON_ERR_ARG, "unknown op");
        }
    });
}

}  // extern "C"
