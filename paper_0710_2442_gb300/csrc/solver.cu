// solver.cu -- CG on the normal equations of the even-odd Schur complement,
// with an FP64 defect correction around a reduced-precision inner CG.
//
// The paper (Sec. 5) only notes that an iterative solver repeats Eq. 3; the
// algorithm here is textbook CG in its residual-tracking form for the normal
// equations (CGNR; Hestenes & Stiefel 1952, Sec. 10):
//
//   bhat_e = b_e + kappa D_eo b_o
//   solve Mhat x_e = bhat_e via Mhat^dag Mhat x_e = Mhat^dag bhat_e
//   x_o = b_o + kappa D_oe x_e
//
// Outer loop (FP64, on the GPU): r = bhat - Mhat x_e with FP64 links and
// FP64 reductions; stop when |r| <= tol |b| (equal to the full-system
// residual |b - M x|, whose odd part vanishes by construction).  Inner loop
// (storage precision F32/F16/BF16, FP32 arithmetic; or FP64 for the plain
// FP64 solve) solves Mhat e = r until |s| <= delta |r| where s is the
// recursively updated inner residual; then x_e += e in FP64.
//
// Reliable updates (default): the inner CG keeps its search direction p
// across outer corrections and only replaces its residual by the recomputed
// FP64 one (the scheme of Sleijpen & van der Vorst 1996 as used for lattice
// QCD mixed-precision solvers); with reliable = 0 every correction restarts CG.
//
// One inner iteration is six launches, all reading their scalars from device
// memory and exiting at once when the solve's done flag is set:
//   t = D_oe p;  q = p - k^2 D_eo t, |q|^2 -> alpha
//   x += alpha p, s -= alpha q, |s|^2 -> convergence test
//   t = D'_oe s;  r = s - k^2 D'_eo t, |r|^2 -> beta      (D' = g5 D g5)
//   p = r + beta p
// A chunk of iterations is captured once into a CUDA graph and replayed; the
// host reads the scalars once per chunk.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <vector>

#include "solver.h"

namespace wl {

void schur_apply(const GaugeField& gf, Prec sp, void* out, const void* in, void* tmp, double kappa, int dag,
                 const RedArgs* red, const int* skip, int grid_cap, cudaStream_t st) {
    HopLaunch a{};
    a.out = tmp;
    a.in = in;
    a.gauge = &gf;
    a.sprec = sp;
    a.out_parity = 1;
    a.dagger = dag;
    a.a = 1.0;
    a.skip = skip;
    launch_hop(a, st);
    HopLaunch b{};
    b.out = out;
    b.in = tmp;
    b.x = in;
    b.xpay = 1;
    b.a = -kappa * kappa;
    b.gauge = &gf;
    b.sprec = sp;
    b.out_parity = 0;
    b.dagger = dag;
    b.red = red;
    b.skip = skip;
    b.grid_cap = red ? grid_cap : 0;
    launch_hop(b, st);
}

namespace {

struct Pinned {
    void* p = nullptr;
    explicit Pinned(size_t n) { WL_CUDA(cudaMallocHost(&p, n)); }
    ~Pinned() { if (p) cudaFreeHost(p); }
};

struct Inner {
    Prec ip, xp;
    Geom g;
    SpinorField xin, s, slow, p, q, r, t;
    bool has_slow;
    void alloc(Prec inner, const Geom& geom) {
        ip = inner;
        xp = inner == P_F64 ? P_F64 : P_F32;
        g = geom;
        has_slow = (ip != xp);
        xin.alloc(xp, 0, 1, g);
        s.alloc(xp, 0, 1, g);
        if (has_slow) slow.alloc(ip, 0, 1, g);
        p.alloc(ip, 0, 1, g);
        q.alloc(ip, 0, 1, g);
        r.alloc(ip, 0, 1, g);
        t.alloc(ip, 1, 1, g);
    }
    void* s_in() { return has_slow ? slow.block(0) : s.block(0); }
};

}  // namespace

SolveStats cg_solve_prepared(SpinorField& x, const SpinorField& b, const GaugeField& g64, const GaugeField& glo,
                             double kappa, const SolveParams& prm, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    SolveStats stats;
    const Geom g = g64.g;
    const int sms = device_sm_count();
    const int grid_cap = 8 * sms;          // blocks of reducing launches (<= Reduction capacity / 2)
    Reduction red;
    red.init(2 * grid_cap, 8, st);
    DevBuf scbuf(sizeof(CGScalars));
    CGScalars* sc = scbuf.as<CGScalars>();
    Pinned hbuf(sizeof(CGScalars) + 8 * sizeof(double));
    CGScalars* h_sc = static_cast<CGScalars*>(hbuf.p);
    double* h_res = reinterpret_cast<double*>(h_sc + 1);
    double* d_res = red.results.as<double>();

    // FP64 work fields
    SpinorField bhat, r64, q64, t64;
    bhat.alloc(P_F64, 0, 1, g);
    r64.alloc(P_F64, 0, 1, g);
    q64.alloc(P_F64, 0, 1, g);
    t64.alloc(P_F64, 1, 1, g);

    // |b|^2 over both parities
    {
        RedArgs ra = red.args(0, FIN_STORE, d_res + 0, nullptr);
        norm2(P_F64, b.block(0), g, ra, grid_cap, st);
        RedArgs rb = red.args(1, FIN_STORE, d_res + 1, nullptr);
        norm2(P_F64, b.block(1), g, rb, grid_cap, st);
    }
    // bhat_e = b_e + kappa D_eo b_o
    {
        HopLaunch h{};
        h.out = bhat.block(0);
        h.in = b.block(1);
        h.x = b.block(0);
        h.xpay = 1;
        h.a = kappa;
        h.gauge = &g64;
        h.sprec = P_F64;
        h.out_parity = 0;
        launch_hop(h, st);
        stats.hop_applications += 1;
    }
    if (!prm.use_initial_guess) WL_CUDA(cudaMemsetAsync(x.block(0), 0, x.pbytes, st));
    WL_CUDA(cudaMemcpyAsync(h_res, d_res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    WL_CUDA(cudaStreamSynchronize(st));
    const double bnorm = std::sqrt(h_res[0] + h_res[1]);
    const double target = prm.tol * bnorm;

    Inner in;
    in.alloc(prm.inner, g);
    double delta = prm.delta;
    if (!(delta > 0.0)) delta = prm.inner == P_F64 ? 0.0 : prm.inner == P_F32 ? 1e-3 : 0.1;

    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    int total_inner = 0;
    int status = 0;
    bool first = true;

    auto iteration = [&](cudaStream_t s) {
        const int* skip = &sc->done;
        RedArgs ra = red.args(2, FIN_CG_ALPHA, nullptr, sc);
        schur_apply(glo, in.ip, in.q.block(0), in.p.block(0), in.t.block(1), kappa, 0, &ra, skip, grid_cap, s);
        RedArgs rs = red.args(3, FIN_CG_RES, nullptr, sc);
        cg_xs_update(in.xp, in.ip, in.xin.block(0), in.p.block(0), in.s.block(0), in.q.block(0),
                     in.has_slow ? in.slow.block(0) : nullptr, g, sc, rs, grid_cap, s);
        RedArgs rb = red.args(4, FIN_CG_BETA, nullptr, sc);
        schur_apply(glo, in.ip, in.r.block(0), in.s_in(), in.t.block(1), kappa, 1, &rb, skip, grid_cap, s);
        cg_p_update(in.ip, in.p.block(0), in.r.block(0), g, sc, s);
    };

    // Tune the operator launches before capture (tuning cannot run inside a
    // captured stream).  The launches below only write scratch fields.
    WL_CUDA(cudaMemsetAsync(in.p.block(0), 0, in.p.pbytes, st));
    for (int dag = 0; dag < 2; dag++)
        schur_apply(glo, in.ip, in.q.block(0), in.p.block(0), in.t.block(1), kappa, dag, nullptr, nullptr, 0, st);
    schur_apply(g64, P_F64, q64.block(0), x.block(0), t64.block(1), kappa, 0, nullptr, nullptr, 0, st);

    const int chunk = prm.chunk > 0 ? prm.chunk : 16;
    if (prm.use_graph) {
        WL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            for (int k = 0; k < chunk; k++) iteration(st);
        } catch (...) {
            cudaGraph_t junk;
            cudaStreamEndCapture(st, &junk);
            if (junk) cudaGraphDestroy(junk);
            throw;
        }
        WL_CUDA(cudaStreamEndCapture(st, &graph));
        WL_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
    }

    try {
        while (true) {
            // r64 = bhat - Mhat x_e (FP64)
            schur_apply(g64, P_F64, q64.block(0), x.block(0), t64.block(1), kappa, 0, nullptr, nullptr, 0, st);
            stats.hop_applications += 2;
            RedArgs rr = red.args(5, FIN_STORE, d_res + 2, nullptr);
            xmy_norm64(r64.block(0), bhat.block(0), q64.block(0), g, rr, grid_cap, st);
            WL_CUDA(cudaMemcpyAsync(h_res + 2, d_res + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            WL_CUDA(cudaStreamSynchronize(st));
            const double rnorm = std::sqrt(h_res[2]);
            if (!std::isfinite(rnorm)) { status = 6; break; }
            if (rnorm <= target) break;
            if (stats.outer_iters >= prm.max_restarts || total_inner >= prm.maxiter) { status = 4; break; }
            stats.outer_iters++;

            // inner start: s = r64, xin = 0, r = Mhat^dag s, p = r (first / restart)
            convert_block(in.xp, in.s.block(0), P_F64, r64.block(0), g, st);
            if (in.has_slow) convert_block(in.ip, in.slow.block(0), P_F64, r64.block(0), g, st);
            WL_CUDA(cudaMemsetAsync(in.xin.block(0), 0, in.xin.pbytes, st));
            // Reset the iteration state; keep gam (|r|^2 that produced p) for
            // a reliable update, which continues p = r + beta p.
            const bool restart = first || !prm.reliable;
            const double stop = std::max(delta * rnorm, target);
            *h_sc = CGScalars{};
            h_sc->stop2 = stop * stop;
            h_sc->snorm2 = rnorm * rnorm;
            h_sc->maxiter = prm.maxiter - total_inner;
            const size_t off = restart ? 0 : offsetof(CGScalars, snorm2);
            WL_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(sc) + off, reinterpret_cast<char*>(h_sc) + off,
                                    sizeof(CGScalars) - off, cudaMemcpyHostToDevice, st));
            RedArgs rg = restart ? red.args(6, FIN_STORE, &sc->gam, nullptr) : red.args(6, FIN_CG_BETA, nullptr, sc);
            schur_apply(glo, in.ip, in.r.block(0), in.s_in(), in.t.block(1), kappa, 1, &rg, nullptr, grid_cap, st);
            stats.hop_applications += 2;
            if (restart) convert_block(in.ip, in.p.block(0), in.ip, in.r.block(0), g, st);
            else cg_p_update(in.ip, in.p.block(0), in.r.block(0), g, sc, st);
            first = false;

            while (true) {
                if (gexec) {
                    WL_CUDA(cudaGraphLaunch(gexec, st));
                } else {
                    for (int k = 0; k < chunk; k++) iteration(st);
                }
                WL_CUDA(cudaMemcpyAsync(h_sc, sc, sizeof(CGScalars), cudaMemcpyDeviceToHost, st));
                WL_CUDA(cudaStreamSynchronize(st));
                if (h_sc->done) break;
            }
            total_inner += h_sc->iter;
            stats.hop_applications += 4 * h_sc->iter;
            axpy(P_F64, x.block(0), in.xp, in.xin.block(0), 1.0, g, st);
            if (h_sc->done == 3) { status = 6; break; }
        }
    } catch (...) {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);

    // x_o = b_o + kappa D_oe x_e
    {
        HopLaunch h{};
        h.out = x.block(1);
        h.in = x.block(0);
        h.x = b.block(1);
        h.xpay = 1;
        h.a = kappa;
        h.gauge = &g64;
        h.sprec = P_F64;
        h.out_parity = 1;
        launch_hop(h, st);
        stats.hop_applications += 1;
    }
    // true residual |b - M x| / |b| over the full lattice, FP64
    {
        SpinorField mx;
        mx.alloc(P_F64, 2, 1, g);
        HopLaunch h{};
        h.out = mx.block(0);
        h.in = x.block(0);
        h.x = x.block(0);
        h.out_pstep = mx.pbytes;
        h.in_pstep = x.pbytes;
        h.x_pstep = x.pbytes;
        h.full = 1;
        h.xpay = 1;
        h.a = -kappa;
        h.gauge = &g64;
        h.sprec = P_F64;
        launch_hop(h, st);
        stats.hop_applications += 2;
        RedArgs r0 = red.args(0, FIN_STORE, d_res + 3, nullptr);
        xmy_norm64(nullptr, b.block(0), mx.block(0), g, r0, grid_cap, st);
        RedArgs r1 = red.args(1, FIN_STORE, d_res + 4, nullptr);
        xmy_norm64(nullptr, b.block(1), mx.block(1), g, r1, grid_cap, st);
        WL_CUDA(cudaMemcpyAsync(h_res + 3, d_res + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        WL_CUDA(cudaStreamSynchronize(st));
        const double rr = std::sqrt(h_res[3] + h_res[4]);
        stats.true_rel_resid = bnorm > 0 ? rr / bnorm : rr;
    }
    stats.inner_iters = total_inner;
    if (status == 0 && !(stats.true_rel_resid <= prm.tol)) status = std::isfinite(stats.true_rel_resid) ? 4 : 6;
    stats.status = status;
    stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return stats;
}

SolveStats cg_solve(double* xc, const double* gauge_canon, const double* bc, const Geom& g, double kappa,
                    const SolveParams& prm, cudaStream_t st) {
    GaugeField g64;
    g64.prec = P_F64;
    g64.recon = 18;
    g64.g = g;
    g64.buf.alloc(gauge_bytes(P_F64, 18, g.stride));
    pack_gauge(g64, gauge_canon, st);
    GaugeField glo;
    const GaugeField* inner_gauge = &g64;
    if (prm.inner != P_F64 || prm.recon != 18) {
        glo.prec = prm.inner;
        glo.recon = prm.recon;
        glo.g = g;
        glo.buf.alloc(gauge_bytes(prm.inner, prm.recon, g.stride));
        pack_gauge(glo, gauge_canon, st);
        inner_gauge = &glo;
    }
    SpinorField b, x;
    b.alloc(P_F64, 2, 1, g);
    x.alloc(P_F64, 2, 1, g);
    pack_spinor(b, 0, bc, st);
    if (prm.use_initial_guess) pack_spinor(x, 0, xc, st);
    SolveStats stats = cg_solve_prepared(x, b, g64, *inner_gauge, kappa, prm, st);
    unpack_spinor(x, 0, xc, st);
    WL_CUDA(cudaStreamSynchronize(st));
    return stats;
}

void Reduction::init(int cap, int ncounters, cudaStream_t st) {
    capacity = cap;
    partials.alloc(sizeof(double) * (size_t)cap * ncounters);
    counters.alloc(sizeof(unsigned int) * ncounters);
    results.alloc(sizeof(double) * 16);
    WL_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(unsigned int) * ncounters, st));
    WL_CUDA(cudaMemsetAsync(results.p, 0, sizeof(double) * 16, st));
}

}  // namespace wl
