// solver.cu -- CG on the normal equations of the even-odd Schur complement,
// with an FP64 defect correction around a reduced-precision inner CG, for one
// or several right-hand sides.
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
// FP64 reductions; a right-hand side is finished when |r| <= tol |b| (equal
// to the full-system residual |b - M x|, whose odd part vanishes by
// construction).  Inner loop (storage precision F32/F16/BF16 with FP32
// arithmetic, or FP64 for the plain FP64 solve) solves Mhat e = r until
// |s| <= delta |r| where s is the recursively updated inner residual; then
// x_e += e in FP64.
//
// Reliable updates (default): the inner CG keeps its search direction p
// across outer corrections and only replaces its residual by the recomputed
// FP64 one (the scheme of Sleijpen & van der Vorst 1996 as used for lattice
// QCD mixed-precision solvers); with reliable = 0 every correction restarts CG.
//
// Several right-hand sides run as independent CGs in lockstep: every launch
// covers all of them (one grid, right-hand sides fastest), each has its own
// scalars and done flag, and a finished one is skipped by every kernel.
//
// One inner iteration is six launches, all reading their scalars from device
// memory and exiting at once when their right-hand side is done:
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
#include <memory>
#include <vector>

#include "blockcg.h"
#include "solver.h"

namespace wl {

namespace {

void schur_launch(const GaugeField& gf, Prec sp, Vec out, Vec in, Vec tmp, int nrhs, double kappa, int dag,
                  const RedArgs* red, const int* skip, int skip_stride, int grid_cap, bool tune_only,
                  cudaStream_t st) {
    HopLaunch a{};
    a.tune_only = tune_only;
    a.out = tmp.p;
    a.in = in.p;
    a.nrhs = nrhs;
    a.out_rstep = tmp.rstep;
    a.in_rstep = in.rstep;
    a.gauge = &gf;
    a.sprec = sp;
    a.out_parity = 1;
    a.dagger = dag;
    a.a = 1.0;
    a.skip = skip;
    a.skip_stride = skip_stride;
    launch_hop(a, st);
    HopLaunch b{};
    b.tune_only = tune_only;
    b.out = out.p;
    b.in = tmp.p;
    b.x = in.p;
    b.nrhs = nrhs;
    b.out_rstep = out.rstep;
    b.in_rstep = tmp.rstep;
    b.x_rstep = in.rstep;
    b.xpay = 1;
    b.a = -kappa * kappa;
    b.gauge = &gf;
    b.sprec = sp;
    b.out_parity = 0;
    b.dagger = dag;
    b.red = red;
    b.skip = skip;
    b.skip_stride = skip_stride;
    b.grid_cap = red ? grid_cap : 0;
    launch_hop(b, st);
}

}  // namespace

void schur_apply(const GaugeField& gf, Prec sp, Vec out, Vec in, Vec tmp, int nrhs, double kappa, int dag,
                 const RedArgs* red, const int* skip, int skip_stride, int grid_cap, cudaStream_t st) {
    schur_launch(gf, sp, out, in, tmp, nrhs, kappa, dag, red, skip, skip_stride, grid_cap, false, st);
}

void schur_tune(const GaugeField& gf, Prec sp, Vec out, Vec in, Vec tmp, int nrhs, int dag, const RedArgs* red,
                int grid_cap, cudaStream_t st) {
    schur_launch(gf, sp, out, in, tmp, nrhs, 0.0, dag, red, nullptr, 0, red ? grid_cap : 0, true, st);
}

namespace {

struct Pinned {
    void* p = nullptr;
    explicit Pinned(size_t n) { WL_CUDA(cudaMallocHost(&p, n)); }
    ~Pinned() { if (p) cudaFreeHost(p); }
};

struct Inner {
    Prec ip, xp;
    SpinorField xin, s, slow, p, q, r, t;
    bool has_slow;
    void alloc(Prec inner, const Geom& g, int nr) {
        ip = inner;
        xp = inner == P_F64 ? P_F64 : P_F32;
        has_slow = (ip != xp);
        xin.alloc(xp, 0, nr, g);
        s.alloc(xp, 0, nr, g);
        if (has_slow) slow.alloc(ip, 0, nr, g);
        p.alloc(ip, 0, nr, g);
        q.alloc(ip, 0, nr, g);
        r.alloc(ip, 0, nr, g);
        t.alloc(ip, 1, nr, g);
    }
    Vec s_in() const { return has_slow ? vec(slow, 0) : vec(s, 0); }
};

constexpr int kSkipStride = sizeof(CGScalars) / sizeof(int);

}  // namespace

std::vector<SolveStats> cg_solve_prepared(SpinorField& x, const SpinorField& b, const GaugeField& g64,
                                          const GaugeField& glo, double kappa, const SolveParams& prm,
                                          cudaStream_t st, const GaugeField* g32) {
    NvtxRange nvtx_solve("wilson cg solve");
    auto t0 = std::chrono::steady_clock::now();
    const int nr = b.nrhs;
    std::vector<SolveStats> stats(nr);
    const Geom g = g64.g;
    const int grid_cap = 8 * device_sm_count();  // blocks per rhs of reducing launches
    Reduction red;
    red.init(grid_cap, 8 * nr, st);               // logical reduction j uses slots j*nr .. j*nr+nr-1
    auto slot = [nr](int j) { return j * nr; };
    DevBuf scbuf(sizeof(CGScalars) * nr);
    CGScalars* sc = scbuf.as<CGScalars>();
    DevBuf resbuf(sizeof(double) * 8 * nr);
    double* d_res = resbuf.as<double>();
    Pinned hbuf(sizeof(CGScalars) * nr + sizeof(double) * 8 * nr);
    CGScalars* h_sc = static_cast<CGScalars*>(hbuf.p);
    double* h_res = reinterpret_cast<double*>(h_sc + nr);
    int hops = 0;

    SpinorField bhat, r64, q64, t64;
    bhat.alloc(P_F64, 0, nr, g);
    r64.alloc(P_F64, 0, nr, g);
    q64.alloc(P_F64, 0, nr, g);
    t64.alloc(P_F64, 1, nr, g);

    // |b_k|^2 over both parities
    norm2(P_F64, vec(b, 0), g, nr, red.args(slot(0), FIN_STORE, d_res, nullptr), grid_cap, st);
    norm2(P_F64, vec(b, 1), g, nr, red.args(slot(1), FIN_STORE, d_res + nr, nullptr), grid_cap, st);
    // bhat_e = b_e + kappa D_eo b_o
    {
        HopLaunch h{};
        h.out = bhat.block(0);
        h.in = b.block(1);
        h.x = b.block(0);
        h.nrhs = nr;
        h.out_rstep = bhat.rstep();
        h.in_rstep = b.rstep();
        h.x_rstep = b.rstep();
        h.xpay = 1;
        h.a = kappa;
        h.gauge = &g64;
        h.sprec = P_F64;
        h.out_parity = 0;
        launch_hop(h, st);
        hops += 1;
    }
    if (!prm.use_initial_guess)
        for (int k = 0; k < nr; k++) WL_CUDA(cudaMemsetAsync(x.block(0, k), 0, x.pbytes, st));
    // |bhat_k|: the scale of the FP32-residual threshold
    norm2(P_F64, vec(bhat, 0), g, nr, red.args(slot(7), FIN_STORE, d_res + 5 * nr, nullptr), grid_cap, st);
    WL_CUDA(cudaMemcpyAsync(h_res, d_res, 6 * nr * sizeof(double), cudaMemcpyDeviceToHost, st));
    WL_CUDA(cudaStreamSynchronize(st));
    std::vector<double> bnorm(nr), target(nr), bhat_norm(nr);
    for (int k = 0; k < nr; k++) {
        bnorm[k] = std::sqrt(h_res[k] + h_res[nr + k]);
        target[k] = prm.tol * bnorm[k];
        bhat_norm[k] = std::sqrt(h_res[5 * nr + k]);
    }
    // FP32 outer residuals (kF32ResidualRel): x and the operator in FP32
    const bool f32_ok = g32 != nullptr && prm.tol < 1e-7 && prm.inner != P_F64;
    SpinorField x32, q32, t32;
    if (f32_ok) {
        x32.alloc(P_F32, 0, nr, g);
        q32.alloc(P_F32, 0, nr, g);
        t32.alloc(P_F32, 1, nr, g);
    }
    std::vector<double> last_rnorm(nr, HUGE_VAL);
    int outer_f32 = 0;

    Inner in;
    in.alloc(prm.inner, g, nr);
    std::unique_ptr<BlockInner> blk;
    if (prm.block_cg && nr > 1) blk = std::make_unique<BlockInner>(in.ip, in.xp, g, nr);
    // The block's own reduction per correction: the caller's delta, else a
    // conservative default (longer block runs in reduced precision lose the
    // orthogonality of their residual basis).
    const double delta_block =
        prm.delta > 0.0 ? prm.delta : prm.inner == P_F64 ? 0.0 : prm.inner == P_F32 ? 1e-3 : 0.1;
    double delta = prm.delta;
    if (!(delta > 0.0)) delta = default_delta(prm.inner);

    // Tune the operator launches before capture (tuning cannot run inside a
    // captured stream).  Tuning launches write only scratch fields; once the
    // configurations are known this launches nothing.
    for (int k = 0; k < nr; k++) WL_CUDA(cudaMemsetAsync(in.p.block(0, k), 0, in.p.pbytes, st));
    {
        // the inner operators as the iterations launch them (second hop
        // reducing: its own launch kind) and without reductions
        const RedArgs rt = red.args(slot(2), FIN_CG_ALPHA, nullptr, sc);
        for (int dag = 0; dag < 2; dag++) {
            schur_tune(glo, in.ip, vec(in.q, 0), vec(in.p, 0), vec(in.t, 1), nr, dag, &rt, grid_cap, st);
            schur_tune(glo, in.ip, vec(in.q, 0), vec(in.p, 0), vec(in.t, 1), nr, dag, nullptr, 0, st);
        }
    }
    schur_tune(g64, P_F64, vec(q64, 0), vec(x, 0), vec(t64, 1), nr, 0, nullptr, 0, st);

    auto iteration = [&](cudaStream_t s) {
        const int* skip = &sc->done;
        RedArgs ra = red.args(slot(2), FIN_CG_ALPHA, nullptr, sc);
        schur_apply(glo, in.ip, vec(in.q, 0), vec(in.p, 0), vec(in.t, 1), nr, kappa, 0, &ra, skip, kSkipStride,
                    grid_cap, s);
        RedArgs rs = red.args(slot(3), FIN_CG_RES, nullptr, sc);
        cg_xs_update(in.xp, in.ip, vec(in.xin, 0), vec(in.p, 0), vec(in.s, 0), vec(in.q, 0),
                     in.has_slow ? vec(in.slow, 0) : Vec{nullptr, 0}, g, nr, sc, rs, grid_cap, s);
        RedArgs rb = red.args(slot(4), FIN_CG_BETA, nullptr, sc);
        schur_apply(glo, in.ip, vec(in.r, 0), in.s_in(), vec(in.t, 1), nr, kappa, 1, &rb, skip, kSkipStride,
                    grid_cap, s);
        cg_p_update(in.ip, vec(in.p, 0), vec(in.r, 0), g, nr, sc, s);
    };

    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const int chunk = prm.chunk > 0 ? prm.chunk : 16;
    if (prm.use_graph) {
        WL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            for (int k = 0; k < chunk; k++) iteration(st);
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(st, &junk);
            if (junk) cudaGraphDestroy(junk);
            throw;
        }
        WL_CUDA(cudaStreamEndCapture(st, &graph));
        WL_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
    }

    std::vector<int> total_inner(nr, 0), finished(nr, 0);
    std::vector<double> best(nr, HUGE_VAL);  // smallest FP64 residual so far
    int outer = 0;
    bool first = true;
    bool force64 = false;  // the next residual is FP64
    bool f32_off = false;  // no more FP32 residuals in this solve
    // device time of the inner iterations: events around each chunk's replay
    cudaEvent_t ev_in0 = nullptr, ev_in1 = nullptr;
    WL_CUDA(cudaEventCreate(&ev_in0));
    WL_CUDA(cudaEventCreate(&ev_in1));
    double inner_ms = 0.0;
    try {
        while (true) {
            // r64 = bhat - Mhat x_e (FP64); the first residual of a solve from
            // x_e = 0 is bhat itself
            NvtxRange nvtx_outer("fp64 correction");
            // FP32 residual while every unfinished right-hand side's expected
            // residual is above kF32ResidualRel |bhat| (never for a convergence
            // decision: see below)
            bool use32 = f32_ok && outer > 0 && !force64 && !f32_off;
            for (int k = 0; k < nr && use32; k++)
                if (!finished[k] && !(last_rnorm[k] * delta > kF32ResidualRel * bhat_norm[k])) use32 = false;
            force64 = false;
            if (outer == 0 && !prm.use_initial_guess) {
                for (int k = 0; k < nr; k++) WL_CUDA(cudaMemsetAsync(q64.block(0, k), 0, q64.pbytes, st));
                xmy_norm64(vec(r64, 0), vec(bhat, 0), vec(q64, 0), g, nr,
                           red.args(slot(5), FIN_STORE, d_res + 2 * nr, nullptr), grid_cap, st);
            } else if (use32) {
                convert(P_F32, vec(x32, 0), P_F64, vec(x, 0), g, nr, st);
                schur_apply(*g32, P_F32, vec(q32, 0), vec(x32, 0), vec(t32, 1), nr, kappa, 0, nullptr, nullptr, 0,
                            0, st);
                hops += 2;
                outer_f32++;
                xmy_norm(P_F32, vec(r64, 0), vec(bhat, 0), vec(q32, 0), g, nr,
                         red.args(slot(5), FIN_STORE, d_res + 2 * nr, nullptr), grid_cap, st);
            } else {
                schur_apply(g64, P_F64, vec(q64, 0), vec(x, 0), vec(t64, 1), nr, kappa, 0, nullptr, nullptr, 0, 0,
                            st);
                hops += 2;
                xmy_norm64(vec(r64, 0), vec(bhat, 0), vec(q64, 0), g, nr,
                           red.args(slot(5), FIN_STORE, d_res + 2 * nr, nullptr), grid_cap, st);
            }
            WL_CUDA(cudaMemcpyAsync(h_res + 2 * nr, d_res + 2 * nr, nr * sizeof(double), cudaMemcpyDeviceToHost,
                                    st));
            WL_CUDA(cudaStreamSynchronize(st));
            std::vector<double> rnorm(nr, 0.0);
            // an FP32 residual at or below its target decides nothing: recompute in
            // FP64; one that has not halved has reached the FP32 noise floor
            if (use32) {
                for (int k = 0; k < nr; k++) {
                    if (finished[k]) continue;
                    const double r32 = std::sqrt(h_res[2 * nr + k]);
                    if (r32 <= target[k]) force64 = true;
                    if (!(r32 <= 0.5 * last_rnorm[k])) f32_off = true;
                }
                if (force64) continue;
            }
            bool all_done = true;
            const bool budget = outer < prm.max_restarts;
            for (int k = 0; k < nr; k++) {
                if (finished[k]) continue;
                rnorm[k] = std::sqrt(h_res[2 * nr + k]);
                last_rnorm[k] = rnorm[k];
                if (!std::isfinite(rnorm[k])) {
                    finished[k] = 1;
                    stats[k].status = 6;
                } else if (rnorm[k] <= target[k]) {
                    finished[k] = 1;
                } else if (total_inner[k] >= prm.maxiter || !budget || rnorm[k] > kDivergence * best[k]) {
                    finished[k] = 1;
                    stats[k].status = 4;
                } else {
                    all_done = false;
                }
                best[k] = std::min(best[k], rnorm[k]);
            }
            if (all_done) break;
            outer++;

            // inner start: s = r64, xin = 0, r = Mhat^dag s, p = r (first / restart) or
            // p = r + beta p (reliable update, keeps the direction)
            convert(in.xp, vec(in.s, 0), P_F64, vec(r64, 0), g, nr, st);
            if (in.has_slow) convert(in.ip, vec(in.slow, 0), P_F64, vec(r64, 0), g, nr, st);
            for (int k = 0; k < nr; k++) WL_CUDA(cudaMemsetAsync(in.xin.block(0, k), 0, in.xin.pbytes, st));
            if (blk) {
                // block CG over the unfinished right-hand sides
                // column k stops after its normal residual fell by max(delta, half the
                // factor its Schur residual still has to fall to reach the target)
                int left = kInnerCap;
                std::vector<double> dk(nr, 1.0);
                for (int k = 0; k < nr; k++) {
                    if (finished[k]) continue;
                    left = std::min(left, prm.maxiter - total_inner[k]);
                    dk[k] = std::max(delta_block, 0.5 * target[k] / rnorm[k]);
                }
                const BlockInner::Result br =
                    blk->run(glo, kappa, in.s_in(), vec(in.p, 0), vec(in.q, 0), vec(in.r, 0), vec(in.t, 1),
                             vec(in.xin, 0), finished, dk, left, chunk, prm.use_graph != 0, prm.reliable != 0,
                             st);
                hops += 2 + 4 * br.iterations;
                for (int k = 0; k < nr; k++)
                    if (!finished[k]) total_inner[k] += br.iterations;
                // The block lost rank (3) or met NaN/Inf in its own arithmetic (4; the
                // sources' NaNs were caught by the FP64 residual above): independent CGs
                // from here on, from a fresh start.  A rank loss keeps the correction made
                // so far; a NaN/Inf drops it.
                // A correction that is not finite everywhere is dropped the same way.
                bool finite = br.status != 4;
                if (finite) {
                    norm2(in.xp, vec(in.xin, 0), g, nr, red.args(slot(7), FIN_STORE, d_res + 5 * nr, nullptr),
                          grid_cap, st);
                    WL_CUDA(cudaMemcpyAsync(h_res + 5 * nr, d_res + 5 * nr, nr * sizeof(double),
                                            cudaMemcpyDeviceToHost, st));
                    WL_CUDA(cudaStreamSynchronize(st));
                    for (int k = 0; k < nr; k++)
                        if (!finished[k] && !std::isfinite(h_res[5 * nr + k])) finite = false;
                }
                if (br.status != 0 || !finite) blk.reset();
                if (finite) axpy(P_F64, vec(x, 0), in.xp, vec(in.xin, 0), 1.0, g, nr, st);
                continue;
            }
            const bool restart = first || !prm.reliable;
            for (int k = 0; k < nr; k++) {
                h_sc[k] = CGScalars{};
                if (finished[k]) {
                    h_sc[k].done = 4;
                    continue;
                }
                const double stop = std::max(delta * rnorm[k], target[k]);
                h_sc[k].stop2 = stop * stop;
                h_sc[k].snorm2 = rnorm[k] * rnorm[k];
                h_sc[k].maxiter = std::min(prm.maxiter - total_inner[k], kInnerCap);
            }
            if (restart) {
                WL_CUDA(cudaMemcpyAsync(sc, h_sc, sizeof(CGScalars) * nr, cudaMemcpyHostToDevice, st));
            } else {
                // keep gam/alpha/beta/pq (the direction's history); reset the rest
                const size_t off = offsetof(CGScalars, snorm2);
                for (int k = 0; k < nr; k++)
                    WL_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(sc + k) + off,
                                            reinterpret_cast<char*>(h_sc + k) + off, sizeof(CGScalars) - off,
                                            cudaMemcpyHostToDevice, st));
            }
            RedArgs rg = red.args(slot(6), restart ? FIN_CG_GAM : FIN_CG_BETA, nullptr, sc);
            schur_apply(glo, in.ip, vec(in.r, 0), in.s_in(), vec(in.t, 1), nr, kappa, 1, &rg, nullptr, 0, grid_cap,
                        st);
            hops += 2;
            if (restart) convert(in.ip, vec(in.p, 0), in.ip, vec(in.r, 0), g, nr, st);
            else cg_p_update(in.ip, vec(in.p, 0), vec(in.r, 0), g, nr, sc, st);
            first = false;

            while (true) {
                WL_CUDA(cudaEventRecord(ev_in0, st));
                if (gexec) {
                    WL_CUDA(cudaGraphLaunch(gexec, st));
                } else {
                    for (int it = 0; it < chunk; it++) iteration(st);
                }
                WL_CUDA(cudaEventRecord(ev_in1, st));
                WL_CUDA(cudaMemcpyAsync(h_sc, sc, sizeof(CGScalars) * nr, cudaMemcpyDeviceToHost, st));
                WL_CUDA(cudaStreamSynchronize(st));
                {
                    float ms = 0.f;
                    WL_CUDA(cudaEventElapsedTime(&ms, ev_in0, ev_in1));
                    inner_ms += ms;
                }
                bool all = true;
                for (int k = 0; k < nr; k++) all = all && h_sc[k].done != 0;
                if (all) break;
            }
            int most = 0;
            for (int k = 0; k < nr; k++) {
                if (finished[k]) continue;
                total_inner[k] += h_sc[k].iter;
                most = std::max(most, h_sc[k].iter);
                if (h_sc[k].done == 3) {
                    finished[k] = 1;
                    stats[k].status = 6;
                }
            }
            hops += 4 * most;
            axpy(P_F64, vec(x, 0), in.xp, vec(in.xin, 0), 1.0, g, nr, st);
        }
    } catch (...) {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        cudaEventDestroy(ev_in0);
        cudaEventDestroy(ev_in1);
        throw;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    cudaEventDestroy(ev_in0);
    cudaEventDestroy(ev_in1);

    // x_o = b_o + kappa D_oe x_e
    {
        HopLaunch h{};
        h.out = x.block(1);
        h.in = x.block(0);
        h.x = b.block(1);
        h.nrhs = nr;
        h.out_rstep = x.rstep();
        h.in_rstep = x.rstep();
        h.x_rstep = b.rstep();
        h.xpay = 1;
        h.a = kappa;
        h.gauge = &g64;
        h.sprec = P_F64;
        h.out_parity = 1;
        launch_hop(h, st);
        hops += 1;
    }
    // true residual |b - M x| / |b| over the full lattice, FP64
    {
        SpinorField mx;
        mx.alloc(P_F64, 2, nr, g);
        HopLaunch h{};
        h.out = mx.block(0);
        h.in = x.block(0);
        h.x = x.block(0);
        h.out_pstep = mx.pbytes;
        h.in_pstep = x.pbytes;
        h.x_pstep = x.pbytes;
        h.nrhs = nr;
        h.out_rstep = mx.rstep();
        h.in_rstep = x.rstep();
        h.x_rstep = x.rstep();
        h.full = 1;
        h.xpay = 1;
        h.a = -kappa;
        h.gauge = &g64;
        h.sprec = P_F64;
        launch_hop(h, st);
        hops += 2;
        xmy_norm64(Vec{nullptr, 0}, vec(b, 0), vec(mx, 0), g, nr,
                   red.args(slot(0), FIN_STORE, d_res + 3 * nr, nullptr), grid_cap, st);
        xmy_norm64(Vec{nullptr, 0}, vec(b, 1), vec(mx, 1), g, nr,
                   red.args(slot(1), FIN_STORE, d_res + 4 * nr, nullptr), grid_cap, st);
        WL_CUDA(cudaMemcpyAsync(h_res + 3 * nr, d_res + 3 * nr, 2 * nr * sizeof(double), cudaMemcpyDeviceToHost,
                                st));
        WL_CUDA(cudaStreamSynchronize(st));
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < nr; k++) {
        SolveStats& s = stats[k];
        const double rr = std::sqrt(h_res[3 * nr + k] + h_res[4 * nr + k]);
        s.true_rel_resid = bnorm[k] > 0 ? rr / bnorm[k] : rr;
        s.inner_iters = total_inner[k];
        s.outer_iters = outer;
        s.hop_applications = hops;
        s.seconds = secs;
        s.inner_seconds = inner_ms * 1e-3;
        s.outer_f32 = outer_f32;
        if (s.status == 0 && !(s.true_rel_resid <= prm.tol)) s.status = std::isfinite(s.true_rel_resid) ? 4 : 6;
    }
    return stats;
}

std::vector<SolveStats> cg_solve(double* xc, const double* gauge_canon, const double* bc, int nrhs, const Geom& g,
                                 double kappa, const SolveParams& prm, cudaStream_t st) {
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
    // FP32 links for the FP32 outer residuals: the inner links when they are FP32
    GaugeField g32f;
    const GaugeField* g32 = nullptr;
    if (prm.inner == P_F32) {
        g32 = inner_gauge;
    } else if (prm.inner != P_F64 && prm.tol < 1e-7) {
        g32f.prec = P_F32;
        g32f.recon = 12;
        g32f.g = g;
        g32f.buf.alloc(gauge_bytes(P_F32, 12, g.stride));
        pack_gauge(g32f, gauge_canon, st);
        g32 = &g32f;
    }
    SpinorField b, x;
    b.alloc(P_F64, 2, nrhs, g);
    x.alloc(P_F64, 2, nrhs, g);
    const size_t per = (size_t)24 * 2 * g.Vh;  // doubles per canonical full field
    for (int k = 0; k < nrhs; k++) {
        pack_spinor(b, k, bc + per * k, st);
        if (prm.use_initial_guess) pack_spinor(x, k, xc + per * k, st);
    }
    std::vector<SolveStats> stats = cg_solve_prepared(x, b, g64, *inner_gauge, kappa, prm, st, g32);
    for (int k = 0; k < nrhs; k++) unpack_spinor(x, k, xc + per * k, st);
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
