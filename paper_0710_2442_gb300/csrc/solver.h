// solver.h -- the even-odd CG solve (host orchestration of device kernels).
#pragma once

#include <vector>

#include "../../include/wilson.h"
#include "blas.h"
#include "internal.h"

namespace wl {

struct SolveParams {
    Prec inner = P_F16;
    int recon = 12;
    double tol = 1e-10;
    int maxiter = 100000;
    int max_restarts = 1000;
    double delta = 0.0;       // 0: default per precision
    int use_initial_guess = 0;
    int reliable = 1;
    int block_cg = 0;           // several right-hand sides: one block CG instead of lockstep CGs
    int chunk = 16;           // iterations per captured graph
    int use_graph = 1;
    int batch_small_vh = 4096;  // batched solves: problems with at most this many sites per parity
                                // run the CTA-resident solver (0: none)
};

// Default inner reduction per FP64 correction (|s| <= delta |r|), by inner
// precision: measured on the 24^3 x 48 solve, F16 is fastest near 0.02 and
// stagnates below about 0.005 (its storage precision), BF16 is fastest at
// 0.1, F32 at 1e-4 .. 1e-5.  FP64: the inner CG runs to the target.
inline double default_delta(Prec ip) {
    return ip == P_F64 ? 0.0 : ip == P_F32 ? 1e-4 : ip == P_F16 ? 0.02 : 0.1;
}

// Inner CG iterations between two FP64 corrections at most.  With reliable
// updates a forced correction only replaces the residual (the direction
// continues), so the cap costs one FP64 residual per 1000 iterations; it
// bounds an inner solve whose delta is below what its precision can reach.
constexpr int kInnerCap = 1000;

// FP32 outer residuals: while every unfinished right-hand side's expected
// residual (its last one times the inner reduction delta) is above this
// fraction of |bhat|, the outer residual r = bhat - Mhat x is computed with
// FP32 fields and links.  Its error is about 1e-7 |Mhat| |x| (the FP32
// rounding of x and of the operator), so cond(Mhat) 1e-7 |bhat|: a few
// percent of |r| at cond = 100, which the defect correction absorbs.  Below
// the threshold, and for every convergence decision, the residual is FP64;
// an FP32 residual that has not fallen below half the previous one (its
// noise floor reached) ends the FP32 residuals of the solve.  Used when the
// target is below 1e-7 (else every residual is FP64).
constexpr double kF32ResidualRel = 1e-4;

// A right-hand side whose FP64 residual grows past this factor times the
// smallest one it has had is diverging (an inner precision too coarse for its
// delta): it stops with WILSON_ERR_NOCONV instead of spending maxiter.
constexpr double kDivergence = 1e3;

struct SolveStats {
    int status = 0;
    int outer_iters = 0;
    int inner_iters = 0;
    int hop_applications = 0;
    double true_rel_resid = 0.0;
    double seconds = 0.0;
    double inner_seconds = 0.0;  // device time of the inner CG iterations (graph replays)
    int outer_f32 = 0;           // FP64 corrections whose residual was computed in FP32
};

// Mhat (dag = 0) or Mhat^dag (dag = 1) on even blocks of nrhs right-hand
// sides: out = in - kappa^2 D_eo D_oe in.  tmp: odd blocks of the same
// precision.  Optional per-rhs |out|^2 reduction and per-rhs skip flags.
void schur_apply(const GaugeField& gf, Prec sp, Vec out, Vec in, Vec tmp, int nrhs, double kappa, int dag,
                 const RedArgs* red, const int* skip, int skip_stride, int grid_cap, cudaStream_t st);
// Tunes the launch configurations of schur_apply's two hops where they are
// not known yet (the tuning launches write out and tmp); launches nothing else.
// red != nullptr tunes the reducing form of the second hop (grid_cap: its
// reduction capacity); red itself is not written.
void schur_tune(const GaugeField& gf, Prec sp, Vec out, Vec in, Vec tmp, int nrhs, int dag, const RedArgs* red,
                int grid_cap, cudaStream_t st);

// Solve M x_k = b_k for the nrhs right-hand sides of b (full F64 fields; x:
// full F64, in/out) with independent CGs run in lockstep.  g64: FP64 links;
// glo: the inner operator's links (may be g64).  Returns one SolveStats per
// right-hand side (outer_iters, hop_applications and seconds are shared).
std::vector<SolveStats> cg_solve_prepared(SpinorField& x, const SpinorField& b, const GaugeField& g64,
                                          const GaugeField& glo, double kappa, const SolveParams& prm,
                                          cudaStream_t st,
                                          const GaugeField* g32 = nullptr);

// The same on canonical complex128 device fields (nrhs fields back to back).
std::vector<SolveStats> cg_solve(double* x, const double* gauge_canon, const double* b, int nrhs, const Geom& g,
                                 double kappa, const SolveParams& prm, cudaStream_t st);

// Many independent solves in one graph launch (batch.cu).
void batch_solve(int n, const wilson_problem* probs, const SolveParams& prm, wilson_solve_stats* stats,
                 wilson_batch_info* info, cudaStream_t st);

}  // namespace wl
