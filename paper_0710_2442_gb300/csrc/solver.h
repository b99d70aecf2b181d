// solver.h -- the even-odd CG solve (host orchestration of device kernels).
#pragma once

#include "blas.h"
#include "internal.h"

namespace wl {

struct SolveParams {
    Prec inner = P_F16;
    int recon = 12;
    double tol = 1e-10;
    int maxiter = 100000;
    int max_restarts = 100;
    double delta = 0.0;       // 0: default per precision
    int use_initial_guess = 0;
    int reliable = 1;
    int chunk = 16;           // iterations per captured graph
    int use_graph = 1;
};

struct SolveStats {
    int status = 0;
    int outer_iters = 0;
    int inner_iters = 0;
    int hop_applications = 0;
    double true_rel_resid = 0.0;
    double seconds = 0.0;
};

// Mhat (dag = 0) or Mhat^dag (dag = 1) on even blocks: out = in - kappa^2 D_eo D_oe in.
// tmp is an odd block of the same precision.  Optional |out|^2 reduction.
void schur_apply(const GaugeField& gf, Prec sp, void* out, const void* in, void* tmp, double kappa, int dag,
                 const RedArgs* red, const int* skip, int grid_cap, cudaStream_t st);

// Solve M x = b on canonical complex128 device fields (x: V spinors, in/out).
SolveStats cg_solve(double* x, const double* gauge_canon, const double* b, const Geom& g, double kappa,
                    const SolveParams& prm, cudaStream_t caller);

// The same solve on already-prepared fields: b full F64, x full F64 (in/out);
// g64: F64 links; glo: the inner operator's links (may be g64).
SolveStats cg_solve_prepared(SpinorField& x, const SpinorField& b, const GaugeField& g64, const GaugeField& glo,
                             double kappa, const SolveParams& prm, cudaStream_t st);

}  // namespace wl
