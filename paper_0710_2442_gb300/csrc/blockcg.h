// blockcg.h -- block CG over the right-hand sides of a multi-RHS solve, as
// the inner solver of the FP64 defect correction (blockcg.cu).
#pragma once

#include <vector>

#include "blas.h"
#include "internal.h"

namespace wl {

constexpr int kBlockMax = 16;  // right-hand sides one block CG can carry

struct BCGState;

// Workspace and captured iteration graph of one solve's block CG.  Every
// run() solves Mhat^dag Mhat E = Mhat^dag s for the active right-hand sides
// (those not flagged in `finished`) until every column's normal residual has
// fallen by its factor delta[k] (or maxiter): on entry s_in holds the quantised FP64
// residual s of every right-hand side; on exit X holds the correction E in
// the accumulation precision xp.  S, W, Z: even fields of the inner
// precision ip (search directions, Mhat S, Mhat^dag Mhat S); T: odd field
// of ip (the operator's intermediate).  The fields must stay the same
// between runs (the iteration is captured once into a CUDA graph).  With
// `reliable`, a run over the same right-hand sides as the previous one keeps
// its search directions (the block form of a reliable update).
class BlockInner {
public:
    BlockInner(Prec ip, Prec xp, const Geom& g, int nrhs);
    ~BlockInner();
    BlockInner(const BlockInner&) = delete;
    BlockInner& operator=(const BlockInner&) = delete;

    struct Result {
        int iterations = 0;
        int status = 0;  // 0: reduced by delta (or iteration cap), 3: breakdown, 4: NaN/Inf
    };
    Result run(const GaugeField& glo, double kappa, Vec s_in, Vec S, Vec W, Vec Z, Vec T, Vec X,
               const std::vector<int>& finished, const std::vector<double>& delta, int maxiter, int chunk,
               bool use_graph, bool reliable, cudaStream_t st);

private:
    void iteration(const GaugeField& glo, double kappa, Vec S, Vec W, Vec Z, Vec T, Vec X, cudaStream_t st);
    void gram(Prec p, Vec a, Vec b, cudaStream_t st);
    void small(int mode, cudaStream_t st);
    void update(int mode, Vec S, Vec X, cudaStream_t st);

    Prec ip_, xp_;
    Geom g_;
    int nr_, nbm_ = kBlockMax, grid_ = 1;
    bool prev_ok_ = false;                // the last run ended normally (its S and C continue)
    std::vector<int> prev_active_;        // its active right-hand sides
    SpinorField q_;                       // orthonormal residual basis (xp)
    DevBuf state_, partials_, counter_, skip_;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
};

}  // namespace wl
