// batch_impl.cuh -- device side of the batched solve (batch.cu): problem
// descriptors and states, the per-problem finishers, the tile-walking hop
// kernels and the CTA-resident small-lattice solver.  The kernels are
// instantiated in batch_hop_lo.cu, batch_hop_64.cu and batch_small_*.cu so
// that they compile in parallel.
#pragma once

#include <cooperative_groups.h>

#include "../../include/wilson.h"
#include "dslash_impl.cuh"
#include "solver.h"

namespace wl {
namespace bt {

constexpr int kTile = 256;  // default half-lattice sites per tile (the run's tile is tuned: 128, 256, 512)

enum BField { BF_B, BF_X, BF_BHAT, BF_R64, BF_Q64, BF_T64, BF_XIN, BF_S, BF_SLOW, BF_P, BF_Q, BF_R, BF_T,
              BF_X32, BF_Q32, BF_T32, BF_N };
enum Phase { PH_OUTER = 0, PH_INNER = 1, PH_DONE = 2 };
enum BFin { BF_NONE = -1, BFIN_ALPHA, BFIN_RES, BFIN_BETA, BFIN_START, BFIN_OUTER, BFIN_BNORM, BFIN_TRUE };

struct BatchProb {
    Geom g;
    char* f[BF_N];        // parity block (half fields) or parity-0 block (full fields)
    long long fp[BF_N];   // parity step of full fields, 0 for half fields
    const char* g64;      // FP64 18-real links
    const char* glo;      // inner links
    const char* g32;      // FP32 12-real links of the FP32 residuals (null: none)
    double kappa, tol, delta;
    int tile0, ntiles;
    int maxiter, max_outer;
    int small;            // 1: solved by one CTA (small_solve_kernel), no tiles
    int keep_x;           // 1: x holds an initial guess
    int res32_ok;         // 1: early corrections may compute their residual in FP32
};

struct BatchState {
    CGScalars sc;
    int phase, next_phase;
    int outer;
    int status;
    int first;
    int pad;
    double bnorm2;
    double rnorm2;
    double best2;  // smallest |r|^2 of the FP64 corrections so far
    double res2;
    unsigned long long t_done;
    int use32;    // the next correction computes its residual with FP32 fields and links
    int f32_off;  // an FP32 residual stopped halving: no more of them
    int n32;      // corrections whose residual was FP32
    int pad2;
};

struct BatchGlobal {
    unsigned long long t_start, t_end;
    int iterations;
    int timed_out;
};

struct BatchArgs {
    const BatchProb* probs;
    BatchState* state;
    const int* tile_prob;
    int ntiles;
    int nprob;
    int tile;  // half-lattice sites per tile
};

struct BOp {
    int f_out, f_in, f_x;   // field ids (f_x < 0: no xpay)
    int out_parity;
    int use64;              // links: FP64 (1), inner (0), or the FP32 residual links (2)
    int coef;               // a = 1, kappa, -kappa^2, -kappa
    int phase;              // only problems in this phase (-1: all)
    int skip_done;          // also skip problems whose inner CG is done
    int fin;                // BFin of the fused reduction (BF_NONE: none)
    int res32;              // only problems whose next residual is FP32 (1), FP64 (0), or all (-1)
    int zero_first;         // the FP64 correction hops: while a problem's iterate is still zero
                            // (its first correction), the hop term is zero and is not computed
    double* partials;       // [ntiles]
    unsigned int* counters; // [nprob]
};

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double coef_of(int c, double kappa) {
    return c == 0 ? 1.0 : c == 1 ? kappa : c == 2 ? -kappa * kappa : -kappa;
}

// The problem's finisher (runs once per problem per reducing launch).
__device__ inline void batch_finish(int op, const BatchProb& P, BatchState& S, double sum) {
    CGScalars& sc = S.sc;
    switch (op) {
        case BFIN_ALPHA:
            sc.pq = sum;
            if (!isfinite(sum)) sc.done = 3;
            else if (!(sum > 0.0)) { sc.alpha = 0.0; if (sc.done == 0) sc.done = 1; }
            else sc.alpha = sc.gam / sum;
            if (sc.done) S.next_phase = PH_OUTER;
            break;
        case BFIN_RES:
            sc.snorm2 = sum;
            sc.iter += 1;
            if (!isfinite(sum)) sc.done = 3;
            else if (sum <= sc.stop2) sc.done = 1;
            else if (sc.iter >= sc.maxiter) sc.done = 2;
            if (sc.done) S.next_phase = PH_OUTER;
            break;
        case BFIN_BETA:
            if (!isfinite(sum)) { sc.done = 3; S.next_phase = PH_OUTER; break; }
            sc.beta = sc.gam > 0.0 ? sum / sc.gam : 0.0;
            sc.gam = sum;
            break;
        case BFIN_START:
            if (!isfinite(sum)) {
                S.status = WILSON_ERR_NUMERIC;
                S.next_phase = PH_DONE;
                S.t_done = globaltimer();
                break;
            }
            sc.beta = (S.first || !(sc.gam > 0.0)) ? 0.0 : sum / sc.gam;
            sc.gam = sum;
            S.first = 0;
            break;
        case BFIN_OUTER: {
            // the correction's residual was FP32 (use32) or FP64; an FP32 one
            // decides no convergence (the inner solve it starts stops at once
            // and the next residual is FP64), and one that has not halved has
            // reached the FP32 noise floor (kF32ResidualRel, solver.h)
            const bool was32 = S.use32 != 0;
            const double prev2 = S.rnorm2;
            S.rnorm2 = sum;
            if (S.outer == 0 || sum < S.best2) S.best2 = sum;
            const double target2 = P.tol * P.tol * S.bnorm2;
            if (was32) {
                S.n32 += 1;
                if (!(sum <= 0.25 * prev2)) S.f32_off = 1;
            }
            if (!isfinite(sum)) {
                S.status = WILSON_ERR_NUMERIC;
                S.next_phase = PH_DONE;
            } else if (sum <= target2 && !was32) {
                S.next_phase = PH_DONE;
            } else if (S.outer >= P.max_outer || sc.iter >= P.maxiter ||
                       (S.outer > 0 && sum > kDivergence * kDivergence * S.best2)) {
                S.status = WILSON_ERR_NOCONV;
                S.next_phase = PH_DONE;
            } else {
                S.outer += 1;
                S.next_phase = PH_INNER;
                const double stop = fmax(P.delta * sqrt(sum), sqrt(target2));
                sc.stop2 = stop * stop;
                sc.snorm2 = sum;
                sc.done = 0;
                sc.maxiter = min(P.maxiter, sc.iter + kInnerCap);  // iter counts the whole solve
                // the next residual in FP32 while the expected one (this one
                // times delta) is above kF32ResidualRel |b|
                S.use32 = P.res32_ok && !S.f32_off &&
                          P.delta * P.delta * sum > kF32ResidualRel * kF32ResidualRel * S.bnorm2;
            }
            if (S.next_phase == PH_DONE) S.t_done = globaltimer();
            break;
        }
        case BFIN_BNORM: S.bnorm2 += sum; break;
        case BFIN_TRUE: S.res2 += sum; break;
    }
}

// Block-uniform decision whether this block works on tile t.  Reads the
// problem's phase and done flag once (thread 0) and broadcasts them.
__device__ __forceinline__ bool tile_active(const BatchArgs& A, const BOp& op, int pid) {
    __shared__ int s_act;
    __syncthreads();  // the previous tile's readers are done with s_act
    if (threadIdx.x == 0) {
        const BatchState& S = A.state[pid];
        int act = 1;
        if (op.phase >= 0 && __ldcg(&S.phase) != op.phase) act = 0;
        if (act && op.skip_done && __ldcg(&S.sc.done)) act = 0;
        if (act && op.res32 >= 0 && __ldcg(&S.use32) != op.res32) act = 0;
        s_act = act;
    }
    __syncthreads();
    return s_act != 0;
}

// Tile partial + per-problem ticket; the problem's last tile finishes.
__device__ inline void tile_reduce(double v, const BatchArgs& A, const BOp& op, int t, int pid) {
    const double bs = block_sum(v);
    __shared__ int s_last;
    const BatchProb& P = A.probs[pid];
    if (threadIdx.x == 0) {
        op.partials[t] = bs;
        __threadfence();
        const unsigned int ticket = atomicAdd(op.counters + pid, 1u);
        s_last = (ticket == (unsigned)P.ntiles - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < P.ntiles; i += blockDim.x) acc += __ldcg(op.partials + P.tile0 + i);
    const double total = block_sum(acc);
    if (threadIdx.x == 0) {
        batch_finish(op.fin, P, A.state[pid], total);
        op.counters[pid] = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// batched hopping term: out = a * D in (+ x), tile by tile
// ---------------------------------------------------------------------------
template <int SP, int GP, int R, bool DAG, int MINB>
__global__ void __launch_bounds__(256, MINB) bhop_kernel(const BatchArgs A, const BOp op) {
    using SF = SpinorFmt<SP>;
    using T = typename SF::real;
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const int pid = __ldg(A.tile_prob + t);
        if (!tile_active(A, op, pid)) continue;
        const BatchProb& Pr = A.probs[pid];
        HopParams P;
        P.g = Pr.g;
        P.gauge = op.use64 == 1 ? Pr.g64 : op.use64 == 2 ? Pr.g32 : Pr.glo;
        const int p = op.out_parity;
        char* out = Pr.f[op.f_out] + p * Pr.fp[op.f_out];
        const char* in = Pr.f[op.f_in] + (1 - p) * Pr.fp[op.f_in];
        const char* x = op.f_x >= 0 ? Pr.f[op.f_x] + p * Pr.fp[op.f_x] : nullptr;
        const T a = (T)coef_of(op.coef, Pr.kappa);
        const Geom& g = P.g;
        // outer is written only by the correction finisher, a later kernel
        const bool zero = op.zero_first && __ldcg(&A.state[pid].outer) == 0;
        double nrm = 0.0;
        const int h0 = (t - Pr.tile0) * A.tile;
        for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
            const int h = h0 + j;
            if (h >= g.Vh) break;
            int c[4], s;
            site_of_half(h, p, g, c, s);
            cpx<T> acc[12];
            if (zero) {
#pragma unroll
                for (int k = 0; k < 12; k++) acc[k] = {T(0), T(0)};
            } else {
                hop_dir<SP, GP, R, DAG, 0, true>(acc, P, in, p, h, c, s);
                hop_dir<SP, GP, R, DAG, 1, false>(acc, P, in, p, h, c, s);
                hop_dir<SP, GP, R, DAG, 2, false>(acc, P, in, p, h, c, s);
                hop_dir<SP, GP, R, DAG, 3, false>(acc, P, in, p, h, c, s);
            }
            if (x) {
                cpx<T> xv[12];
                SF::load(x, g.stride, h, xv);
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    acc[k].re = fma(a, acc[k].re, xv[k].re);
                    acc[k].im = fma(a, acc[k].im, xv[k].im);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) acc[k] = cscale(a, acc[k]);
            }
            if (op.fin != BF_NONE) {
                T n2 = 0;
#pragma unroll
                for (int k = 0; k < 12; k++) n2 += cnorm2(acc[k]);
                nrm += (double)n2;
            }
            SF::store(out, g.stride, h, acc);
        }
        if (op.fin != BF_NONE) tile_reduce(nrm, A, op, t, pid);
    }
}

// The same on the paired-FP32 stencil (F32 / F16 / BF16 spinors; see
// hop_kernel_p): fewer instructions per site for the same arithmetic.
template <int SP, int GP, int R, bool DAG, int MINB>
__global__ void __launch_bounds__(256, MINB) bhop_kernel_p(const BatchArgs A, const BOp op) {
    using SF = SpinorFmt<SP>;
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const int pid = __ldg(A.tile_prob + t);
        if (!tile_active(A, op, pid)) continue;
        const BatchProb& Pr = A.probs[pid];
        HopParams P;
        P.g = Pr.g;
        P.gauge = op.use64 == 2 ? Pr.g32 : Pr.glo;
        const int p = op.out_parity;
        char* out = Pr.f[op.f_out] + p * Pr.fp[op.f_out];
        const char* in = Pr.f[op.f_in] + (1 - p) * Pr.fp[op.f_in];
        const char* x = op.f_x >= 0 ? Pr.f[op.f_x] + p * Pr.fp[op.f_x] : nullptr;
        const float a = (float)coef_of(op.coef, Pr.kappa);
        const Geom& g = P.g;
        double nrm = 0.0;
        const int h0 = (t - Pr.tile0) * A.tile;
        for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
            const int h = h0 + j;
            if (h >= g.Vh) break;
            int c[4], s;
            site_of_half(h, p, g, c, s);
            PSpinor acc;
            hop_dir_p<SP, GP, R, DAG, 0, true>(acc, P, in, p, h, c, s);
            hop_dir_p<SP, GP, R, DAG, 1, false>(acc, P, in, p, h, c, s);
            hop_dir_p<SP, GP, R, DAG, 2, false>(acc, P, in, p, h, c, s);
            hop_dir_p<SP, GP, R, DAG, 3, false>(acc, P, in, p, h, c, s);
            const float2 Af = bc2(a);
            if (x) {
                PSpinor xq;
                float xs;
                SF::load_packed(x, g.stride, h, xq, xs);
                const float2 X = bc2(xs);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    acc.re01[cc] = fma2(Af, acc.re01[cc], mul2(X, xq.re01[cc]));
                    acc.im01[cc] = fma2(Af, acc.im01[cc], mul2(X, xq.im01[cc]));
                    acc.re23[cc] = fma2(Af, acc.re23[cc], mul2(X, xq.re23[cc]));
                    acc.im23[cc] = fma2(Af, acc.im23[cc], mul2(X, xq.im23[cc]));
                }
            } else {
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    acc.re01[cc] = mul2(Af, acc.re01[cc]);
                    acc.im01[cc] = mul2(Af, acc.im01[cc]);
                    acc.re23[cc] = mul2(Af, acc.re23[cc]);
                    acc.im23[cc] = mul2(Af, acc.im23[cc]);
                }
            }
            if (op.fin != BF_NONE) {
                float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    n2 = fma2(acc.re01[cc], acc.re01[cc], n2);
                    n2 = fma2(acc.im01[cc], acc.im01[cc], n2);
                    n2 = fma2(acc.re23[cc], acc.re23[cc], n2);
                    n2 = fma2(acc.im23[cc], acc.im23[cc], n2);
                }
                nrm += (double)n2.x + (double)n2.y;
            }
            SF::store_packed(out, g.stride, h, acc);
        }
        if (op.fin != BF_NONE) tile_reduce(nrm, A, op, t, pid);
    }
}

// ---------------------------------------------------------------------------
// Cluster-resident solve of a small problem.  The paper's first layout keeps
// a whole iterative solver in the SPEs' local stores (Sec. 5, "Data in
// on-chip memory"); the GB300 analogue for lattices of a few thousand sites
// is a thread-block cluster (or one block) that runs the complete solve (the
// same FP64-corrected CG as the rest of the batch) on its own SMs, with the
// problem's fields resident in L2 and cluster barriers in place of kernel
// boundaries: no launch per step, no device-wide synchronisation, and the
// problem finishes on its own clock instead of advancing in lockstep with the
// largest lattice of the batch.  Loads that may see data written earlier in
// the same launch go to L2 (COH = true).
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 256;

__device__ inline double cta_sum(double v) {  // block-wide sum, valid in every thread
    __shared__ double s_bc;
    const double t = block_sum(v);
    if (threadIdx.x == 0) s_bc = t;
    __syncthreads();
    const double r = s_bc;
    __syncthreads();
    return r;
}

// The barrier of a solve that runs on a cluster of CL thread blocks (one
// block: __syncthreads).  The cluster barrier has release/acquire semantics,
// so global writes before it are visible to the cluster's other blocks
// after it (their loads of such data go to L2: COH loads).
template <int CL>
__device__ __forceinline__ void solve_sync() {
    if constexpr (CL == 1) __syncthreads();
    else cooperative_groups::this_cluster().sync();
}

// Sum over the solve's threads, the same value in every thread.  On a
// cluster each block's sum is read by every block from the others' shared
// memory (distributed shared memory) in rank order, so all blocks add the
// same numbers in the same order and take the same decisions.
template <int CL>
__device__ inline double solve_sum(double v) {
    if constexpr (CL == 1) {
        return cta_sum(v);
    } else {
        namespace cg = cooperative_groups;
        __shared__ double s_part, s_tot;
        const double t = block_sum(v);
        if (threadIdx.x == 0) s_part = t;
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int r = 0; r < CL; r++) tot += *cl.map_shared_rank(&s_part, r);
            s_tot = tot;
        }
        cl.sync();  // every block has read s_part before it is written again
        return s_tot;
    }
}

// out (parity p) = a * D in + x over the problem's sites, thread tid of nt;
// returns |out|^2.  Ends with the solve's barrier, so out is visible to all
// of its threads.
template <int SP, int GP, int R, bool DAG, int CL>
__device__ double cta_hop(const Geom& g, const char* gauge, char* out, const char* in, const char* x, double a,
                          int p, int tid, int nt) {
    using SF = SpinorFmt<SP>;
    using T = typename SF::real;
    HopParams P;
    P.g = g;
    P.gauge = gauge;
    const T at = (T)a;
    double nrm = 0.0;
    for (int h = tid; h < g.Vh; h += nt) {
        int c[4], s;
        site_of_half(h, p, g, c, s);
        cpx<T> acc[12];
        hop_dir<SP, GP, R, DAG, 0, true, true>(acc, P, in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 1, false, true>(acc, P, in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 2, false, true>(acc, P, in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 3, false, true>(acc, P, in, p, h, c, s);
        if (x) {
            cpx<T> xv[12];
            SF::template load<true>(x, g.stride, h, xv);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                acc[k].re = fma(at, acc[k].re, xv[k].re);
                acc[k].im = fma(at, acc[k].im, xv[k].im);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 12; k++) acc[k] = cscale(at, acc[k]);
        }
        T n2 = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) n2 += cnorm2(acc[k]);
        nrm += (double)n2;
        SF::store(out, g.stride, h, acc);
    }
    return solve_sum<CL>(nrm);
}

// The whole solve of problem ids[blockIdx.x / CL], on CL blocks.
template <int IP, int CL>
__device__ __forceinline__ void small_solve_body(const BatchArgs& A, const int* ids, const BatchGlobal* G,
                                                 unsigned long long budget_ns) {
    using TI = typename SpinorFmt<IP>::real;
    const int pid = ids[blockIdx.x / CL];
    const BatchProb& Pr = A.probs[pid];
    BatchState& S = A.state[pid];
    const Geom g = Pr.g;
    const double kappa = Pr.kappa, k2 = kappa * kappa;
    char* const* f = Pr.f;
    const char* b_e = f[BF_B];
    const char* b_o = f[BF_B] + Pr.fp[BF_B];
    char* x_e = f[BF_X];
    char* x_o = f[BF_X] + Pr.fp[BF_X];
    const int tid = (int)(blockIdx.x % CL) * (int)blockDim.x + (int)threadIdx.x, nt = CL * (int)blockDim.x;
    // the wall-clock budget, decided the same way in every block of the solve
    auto late = [&]() { return solve_sum<CL>(globaltimer() - G->t_start > budget_ns ? 1.0 : 0.0) > 0.0; };

    // set-up: zeroed iterates, |b|^2, bhat_e = b_e + kappa D_eo b_o
    for (int h = tid; h < g.Vh; h += nt) {
        cpx<double> z64[12];
        cpx<float> z32[12];
        cpx<TI> zl[12];
#pragma unroll
        for (int k = 0; k < 12; k++) {
            z64[k] = {0.0, 0.0};
            z32[k] = {0.f, 0.f};
            zl[k] = {(TI)0.f, (TI)0.f};
        }
        if (!Pr.keep_x) SpinorFmt<P_F64>::store(x_e, g.stride, h, z64);
        SpinorFmt<P_F32>::store(f[BF_XIN], g.stride, h, z32);
        SpinorFmt<IP>::store(f[BF_P], g.stride, h, zl);
    }
    double nb = 0.0;
    for (int h = tid; h < g.Vh; h += nt) {
        cpx<double> v[12], w[12];
        SpinorFmt<P_F64>::load<true>(b_e, g.stride, h, v);
        SpinorFmt<P_F64>::load<true>(b_o, g.stride, h, w);
#pragma unroll
        for (int k = 0; k < 12; k++) nb += cnorm2(v[k]) + cnorm2(w[k]);
    }
    const double bnorm2 = solve_sum<CL>(nb);
    cta_hop<P_F64, P_F64, 18, false, CL>(g, Pr.g64, f[BF_BHAT], b_o, b_e, kappa, 0, tid, nt);
    const double target2 = Pr.tol * Pr.tol * bnorm2;

    int iter = 0, outer = 0, status = 0;
    double gam = 0.0, best2 = HUGE_VAL;  // best2: smallest |r|^2 of the FP64 corrections
    bool first = true;
    while (true) {
        // x_e += xin; r = bhat - Mhat x_e (FP64)
        for (int h = tid; h < g.Vh; h += nt) {
            cpx<double> xv[12];
            cpx<float> ev[12];
            SpinorFmt<P_F64>::load<true>(x_e, g.stride, h, xv);
            SpinorFmt<P_F32>::load<true>(f[BF_XIN], g.stride, h, ev);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                xv[k].re += (double)ev[k].re;
                xv[k].im += (double)ev[k].im;
            }
            SpinorFmt<P_F64>::store(x_e, g.stride, h, xv);
        }
        solve_sync<CL>();
        cta_hop<P_F64, P_F64, 18, false, CL>(g, Pr.g64, f[BF_T64], x_e, nullptr, 1.0, 1, tid, nt);
        cta_hop<P_F64, P_F64, 18, false, CL>(g, Pr.g64, f[BF_Q64], f[BF_T64], x_e, -k2, 0, tid, nt);
        double rn = 0.0;
        for (int h = tid; h < g.Vh; h += nt) {
            cpx<double> bv[12], qv[12];
            SpinorFmt<P_F64>::load<true>(f[BF_BHAT], g.stride, h, bv);
            SpinorFmt<P_F64>::load<true>(f[BF_Q64], g.stride, h, qv);
            cpx<float> sv[12];
            cpx<TI> lv[12], zl[12];
            cpx<float> z32[12];
#pragma unroll
            for (int k = 0; k < 12; k++) {
                bv[k] = csub(bv[k], qv[k]);
                rn += cnorm2(bv[k]);
                sv[k] = {(float)bv[k].re, (float)bv[k].im};
                lv[k] = {(TI)bv[k].re, (TI)bv[k].im};
                z32[k] = {0.f, 0.f};
            }
            // s = r, slow = r, xin = 0 (used only if the solve goes on)
            SpinorFmt<P_F32>::store(f[BF_S], g.stride, h, sv);
            SpinorFmt<IP>::store(f[BF_SLOW], g.stride, h, lv);
            SpinorFmt<P_F32>::store(f[BF_XIN], g.stride, h, z32);
        }
        const double rn2 = solve_sum<CL>(rn);
        if (!isfinite(rn2)) { status = WILSON_ERR_NUMERIC; break; }
        if (rn2 <= target2) break;
        if (outer >= Pr.max_outer || iter >= Pr.maxiter || rn2 > kDivergence * kDivergence * best2) {
            status = WILSON_ERR_NOCONV;
            break;
        }
        best2 = fmin(best2, rn2);
        if (late()) { status = WILSON_ERR_TIMEOUT; break; }
        outer++;
        // r' = Mhat'^dag s; p = r' + beta p (beta = 0 at the start)
        cta_hop<IP, IP, 12, true, CL>(g, Pr.glo, f[BF_T], f[BF_SLOW], nullptr, 1.0, 1, tid, nt);
        const double rr0 = cta_hop<IP, IP, 12, true, CL>(g, Pr.glo, f[BF_R], f[BF_T], f[BF_SLOW], -k2, 0, tid, nt);
        if (!isfinite(rr0)) { status = WILSON_ERR_NUMERIC; break; }
        double beta = (first || !(gam > 0.0)) ? 0.0 : rr0 / gam;
        gam = rr0;
        first = false;
        const double stop = fmax(Pr.delta * sqrt(rn2), sqrt(target2));
        const double stop2 = stop * stop;
        const int iter_cap = min(Pr.maxiter, iter + kInnerCap);
        while (true) {
            for (int h = tid; h < g.Vh; h += nt) {
                cpx<TI> pv[12], rv[12];
                SpinorFmt<IP>::template load<true>(f[BF_P], g.stride, h, pv);
                SpinorFmt<IP>::template load<true>(f[BF_R], g.stride, h, rv);
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    pv[k].re = fma((TI)beta, pv[k].re, rv[k].re);
                    pv[k].im = fma((TI)beta, pv[k].im, rv[k].im);
                }
                SpinorFmt<IP>::store(f[BF_P], g.stride, h, pv);
            }
            solve_sync<CL>();
            cta_hop<IP, IP, 12, false, CL>(g, Pr.glo, f[BF_T], f[BF_P], nullptr, 1.0, 1, tid, nt);
            const double pq = cta_hop<IP, IP, 12, false, CL>(g, Pr.glo, f[BF_Q], f[BF_T], f[BF_P], -k2, 0, tid, nt);
            if (!isfinite(pq)) { status = WILSON_ERR_NUMERIC; break; }
            if (!(pq > 0.0)) break;
            const float alpha = (float)(gam / pq);
            double sn = 0.0;
            for (int h = tid; h < g.Vh; h += nt) {
                cpx<float> xv[12], sv[12];
                cpx<TI> pv[12], qv[12], lv[12];
                SpinorFmt<P_F32>::load<true>(f[BF_XIN], g.stride, h, xv);
                SpinorFmt<P_F32>::load<true>(f[BF_S], g.stride, h, sv);
                SpinorFmt<IP>::template load<true>(f[BF_P], g.stride, h, pv);
                SpinorFmt<IP>::template load<true>(f[BF_Q], g.stride, h, qv);
                float n2 = 0.f;
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    xv[k].re = fmaf(alpha, (float)pv[k].re, xv[k].re);
                    xv[k].im = fmaf(alpha, (float)pv[k].im, xv[k].im);
                    sv[k].re = fmaf(-alpha, (float)qv[k].re, sv[k].re);
                    sv[k].im = fmaf(-alpha, (float)qv[k].im, sv[k].im);
                    n2 += cnorm2(sv[k]);
                    lv[k] = {(TI)sv[k].re, (TI)sv[k].im};
                }
                sn += (double)n2;
                SpinorFmt<P_F32>::store(f[BF_XIN], g.stride, h, xv);
                SpinorFmt<P_F32>::store(f[BF_S], g.stride, h, sv);
                SpinorFmt<IP>::store(f[BF_SLOW], g.stride, h, lv);
            }
            const double ss = solve_sum<CL>(sn);
            iter++;
            if (!isfinite(ss)) { status = WILSON_ERR_NUMERIC; break; }
            if (ss <= stop2 || iter >= iter_cap) break;
            if ((iter & 15) == 0 && late()) break;
            cta_hop<IP, IP, 12, true, CL>(g, Pr.glo, f[BF_T], f[BF_SLOW], nullptr, 1.0, 1, tid, nt);
            const double rr = cta_hop<IP, IP, 12, true, CL>(g, Pr.glo, f[BF_R], f[BF_T], f[BF_SLOW], -k2, 0, tid, nt);
            if (!isfinite(rr)) { status = WILSON_ERR_NUMERIC; break; }
            beta = gam > 0.0 ? rr / gam : 0.0;
            gam = rr;
        }
        if (status) break;
    }
    // x_o = b_o + kappa D_oe x_e; true residual |b - M x|^2 over both parities
    cta_hop<P_F64, P_F64, 18, false, CL>(g, Pr.g64, x_o, x_e, b_o, kappa, 1, tid, nt);
    cta_hop<P_F64, P_F64, 18, false, CL>(g, Pr.g64, f[BF_Q64], x_o, x_e, -kappa, 0, tid, nt);
    cta_hop<P_F64, P_F64, 18, false, CL>(g, Pr.g64, f[BF_T64], x_e, x_o, -kappa, 1, tid, nt);
    double rs = 0.0;
    for (int h = tid; h < g.Vh; h += nt) {
        cpx<double> a[12], m[12];
        SpinorFmt<P_F64>::load<true>(b_e, g.stride, h, a);
        SpinorFmt<P_F64>::load<true>(f[BF_Q64], g.stride, h, m);
#pragma unroll
        for (int k = 0; k < 12; k++) rs += cnorm2(csub(a[k], m[k]));
        SpinorFmt<P_F64>::load<true>(b_o, g.stride, h, a);
        SpinorFmt<P_F64>::load<true>(f[BF_T64], g.stride, h, m);
#pragma unroll
        for (int k = 0; k < 12; k++) rs += cnorm2(csub(a[k], m[k]));
    }
    const double res2 = solve_sum<CL>(rs);
    if (tid == 0) {
        S.sc.iter = iter;
        S.outer = outer;
        S.status = status;
        S.bnorm2 = bnorm2;
        S.res2 = res2;
        S.t_done = globaltimer();
        S.phase = S.next_phase = PH_DONE;
    }
}

// One block per small problem, or a cluster of kSmallCluster blocks on as
// many SMs (the solve's parallel width grows, its barriers become cluster
// barriers and its sums go through distributed shared memory).
constexpr int kSmallCluster = 4;

template <int IP>
__global__ void __launch_bounds__(kSmallThreads, 1) small_solve_kernel(const BatchArgs A, const int* ids,
                                                                       const BatchGlobal* G,
                                                                       unsigned long long budget_ns) {
    small_solve_body<IP, 1>(A, ids, G, budget_ns);
}

template <int IP>
__global__ void __cluster_dims__(kSmallCluster, 1, 1) __launch_bounds__(kSmallThreads, 1)
    small_solve_cluster_kernel(const BatchArgs A, const int* ids, const BatchGlobal* G, unsigned long long budget_ns) {
    small_solve_body<IP, kSmallCluster>(A, ids, G, budget_ns);
}

// The batched hop of F16 / BF16 storage on the pipelined site (pipe_site):
// each thread copies the next hops' raw data into its own shared-memory slots
// (batch variant 22; TB threads per block, D hops ahead, NREG registers).
template <int SP, bool DAG, int NREG, int D, int TB>
__global__ void __launch_bounds__(TB) __maxnreg__(NREG) bhop_kernel_pipe(const BatchArgs A, const BOp op) {
    using SF = SpinorFmt<SP>;
    extern __shared__ __align__(16) unsigned char bpipe_smem[];
    uint4* sp = reinterpret_cast<uint4*>(bpipe_smem);      // [D][3][TB] spinor chunks
    uint2* lk = reinterpret_cast<uint2*>(sp + D * 3 * TB);  // [D][3][TB] link chunks
    float* scs = reinterpret_cast<float*>(lk + D * 3 * TB); // [D][TB] scales
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const int pid = __ldg(A.tile_prob + t);
        if (!tile_active(A, op, pid)) continue;
        const BatchProb& Pr = A.probs[pid];
        const Geom& g = Pr.g;
        const int p = op.out_parity;
        char* out = Pr.f[op.f_out] + p * Pr.fp[op.f_out];
        const char* in = Pr.f[op.f_in] + (1 - p) * Pr.fp[op.f_in];
        const char* x = op.f_x >= 0 ? Pr.f[op.f_x] + p * Pr.fp[op.f_x] : nullptr;
        const float2 Af = bc2((float)coef_of(op.coef, Pr.kappa));
        double nrm = 0.0;
        const int h0 = (t - Pr.tile0) * A.tile;
        for (int j = threadIdx.x; j < A.tile; j += TB) {
            const int h = h0 + j;
            if (h >= g.Vh) break;
            PSpinor acc;
            pipe_site<SP, DAG, D, TB>(acc, in, Pr.glo, g, p, h, sp, lk, scs, threadIdx.x);
            if (x) {
                PSpinor xq;
                float xs;
                SF::load_packed(x, g.stride, h, xq, xs);
                const float2 X = bc2(xs);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    acc.re01[cc] = fma2(Af, acc.re01[cc], mul2(X, xq.re01[cc]));
                    acc.im01[cc] = fma2(Af, acc.im01[cc], mul2(X, xq.im01[cc]));
                    acc.re23[cc] = fma2(Af, acc.re23[cc], mul2(X, xq.re23[cc]));
                    acc.im23[cc] = fma2(Af, acc.im23[cc], mul2(X, xq.im23[cc]));
                }
            } else {
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    acc.re01[cc] = mul2(Af, acc.re01[cc]);
                    acc.im01[cc] = mul2(Af, acc.im01[cc]);
                    acc.re23[cc] = mul2(Af, acc.re23[cc]);
                    acc.im23[cc] = mul2(Af, acc.im23[cc]);
                }
            }
            if (op.fin != BF_NONE) {
                float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    n2 = fma2(acc.re01[cc], acc.re01[cc], n2);
                    n2 = fma2(acc.im01[cc], acc.im01[cc], n2);
                    n2 = fma2(acc.re23[cc], acc.re23[cc], n2);
                    n2 = fma2(acc.im23[cc], acc.im23[cc], n2);
                }
                nrm += (double)n2.x + (double)n2.y;
            }
            SF::store_packed(out, g.stride, h, acc);
        }
        if (op.fin != BF_NONE) tile_reduce(nrm, A, op, t, pid);
    }
}

// ---------------------------------------------------------------------------
// launchers (instantiated in their own translation units)
// ---------------------------------------------------------------------------
// Batched hop: variants 0-2 the scalar stencil (register budgets), 3-5 the
// paired-FP32 stencil (F32 / F16 / BF16 spinors only), 22 the pipelined
// F16 / BF16 stencil (64- or 128-thread blocks).
constexpr int kBatchPipeVariant = 22;  // the pipelined F16 / BF16 stencil (as hop variant 22)
constexpr int kBatchPipeDepth = 3;     // hops copied ahead
template <int SP, int GP>
void launch_bhop(const BatchArgs& A, const BOp& o, int dag, int v, int block, int blocks, cudaStream_t st) {
    constexpr int R = wide_regs(SP) ? 18 : 12;
#define WL_BHOP(V)                                                                                        \
    if (dag) bhop_kernel<SP, GP, R, true, hop_variant_minb(V, SP)><<<blocks, block, 0, st>>>(A, o);     \
    else bhop_kernel<SP, GP, R, false, hop_variant_minb(V, SP)><<<blocks, block, 0, st>>>(A, o);
#define WL_BHOP_P(V)                                                                                      \
    if (dag) bhop_kernel_p<SP, GP, 12, true, hop_variant_minb(V, SP)><<<blocks, block, 0, st>>>(A, o);  \
    else bhop_kernel_p<SP, GP, 12, false, hop_variant_minb(V, SP)><<<blocks, block, 0, st>>>(A, o);
    if constexpr ((SP == P_F16 || SP == P_BF16) && GP == SP) {
        if (v == kBatchPipeVariant) {
            constexpr size_t per_thread = (size_t)kBatchPipeDepth * (3 * 16 + 3 * 8 + 4);
            constexpr int D = kBatchPipeDepth;
            if (block == 64) {
                if (dag) bhop_kernel_pipe<SP, true, 96, D, 64><<<blocks, 64, per_thread * 64, st>>>(A, o);
                else bhop_kernel_pipe<SP, false, 96, D, 64><<<blocks, 64, per_thread * 64, st>>>(A, o);
            } else {
                WL_REQUIRE(block == 128, "the pipelined batch hop takes 64- or 128-thread blocks");
                if (dag) bhop_kernel_pipe<SP, true, 96, D, 128><<<blocks, 128, per_thread * 128, st>>>(A, o);
                else bhop_kernel_pipe<SP, false, 96, D, 128><<<blocks, 128, per_thread * 128, st>>>(A, o);
            }
            return;
        }
    }
    if constexpr (float_storage(SP)) {
        if (v == 3) { WL_BHOP_P(3) return; }
        if (v == 4) { WL_BHOP_P(4) return; }
        if (v == 5) { WL_BHOP_P(5) return; }
    }
    if (v % 3 == 1) { WL_BHOP(1) } else if (v % 3 == 2) { WL_BHOP(2) } else { WL_BHOP(0) }
#undef WL_BHOP
#undef WL_BHOP_P
}

extern template void launch_bhop<P_F32, P_F32>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);
extern template void launch_bhop<P_F16, P_F16>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);
extern template void launch_bhop<P_BF16, P_BF16>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);
extern template void launch_bhop<P_F64, P_F64>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);

// The CTA-resident solves of nprob small problems (ids: their indices), inner
// precision IP.  Instantiated one inner precision per translation unit
// (batch_small_*.cu).
template <int IP>
void launch_small_ip(bool cluster, const BatchArgs& A, const int* ids, const BatchGlobal* G,
                     unsigned long long budget_ns, int nprob, cudaStream_t st) {
    if (cluster)
        small_solve_cluster_kernel<IP><<<nprob * kSmallCluster, kSmallThreads, 0, st>>>(A, ids, G, budget_ns);
    else small_solve_kernel<IP><<<nprob, kSmallThreads, 0, st>>>(A, ids, G, budget_ns);
}

extern template void launch_small_ip<P_F32>(bool, const BatchArgs&, const int*, const BatchGlobal*,
                                            unsigned long long, int, cudaStream_t);
extern template void launch_small_ip<P_F16>(bool, const BatchArgs&, const int*, const BatchGlobal*,
                                            unsigned long long, int, cudaStream_t);
extern template void launch_small_ip<P_BF16>(bool, const BatchArgs&, const int*, const BatchGlobal*,
                                             unsigned long long, int, cudaStream_t);

}  // namespace bt
}  // namespace wl
