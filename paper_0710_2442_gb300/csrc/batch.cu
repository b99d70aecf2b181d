// batch.cu -- many independent solves on lattices of different sizes in one
// CUDA graph launch (wilson_batch_solve).
//
// Every problem keeps its own lattice, links, kappa, fields and CG scalars.
// The half lattices of all problems are cut into tiles of kTile sites; a
// tile table maps every tile to its problem, and every kernel of the batch is
// a persistent grid that walks the tile table, so one launch serves all
// problems whatever their sizes.  Per-problem reductions are tile partials
// summed in a fixed order by the problem's last tile (no block waits for
// another).
//
// Each problem runs the solver of solver.cu (CGNR on the even Schur
// complement; FP64 outer corrections with reliable updates around an inner
// CG in reduced storage precision) as a device-side state machine:
//
//   OUTER:  x_e += e;  r = bhat - Mhat x_e (FP64);  finished if |r| <= tol |b|
//           (or out of budget), else s = r, e = 0, r' = Mhat'^dag s,
//           p = r' + beta p  -> INNER
//   INNER:  one CG iteration (six kernels as in solver.cu) -> OUTER when
//           |s| <= delta |r| (or maxiter)
//
// The graph is: prologue (|b|^2, bhat, zeroed iterates) -> a device-side
// while loop whose body runs the OUTER kernels and the INNER kernels as two
// parallel branches (disjoint problems) and then a one-block commit kernel
// that advances every problem's phase and sets the loop condition -> epilogue
// (x_o = b_o + kappa D_oe x_e, true residuals, completion times).  The commit
// kernel stops the loop after a hard number of iterations or a wall-clock
// budget even if some problem has not finished, so the launch always ends.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/wilson.h"
#include "dslash_impl.cuh"
#include "solver.h"

namespace wl {

namespace {

constexpr int kTile = 256;  // half-lattice sites per tile

enum BField { BF_B, BF_X, BF_BHAT, BF_R64, BF_Q64, BF_T64, BF_XIN, BF_S, BF_SLOW, BF_P, BF_Q, BF_R, BF_T, BF_N };
enum Phase { PH_OUTER = 0, PH_INNER = 1, PH_DONE = 2 };
enum BFin { BF_NONE = -1, BFIN_ALPHA, BFIN_RES, BFIN_BETA, BFIN_START, BFIN_OUTER, BFIN_BNORM, BFIN_TRUE };

struct BatchProb {
    Geom g;
    char* f[BF_N];        // parity block (half fields) or parity-0 block (full fields)
    long long fp[BF_N];   // parity step of full fields, 0 for half fields
    const char* g64;      // FP64 18-real links
    const char* glo;      // inner links
    double kappa, tol, delta;
    int tile0, ntiles;
    int maxiter, max_outer;
    int small;            // 1: solved by one CTA (small_solve_kernel), no tiles
    int keep_x;           // 1: x holds an initial guess
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
};

struct BOp {
    int f_out, f_in, f_x;   // field ids (f_x < 0: no xpay)
    int out_parity;
    int use64;              // links: FP64 (1) or inner (0)
    int coef;               // a = 1, kappa, -kappa^2, -kappa
    int phase;              // only problems in this phase (-1: all)
    int skip_done;          // also skip problems whose inner CG is done
    int fin;                // BFin of the fused reduction (BF_NONE: none)
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
__device__ void batch_finish(int op, const BatchProb& P, BatchState& S, double sum) {
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
            S.rnorm2 = sum;
            if (S.outer == 0 || sum < S.best2) S.best2 = sum;
            const double target2 = P.tol * P.tol * S.bnorm2;
            if (!isfinite(sum)) {
                S.status = WILSON_ERR_NUMERIC;
                S.next_phase = PH_DONE;
            } else if (sum <= target2) {
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
        s_act = act;
    }
    __syncthreads();
    return s_act != 0;
}

// Tile partial + per-problem ticket; the problem's last tile finishes.
__device__ void tile_reduce(double v, const BatchArgs& A, const BOp& op, int t, int pid) {
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
        P.gauge = op.use64 ? Pr.g64 : Pr.glo;
        const int p = op.out_parity;
        char* out = Pr.f[op.f_out] + p * Pr.fp[op.f_out];
        const char* in = Pr.f[op.f_in] + (1 - p) * Pr.fp[op.f_in];
        const char* x = op.f_x >= 0 ? Pr.f[op.f_x] + p * Pr.fp[op.f_x] : nullptr;
        const T a = (T)coef_of(op.coef, Pr.kappa);
        const Geom& g = P.g;
        double nrm = 0.0;
        const int h0 = (t - Pr.tile0) * kTile;
        for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
            const int h = h0 + j;
            if (h >= g.Vh) break;
            int c[4], s;
            site_of_half(h, p, g, c, s);
            cpx<T> acc[12];
            hop_dir<SP, GP, R, DAG, 0, true>(acc, P, in, p, h, c, s);
            hop_dir<SP, GP, R, DAG, 1, false>(acc, P, in, p, h, c, s);
            hop_dir<SP, GP, R, DAG, 2, false>(acc, P, in, p, h, c, s);
            hop_dir<SP, GP, R, DAG, 3, false>(acc, P, in, p, h, c, s);
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
        P.gauge = Pr.glo;
        const int p = op.out_parity;
        char* out = Pr.f[op.f_out] + p * Pr.fp[op.f_out];
        const char* in = Pr.f[op.f_in] + (1 - p) * Pr.fp[op.f_in];
        const char* x = op.f_x >= 0 ? Pr.f[op.f_x] + p * Pr.fp[op.f_x] : nullptr;
        const float a = (float)coef_of(op.coef, Pr.kappa);
        const Geom& g = P.g;
        double nrm = 0.0;
        const int h0 = (t - Pr.tile0) * kTile;
        for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
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
// batched BLAS-1 kernels (all tile-walking, phase-filtered)
// ---------------------------------------------------------------------------
#define WL_TILE_LOOP_BEGIN                                                   \
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {                 \
        const int pid = __ldg(A.tile_prob + t);                              \
        if (!tile_active(A, op, pid)) continue;                              \
        const BatchProb& Pr = A.probs[pid];                                  \
        const Geom& g = Pr.g;                                                \
        const int h0 = (t - Pr.tile0) * kTile;
#define WL_TILE_LOOP_END }

// xin += alpha p; s -= alpha q; slow = s; |s|^2   (INNER)
template <int IP>
__global__ void __launch_bounds__(256) bxs_kernel(const BatchArgs A, const BOp op) {
    using TP = typename SpinorFmt<IP>::real;
    WL_TILE_LOOP_BEGIN
    const float alpha = (float)__ldcg(&A.state[pid].sc.alpha);
    double nrm = 0.0;
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<float> xv[12], sv[12];
        cpx<TP> pv[12], qv[12];
        SpinorFmt<P_F32>::load(Pr.f[BF_XIN], g.stride, h, xv);
        SpinorFmt<P_F32>::load(Pr.f[BF_S], g.stride, h, sv);
        SpinorFmt<IP>::load(Pr.f[BF_P], g.stride, h, pv);
        SpinorFmt<IP>::load(Pr.f[BF_Q], g.stride, h, qv);
        float n2 = 0.f;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            xv[k].re = fmaf(alpha, (float)pv[k].re, xv[k].re);
            xv[k].im = fmaf(alpha, (float)pv[k].im, xv[k].im);
            sv[k].re = fmaf(-alpha, (float)qv[k].re, sv[k].re);
            sv[k].im = fmaf(-alpha, (float)qv[k].im, sv[k].im);
            n2 += cnorm2(sv[k]);
        }
        nrm += (double)n2;
        SpinorFmt<P_F32>::store(Pr.f[BF_XIN], g.stride, h, xv);
        SpinorFmt<P_F32>::store(Pr.f[BF_S], g.stride, h, sv);
        cpx<TP> sl[12];
#pragma unroll
        for (int k = 0; k < 12; k++) sl[k] = {(TP)sv[k].re, (TP)sv[k].im};
        SpinorFmt<IP>::store(Pr.f[BF_SLOW], g.stride, h, sl);
    }
    tile_reduce(nrm, A, op, t, pid);
    WL_TILE_LOOP_END
}

// p = r + beta p
template <int IP>
__global__ void __launch_bounds__(256) bp_kernel(const BatchArgs A, const BOp op) {
    using TP = typename SpinorFmt<IP>::real;
    WL_TILE_LOOP_BEGIN
    const TP beta = (TP)__ldcg(&A.state[pid].sc.beta);
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<TP> pv[12], rv[12];
        SpinorFmt<IP>::load(Pr.f[BF_P], g.stride, h, pv);
        SpinorFmt<IP>::load(Pr.f[BF_R], g.stride, h, rv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            pv[k].re = fma(beta, pv[k].re, rv[k].re);
            pv[k].im = fma(beta, pv[k].im, rv[k].im);
        }
        SpinorFmt<IP>::store(Pr.f[BF_P], g.stride, h, pv);
    }
    WL_TILE_LOOP_END
}

// x_e += xin (FP64 += FP32)   (OUTER)
__global__ void __launch_bounds__(256) baxpy_kernel(const BatchArgs A, const BOp op) {
    WL_TILE_LOOP_BEGIN
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<double> xv[12];
        cpx<float> ev[12];
        SpinorFmt<P_F64>::load(Pr.f[BF_X], g.stride, h, xv);
        SpinorFmt<P_F32>::load(Pr.f[BF_XIN], g.stride, h, ev);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            xv[k].re += (double)ev[k].re;
            xv[k].im += (double)ev[k].im;
        }
        SpinorFmt<P_F64>::store(Pr.f[BF_X], g.stride, h, xv);
    }
    WL_TILE_LOOP_END
}

// r64 = bhat - q64, |r64|^2   (OUTER)
__global__ void __launch_bounds__(256) bxmy_kernel(const BatchArgs A, const BOp op) {
    WL_TILE_LOOP_BEGIN
    double nrm = 0.0;
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<double> bv[12], qv[12];
        SpinorFmt<P_F64>::load(Pr.f[BF_BHAT], g.stride, h, bv);
        SpinorFmt<P_F64>::load(Pr.f[BF_Q64], g.stride, h, qv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            bv[k] = csub(bv[k], qv[k]);
            nrm += cnorm2(bv[k]);
        }
        SpinorFmt<P_F64>::store(Pr.f[BF_R64], g.stride, h, bv);
    }
    tile_reduce(nrm, A, op, t, pid);
    WL_TILE_LOOP_END
}

// s = r64 (F32), slow = r64 (inner), xin = 0   (OUTER)
template <int IP>
__global__ void __launch_bounds__(256) bprep_kernel(const BatchArgs A, const BOp op) {
    using TP = typename SpinorFmt<IP>::real;
    WL_TILE_LOOP_BEGIN
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<double> rv[12];
        SpinorFmt<P_F64>::load(Pr.f[BF_R64], g.stride, h, rv);
        cpx<float> sv[12], z[12];
        cpx<TP> lv[12];
#pragma unroll
        for (int k = 0; k < 12; k++) {
            sv[k] = {(float)rv[k].re, (float)rv[k].im};
            lv[k] = {(TP)rv[k].re, (TP)rv[k].im};
            z[k] = {0.f, 0.f};
        }
        SpinorFmt<P_F32>::store(Pr.f[BF_S], g.stride, h, sv);
        SpinorFmt<IP>::store(Pr.f[BF_SLOW], g.stride, h, lv);
        SpinorFmt<P_F32>::store(Pr.f[BF_XIN], g.stride, h, z);
    }
    WL_TILE_LOOP_END
}

// |v|^2 of an FP64 field (parity op.out_parity); |b - m|^2 with op.f_x = m
__global__ void __launch_bounds__(256) bnorm_kernel(const BatchArgs A, const BOp op) {
    WL_TILE_LOOP_BEGIN
    const char* v = Pr.f[op.f_in] + op.out_parity * Pr.fp[op.f_in];
    const char* m = op.f_x >= 0 ? Pr.f[op.f_x] + op.out_parity * Pr.fp[op.f_x] : nullptr;
    double nrm = 0.0;
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<double> vv[12];
        SpinorFmt<P_F64>::load(v, g.stride, h, vv);
        if (m) {
            cpx<double> mv[12];
            SpinorFmt<P_F64>::load(m, g.stride, h, mv);
#pragma unroll
            for (int k = 0; k < 12; k++) vv[k] = csub(vv[k], mv[k]);
        }
#pragma unroll
        for (int k = 0; k < 12; k++) nrm += cnorm2(vv[k]);
    }
    tile_reduce(nrm, A, op, t, pid);
    WL_TILE_LOOP_END
}

// zero x_e (unless a guess is given), xin, p; reset the state machine
template <int IP>
__global__ void __launch_bounds__(256) binit_kernel(const BatchArgs A, const BOp op, int keep_x, BatchGlobal* G) {
    using TP = typename SpinorFmt<IP>::real;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        G->t_start = globaltimer();
        G->iterations = 0;
        G->timed_out = 0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nprob; i += gridDim.x * blockDim.x) {
        BatchState& S = A.state[i];
        S = BatchState{};
        // small problems are solved by their own CTA: the loop skips them
        S.phase = S.next_phase = A.probs[i].small ? PH_DONE : PH_OUTER;
        S.first = 1;
        S.sc.maxiter = A.probs[i].maxiter;
    }
    WL_TILE_LOOP_BEGIN
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<double> z64[12];
        cpx<float> z32[12];
        cpx<TP> zl[12];
#pragma unroll
        for (int k = 0; k < 12; k++) {
            z64[k] = {0.0, 0.0};
            z32[k] = {0.f, 0.f};
            zl[k] = {(TP)0.f, (TP)0.f};
        }
        if (!keep_x) SpinorFmt<P_F64>::store(Pr.f[BF_X], g.stride, h, z64);
        SpinorFmt<P_F32>::store(Pr.f[BF_XIN], g.stride, h, z32);
        SpinorFmt<IP>::store(Pr.f[BF_P], g.stride, h, zl);
    }
    WL_TILE_LOOP_END
}

// One block: advance every problem's phase, decide whether the loop goes on.
__global__ void bcommit_kernel(BatchState* state, int nprob, BatchGlobal* G, cudaGraphConditionalHandle handle,
                               int use_handle, int max_iterations, unsigned long long budget_ns) {
    __shared__ int s_active;
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nprob; i += blockDim.x) {
        BatchState& S = state[i];
        S.phase = S.next_phase;
        if (S.phase != PH_DONE) atomicOr(&s_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int it = G->iterations + 1;
        G->iterations = it;
        int go = s_active;
        if (go && (it >= max_iterations || globaltimer() - G->t_start > budget_ns)) {
            G->timed_out = 1;
            go = 0;
        }
        if (use_handle) cudaGraphSetConditional(handle, go ? 1u : 0u);
    }
}

__global__ void bfinal_kernel(BatchGlobal* G) { G->t_end = globaltimer(); }

// ---------------------------------------------------------------------------
// CTA-resident solve of a small problem.  The paper's first layout keeps a
// whole iterative solver in the SPEs' local stores (Sec. 5, "Data in on-chip
// memory"); the GB300 analogue for lattices of a few thousand sites is one
// thread block that runs the complete solve (the same FP64-corrected CG as
// the rest of the batch) on its own SM, with the problem's fields resident in
// L1/L2 and block barriers in place of kernel boundaries: no launch per step,
// no device-wide synchronisation, and the problem finishes on its own clock
// instead of advancing in lockstep with the largest lattice of the batch.
// Loads that may see data written earlier in the same launch use the
// coherent path (COH = true).
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 256;

__device__ double cta_sum(double v) {  // block-wide sum, valid in every thread
    __shared__ double s_bc;
    const double t = block_sum(v);
    if (threadIdx.x == 0) s_bc = t;
    __syncthreads();
    const double r = s_bc;
    __syncthreads();
    return r;
}

// out (parity p) = a * D in + x over the problem's sites; returns |out|^2.
// Ends with a block barrier, so out is visible to the whole block.
template <int SP, int GP, int R, bool DAG>
__device__ double cta_hop(const Geom& g, const char* gauge, char* out, const char* in, const char* x, double a,
                          int p) {
    using SF = SpinorFmt<SP>;
    using T = typename SF::real;
    HopParams P;
    P.g = g;
    P.gauge = gauge;
    const T at = (T)a;
    double nrm = 0.0;
    for (int h = threadIdx.x; h < g.Vh; h += blockDim.x) {
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
    return cta_sum(nrm);
}

template <int IP>
__global__ void __launch_bounds__(kSmallThreads, 1) small_solve_kernel(const BatchArgs A, const int* ids,
                                                                       const BatchGlobal* G,
                                                                       unsigned long long budget_ns) {
    using TI = typename SpinorFmt<IP>::real;
    const int pid = ids[blockIdx.x];
    const BatchProb& Pr = A.probs[pid];
    BatchState& S = A.state[pid];
    const Geom g = Pr.g;
    const double kappa = Pr.kappa, k2 = kappa * kappa;
    char* const* f = Pr.f;
    const char* b_e = f[BF_B];
    const char* b_o = f[BF_B] + Pr.fp[BF_B];
    char* x_e = f[BF_X];
    char* x_o = f[BF_X] + Pr.fp[BF_X];
    const int tid = threadIdx.x, nt = blockDim.x;

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
    const double bnorm2 = cta_sum(nb);
    cta_hop<P_F64, P_F64, 18, false>(g, Pr.g64, f[BF_BHAT], b_o, b_e, kappa, 0);
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
        __syncthreads();
        cta_hop<P_F64, P_F64, 18, false>(g, Pr.g64, f[BF_T64], x_e, nullptr, 1.0, 1);
        cta_hop<P_F64, P_F64, 18, false>(g, Pr.g64, f[BF_Q64], f[BF_T64], x_e, -k2, 0);
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
        const double rn2 = cta_sum(rn);
        if (!isfinite(rn2)) { status = WILSON_ERR_NUMERIC; break; }
        if (rn2 <= target2) break;
        if (outer >= Pr.max_outer || iter >= Pr.maxiter || rn2 > kDivergence * kDivergence * best2) {
            status = WILSON_ERR_NOCONV;
            break;
        }
        best2 = fmin(best2, rn2);
        if (globaltimer() - G->t_start > budget_ns) { status = WILSON_ERR_TIMEOUT; break; }
        outer++;
        // r' = Mhat'^dag s; p = r' + beta p (beta = 0 at the start)
        cta_hop<IP, IP, 12, true>(g, Pr.glo, f[BF_T], f[BF_SLOW], nullptr, 1.0, 1);
        const double rr0 = cta_hop<IP, IP, 12, true>(g, Pr.glo, f[BF_R], f[BF_T], f[BF_SLOW], -k2, 0);
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
            __syncthreads();
            cta_hop<IP, IP, 12, false>(g, Pr.glo, f[BF_T], f[BF_P], nullptr, 1.0, 1);
            const double pq = cta_hop<IP, IP, 12, false>(g, Pr.glo, f[BF_Q], f[BF_T], f[BF_P], -k2, 0);
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
            const double ss = cta_sum(sn);
            iter++;
            if (!isfinite(ss)) { status = WILSON_ERR_NUMERIC; break; }
            if (ss <= stop2 || iter >= iter_cap) break;
            if ((iter & 15) == 0 && globaltimer() - G->t_start > budget_ns) break;
            cta_hop<IP, IP, 12, true>(g, Pr.glo, f[BF_T], f[BF_SLOW], nullptr, 1.0, 1);
            const double rr = cta_hop<IP, IP, 12, true>(g, Pr.glo, f[BF_R], f[BF_T], f[BF_SLOW], -k2, 0);
            if (!isfinite(rr)) { status = WILSON_ERR_NUMERIC; break; }
            beta = gam > 0.0 ? rr / gam : 0.0;
            gam = rr;
        }
        if (status) break;
    }
    // x_o = b_o + kappa D_oe x_e; true residual |b - M x|^2 over both parities
    cta_hop<P_F64, P_F64, 18, false>(g, Pr.g64, x_o, x_e, b_o, kappa, 1);
    cta_hop<P_F64, P_F64, 18, false>(g, Pr.g64, f[BF_Q64], x_o, x_e, -kappa, 0);
    cta_hop<P_F64, P_F64, 18, false>(g, Pr.g64, f[BF_T64], x_e, x_o, -kappa, 1);
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
    const double res2 = cta_sum(rs);
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct HostProb {
    Geom g;
    GaugeField g64, glo;
    SpinorField f[BF_N];
    double kappa;
};

template <class F>
void dispatch_low(Prec p, F&& f) {
    switch (p) {
        case P_F16: f(std::integral_constant<int, P_F16>{}); break;
        case P_BF16: f(std::integral_constant<int, P_BF16>{}); break;
        case P_F32: f(std::integral_constant<int, P_F32>{}); break;
        default: throw Error(7, "batched solve: inner precision must be F32, F16 or BF16");
    }
}

}  // namespace

struct BatchRun {
    int nprob = 0, ntiles = 0, sms = 1;
    Prec ip = P_F16;
    std::vector<int> members;  // global problem ids of this run's problems (local order)
    DevBuf probs, state, tile_prob, global, partials, counters, ids;
    BatchArgs A{};
    int grid = 1;
    LaunchConfig hop_lo{128, 1}, hop_64{128, 0};
    cudaGraphConditionalHandle handle{};
    BatchGlobal* G() const { return global.as<BatchGlobal>(); }

    BOp op(int f_out, int f_in, int f_x, int parity, int use64, int coef, int phase, int skip_done, int fin,
           int rslot) const {
        BOp o;
        o.f_out = f_out;
        o.f_in = f_in;
        o.f_x = f_x;
        o.out_parity = parity;
        o.use64 = use64;
        o.coef = coef;
        o.phase = phase;
        o.skip_done = skip_done;
        o.fin = fin;
        o.partials = partials.as<double>() + (size_t)rslot * ntiles;
        o.counters = counters.as<unsigned int>() + (size_t)rslot * nprob;
        return o;
    }

    template <int SP, int GP>
    void hop_t(const BOp& o, int dag, const LaunchConfig& c, cudaStream_t st) const {
        const int v = c.variant;
        const int blocks = grid;
#define WL_BHOP(V)                                                                                  \
    if (dag) bhop_kernel<SP, GP, (SP == P_F64 ? 18 : 12), true, hop_variant_minb(V, SP)>           \
                 <<<blocks, c.block, 0, st>>>(A, o);                                                \
    else bhop_kernel<SP, GP, (SP == P_F64 ? 18 : 12), false, hop_variant_minb(V, SP)>              \
             <<<blocks, c.block, 0, st>>>(A, o);
#define WL_BHOP_P(V)                                                                                \
    if (dag) bhop_kernel_p<SP, GP, 12, true, hop_variant_minb(V, SP)><<<blocks, c.block, 0, st>>>(A, o); \
    else bhop_kernel_p<SP, GP, 12, false, hop_variant_minb(V, SP)><<<blocks, c.block, 0, st>>>(A, o);
        // variants 0-2: scalar stencil, 3-5: paired-FP32 stencil (not for FP64)
        if constexpr (SP != P_F64) {
            if (v == 3) { WL_BHOP_P(3) return; }
            if (v == 4) { WL_BHOP_P(4) return; }
            if (v == 5) { WL_BHOP_P(5) return; }
        }
        if (v % 3 == 1) { WL_BHOP(1) } else if (v % 3 == 2) { WL_BHOP(2) } else { WL_BHOP(0) }
#undef WL_BHOP
#undef WL_BHOP_P
    }
    void hop(const BOp& o, int dag, cudaStream_t st) const {
        if (o.use64) {
            hop_t<P_F64, P_F64>(o, dag, hop_64, st);
        } else {
            dispatch_low(ip, [&](auto I) { hop_t<decltype(I)::value, decltype(I)::value>(o, dag, hop_lo, st); });
        }
        WL_LAUNCH_CHECK();
    }
};

namespace {

void build_problem(HostProb& P, const wilson_problem& in, Prec ip, const SolveParams& prm, cudaStream_t st) {
    P.g = make_geom(in.L.dims, in.L.bc_phase);
    P.kappa = in.kappa;
    P.g64.prec = P_F64;
    P.g64.recon = 18;
    P.g64.g = P.g;
    P.g64.buf.alloc(gauge_bytes(P_F64, 18, P.g.stride));
    pack_gauge(P.g64, in.gauge, st);
    P.glo.prec = ip;
    P.glo.recon = 12;
    P.glo.g = P.g;
    P.glo.buf.alloc(gauge_bytes(ip, 12, P.g.stride));
    pack_gauge(P.glo, in.gauge, st);
    P.f[BF_B].alloc(P_F64, 2, 1, P.g);
    P.f[BF_X].alloc(P_F64, 2, 1, P.g);
    P.f[BF_BHAT].alloc(P_F64, 0, 1, P.g);
    P.f[BF_R64].alloc(P_F64, 0, 1, P.g);
    P.f[BF_Q64].alloc(P_F64, 0, 1, P.g);
    P.f[BF_T64].alloc(P_F64, 1, 1, P.g);
    P.f[BF_XIN].alloc(P_F32, 0, 1, P.g);
    P.f[BF_S].alloc(P_F32, 0, 1, P.g);
    P.f[BF_SLOW].alloc(ip, 0, 1, P.g);
    P.f[BF_P].alloc(ip, 0, 1, P.g);
    P.f[BF_Q].alloc(ip, 0, 1, P.g);
    P.f[BF_R].alloc(ip, 0, 1, P.g);
    P.f[BF_T].alloc(ip, 1, 1, P.g);
    pack_spinor(P.f[BF_B], 0, in.b, st);
    if (prm.use_initial_guess) pack_spinor(P.f[BF_X], 0, in.x, st);
}

// Device descriptors, states and the tile table of one run.
std::unique_ptr<BatchRun> make_run(const std::vector<HostProb>& hp, const std::vector<int>& members, bool small,
                                   const SolveParams& prm, cudaStream_t st) {
    auto R = std::make_unique<BatchRun>();
    R->members = members;
    R->nprob = (int)members.size();
    R->ip = prm.inner;
    R->sms = device_sm_count();
    std::vector<BatchProb> desc(R->nprob);
    std::vector<int> tiles, ids;
    for (int j = 0; j < R->nprob; j++) {
        const HostProb& P = hp[members[j]];
        BatchProb& D = desc[j];
        std::memset(&D, 0, sizeof(D));
        D.g = P.g;
        for (int f = 0; f < BF_N; f++) {
            const int parity = P.f[f].subset == 2 ? 0 : P.f[f].subset;
            D.f[f] = static_cast<char*>(P.f[f].block(parity));
            D.fp[f] = P.f[f].subset == 2 ? P.f[f].pbytes : 0;
        }
        D.g64 = P.g64.buf.as<const char>();
        D.glo = P.glo.buf.as<const char>();
        D.kappa = P.kappa;
        D.tol = prm.tol;
        D.delta = prm.delta > 0 ? prm.delta : default_delta(R->ip);
        D.maxiter = prm.maxiter;
        D.max_outer = prm.max_restarts;
        D.keep_x = prm.use_initial_guess;
        D.small = small ? 1 : 0;
        D.tile0 = (int)tiles.size();
        D.ntiles = small ? 0 : (P.g.Vh + kTile - 1) / kTile;
        for (int t = 0; t < D.ntiles; t++) tiles.push_back(j);
        ids.push_back(j);
    }
    R->ntiles = (int)tiles.size();
    constexpr int kRed = 6;  // reduction slots: prologue/epilogue, A4, A7, B2, B3, B5
    R->probs.alloc(sizeof(BatchProb) * R->nprob);
    R->state.alloc(sizeof(BatchState) * R->nprob);
    R->tile_prob.alloc(sizeof(int) * std::max(R->ntiles, 1));
    R->ids.alloc(sizeof(int) * R->nprob);
    R->global.alloc(sizeof(BatchGlobal));
    R->partials.alloc(sizeof(double) * (size_t)kRed * std::max(R->ntiles, 1));
    R->counters.alloc(sizeof(unsigned int) * (size_t)kRed * R->nprob);
    WL_CUDA(cudaMemcpyAsync(R->probs.p, desc.data(), sizeof(BatchProb) * R->nprob, cudaMemcpyHostToDevice, st));
    WL_CUDA(cudaMemcpyAsync(R->ids.p, ids.data(), sizeof(int) * R->nprob, cudaMemcpyHostToDevice, st));
    if (R->ntiles)
        WL_CUDA(cudaMemcpyAsync(R->tile_prob.p, tiles.data(), sizeof(int) * R->ntiles, cudaMemcpyHostToDevice, st));
    WL_CUDA(cudaMemsetAsync(R->counters.p, 0, sizeof(unsigned int) * kRed * R->nprob, st));
    WL_CUDA(cudaMemsetAsync(R->state.p, 0, sizeof(BatchState) * R->nprob, st));
    WL_CUDA(cudaMemsetAsync(R->global.p, 0, sizeof(BatchGlobal), st));
    R->A.probs = R->probs.as<BatchProb>();
    R->A.state = R->state.as<BatchState>();
    R->A.tile_prob = R->tile_prob.as<int>();
    R->A.ntiles = R->ntiles;
    R->A.nprob = R->nprob;
    // blocks per SM of the tile-walking kernels; 0 (default): one block per
    // tile, so that the block scheduler can interleave the classes' kernels
    // tile by tile in priority order
    int per_sm = 0;
    if (const char* e = std::getenv("WILSON_BATCH_GRID_PER_SM")) per_sm = std::max(0, std::atoi(e));
    R->grid = std::max(1, per_sm ? std::min(R->ntiles, per_sm * R->sms) : R->ntiles);
    return R;
}

// Give every kernel node of g the launch priority prio.
void set_kernel_priority(cudaGraph_t g, int prio) {
    size_t n = 0;
    WL_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    WL_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        WL_CUDA(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeAttrValue v{};
        v.priority = prio;
        WL_CUDA(cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &v));
    }
}

// Group the loop problems by lattice size: one class per distinct half
// volume, merged into at most max_classes classes of neighbouring sizes.
std::vector<std::vector<int>> size_classes(const std::vector<HostProb>& hp, const std::vector<int>& ids,
                                           int max_classes) {
    std::vector<int> sizes;
    for (int i : ids) sizes.push_back(hp[i].g.Vh);
    std::sort(sizes.begin(), sizes.end());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    const int nd = (int)sizes.size();
    const int nc = std::max(1, std::min(max_classes, nd));
    std::vector<std::vector<int>> cls(nc);
    for (int i : ids) {
        const int rank = (int)(std::lower_bound(sizes.begin(), sizes.end(), hp[i].g.Vh) - sizes.begin());
        cls[(long long)rank * nc / std::max(nd, 1)].push_back(i);
    }
    cls.erase(std::remove_if(cls.begin(), cls.end(), [](const std::vector<int>& c) { return c.empty(); }), cls.end());
    return cls;
}

}  // namespace

// Build, run and tear down one batch; fills stats[n] and info.
void batch_solve(int n, const wilson_problem* probs, const SolveParams& prm, wilson_solve_stats* stats,
                 wilson_batch_info* info, cudaStream_t st) {
    NvtxRange nvtx_batch("wilson batch solve");
    auto t0 = std::chrono::steady_clock::now();
    const Prec ip = prm.inner;
    std::vector<HostProb> hp(n);
    for (int i = 0; i < n; i++) build_problem(hp[i], probs[i], ip, prm, st);

    // Problems with at most small_vh sites per parity get their own CTA; the
    // others run device loops, one per class of lattice sizes.
    int small_vh = prm.batch_small_vh;
    if (const char* e = std::getenv("WILSON_BATCH_SMALL_VH")) small_vh = std::atoi(e);
    int max_classes = 4;
    if (const char* e = std::getenv("WILSON_BATCH_CLASSES"))
        if (std::atoi(e) > 0) max_classes = std::atoi(e);
    std::vector<int> small_ids, loop_ids;
    for (int i = 0; i < n; i++) (hp[i].g.Vh <= small_vh ? small_ids : loop_ids).push_back(i);
    std::vector<std::unique_ptr<BatchRun>> loops;
    for (const auto& c : size_classes(hp, loop_ids, max_classes)) loops.push_back(make_run(hp, c, false, prm, st));
    std::unique_ptr<BatchRun> smallrun;
    if (!small_ids.empty()) smallrun = make_run(hp, small_ids, true, prm, st);

    // Loop limits: an iteration cap every problem's own caps fit into, and a
    // wall-clock budget.  WILSON_BATCH_MAX_LOOP / WILSON_BATCH_BUDGET_MS lower
    // them (used by the tests that make the limit run out).
    int max_iter = std::min(2 * prm.maxiter + 4 * prm.max_restarts + 16, 4000000);
    unsigned long long budget_ns = 60ULL * 1000000000ULL;
    if (const char* e = std::getenv("WILSON_BATCH_MAX_LOOP"))
        if (std::atoi(e) > 0) max_iter = std::min(max_iter, std::atoi(e));
    if (const char* e = std::getenv("WILSON_BATCH_BUDGET_MS"))
        if (std::atoll(e) > 0) budget_ns = std::min(budget_ns, (unsigned long long)std::atoll(e) * 1000000ULL);

    // tune the batched hop kernels of every loop class (non-reducing launches on scratch fields)
    std::vector<LaunchConfig> cands, cands64;
    for (const LaunchConfig& c : hop_candidates()) {
        cands.push_back(c);
        if (c.variant < 3) cands64.push_back(c);
    }
    for (auto& R : loops) {
        char key[96];
        snprintf(key, sizeof(key), "bhop:lo%d:n%d:t%d", (int)ip, R->nprob, R->ntiles);
        const BOp o = R->op(BF_Q, BF_T, BF_P, 0, 0, 2, -1, 0, BF_NONE, 0);
        BatchRun* Rp = R.get();
        R->hop_lo = tune_launch(key, cands, LaunchConfig{128, 1}, st, [&](const LaunchConfig& c) {
            dispatch_low(ip, [&](auto I) { Rp->hop_t<decltype(I)::value, decltype(I)::value>(o, 0, c, st); });
        });
        snprintf(key, sizeof(key), "bhop:f64:n%d:t%d", R->nprob, R->ntiles);
        const BOp o64 = R->op(BF_Q64, BF_T64, BF_X, 0, 1, 2, -1, 0, BF_NONE, 0);
        R->hop_64 = tune_launch(key, cands64, LaunchConfig{128, 0}, st,
                                [&](const LaunchConfig& c) { Rp->hop_t<P_F64, P_F64>(o64, 0, c, st); });
    }

    cudaStream_t st2 = nullptr, st3 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, fork3 = nullptr, join3 = nullptr;
    WL_CUDA(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    WL_CUDA(cudaStreamCreateWithFlags(&st3, cudaStreamNonBlocking));
    WL_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    WL_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    WL_CUDA(cudaEventCreateWithFlags(&fork3, cudaEventDisableTiming));
    WL_CUDA(cudaEventCreateWithFlags(&join3, cudaEventDisableTiming));
    struct Cleanup {
        cudaStream_t s[2];
        cudaEvent_t e[4];
        ~Cleanup() {
            for (cudaStream_t x : s)
                if (x) cudaStreamDestroy(x);
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } cleanup{{st2, st3}, {fork, join, fork3, join3}};

    auto blas = [&](const BatchRun& R, auto kernel, const BOp& o, cudaStream_t s) {
        kernel<<<R.grid, 256, 0, s>>>(R.A, o);
        WL_LAUNCH_CHECK();
    };
    auto prologue = [&](const BatchRun& R, cudaStream_t s) {
        dispatch_low(ip, [&](auto I) {
            binit_kernel<decltype(I)::value><<<R.grid, 256, 0, s>>>(
                R.A, R.op(0, 0, -1, 0, 0, 0, -1, 0, BF_NONE, 0), prm.use_initial_guess, R.G());
        });
        WL_LAUNCH_CHECK();
        if (!R.ntiles) return;
        blas(R, bnorm_kernel, R.op(0, BF_B, -1, 0, 0, 0, -1, 0, BFIN_BNORM, 0), s);
        blas(R, bnorm_kernel, R.op(0, BF_B, -1, 1, 0, 0, -1, 0, BFIN_BNORM, 0), s);
        // bhat_e = b_e + kappa D_eo b_o
        R.hop(R.op(BF_BHAT, BF_B, BF_B, 0, 1, 1, -1, 0, BF_NONE, 0), 0, s);
    };
    auto body = [&](const BatchRun& R, int use_handle, cudaStream_t s) {
        WL_CUDA(cudaEventRecord(fork, s));
        WL_CUDA(cudaStreamWaitEvent(st2, fork, 0));
        // branch A (OUTER problems) on s
        blas(R, baxpy_kernel, R.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0, BF_NONE, 1), s);
        R.hop(R.op(BF_T64, BF_X, -1, 1, 1, 0, PH_OUTER, 0, BF_NONE, 1), 0, s);
        R.hop(R.op(BF_Q64, BF_T64, BF_X, 0, 1, 2, PH_OUTER, 0, BF_NONE, 1), 0, s);
        blas(R, bxmy_kernel, R.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0, BFIN_OUTER, 1), s);
        dispatch_low(ip, [&](auto I) {
            bprep_kernel<decltype(I)::value><<<R.grid, 256, 0, s>>>(R.A, R.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0,
                                                                              BF_NONE, 2));
        });
        WL_LAUNCH_CHECK();
        R.hop(R.op(BF_T, BF_SLOW, -1, 1, 0, 0, PH_OUTER, 0, BF_NONE, 2), 1, s);
        R.hop(R.op(BF_R, BF_T, BF_SLOW, 0, 0, 2, PH_OUTER, 0, BFIN_START, 2), 1, s);
        dispatch_low(ip, [&](auto I) {
            bp_kernel<decltype(I)::value><<<R.grid, 256, 0, s>>>(R.A, R.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0, BF_NONE,
                                                                           2));
        });
        WL_LAUNCH_CHECK();
        // branch B (INNER problems) on st2
        R.hop(R.op(BF_T, BF_P, -1, 1, 0, 0, PH_INNER, 1, BF_NONE, 3), 0, st2);
        R.hop(R.op(BF_Q, BF_T, BF_P, 0, 0, 2, PH_INNER, 1, BFIN_ALPHA, 3), 0, st2);
        dispatch_low(ip, [&](auto I) {
            bxs_kernel<decltype(I)::value><<<R.grid, 256, 0, st2>>>(R.A, R.op(0, 0, -1, 0, 0, 0, PH_INNER, 1,
                                                                              BFIN_RES, 4));
        });
        WL_LAUNCH_CHECK();
        R.hop(R.op(BF_T, BF_SLOW, -1, 1, 0, 0, PH_INNER, 1, BF_NONE, 5), 1, st2);
        R.hop(R.op(BF_R, BF_T, BF_SLOW, 0, 0, 2, PH_INNER, 1, BFIN_BETA, 5), 1, st2);
        dispatch_low(ip, [&](auto I) {
            bp_kernel<decltype(I)::value><<<R.grid, 256, 0, st2>>>(R.A, R.op(0, 0, -1, 0, 0, 0, PH_INNER, 1,
                                                                             BF_NONE, 5));
        });
        WL_LAUNCH_CHECK();
        WL_CUDA(cudaEventRecord(join, st2));
        WL_CUDA(cudaStreamWaitEvent(s, join, 0));
        bcommit_kernel<<<1, 256, 0, s>>>(R.A.state, R.nprob, R.G(), R.handle, use_handle, max_iter, budget_ns);
        WL_LAUNCH_CHECK();
    };
    auto epilogue = [&](const BatchRun& R, cudaStream_t s) {
        if (R.ntiles) {
            // x_o = b_o + kappa D_oe x_e
            R.hop(R.op(BF_X, BF_X, BF_B, 1, 1, 1, -1, 0, BF_NONE, 0), 0, s);
            // M x per parity into q64 (even) and t64 (odd); |b - M x|^2
            R.hop(R.op(BF_Q64, BF_X, BF_X, 0, 1, 3, -1, 0, BF_NONE, 0), 0, s);
            R.hop(R.op(BF_T64, BF_X, BF_X, 1, 1, 3, -1, 0, BF_NONE, 0), 0, s);
            blas(R, bnorm_kernel, R.op(0, BF_B, BF_Q64, 0, 0, 0, -1, 0, BFIN_TRUE, 0), s);
            blas(R, bnorm_kernel, R.op(0, BF_B, BF_T64, 1, 0, 0, -1, 0, BFIN_TRUE, 0), s);
        }
        bfinal_kernel<<<1, 1, 0, s>>>(R.G());
        WL_LAUNCH_CHECK();
    };
    // the small problems' CTA-resident solves, concurrent with the loops
    auto small_fork = [&](cudaStream_t s) {
        if (!smallrun) return;
        WL_CUDA(cudaEventRecord(fork3, s));
        WL_CUDA(cudaStreamWaitEvent(st3, fork3, 0));
        dispatch_low(ip, [&](auto I) {
            small_solve_kernel<decltype(I)::value><<<smallrun->nprob, kSmallThreads, 0, st3>>>(
                smallrun->A, smallrun->ids.as<int>(), smallrun->G(), budget_ns);
        });
        WL_LAUNCH_CHECK();
        WL_CUDA(cudaEventRecord(join3, st3));
    };
    auto small_join = [&](cudaStream_t s) {
        if (smallrun) WL_CUDA(cudaStreamWaitEvent(s, join3, 0));
    };

    // ------------------------------------------------------------------ graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraph_t> bodies;
    // WILSON_BATCH_HOST_LOOP=1 selects the host-driven loop (the path taken
    // where conditional graph nodes are unavailable)
    int use_cond = 1;
    if (const char* e = std::getenv("WILSON_BATCH_HOST_LOOP")) use_cond = std::atoi(e) ? 0 : 1;
    WL_CUDA(cudaGraphCreate(&graph, 0));
    for (auto& R : loops)
        if (use_cond &&
            cudaGraphConditionalHandleCreate(&R->handle, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            cudaGetLastError();
            use_cond = 0;
        }
    // The classes' loops share the SMs.  Blocks of a smaller class's kernels
    // are scheduled ahead of pending blocks of larger classes (graph node
    // priorities), so small lattices finish at their own pace instead of
    // queueing behind the largest lattice's sweeps.  WILSON_BATCH_PRIORITY=0
    // turns this off.
    int prio_least = 0, prio_greatest = 0;
    WL_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    int prioritise = loops.size() > 1 && prio_greatest < prio_least;
    if (const char* e = std::getenv("WILSON_BATCH_PRIORITY")) prioritise = prioritise && std::atoi(e) != 0;
    auto class_priority = [&](int c) { return std::min(prio_least, prio_greatest + c); };
    int graph_launches = 0;
    try {
        if (use_cond) {
            WL_CUDA(cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            for (auto& R : loops) prologue(*R, st);
            if (smallrun) prologue(*smallrun, st);
            small_fork(st);
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            WL_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
            const std::vector<cudaGraphNode_t> prologue_tail(deps, deps + ndeps);
            // one device-side while loop per size class, as parallel branches
            std::vector<cudaGraphNode_t> cnodes;
            for (auto& R : loops) {
                cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
                cp.conditional.handle = R->handle;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                cudaGraphNode_t cnode;
                WL_CUDA(cudaGraphAddNode(&cnode, graph, prologue_tail.data(), nullptr, prologue_tail.size(), &cp));
                cnodes.push_back(cnode);
                bodies.push_back(cp.conditional.phGraph_out[0]);
            }
            if (!cnodes.empty())
                WL_CUDA(cudaStreamUpdateCaptureDependencies(st, cnodes.data(), nullptr, cnodes.size(),
                                                            cudaStreamSetCaptureDependencies));
            small_join(st);
            for (auto& R : loops) epilogue(*R, st);
            if (smallrun) epilogue(*smallrun, st);
            cudaGraph_t out = nullptr;
            WL_CUDA(cudaStreamEndCapture(st, &out));
            for (size_t c = 0; c < loops.size(); c++) {
                WL_CUDA(cudaStreamBeginCaptureToGraph(st, bodies[c], nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal));
                body(*loops[c], 1, st);
                WL_CUDA(cudaStreamEndCapture(st, &out));
                if (prioritise) set_kernel_priority(bodies[c], class_priority((int)c));
            }
            WL_CUDA(cudaGraphInstantiate(&exec, graph, prioritise ? cudaGraphInstantiateFlagUseNodePriority : 0));
            WL_CUDA(cudaGraphLaunch(exec, st));
            graph_launches = 1;
        } else {
            // without conditional nodes: prologues, then per class graphs of 8
            // body iterations replayed while the class is active, then epilogues
            WL_CUDA(cudaGraphDestroy(graph));
            graph = nullptr;
            for (auto& R : loops) prologue(*R, st);
            if (smallrun) prologue(*smallrun, st);
            small_fork(st);
            for (auto& R : loops) {
                cudaGraph_t g8 = nullptr;
                cudaGraphExec_t e8 = nullptr;
                WL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                for (int k = 0; k < 8; k++) body(*R, 0, st);
                WL_CUDA(cudaStreamEndCapture(st, &g8));
                WL_CUDA(cudaGraphInstantiate(&e8, g8, 0));
                std::vector<BatchState> hs(R->nprob);
                BatchGlobal hgl{};
                for (int launches = 0;; launches++) {
                    WL_CUDA(cudaGraphLaunch(e8, st));
                    graph_launches++;
                    WL_CUDA(cudaMemcpyAsync(hs.data(), R->state.p, sizeof(BatchState) * R->nprob,
                                            cudaMemcpyDeviceToHost, st));
                    WL_CUDA(cudaMemcpyAsync(&hgl, R->global.p, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
                    WL_CUDA(cudaStreamSynchronize(st));
                    bool active = false;
                    for (auto& x : hs) active = active || x.phase != PH_DONE;
                    if (!active || hgl.timed_out || (launches + 1) * 8 >= max_iter) break;
                }
                cudaGraphExecDestroy(e8);
                cudaGraphDestroy(g8);
            }
            small_join(st);
            for (auto& R : loops) epilogue(*R, st);
            if (smallrun) epilogue(*smallrun, st);
        }
        WL_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(st, &junk);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);

    // results, problem by problem (latencies from the earliest run start)
    std::vector<BatchRun*> runs;
    for (auto& R : loops) runs.push_back(R.get());
    if (smallrun) runs.push_back(smallrun.get());
    std::vector<BatchGlobal> hg(runs.size());
    unsigned long long t_first = ~0ULL, t_last = 0;
    int iters = 0, timed_out = 0, tiles = 0;
    for (size_t r = 0; r < runs.size(); r++) {
        WL_CUDA(cudaMemcpy(&hg[r], runs[r]->global.p, sizeof(BatchGlobal), cudaMemcpyDeviceToHost));
        t_first = std::min(t_first, hg[r].t_start);
        t_last = std::max(t_last, hg[r].t_end);
        tiles += runs[r]->ntiles;
        if (runs[r] != smallrun.get()) {
            iters = std::max(iters, hg[r].iterations);
            timed_out |= hg[r].timed_out;
        }
    }
    for (size_t r = 0; r < runs.size(); r++) {
        const BatchRun& R = *runs[r];
        std::vector<BatchState> hs(R.nprob);
        WL_CUDA(cudaMemcpy(hs.data(), R.state.p, sizeof(BatchState) * R.nprob, cudaMemcpyDeviceToHost));
        for (int j = 0; j < R.nprob; j++) {
            const int i = R.members[j];
            unpack_spinor(hp[i].f[BF_X], 0, probs[i].x, st);
            const BatchState& S = hs[j];
            wilson_solve_stats& o = stats[i];
            const double bn = std::sqrt(S.bnorm2);
            o.true_rel_resid = bn > 0 ? std::sqrt(S.res2) / bn : std::sqrt(S.res2);
            o.inner_iters = S.sc.iter;
            o.outer_iters = S.outer;
            o.hop_applications = 4 * S.sc.iter + 4 * (S.outer + 1) + 4;
            o.seconds = S.phase == PH_DONE && S.t_done >= t_first ? (double)(S.t_done - t_first) * 1e-9 : -1.0;
            int status = S.status;
            if (status == 0 && S.phase != PH_DONE) status = hg[r].timed_out ? WILSON_ERR_TIMEOUT : WILSON_ERR_NOCONV;
            if (status == 0 && !(o.true_rel_resid <= prm.tol)) status = WILSON_ERR_NOCONV;
            o.status = status;
        }
    }
    WL_CUDA(cudaStreamSynchronize(st));
    if (info) {
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->device_seconds = t_last > t_first ? (double)(t_last - t_first) * 1e-9 : 0.0;
        info->iterations = iters;
        info->graph_launches = graph_launches;
        info->device_loop = use_cond;
        info->timed_out = timed_out;
        info->tiles = tiles;
    }
}

}  // namespace wl
