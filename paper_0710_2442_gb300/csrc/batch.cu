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
            const double target2 = P.tol * P.tol * S.bnorm2;
            if (!isfinite(sum)) {
                S.status = WILSON_ERR_NUMERIC;
                S.next_phase = PH_DONE;
            } else if (sum <= target2) {
                S.next_phase = PH_DONE;
            } else if (S.outer >= P.max_outer || sc.iter >= P.maxiter) {
                S.status = WILSON_ERR_NOCONV;
                S.next_phase = PH_DONE;
            } else {
                S.outer += 1;
                S.next_phase = PH_INNER;
                const double stop = fmax(P.delta * sqrt(sum), sqrt(target2));
                sc.stop2 = stop * stop;
                sc.snorm2 = sum;
                sc.done = 0;
                sc.maxiter = P.maxiter;
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
        S.phase = S.next_phase = PH_OUTER;
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
    std::vector<HostProb> hp;
    DevBuf probs, state, tile_prob, global, partials, counters;
    BatchArgs A{};
    int grid = 1;
    LaunchConfig hop_lo{128, 1}, hop_64{128, 0};

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
        // the batch walker uses the scalar stencil: register variants only
        if (v % 3 == 1) { WL_BHOP(1) } else if (v % 3 == 2) { WL_BHOP(2) } else { WL_BHOP(0) }
#undef WL_BHOP
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

}  // namespace

// Build, run and tear down one batch; fills stats[n] and info.
void batch_solve(int n, const wilson_problem* probs, const SolveParams& prm, wilson_solve_stats* stats,
                 wilson_batch_info* info, cudaStream_t st) {
    NvtxRange nvtx_batch("wilson batch solve");
    auto t0 = std::chrono::steady_clock::now();
    BatchRun B;
    B.nprob = n;
    B.ip = prm.inner;
    B.sms = device_sm_count();
    B.hp.resize(n);
    std::vector<BatchProb> desc(n);
    std::vector<int> tiles;
    for (int i = 0; i < n; i++) {
        build_problem(B.hp[i], probs[i], B.ip, prm, st);
        HostProb& P = B.hp[i];
        BatchProb& D = desc[i];
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
        D.delta = prm.delta > 0 ? prm.delta : (B.ip == P_F32 ? 1e-3 : 0.1);
        D.maxiter = prm.maxiter;
        D.max_outer = prm.max_restarts;
        D.tile0 = (int)tiles.size();
        D.ntiles = (P.g.Vh + kTile - 1) / kTile;
        for (int t = 0; t < D.ntiles; t++) tiles.push_back(i);
    }
    B.ntiles = (int)tiles.size();
    B.probs.alloc(sizeof(BatchProb) * n);
    B.state.alloc(sizeof(BatchState) * n);
    B.tile_prob.alloc(sizeof(int) * B.ntiles);
    B.global.alloc(sizeof(BatchGlobal));
    constexpr int kRed = 6;  // reduction slots: prologue/epilogue, A4, A7, B2, B3, B5
    B.partials.alloc(sizeof(double) * (size_t)kRed * B.ntiles);
    B.counters.alloc(sizeof(unsigned int) * (size_t)kRed * n);
    WL_CUDA(cudaMemcpyAsync(B.probs.p, desc.data(), sizeof(BatchProb) * n, cudaMemcpyHostToDevice, st));
    WL_CUDA(cudaMemcpyAsync(B.tile_prob.p, tiles.data(), sizeof(int) * B.ntiles, cudaMemcpyHostToDevice, st));
    WL_CUDA(cudaMemsetAsync(B.counters.p, 0, sizeof(unsigned int) * kRed * n, st));
    WL_CUDA(cudaMemsetAsync(B.state.p, 0, sizeof(BatchState) * n, st));
    B.A.probs = B.probs.as<BatchProb>();
    B.A.state = B.state.as<BatchState>();
    B.A.tile_prob = B.tile_prob.as<int>();
    B.A.ntiles = B.ntiles;
    B.A.nprob = n;
    B.grid = std::max(1, std::min(B.ntiles, 8 * B.sms));
    BatchGlobal* G = B.global.as<BatchGlobal>();

    // tune the two batched hop kernels (non-reducing launches on scratch fields)
    {
        char key[96];
        snprintf(key, sizeof(key), "bhop:lo%d:n%d:t%d", (int)B.ip, n, B.ntiles);
        const BOp o = B.op(BF_Q, BF_T, BF_P, 0, 0, 2, -1, 0, BF_NONE, 0);
        std::vector<LaunchConfig> cands;
        for (const LaunchConfig& c : hop_candidates())
            if (c.variant < 3) cands.push_back(c);
        B.hop_lo = tune_launch(key, cands, LaunchConfig{128, 1}, st, [&](const LaunchConfig& c) {
            dispatch_low(B.ip, [&](auto I) { B.hop_t<decltype(I)::value, decltype(I)::value>(o, 0, c, st); });
        });
        snprintf(key, sizeof(key), "bhop:f64:n%d:t%d", n, B.ntiles);
        const BOp o64 = B.op(BF_Q64, BF_T64, BF_X, 0, 1, 2, -1, 0, BF_NONE, 0);
        B.hop_64 = tune_launch(key, cands, LaunchConfig{128, 0}, st, [&](const LaunchConfig& c) {
            B.hop_t<P_F64, P_F64>(o64, 0, c, st);
        });
    }

    const int bgrid = B.grid;
    auto blas = [&](auto kernel, const BOp& o) {
        kernel<<<bgrid, 256, 0, st>>>(B.A, o);
        WL_LAUNCH_CHECK();
    };
    cudaStream_t st2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    WL_CUDA(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    WL_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    WL_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    struct Cleanup {
        cudaStream_t s;
        cudaEvent_t a, b;
        ~Cleanup() {
            if (s) cudaStreamDestroy(s);
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } cleanup{st2, fork, join};

    // ------------------------------------------------------------------ graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle{};
    int use_cond = 1;
    // Loop limits: an iteration cap every problem's own caps fit into, and a
    // wall-clock budget.  WILSON_BATCH_MAX_LOOP / WILSON_BATCH_BUDGET_MS lower
    // them (used by the tests that make the limit run out).
    int max_iter = std::min(2 * prm.maxiter + 4 * prm.max_restarts + 16, 4000000);
    unsigned long long budget_ns = 60ULL * 1000000000ULL;
    if (const char* e = std::getenv("WILSON_BATCH_MAX_LOOP"))
        if (std::atoi(e) > 0) max_iter = std::min(max_iter, std::atoi(e));
    if (const char* e = std::getenv("WILSON_BATCH_BUDGET_MS"))
        if (std::atoll(e) > 0) budget_ns = std::min(budget_ns, (unsigned long long)std::atoll(e) * 1000000ULL);
    WL_CUDA(cudaGraphCreate(&graph, 0));
    if (cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGetLastError();
        use_cond = 0;
    }
    auto prologue = [&](cudaStream_t s) {
        dispatch_low(B.ip, [&](auto I) {
            binit_kernel<decltype(I)::value><<<bgrid, 256, 0, s>>>(B.A, B.op(0, 0, -1, 0, 0, 0, -1, 0, BF_NONE, 0),
                                                                   prm.use_initial_guess, G);
        });
        WL_LAUNCH_CHECK();
        blas(bnorm_kernel, B.op(0, BF_B, -1, 0, 0, 0, -1, 0, BFIN_BNORM, 0));
        blas(bnorm_kernel, B.op(0, BF_B, -1, 1, 0, 0, -1, 0, BFIN_BNORM, 0));
        // bhat_e = b_e + kappa D_eo b_o
        B.hop(B.op(BF_BHAT, BF_B, BF_B, 0, 1, 1, -1, 0, BF_NONE, 0), 0, s);
    };
    auto body = [&](cudaStream_t s) {
        WL_CUDA(cudaEventRecord(fork, s));
        WL_CUDA(cudaStreamWaitEvent(st2, fork, 0));
        // branch A (OUTER problems) on s
        blas(baxpy_kernel, B.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0, BF_NONE, 1));
        B.hop(B.op(BF_T64, BF_X, -1, 1, 1, 0, PH_OUTER, 0, BF_NONE, 1), 0, s);
        B.hop(B.op(BF_Q64, BF_T64, BF_X, 0, 1, 2, PH_OUTER, 0, BF_NONE, 1), 0, s);
        blas(bxmy_kernel, B.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0, BFIN_OUTER, 1));
        dispatch_low(B.ip, [&](auto I) {
            bprep_kernel<decltype(I)::value><<<bgrid, 256, 0, s>>>(B.A, B.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0,
                                                                             BF_NONE, 2));
        });
        WL_LAUNCH_CHECK();
        B.hop(B.op(BF_T, BF_SLOW, -1, 1, 0, 0, PH_OUTER, 0, BF_NONE, 2), 1, s);
        B.hop(B.op(BF_R, BF_T, BF_SLOW, 0, 0, 2, PH_OUTER, 0, BFIN_START, 2), 1, s);
        dispatch_low(B.ip, [&](auto I) {
            bp_kernel<decltype(I)::value><<<bgrid, 256, 0, s>>>(B.A, B.op(0, 0, -1, 0, 0, 0, PH_OUTER, 0, BF_NONE, 2));
        });
        WL_LAUNCH_CHECK();
        // branch B (INNER problems) on st2
        B.hop(B.op(BF_T, BF_P, -1, 1, 0, 0, PH_INNER, 1, BF_NONE, 3), 0, st2);
        B.hop(B.op(BF_Q, BF_T, BF_P, 0, 0, 2, PH_INNER, 1, BFIN_ALPHA, 3), 0, st2);
        dispatch_low(B.ip, [&](auto I) {
            bxs_kernel<decltype(I)::value><<<bgrid, 256, 0, st2>>>(B.A, B.op(0, 0, -1, 0, 0, 0, PH_INNER, 1,
                                                                             BFIN_RES, 4));
        });
        WL_LAUNCH_CHECK();
        B.hop(B.op(BF_T, BF_SLOW, -1, 1, 0, 0, PH_INNER, 1, BF_NONE, 5), 1, st2);
        B.hop(B.op(BF_R, BF_T, BF_SLOW, 0, 0, 2, PH_INNER, 1, BFIN_BETA, 5), 1, st2);
        dispatch_low(B.ip, [&](auto I) {
            bp_kernel<decltype(I)::value><<<bgrid, 256, 0, st2>>>(B.A, B.op(0, 0, -1, 0, 0, 0, PH_INNER, 1,
                                                                            BF_NONE, 5));
        });
        WL_LAUNCH_CHECK();
        WL_CUDA(cudaEventRecord(join, st2));
        WL_CUDA(cudaStreamWaitEvent(s, join, 0));
        bcommit_kernel<<<1, 256, 0, s>>>(B.A.state, n, G, handle, use_cond, max_iter, budget_ns);
        WL_LAUNCH_CHECK();
    };
    auto epilogue = [&](cudaStream_t s) {
        // x_o = b_o + kappa D_oe x_e
        B.hop(B.op(BF_X, BF_X, BF_B, 1, 1, 1, -1, 0, BF_NONE, 0), 0, s);
        // M x per parity into q64 (even) and t64 (odd); |b - M x|^2
        B.hop(B.op(BF_Q64, BF_X, BF_X, 0, 1, 3, -1, 0, BF_NONE, 0), 0, s);
        B.hop(B.op(BF_T64, BF_X, BF_X, 1, 1, 3, -1, 0, BF_NONE, 0), 0, s);
        blas(bnorm_kernel, B.op(0, BF_B, BF_Q64, 0, 0, 0, -1, 0, BFIN_TRUE, 0));
        blas(bnorm_kernel, B.op(0, BF_B, BF_T64, 1, 0, 0, -1, 0, BFIN_TRUE, 0));
        bfinal_kernel<<<1, 1, 0, s>>>(G);
        WL_LAUNCH_CHECK();
    };

    int graph_launches = 0;
    try {
        if (use_cond) {
            WL_CUDA(cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            prologue(st);
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            WL_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode;
            WL_CUDA(cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp));
            cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
            WL_CUDA(cudaStreamUpdateCaptureDependencies(st, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
            epilogue(st);
            cudaGraph_t out = nullptr;
            WL_CUDA(cudaStreamEndCapture(st, &out));
            // the loop body, captured into the conditional node's child graph
            WL_CUDA(cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            body(st);
            WL_CUDA(cudaStreamEndCapture(st, &out));
            WL_CUDA(cudaGraphInstantiate(&exec, graph, 0));
            WL_CUDA(cudaGraphLaunch(exec, st));
            graph_launches = 1;
        } else {
            // without conditional nodes: prologue, then graphs of 8 body
            // iterations replayed while some problem is active, then epilogue
            prologue(st);
            WL_CUDA(cudaGraphDestroy(graph));
            graph = nullptr;
            WL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < 8; k++) body(st);
            WL_CUDA(cudaStreamEndCapture(st, &graph));
            WL_CUDA(cudaGraphInstantiate(&exec, graph, 0));
            std::vector<BatchState> hs(n);
            while (true) {
                WL_CUDA(cudaGraphLaunch(exec, st));
                graph_launches++;
                WL_CUDA(cudaMemcpyAsync(hs.data(), B.state.p, sizeof(BatchState) * n, cudaMemcpyDeviceToHost, st));
                WL_CUDA(cudaStreamSynchronize(st));
                bool active = false;
                for (auto& s : hs) active = active || s.phase != PH_DONE;
                if (!active || graph_launches * 8 >= max_iter) break;
            }
            epilogue(st);
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

    std::vector<BatchState> hs(n);
    BatchGlobal hg;
    WL_CUDA(cudaMemcpy(hs.data(), B.state.p, sizeof(BatchState) * n, cudaMemcpyDeviceToHost));
    WL_CUDA(cudaMemcpy(&hg, B.global.p, sizeof(BatchGlobal), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; i++) {
        unpack_spinor(B.hp[i].f[BF_X], 0, probs[i].x, st);
        const BatchState& S = hs[i];
        wilson_solve_stats& o = stats[i];
        const double bn = std::sqrt(S.bnorm2);
        o.true_rel_resid = bn > 0 ? std::sqrt(S.res2) / bn : std::sqrt(S.res2);
        o.inner_iters = S.sc.iter;
        o.outer_iters = S.outer;
        o.hop_applications = 4 * S.sc.iter + 4 * (S.outer + 1) + 4;
        o.seconds = S.phase == PH_DONE && S.t_done >= hg.t_start ? (double)(S.t_done - hg.t_start) * 1e-9 : -1.0;
        int status = S.status;
        if (status == 0 && S.phase != PH_DONE) status = hg.timed_out ? WILSON_ERR_TIMEOUT : WILSON_ERR_NOCONV;
        if (status == 0 && !(o.true_rel_resid <= prm.tol)) status = WILSON_ERR_NOCONV;
        o.status = status;
    }
    WL_CUDA(cudaStreamSynchronize(st));
    if (info) {
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->device_seconds = (double)(hg.t_end - hg.t_start) * 1e-9;
        info->iterations = hg.iterations;
        info->graph_launches = graph_launches;
        info->device_loop = use_cond;
        info->timed_out = hg.timed_out;
        info->tiles = B.ntiles;
    }
}

}  // namespace wl
