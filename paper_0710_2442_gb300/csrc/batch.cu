// batch.cu -- many independent solves on lattices of different sizes in one
// CUDA graph launch (wilson_batch_solve): host orchestration and the batched
// BLAS-1 kernels.  The problem states, finishers, hop kernels and the
// CTA-resident solver are in batch_impl.cuh.
//
// Every problem keeps its own lattice, links, kappa, fields and CG scalars.
// Problems with at most SolveParams::batch_small_vh sites per parity are each
// solved by one thread block (small_solve_kernel).  The others are grouped
// by lattice size into classes; each class's half lattices are cut into
// tiles of a tuned number of sites (128, 256 or 512; the autotuner times
// the class's inner hop with each), a tile table maps every tile to its problem, and
// every kernel of the class walks the tile table (one block per tile by
// default), so one launch serves all its problems whatever their sizes.
// Per-problem reductions are tile partials summed in a fixed order by the
// problem's last tile (no block waits for another).
//
// Each problem runs the solver of solver.cu (CGNR on the even Schur
// complement; FP64 outer corrections with reliable updates around an inner
// CG in reduced storage precision) as a device-side state machine:
//
//   OUTER:  x_e += e;  r = bhat - Mhat x_e (FP64);  finished if |r| <= tol |b|
//           (or out of budget), else s = r, e = 0, r' = Mhat'^dag s,
//           p = r' + beta p  -> INNER
//   INNER:  one CG iteration (six kernels as in solver.cu) -> OUTER when
//           |s| <= delta |r| (or the per-correction iteration cap)
//
// The graph is: prologue (|b|^2, bhat, zeroed iterates) -> the small
// problems' CTA solves and, per class, a device-side while loop (conditional
// node) whose body runs the OUTER kernels and the INNER kernels as two
// parallel branches (disjoint problems) and then a one-block commit kernel
// that advances the class's problems and sets its loop condition; smaller
// classes' kernels carry higher graph-node priorities -> epilogue (x_o =
// b_o + kappa D_oe x_e, true residuals, completion times).  Each commit
// kernel stops its loop after a hard number of iterations or a wall-clock
// budget even if some problem has not finished, so the launch always ends.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "batch_impl.cuh"

namespace wl {

namespace bt {

// ---------------------------------------------------------------------------
// batched BLAS-1 kernels (all tile-walking, phase-filtered)
// ---------------------------------------------------------------------------
#define WL_TILE_LOOP_BEGIN                                                   \
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {                 \
        const int pid = __ldg(A.tile_prob + t);                              \
        if (!tile_active(A, op, pid)) continue;                              \
        const BatchProb& Pr = A.probs[pid];                                  \
        const Geom& g = Pr.g;                                                \
        const int h0 = (t - Pr.tile0) * A.tile;
#define WL_TILE_LOOP_END }

// xin += alpha p; s -= alpha q; slow = s; |s|^2   (INNER)
template <int IP>
__global__ void __launch_bounds__(256) bxs_kernel(const BatchArgs A, const BOp op) {
    using TP = typename SpinorFmt<IP>::real;
    WL_TILE_LOOP_BEGIN
    const float alpha = (float)__ldcg(&A.state[pid].sc.alpha);
    double nrm = 0.0;
    for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
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
    for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
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

// x_e += xin (FP64 += FP32), and an FP32 copy of x_e when the problem's
// residual is FP32 this correction   (OUTER)
__global__ void __launch_bounds__(256) baxpy_kernel(const BatchArgs A, const BOp op) {
    WL_TILE_LOOP_BEGIN
    const bool x32 = __ldcg(&A.state[pid].use32) != 0;  // set by the previous finisher
    for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
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
        if (x32) {
            cpx<float> xf[12];
#pragma unroll
            for (int k = 0; k < 12; k++) xf[k] = {(float)xv[k].re, (float)xv[k].im};
            SpinorFmt<P_F32>::store(Pr.f[BF_X32], g.stride, h, xf);
        }
    }
    WL_TILE_LOOP_END
}

// r64 = bhat - q, |r64|^2, q = Mhat x in FP64 (q64) or FP32 (q32)   (OUTER)
__global__ void __launch_bounds__(256) bxmy_kernel(const BatchArgs A, const BOp op) {
    WL_TILE_LOOP_BEGIN
    const bool q32 = __ldcg(&A.state[pid].use32) != 0;
    double nrm = 0.0;
    for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
        const int h = h0 + j;
        if (h >= g.Vh) break;
        cpx<double> bv[12], qv[12];
        SpinorFmt<P_F64>::load(Pr.f[BF_BHAT], g.stride, h, bv);
        if (q32) {
            cpx<float> qf[12];
            SpinorFmt<P_F32>::load(Pr.f[BF_Q32], g.stride, h, qf);
#pragma unroll
            for (int k = 0; k < 12; k++) qv[k] = {(double)qf[k].re, (double)qf[k].im};
        } else {
            SpinorFmt<P_F64>::load(Pr.f[BF_Q64], g.stride, h, qv);
        }
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
    for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
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
    for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
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
    for (int j = threadIdx.x; j < A.tile; j += blockDim.x) {
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
    GaugeField g64, glo, g32;
    SpinorField f[BF_N];
    double kappa;
    bool res32_ok = false;  // FP32 residuals for the early corrections
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

}  // namespace bt

using namespace bt;

struct BatchRun {
    int nprob = 0, ntiles = 0, sms = 1, tile = kTile;
    Prec ip = P_F16;
    std::vector<int> members;  // global problem ids of this run's problems (local order)
    DevBuf probs, state, tile_prob, global, partials, counters, ids;
    BatchArgs A{};
    int grid = 1;
    LaunchConfig hop_lo{128, 1}, hop_64{128, 0}, hop_32{128, 3};
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
        o.res32 = -1;
        o.zero_first = 0;
        o.partials = partials.as<double>() + (size_t)rslot * ntiles;
        o.counters = counters.as<unsigned int>() + (size_t)rslot * nprob;
        return o;
    }

    template <int SP, int GP>
    void hop_t(const BOp& o, int dag, const LaunchConfig& c, cudaStream_t st) const {
        launch_bhop<SP, GP>(A, o, dag, c.variant, c.block, grid, st);
    }
    void hop(const BOp& o, int dag, cudaStream_t st) const {
        if (o.use64 == 1) {
            hop_t<P_F64, P_F64>(o, dag, hop_64, st);
        } else if (o.use64 == 2) {
            hop_t<P_F32, P_F32>(o, dag, hop_32, st);
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
    // FP32 residuals of the early corrections (solver.h, kF32ResidualRel):
    // FP32 links (the inner ones when the inner solve is FP32) and fields
    P.res32_ok = prm.tol < 1e-7 && ip != P_F64;
    if (P.res32_ok) {
        if (ip != P_F32) {
            P.g32.prec = P_F32;
            P.g32.recon = 12;
            P.g32.g = P.g;
            P.g32.buf.alloc(gauge_bytes(P_F32, 12, P.g.stride));
            pack_gauge(P.g32, in.gauge, st);
        }
        P.f[BF_X32].alloc(P_F32, 0, 1, P.g);
        P.f[BF_Q32].alloc(P_F32, 0, 1, P.g);
        P.f[BF_T32].alloc(P_F32, 1, 1, P.g);
        WL_CUDA(cudaMemsetAsync(P.f[BF_X32].buf.p, 0, P.f[BF_X32].buf.bytes, st));  // read by tuning launches
    }
    pack_spinor(P.f[BF_B], 0, in.b, st);
    if (prm.use_initial_guess) pack_spinor(P.f[BF_X], 0, in.x, st);
}

// Device descriptors, states and the tile table of one run.
std::unique_ptr<BatchRun> make_run(const std::vector<HostProb>& hp, const std::vector<int>& members, bool small,
                                   const SolveParams& prm, cudaStream_t st, int tile = kTile) {
    auto R = std::make_unique<BatchRun>();
    R->tile = tile;
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
        D.g32 = !P.res32_ok ? nullptr : P.glo.prec == P_F32 ? D.glo : P.g32.buf.as<const char>();
        D.res32_ok = P.res32_ok && !small;
        D.kappa = P.kappa;
        D.tol = prm.tol;
        D.delta = prm.delta > 0 ? prm.delta : default_delta(R->ip);
        D.maxiter = prm.maxiter;
        D.max_outer = prm.max_restarts;
        D.keep_x = prm.use_initial_guess;
        D.small = small ? 1 : 0;
        D.tile0 = (int)tiles.size();
        D.ntiles = small ? 0 : (P.g.Vh + tile - 1) / tile;
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
    R->A.tile = tile;
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
    // Each class's tile size: WILSON_BATCH_TILE pins it; otherwise the
    // autotuner times the class's inner hop (a non-reducing xpay hop of the
    // inner precision) on tile tables of 128, 256 and 512 sites.
    int tile_pin = 0;
    if (const char* e = std::getenv("WILSON_BATCH_TILE")) tile_pin = std::atoi(e);
    WL_REQUIRE(tile_pin == 0 || tile_pin == 128 || tile_pin == 256 || tile_pin == 512,
               "WILSON_BATCH_TILE must be 128, 256 or 512");
    std::vector<std::unique_ptr<BatchRun>> loops;
    for (const auto& c : size_classes(hp, loop_ids, max_classes)) {
        if (tile_pin) {
            loops.push_back(make_run(hp, c, false, prm, st, tile_pin));
            continue;
        }
        // 256 first, and another tile only if its hop is more than 5 % faster:
        // an isolated hop does not see what more tiles cost inside the graph
        // (more blocks for every phase-filtered kernel of the class, sharing
        // the GPU with the other classes).  Measured on the 64-problem batch:
        // 128-site tiles for the 16^3 x 32 class, picked on a 0.5 % faster
        // hop, made the whole batch 5.6 % slower (0.266 against 0.252 s).
        std::unique_ptr<BatchRun> cand[3];
        const int tiles[3] = {256, 128, 512};
        long long vh = 0;
        for (int i : c) vh += hp[i].g.Vh;
        for (int k = 0; k < 3; k++) cand[k] = make_run(hp, c, false, prm, st, tiles[k]);
        char key[96];
        snprintf(key, sizeof(key), "btile:lo%d:n%d:vh%lld", (int)ip, (int)c.size(), vh);
        // LaunchConfig.block carries the tile size here
        const LaunchConfig pick = tune_launch(
            key, {LaunchConfig{256, 0}, LaunchConfig{128, 0}, LaunchConfig{512, 0}}, LaunchConfig{kTile, 0}, st,
            [&](const LaunchConfig& t) {
                const BatchRun& Rt = *cand[t.block == 256 ? 0 : t.block == 128 ? 1 : 2];
                const BOp o = Rt.op(BF_Q, BF_T, BF_P, 0, 0, 2, -1, 0, BF_NONE, 0);
                dispatch_low(ip, [&](auto I) {
                    Rt.hop_t<decltype(I)::value, decltype(I)::value>(o, 0, LaunchConfig{128, 4}, st);
                });
            },
            0.05);
        loops.push_back(std::move(cand[pick.block == 256 ? 0 : pick.block == 128 ? 1 : 2]));
    }
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
    // F16 / BF16 inner hops: the pipelined stencil first, so that another candidate
    // replaces it only when more than the tuner's margin faster (inside the
    // graph the pipelined hop wins by more than it does alone: the 64-problem
    // batch took 0.221 s with it on every class, 0.226 s on isolated choices)
    std::vector<LaunchConfig> cands_lo;
    if (ip == P_F16 || ip == P_BF16)
        for (int block : {64, 128}) cands_lo.push_back(LaunchConfig{block, kBatchPipeVariant});
    cands_lo.insert(cands_lo.end(), cands.begin(), cands.end());
    // WILSON_BATCH_HOP=v:block pins the inner hop's launch (one of cands_lo)
    LaunchConfig hop_pin{0, -1};
    if (const char* e = std::getenv("WILSON_BATCH_HOP")) {
        int v = -1, b = 0;
        WL_REQUIRE(std::sscanf(e, "%d:%d", &v, &b) == 2, "WILSON_BATCH_HOP must be variant:block");
        bool listed = false;
        for (const LaunchConfig& c : cands_lo) listed = listed || (c.variant == v && c.block == b);
        WL_REQUIRE(listed, "WILSON_BATCH_HOP names no candidate of this batch's inner hop");
        hop_pin = LaunchConfig{b, v};
    }
    for (auto& R : loops) {
        char key[96];
        snprintf(key, sizeof(key), "bhop:lo%d:n%d:t%d", (int)ip, R->nprob, R->ntiles);
        const BOp o = R->op(BF_Q, BF_T, BF_P, 0, 0, 2, -1, 0, BF_NONE, 0);
        BatchRun* Rp = R.get();
        R->hop_lo = tune_launch(key, cands_lo, LaunchConfig{128, 1}, st, [&](const LaunchConfig& c) {
            dispatch_low(ip, [&](auto I) { Rp->hop_t<decltype(I)::value, decltype(I)::value>(o, 0, c, st); });
        });
        if (hop_pin.variant >= 0) R->hop_lo = hop_pin;
        snprintf(key, sizeof(key), "bhop:f64:n%d:t%d", R->nprob, R->ntiles);
        const BOp o64 = R->op(BF_Q64, BF_T64, BF_X, 0, 1, 2, -1, 0, BF_NONE, 0);
        R->hop_64 = tune_launch(key, cands64, LaunchConfig{128, 0}, st,
                                [&](const LaunchConfig& c) { Rp->hop_t<P_F64, P_F64>(o64, 0, c, st); });
        bool any32 = false;
        for (int i : R->members) any32 = any32 || hp[i].res32_ok;
        if (any32) {
            snprintf(key, sizeof(key), "bhop:f32res:n%d:t%d", R->nprob, R->ntiles);
            const BOp o32 = R->op(BF_Q32, BF_T32, BF_X32, 0, 2, 2, -1, 0, BF_NONE, 0);
            R->hop_32 = tune_launch(key, cands, LaunchConfig{128, 3}, st,
                                    [&](const LaunchConfig& c) { Rp->hop_t<P_F32, P_F32>(o32, 0, c, st); });
        }
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
        // without an initial guess the iterate is zero during a problem's
        // first correction (the prologue zeroes it): those two hops write 0
        // and x without the stencil
        BOp t64 = R.op(BF_T64, BF_X, -1, 1, 1, 0, PH_OUTER, 0, BF_NONE, 1);
        BOp q64 = R.op(BF_Q64, BF_T64, BF_X, 0, 1, 2, PH_OUTER, 0, BF_NONE, 1);
        t64.zero_first = q64.zero_first = prm.use_initial_guess ? 0 : 1;
        t64.res32 = q64.res32 = 0;
        R.hop(t64, 0, s);
        R.hop(q64, 0, s);
        // the problems whose residual is FP32 this correction: the same two hops
        // on the FP32 copy of x with FP32 links
        BOp t32 = R.op(BF_T32, BF_X32, -1, 1, 2, 0, PH_OUTER, 0, BF_NONE, 1);
        BOp q32 = R.op(BF_Q32, BF_T32, BF_X32, 0, 2, 2, PH_OUTER, 0, BF_NONE, 1);
        t32.res32 = q32.res32 = 1;
        R.hop(t32, 0, s);
        R.hop(q32, 0, s);
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
        // a cluster of blocks per small problem unless WILSON_BATCH_SMALL_CLUSTER=1
        bool cluster = true;
        if (const char* e = std::getenv("WILSON_BATCH_SMALL_CLUSTER")) cluster = std::atoi(e) != 1;
        dispatch_low(ip, [&](auto I) {
            launch_small_ip<decltype(I)::value>(cluster, smallrun->A, smallrun->ids.as<int>(), smallrun->G(),
                                                budget_ns, smallrun->nprob, st3);
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
            o.hop_applications = 4 * S.sc.iter + 4 * (S.outer + 1) + (prm.use_initial_guess ? 4 : 2);
            o.seconds = S.phase == PH_DONE && S.t_done >= t_first ? (double)(S.t_done - t_first) * 1e-9 : -1.0;
            o.inner_seconds = 0.0;
            o.outer_f32 = S.n32;
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
