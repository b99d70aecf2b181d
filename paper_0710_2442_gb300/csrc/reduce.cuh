// reduce.cuh -- deterministic FP64 global reductions fused into kernels.
//
// Every block reduces its threads' FP64 values by warp shuffles and a
// shared-memory pass, writes one partial per block, and takes a ticket from a
// global counter.  The block that draws the last ticket sums all partials in
// a fixed order (thread t adds partials t, t+B, ...; then the same shuffle
// tree), so the result does not depend on block scheduling, and then runs
// the finisher that turns the sum into solver scalars.  It also resets the
// counter, so the same reducer can be reused by the next launch on the
// stream.  No block ever waits for another one.
#pragma once

#include "common.cuh"

namespace wl {

enum FinOp {
    FIN_STORE = 0,     // result[0] = sum
    FIN_CG_ALPHA = 1,  // |q|^2: alpha = gam / |q|^2
    FIN_CG_RES = 2,    // |s|^2: convergence test, iteration count
    FIN_CG_BETA = 3,   // |r|^2: beta = |r|^2 / gam, gam = |r|^2
    FIN_ADD = 4,       // result[0] += sum
    FIN_CG_GAM = 5     // |r|^2: gam = |r|^2 (start of a CG)
};

// Scalars of one CG solve, kept on the device so that iterations never wait
// for the host.
struct CGScalars {
    double gam;      // |r|^2 of the normal-equation residual r = Mhat^dag s
    double alpha;
    double beta;
    double pq;       // |Mhat p|^2
    double snorm2;   // |s|^2, recursively updated Schur residual
    double stop2;    // the inner iteration ends when snorm2 <= stop2
    int done;        // 1: converged (snorm2 <= stop2), 2: maxiter, 3: NaN/Inf, 4: finished earlier
    int iter;        // iterations completed since the counter was last reset
    int maxiter;     // iteration cap for this inner solve
    int pad;
};

// A reduction may have several independent slots (one per right-hand side):
// slot k uses partials[k * slot_cap ...], counter[k], result[k] and sc[k].
struct RedArgs {
    double* partials;       // slot_cap partials per slot (slot_cap >= blocks per slot)
    unsigned int* counter;  // one per slot: 0 before the launch; reset to 0 by the last block
    double* result;         // FIN_STORE / FIN_ADD targets (one per slot)
    CGScalars* sc;          // FIN_CG_* targets (one per slot)
    int op;
    int slot_cap;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the value is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();  // protects sm against a previous use
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nwarps ? sm[lane] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

__device__ inline void run_finisher(const RedArgs& r, int slot, double sum) {
    CGScalars* sc = r.sc ? r.sc + slot : nullptr;
    switch (r.op) {
        case FIN_STORE: r.result[slot] = sum; break;
        case FIN_ADD: r.result[slot] += sum; break;
        case FIN_CG_ALPHA:
            sc->pq = sum;
            if (!(sum > 0.0) || !isfinite(sum)) {
                sc->alpha = 0.0;
                if (!isfinite(sum)) sc->done = 3;
                else if (sc->done == 0) sc->done = 1;  // Mhat p = 0: nothing left to do
            } else {
                sc->alpha = sc->gam / sum;
            }
            break;
        case FIN_CG_RES:
            sc->snorm2 = sum;
            sc->iter += 1;
            if (!isfinite(sum)) sc->done = 3;
            else if (sum <= sc->stop2) sc->done = 1;
            else if (sc->iter >= sc->maxiter) sc->done = 2;
            break;
        case FIN_CG_GAM:
            sc->gam = sum;
            if (!isfinite(sum)) sc->done = 3;
            break;
        case FIN_CG_BETA:
            if (!isfinite(sum)) { sc->done = 3; sc->beta = 0.0; break; }
            sc->beta = sc->gam > 0.0 ? sum / sc->gam : 0.0;
            sc->gam = sum;
            break;
    }
}

// Called by all threads of every block that reduces into `slot` (uniformly):
// nblocks blocks contribute to the slot, this block is number bid of them.
__device__ inline void grid_reduce(double v, const RedArgs& r, int slot, unsigned int nblocks, unsigned int bid) {
    const double bs = block_sum(v);
    __shared__ int s_last;
    double* part = r.partials + (size_t)slot * r.slot_cap;
    if (threadIdx.x == 0) {
        part[bid] = bs;
        __threadfence();
        const unsigned int ticket = atomicAdd(r.counter + slot, 1u);
        s_last = (ticket == nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // Each thread adds its strided partials in index order; the loads are
    // issued eight at a time so that their L2 latencies overlap (the order of
    // the additions, and so the result, is that of the plain loop).
    double acc = 0.0;
    const unsigned int step = blockDim.x;
    unsigned int i = threadIdx.x;
    for (; i + 7 * step < nblocks; i += 8 * step) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = __ldcg(part + i + k * step);
#pragma unroll
        for (int k = 0; k < 8; k++) acc += v[k];
    }
    for (; i < nblocks; i += step) acc += __ldcg(part + i);
    const double total = block_sum(acc);
    if (threadIdx.x == 0) {
        run_finisher(r, slot, total);
        r.counter[slot] = 0u;
        __threadfence();
    }
}

// Single-slot form: every block of the grid contributes.
__device__ inline void grid_reduce(double v, const RedArgs& r) {
    grid_reduce(v, r, 0, gridDim.x * gridDim.y, blockIdx.x + gridDim.x * blockIdx.y);
}

}  // namespace wl
