// dslash_pipe.cuh -- the pipelined hopping-term kernels for F16 / BF16
// storage (Sec. 5, Eq. 3; hop variants 20-22 and 27, 28), instantiated one
// storage type per translation unit (dslash_pipe_f16.cu, dslash_pipe_bf16.cu)
// so that they compile in parallel.
#pragma once

#include <cuda_pipeline.h>

#include "dslash_impl.cuh"

namespace wl {

namespace {

// ---------------------------------------------------------------------------
// F16 / BF16 hop with the neighbour data copied ahead into shared memory
// (variants 20-22: 2 / 3 / 3 hops ahead at 80 / 80 / 96 registers).  The F16
// hop's exact loads alone run at 0.93 of the copy bandwidth, the packed-
// projection kernel at 0.6: its arithmetic waits on loads it cannot keep in
// flight at the occupancy its registers allow.  Here each thread issues the raw
// data of a hop (3 spinor chunks, the scale, 3 link chunks) with asynchronous
// copies (cp.async) into its own shared-memory slots, D hops ahead, so the
// loads in flight hold no registers (pipe_site, shared with the batch's tile
// kernel).  Before computing hop j the thread waits for that hop's copy group
// (a hardware wait, no spin); after computing it, it reuses the slot for
// hop j + D.  Slots are laid out [slot][chunk][thread] (conflict-free warp accesses);
// a thread reads only what it copied, so no barrier is needed.  The arithmetic
// is that of the packed-projection kernel for F16, of the paired kernel for
// BF16 (exact conversion, projection in FP32).  A thread past the lattice's end
// runs site 0 and stores nothing, so the warp does not diverge inside the
// pipeline.
// ---------------------------------------------------------------------------
// TB: the block size (the launch's blockDim.x), a compile-time constant so
// that every slot offset is an immediate; NREG: the register budget.
template <int SP, bool DAG, int NREG, int D, int TB>
__global__ void __launch_bounds__(TB) __maxnreg__(NREG) hop_kernel_pipe(const HopParams P) {
    using SF = SpinorFmt<SP>;
    extern __shared__ __align__(16) unsigned char pipe_smem[];
    constexpr int T = TB;
    const int t = threadIdx.x;
    uint4* sp = reinterpret_cast<uint4*>(pipe_smem);     // [D][3][T] spinor chunks
    uint2* lk = reinterpret_cast<uint2*>(sp + D * 3 * T);  // [D][3][T] link chunks
    float* scs = reinterpret_cast<float*>(lk + D * 3 * T); // [D][T] scales
    const int k = blockIdx.x % P.nrhs;
    const int sb = blockIdx.x / P.nrhs;
    const int nb = gridDim.x / P.nrhs;
    const int p = P.full ? (int)blockIdx.y : P.out_parity;
    pdl_wait();
    if (P.skip && __ldcg(P.skip + (size_t)k * P.skip_stride)) return;
    const int pin = 1 - p;
    char* out = P.out + (P.full ? p * P.out_pstep : 0) + k * P.out_rstep;
    const char* in = P.in + (P.full ? pin * P.in_pstep : 0) + k * P.in_rstep;
    const char* x = P.x ? P.x + (P.full ? p * P.x_pstep : 0) + k * P.x_rstep : nullptr;
    const Geom& g = P.g;
    const float a = (float)P.a;
    double nrm = 0.0;
    for (int h0 = sb * T + t; h0 - t < g.Vh; h0 += nb * T) {
        const bool ok = h0 < g.Vh;
        const int h = ok ? h0 : 0;
        PSpinor acc;
        pipe_site<SP, DAG, D, T>(acc, in, P.gauge, g, p, h, sp, lk, scs, t);
        if (!ok) continue;
        if (P.xpay) {
            PSpinor xq;
            float xs;
            SF::load_packed(x, g.stride, h, xq, xs);
            const float2 Af = bc2(a), X = bc2(xs);
#pragma unroll
            for (int cc = 0; cc < 3; cc++) {
                acc.re01[cc] = fma2(Af, acc.re01[cc], mul2(X, xq.re01[cc]));
                acc.im01[cc] = fma2(Af, acc.im01[cc], mul2(X, xq.im01[cc]));
                acc.re23[cc] = fma2(Af, acc.re23[cc], mul2(X, xq.re23[cc]));
                acc.im23[cc] = fma2(Af, acc.im23[cc], mul2(X, xq.im23[cc]));
            }
        } else if (P.a != 1.0) {
            const float2 Af = bc2(a);
#pragma unroll
            for (int cc = 0; cc < 3; cc++) {
                acc.re01[cc] = mul2(Af, acc.re01[cc]);
                acc.im01[cc] = mul2(Af, acc.im01[cc]);
                acc.re23[cc] = mul2(Af, acc.re23[cc]);
                acc.im23[cc] = mul2(Af, acc.im23[cc]);
            }
        }
        if (P.reduce) {
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
        if (P.nrhs > 1) SF::template store_packed<true>(out, g.stride, h, acc);
        else SF::store_packed(out, g.stride, h, acc);
    }
    pdl_trigger();
    if (P.reduce) grid_reduce(nrm, P.red, k, nb * gridDim.y, sb + nb * blockIdx.y);
}

template <int SP, bool DAG, int V, int TB>
void launch_pipe_tb(const HopParams& P, int site_blocks, int ny, cudaStream_t st) {
    constexpr int NREG = V == 22 ? 96 : 80, D = V == 20 ? 2 : 3;
    constexpr size_t per_thread = (size_t)D * (3 * 16 + 3 * 8 + 4);
    auto k = hop_kernel_pipe<SP, DAG, NREG, D, TB>;
    static bool opted[64] = {};  // the larger dynamic shared memory, once per device
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    if (!opted[dev]) {
        WL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per_thread * TB)));
        opted[dev] = true;
    }
    launch_dep_smem(k, dim3(site_blocks * P.nrhs, ny), dim3(TB), per_thread * TB, st, P);
}
template <int SP, bool DAG, int V>
void launch_pipe_v(const HopParams& P, int block, int site_blocks, int ny, cudaStream_t st) {
    if (block == 64) launch_pipe_tb<SP, DAG, V, 64>(P, site_blocks, ny, st);
    else if (block == 128) launch_pipe_tb<SP, DAG, V, 128>(P, site_blocks, ny, st);
    else if (block == 256) launch_pipe_tb<SP, DAG, V, 256>(P, site_blocks, ny, st);
    else throw Error(WILSON_ERR_ARG, "the pipelined F16 hop takes blocks of 64, 128 or 256 threads");
}

// Two right-hand sides per thread on the pipelined F16 / BF16 stencil
// (variants 27, 28).  A thread computes one site for right-hand sides k0 and k0 + 1: per
// hop it copies the link once and both neighbour spinors (chunks and scales)
// into its slots, decodes the link once and applies it to both, so the link's
// copy, conversion and third-row reconstruction are shared.  Slots: spinor
// chunks [D][2][3][T], scales [D][2][T], link chunks [D][3][T].  Skip flags,
// the epilogue and the per-RHS reductions as in hop_kernel_pm.
template <int SP, bool DAG, int D, int T>
__device__ __forceinline__ void pipe2_site(PSpinor (&acc)[2], const char* in0, long long rstep,
                                              const char* gauge, const Geom& g, int p, int h, uint4* sp, uint2* lk,
                                              float* scs, int t) {
    using GF = GaugeFmt<SP, 12>;
    const int pin = 1 - p;
    int hn[8];
    unsigned wrap = 0;
    {
        int c[4], s;
        site_of_half(h, p, g, c, s);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            const int L = g.L[mu];
            const int smu = mu == 0 ? 1 : mu == 1 ? g.L[0] : mu == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
            const bool wf = c[mu] == L - 1, wb = c[mu] == 0;
            hn[2 * mu] = (wf ? s - (L - 1) * smu : s + smu) >> 1;
            hn[2 * mu + 1] = (wb ? s + (L - 1) * smu : s - smu) >> 1;
            wrap |= (unsigned)wf << (2 * mu) | (unsigned)wb << (2 * mu + 1);
        }
    }
    auto issue = [&](int j) {
        const int slot = j % D;
        const int n = hn[j];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const char* in = in0 + r * rstep;
            const uint4* gs = reinterpret_cast<const uint4*>(in) + n;
#pragma unroll
            for (int kk = 0; kk < 3; kk++)
                __pipeline_memcpy_async(&sp[((slot * 2 + r) * 3 + kk) * T + t], gs + (size_t)kk * g.stride, 16);
            __pipeline_memcpy_async(&scs[(slot * 2 + r) * T + t],
                                    reinterpret_cast<const float*>(in + 48LL * g.stride) + n, 4);
        }
        const int blk = ((j & 1) ? pin : p) * 4 + (j >> 1);
        const uint2* gl = reinterpret_cast<const uint2*>(gauge) + (size_t)blk * 3 * g.stride + ((j & 1) ? n : h);
#pragma unroll
        for (int kk = 0; kk < 3; kk++)
            __pipeline_memcpy_async(&lk[(slot * 3 + kk) * T + t], gl + (size_t)kk * g.stride, 8);
        __pipeline_commit();
    };
#pragma unroll
    for (int j = 0; j < D; j++) issue(j);
#define WL_PIPE2_HOP(J)                                                                                         \
    {                                                                                                           \
        __pipeline_wait_prior(D - 1);                                                                           \
        constexpr int slot = (J) % D;                                                                           \
        cpx<float> U[3][3];                                                                                     \
        GF::decode(&lk[slot * 3 * T + t], T, U);                                                                \
        _Pragma("unroll") for (int r = 0; r < 2; r++) {                                                         \
            uint4 d[3];                                                                                         \
            _Pragma("unroll") for (int kk = 0; kk < 3; kk++) d[kk] = sp[((slot * 2 + r) * 3 + kk) * T + t];     \
            pipe_hop<SP, DAG, (J)>(acc[r], d, scs[(slot * 2 + r) * T + t], U, wrap, g);                         \
        }                                                                                                       \
        if ((J) + D < 8) issue((J) + D);                                                                        \
        else __pipeline_commit();                                                                               \
    }
    WL_PIPE2_HOP(0) WL_PIPE2_HOP(1) WL_PIPE2_HOP(2) WL_PIPE2_HOP(3)
    WL_PIPE2_HOP(4) WL_PIPE2_HOP(5) WL_PIPE2_HOP(6) WL_PIPE2_HOP(7)
#undef WL_PIPE2_HOP
}

template <int SP, bool DAG, int NREG, int D, int TB>
__global__ void __launch_bounds__(TB) __maxnreg__(NREG) hop_kernel_pipe2(const HopParams P) {
    using SF = SpinorFmt<SP>;
    extern __shared__ __align__(16) unsigned char pipe2_smem[];
    constexpr int T = TB;
    const int t = threadIdx.x;
    uint4* sp = reinterpret_cast<uint4*>(pipe2_smem);       // [D][2][3][T] spinor chunks
    uint2* lk = reinterpret_cast<uint2*>(sp + D * 6 * T);    // [D][3][T] link chunks
    float* scs = reinterpret_cast<float*>(lk + D * 3 * T);   // [D][2][T] scales
    const int ng = P.nrhs / 2;
    const int grp = blockIdx.x % ng;
    const int sb = blockIdx.x / ng;
    const int nb = gridDim.x / ng;
    const int k0 = grp * 2;
    pdl_wait();
    unsigned act = 0;
#pragma unroll
    for (int r = 0; r < 2; r++)
        if (!P.skip || !__ldcg(P.skip + (size_t)(k0 + r) * P.skip_stride)) act |= 1u << r;
    if (!act) return;
    const int p = P.full ? (int)blockIdx.y : P.out_parity;
    const int pin = 1 - p;
    char* out = P.out + (P.full ? p * P.out_pstep : 0) + k0 * P.out_rstep;
    const char* in = P.in + (P.full ? pin * P.in_pstep : 0) + k0 * P.in_rstep;
    const char* x = P.x ? P.x + (P.full ? p * P.x_pstep : 0) + k0 * P.x_rstep : nullptr;
    const Geom& g = P.g;
    const float a = (float)P.a;
    double nrm[2] = {0.0, 0.0};
    for (int h0 = sb * T + t; h0 - t < g.Vh; h0 += nb * T) {
        const bool ok = h0 < g.Vh;
        const int h = ok ? h0 : 0;
        PSpinor acc[2];
        pipe2_site<SP, DAG, D, T>(acc, in, P.in_rstep, P.gauge, g, p, h, sp, lk, scs, t);
        if (!ok) continue;
#pragma unroll
        for (int r = 0; r < 2; r++) {
            PSpinor& A = acc[r];
            if (P.xpay) {
                PSpinor xq;
                float xs;
                SF::load_packed(x + r * P.x_rstep, g.stride, h, xq, xs);
                const float2 Af = bc2(a), X = bc2(xs);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    A.re01[cc] = fma2(Af, A.re01[cc], mul2(X, xq.re01[cc]));
                    A.im01[cc] = fma2(Af, A.im01[cc], mul2(X, xq.im01[cc]));
                    A.re23[cc] = fma2(Af, A.re23[cc], mul2(X, xq.re23[cc]));
                    A.im23[cc] = fma2(Af, A.im23[cc], mul2(X, xq.im23[cc]));
                }
            } else if (P.a != 1.0) {
                const float2 Af = bc2(a);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    A.re01[cc] = mul2(Af, A.re01[cc]);
                    A.im01[cc] = mul2(Af, A.im01[cc]);
                    A.re23[cc] = mul2(Af, A.re23[cc]);
                    A.im23[cc] = mul2(Af, A.im23[cc]);
                }
            }
            if (P.reduce) {
                float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    n2 = fma2(A.re01[cc], A.re01[cc], n2);
                    n2 = fma2(A.im01[cc], A.im01[cc], n2);
                    n2 = fma2(A.re23[cc], A.re23[cc], n2);
                    n2 = fma2(A.im23[cc], A.im23[cc], n2);
                }
                nrm[r] += (double)n2.x + (double)n2.y;
            }
            if (act >> r & 1u) SF::template store_packed<true>(out + r * P.out_rstep, g.stride, h, A);
        }
    }
    pdl_trigger();
    if (P.reduce) {
#pragma unroll
        for (int r = 0; r < 2; r++)
            if (act >> r & 1u) grid_reduce(nrm[r], P.red, k0 + r, nb * gridDim.y, sb + nb * blockIdx.y);
    }
}

template <int SP, bool DAG, int D, int TB>
void launch_pipe2_tb(const HopParams& P, int site_blocks, int ny, cudaStream_t st) {
    constexpr size_t per_thread = (size_t)D * (2 * (3 * 16 + 4) + 3 * 8);
    auto k = hop_kernel_pipe2<SP, DAG, 128, D, TB>;
    static bool opted[64] = {};  // the larger dynamic shared memory, once per device
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    if (!opted[dev]) {
        WL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per_thread * TB)));
        opted[dev] = true;
    }
    launch_dep_smem(k, dim3(site_blocks * (P.nrhs / 2), ny), dim3(TB), per_thread * TB, st, P);
}
template <int SP, bool DAG, int D>
void launch_pipe2_d(const HopParams& P, int block, int site_blocks, int ny, cudaStream_t st) {
    if (block == 64) launch_pipe2_tb<SP, DAG, D, 64>(P, site_blocks, ny, st);
    else if (block == 128) launch_pipe2_tb<SP, DAG, D, 128>(P, site_blocks, ny, st);
    else if (block == 256) launch_pipe2_tb<SP, DAG, D, 256>(P, site_blocks, ny, st);
    else throw Error(WILSON_ERR_ARG, "the pipelined F16 hop takes blocks of 64, 128 or 256 threads");
}


}  // namespace

// Variants 20-22: one right-hand side per thread (D = 2 / 3 / 3 hops ahead
// at 80 / 80 / 96 registers).
template <int SP>
void launch_hop_pipe(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant,
                     cudaStream_t st) {
    if (dag) {
        if (variant == 20) launch_pipe_v<SP, true, 20>(P, block, site_blocks, ny, st);
        else if (variant == 21) launch_pipe_v<SP, true, 21>(P, block, site_blocks, ny, st);
        else launch_pipe_v<SP, true, 22>(P, block, site_blocks, ny, st);
    } else {
        if (variant == 20) launch_pipe_v<SP, false, 20>(P, block, site_blocks, ny, st);
        else if (variant == 21) launch_pipe_v<SP, false, 21>(P, block, site_blocks, ny, st);
        else launch_pipe_v<SP, false, 22>(P, block, site_blocks, ny, st);
    }
}

// Variants 27, 28: two right-hand sides per thread.
template <int SP>
void launch_hop_pipe2(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant,
                      cudaStream_t st) {
    WL_REQUIRE(P.nrhs >= 2 && P.nrhs % 2 == 0, "the two-RHS pipelined hop needs an even number of right-hand sides");
    const bool d3 = variant == kHopPipe2Variant + 1;
    if (dag) d3 ? launch_pipe2_d<SP, true, 3>(P, block, site_blocks, ny, st)
                : launch_pipe2_d<SP, true, 2>(P, block, site_blocks, ny, st);
    else d3 ? launch_pipe2_d<SP, false, 3>(P, block, site_blocks, ny, st)
            : launch_pipe2_d<SP, false, 2>(P, block, site_blocks, ny, st);
}

}  // namespace wl
