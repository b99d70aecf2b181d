// dslash_spt.cu -- more launch shapes of the paired-FP32 hopping-term kernel
// (Sec. 5, Eq. 3) for the autotuner: several sites per thread, and for F16
// storage the spin projection done on the stored halves (hop variants 12-17).
//
// Sites per thread (SPT).  A thread computes SPT output sites, blockDim.x
// apart (so every warp access stays coalesced), direction by direction: the
// SPT neighbour loads of a direction are independent, so a thread has SPT
// times the loads in flight of the one-site kernel, at the cost of SPT
// accumulators.  The block covers SPT * blockDim.x consecutive sites.  A
// thread whose second site lies beyond the lattice computes a valid site
// (site 0) in its place and neither stores nor reduces it, so the warp never
// diverges inside the stencil.
//
// Packed-half projection (F16 only).  The stored chunk of colour c holds
// the half2 words (s0.re, s1.re), (s0.im, s1.im), (s2.re, s3.re),
// (s2.im, s3.im), and the projected half spinor pairs (h0.re, h1.re) and
// (h0.im, h1.im) are one packed FMA of them each (a sign and a swap of the
// halves).  Projecting before the conversion to FP32 converts 12 instead of
// 24 values per hop and drops the 6 FP32 projection FMAs; the sum of two
// stored values is rounded once to F16 (about 1e-4 of relative L2 error on
// top of the 2.5e-4 of F16 storage).  The SU(3) products, the accumulation
// and the scale stay FP32 as in hop_kernel_p.
//
// Variants: 12 = SPT 2 at 128 registers, 13 = SPT 2 at 255, 14 = SPT 4 at
// 255; 15, 16, 17 = the F16 projection at 128, 85 and 64 registers.  The
// pipelined kernels (20-22, 27, 28) live in dslash_pipe.cuh.
#include "dslash_impl.cuh"

namespace wl {

namespace {

// One direction mu of the stencil with the F16 packed projection; otherwise
// the arithmetic of hop_dir_p.
template <int GP, int R, bool DAG, int MU, bool FIRST>
__device__ __forceinline__ void hop_dir_ph(PSpinor& acc, const HopParams& P, const char* in, int p, int h,
                                           const int c[4], int s) {
    using SF = SpinorFmt<P_F16>;
    using GF = GaugeFmt<GP, R>;
    const Geom& g = P.g;
    const int L = g.L[MU];
    const int smu = MU == 0 ? 1 : MU == 1 ? g.L[0] : MU == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
    constexpr int SF_ = DAG ? -1 : 1;
#pragma unroll
    for (int dir = 0; dir < 2; dir++) {
        const bool fwd = dir == 0;
        const bool wrap = fwd ? c[MU] == L - 1 : c[MU] == 0;
        const int sn = fwd ? (wrap ? s - (L - 1) * smu : s + smu) : (wrap ? s + (L - 1) * smu : s - smu);
        const int hn = sn >> 1;
        uint4 d[3];
        const uint4* b = static_cast<const uint4*>(static_cast<const void*>(in)) + hn;
#pragma unroll
        for (int cc = 0; cc < 3; cc++) d[cc] = __ldg(b + (size_t)cc * g.stride);
        const float sc = SF::load_scale(in, g.stride, hn);
        cpx<float> U[3][3];
        GF::load(P.gauge, g.stride, (fwd ? p : 1 - p) * 4 + MU, fwd ? h : hn, U);
        PHalf hh, w;
        if (fwd) project_f16_packed<MU, SF_>(d, hh);
        else project_f16_packed<MU, -SF_>(d, hh);
        if (wrap) apply_phase_p(hh, (float)g.ph[MU][0], fwd ? (float)g.ph[MU][1] : -(float)g.ph[MU][1]);
        if (fwd) {
            su3_mul_p<false>(U, hh, w);
            expand_p<MU, SF_, FIRST>(acc, w, sc);
        } else {
            su3_mul_p<true>(U, hh, w);
            expand_p<MU, -SF_, false>(acc, w, sc);
        }
    }
}

template <int SP, int GP, int R, bool DAG, bool HP, int MU, bool FIRST>
__device__ __forceinline__ void hop_dir_any(PSpinor& acc, const HopParams& P, const char* in, int p, int h,
                                            const int c[4], int s) {
    if constexpr (HP) hop_dir_ph<GP, R, DAG, MU, FIRST>(acc, P, in, p, h, c, s);
    else hop_dir_p<SP, GP, R, DAG, MU, FIRST>(acc, P, in, p, h, c, s);
}

template <int SP, int GP, int R, bool DAG, int MINB, int SPT, bool HP>
__global__ void __launch_bounds__(256, MINB) hop_kernel_ps(const HopParams P) {
    using SF = SpinorFmt<SP>;
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
    const int T = blockDim.x;
    const float a = (float)P.a;
    double nrm = 0.0;
    // block-uniform trip count: the block iterates while its first site is inside
    for (int h0 = sb * T * SPT + threadIdx.x; h0 - (int)threadIdx.x < g.Vh; h0 += nb * T * SPT) {
        int hs[SPT], cs[SPT][4], ss[SPT];
        bool ok[SPT];
#pragma unroll
        for (int q = 0; q < SPT; q++) {
            const int hq = h0 + q * T;
            ok[q] = hq < g.Vh;
            hs[q] = ok[q] ? hq : 0;
            site_of_half(hs[q], p, g, cs[q], ss[q]);
        }
        PSpinor acc[SPT];
#pragma unroll
        for (int q = 0; q < SPT; q++) hop_dir_any<SP, GP, R, DAG, HP, 0, true>(acc[q], P, in, p, hs[q], cs[q], ss[q]);
#pragma unroll
        for (int q = 0; q < SPT; q++) hop_dir_any<SP, GP, R, DAG, HP, 1, false>(acc[q], P, in, p, hs[q], cs[q], ss[q]);
#pragma unroll
        for (int q = 0; q < SPT; q++) hop_dir_any<SP, GP, R, DAG, HP, 2, false>(acc[q], P, in, p, hs[q], cs[q], ss[q]);
#pragma unroll
        for (int q = 0; q < SPT; q++) hop_dir_any<SP, GP, R, DAG, HP, 3, false>(acc[q], P, in, p, hs[q], cs[q], ss[q]);
#pragma unroll
        for (int q = 0; q < SPT; q++) {
            if (!ok[q]) continue;
            PSpinor& A = acc[q];
            const int h = hs[q];
            if (P.xpay) {
                PSpinor xq;
                float xs;
                SF::load_packed(x, g.stride, h, xq, xs);
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
                nrm += (double)n2.x + (double)n2.y;
            }
            if (P.nrhs > 1) SF::template store_packed<true>(out, g.stride, h, A);
            else SF::store_packed(out, g.stride, h, A);
        }
    }
    pdl_trigger();
    if (P.reduce) grid_reduce(nrm, P.red, k, nb * gridDim.y, sb + nb * blockIdx.y);
}

template <int SP, int GP, int R, bool DAG, int V>
void launch_ps_v(const HopParams& P, int block, int site_blocks, int ny, cudaStream_t st) {
    constexpr int MINB = hop_variant_minb(V, SP), SPT = hop_variant_spt(V);
    constexpr bool HP = hop_variant_hproj(V);
    const dim3 grid(site_blocks * P.nrhs, ny);
    if constexpr (HP && SP != P_F16) {
        throw Error(7, "the packed-half projection variants need F16 storage");
    } else {
        launch_dep(hop_kernel_ps<SP, GP, R, DAG, MINB, SPT, HP>, grid, dim3(block), st, P);
    }
}

template <int SP, int GP, int R, bool DAG>
void launch_ps_dag(const HopParams& P, int block, int site_blocks, int ny, int variant, cudaStream_t st) {
    switch (variant) {
        case 12: launch_ps_v<SP, GP, R, DAG, 12>(P, block, site_blocks, ny, st); break;
        case 13: launch_ps_v<SP, GP, R, DAG, 13>(P, block, site_blocks, ny, st); break;
        case 14: launch_ps_v<SP, GP, R, DAG, 14>(P, block, site_blocks, ny, st); break;
        case 15: launch_ps_v<SP, GP, R, DAG, 15>(P, block, site_blocks, ny, st); break;
        case 16: launch_ps_v<SP, GP, R, DAG, 16>(P, block, site_blocks, ny, st); break;
        case 17: launch_ps_v<SP, GP, R, DAG, 17>(P, block, site_blocks, ny, st); break;
        case 20:
        case 21:
        case 22:
            if constexpr ((SP == P_F16 || SP == P_BF16) && GP == SP && R == 12) {
                launch_hop_pipe<SP>(P, block, site_blocks, ny, DAG, variant, st);
                break;
            }
            throw Error(7, "the pipelined hop variants need F16/BF16 spinors and 12-real links");
        default: throw Error(7, "unknown sites-per-thread hop variant");
    }
}

}  // namespace


template <int SP, int GP, int R>
void launch_hop_ps(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant, cudaStream_t st) {
    if (dag) launch_ps_dag<SP, GP, R, true>(P, block, site_blocks, ny, variant, st);
    else launch_ps_dag<SP, GP, R, false>(P, block, site_blocks, ny, variant, st);
}

template void launch_hop_ps<P_F32, P_F32, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_ps<P_F32, P_F32, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_ps<P_F16, P_F16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_ps<P_F16, P_F16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_ps<P_BF16, P_BF16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_ps<P_BF16, P_BF16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);

}  // namespace wl
