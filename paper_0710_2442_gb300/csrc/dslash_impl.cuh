// dslash_impl.cuh -- the Wilson hopping term (QCD on the Cell BE, Sec. 5,
// Eq. 3) as a CUDA stencil on SoA fields.  Included by the per-precision
// translation units (dslash_f64.cu, dslash_f32.cu, dslash_lowp.cu), which
// instantiate the kernels so that they compile in parallel.
//
// One thread computes one output site of one parity.  For each of the 8 hops
// it loads the neighbour spinor (coalesced 16-byte loads), projects it to a
// half spinor with (1 -/+ g_mu) in the DeGrand-Rossi basis (6 complex adds),
// applies the boundary phase when the hop wraps, loads the link (12 or 18
// reals; 12 are completed by the conjugate cross product), multiplies the two
// colour vectors by U or U^dag (2 x 66 flops), and expands the product back
// into the 4-spinor accumulator (12 complex adds).  That is the 1320
// flops/site of Sec. 5.  For F16/BF16 spinors the neighbour's per-site scale
// is applied in the accumulation (acc = fma(scale, w, acc)), which costs no
// extra instruction.  The epilogue scales, optionally adds a field of the
// output parity (out = x + a D in), stores at the storage precision and
// optionally reduces |out|^2 into a deterministic FP64 grid reduction.
//
// The "dagger" variant swaps the two projectors.  Since g_5 (1 -/+ g_mu) g_5
// = (1 +/- g_mu), it applies g_5 D g_5 = D^dag, which gives the adjoint
// Schur operator Mhat^dag = 1 - kappa^2 D'_eo D'_oe without any g_5 passes.
//
// MINB selects the register budget: __launch_bounds__(256, MINB) caps a
// thread at 65536 / (256 * MINB) registers, trading per-thread load
// parallelism for resident warps; the autotuner picks the variant.
//
// Kernel families (the variant numbers the autotuner and WILSON_HOP_VARIANT
// use):
//   hop_kernel     0..2  scalar stencil (and every FP64 launch)
//   hop_kernel_p   3..5  the same stencil on paired FP32 instructions
//   hop_kernel_pm  6..9  several right-hand sides per thread (register-blocked)
//   hop_kernel_rl  10    links staged in shared memory, loop over right-hand sides
//   hop_kernel_mma 11    link x half-spinor products on the tensor cores, one
//                        warp per site and 16 right-hand sides (dslash_mma.cu)
//   hop_kernel_ps  12-17 the paired stencil with 2 or 4 sites per thread, and
//                        for F16 the projection on packed halves (dslash_spt.cu)
//   hop_kernel_pm  18-19 the register-blocked form with the F16 packed projection
//   hop_kernel_pipe 20-22 F16/BF16 with the neighbour data copied ahead (dslash_pipe.cuh)
//   hop_kernel / hop_kernel_p 23-25 with L2 prefetches of the site's links
//                        (and neighbour spinors) when a thread takes its site
//   hop_kernel_slab 26   t-slab streaming: neighbouring slices of a tile staged
//                        in shared memory by bulk copies (dslash_slab.cu)
//   hop_kernel_pipe2 27-28 the same pipeline with two right-hand sides per
//                        thread sharing each hop's link (dslash_pipe.cuh)
// Multi-RHS launches of the first two run the right-hand sides of a site
// tile as consecutive blocks.  Every kernel starts with the programmatic-
// dependent-launch wait, so it can be launched with that attribute.
#pragma once

#include <cuda_pipeline.h>

#include "internal.h"

namespace wl {

// Half-spinor projection (1 - S g_mu) psi, DeGrand-Rossi basis.  Only the
// upper two spin components are independent; the lower two are recovered in
// expand().  v[k], k = spin*3 + colour; h[k], k = halfspin*3 + colour.
template <int MU, int S, class T>
__device__ __forceinline__ void project(const cpx<T> v[12], cpx<T> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<T> p0 = v[c], p1 = v[3 + c], p2 = v[6 + c], p3 = v[9 + c];
        cpx<T> h0, h1;
        if (MU == 0) {  // (1 - S g_1):  h0 = p0 - S i p3,  h1 = p1 - S i p2
            h0 = S > 0 ? csub(p0, ci(p3)) : cadd(p0, ci(p3));
            h1 = S > 0 ? csub(p1, ci(p2)) : cadd(p1, ci(p2));
        } else if (MU == 1) {  // h0 = p0 + S p3,  h1 = p1 - S p2
            h0 = S > 0 ? cadd(p0, p3) : csub(p0, p3);
            h1 = S > 0 ? csub(p1, p2) : cadd(p1, p2);
        } else if (MU == 2) {  // h0 = p0 - S i p2,  h1 = p1 + S i p3
            h0 = S > 0 ? csub(p0, ci(p2)) : cadd(p0, ci(p2));
            h1 = S > 0 ? cadd(p1, ci(p3)) : csub(p1, ci(p3));
        } else {  // h0 = p0 - S p2,  h1 = p1 - S p3
            h0 = S > 0 ? csub(p0, p2) : cadd(p0, p2);
            h1 = S > 0 ? csub(p1, p3) : cadd(p1, p3);
        }
        h[c] = h0;
        h[3 + c] = h1;
    }
}

// acc (+)= sc * [(1 - S g_mu)-image of the half spinor w]: the full 4-spinor
// is (w0, w1, lower2, lower3) with the lower components fixed by the
// projector.  sc is the neighbour's storage scale (the constant 1 for
// unscaled formats, where the fma folds to an add).
template <int MU, int S, bool FIRST, class T>
__device__ __forceinline__ void expand(cpx<T> acc[12], const cpx<T> w[6], T sc) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<T> w0 = w[c], w1 = w[3 + c];
        cpx<T> l2, l3;
        if (MU == 0) {  // lower = (S i w1, S i w0)
            l2 = S > 0 ? ci(w1) : cneg(ci(w1));
            l3 = S > 0 ? ci(w0) : cneg(ci(w0));
        } else if (MU == 1) {  // (-S w1, S w0)
            l2 = S > 0 ? cneg(w1) : w1;
            l3 = S > 0 ? w0 : cneg(w0);
        } else if (MU == 2) {  // (S i w0, -S i w1)
            l2 = S > 0 ? ci(w0) : cneg(ci(w0));
            l3 = S > 0 ? cneg(ci(w1)) : ci(w1);
        } else {  // (-S w0, -S w1)
            l2 = S > 0 ? cneg(w0) : w0;
            l3 = S > 0 ? cneg(w1) : w1;
        }
        if (FIRST) {
            acc[c] = cscale(sc, w0);
            acc[3 + c] = cscale(sc, w1);
            acc[6 + c] = cscale(sc, l2);
            acc[9 + c] = cscale(sc, l3);
        } else {
#define WL_ACC(k, v)                          \
    acc[k].re = fma(sc, (v).re, acc[k].re);   \
    acc[k].im = fma(sc, (v).im, acc[k].im);
            WL_ACC(c, w0)
            WL_ACC(3 + c, w1)
            WL_ACC(6 + c, l2)
            WL_ACC(9 + c, l3)
#undef WL_ACC
        }
    }
}

// w = U h (ADJ = false) or U^dag h (ADJ = true), for both half-spin rows.
template <bool ADJ, class T>
__device__ __forceinline__ void su3_mul(const cpx<T> U[3][3], const cpx<T> h[6], cpx<T> w[6]) {
#pragma unroll
    for (int a = 0; a < 2; a++) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            cpx<T> r;
            if (!ADJ) {
                r = cmul(U[i][0], h[3 * a + 0]);
                r = cfma(U[i][1], h[3 * a + 1], r);
                r = cfma(U[i][2], h[3 * a + 2], r);
            } else {
                r = cjmul(U[0][i], h[3 * a + 0]);
                r = cjfma(U[1][i], h[3 * a + 1], r);
                r = cjfma(U[2][i], h[3 * a + 2], r);
            }
            w[3 * a + i] = r;
        }
    }
}

struct HopParams {
    char* out;
    const char* in;
    const char* x;
    long long out_pstep, in_pstep, x_pstep;
    long long out_rstep, in_rstep, x_rstep;
    int nrhs;
    int skip_stride;
    const char* gauge;
    Geom g;
    int out_parity;
    int full;
    int xpay;
    double a;
    RedArgs red;
    int reduce;
    const int* skip;
};

// One direction mu: forward and backward hop into acc.
template <int SP, int GP, int R, bool DAG, int MU, bool FIRST, bool COH = false>
__device__ __forceinline__ void hop_dir(cpx<typename SpinorFmt<SP>::real> acc[12], const HopParams& P,
                                        const char* in, int p, int h, const int c[4], int s) {
    using SF = SpinorFmt<SP>;
    using GF = GaugeFmt<GP, R>;
    using T = typename SF::real;
    const Geom& g = P.g;
    const int L = g.L[MU];
    const int smu = MU == 0 ? 1 : MU == 1 ? g.L[0] : MU == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
    constexpr int SF_ = DAG ? -1 : 1;  // projector sign of the forward hop
    // ---- forward: (1 - S g_mu) eta U_{x,mu} psi_{x+mu}
    {
        const bool wrap = c[MU] == L - 1;
        const int sn = wrap ? s - (L - 1) * smu : s + smu;
        cpx<T> v[12], hs[6], w[6], U[3][3];
        T sc;
        SF::template load_raw<COH>(in, g.stride, sn >> 1, v, sc);
        GF::load(P.gauge, g.stride, p * 4 + MU, h, U);
        project<MU, SF_>(v, hs);
        if (wrap) {
            const cpx<T> eta = {(T)g.ph[MU][0], (T)g.ph[MU][1]};
#pragma unroll
            for (int k = 0; k < 6; k++) hs[k] = cmul(eta, hs[k]);
        }
        su3_mul<false>(U, hs, w);
        expand<MU, SF_, FIRST>(acc, w, sc);
    }
    // ---- backward: (1 + S g_mu) eta* U^dag_{x-mu,mu} psi_{x-mu}
    {
        const bool wrap = c[MU] == 0;
        const int sn = wrap ? s + (L - 1) * smu : s - smu;
        const int hn = sn >> 1;
        cpx<T> v[12], hs[6], w[6], U[3][3];
        T sc;
        SF::template load_raw<COH>(in, g.stride, hn, v, sc);
        GF::load(P.gauge, g.stride, (1 - p) * 4 + MU, hn, U);
        project<MU, -SF_>(v, hs);
        if (wrap) {
            const cpx<T> eta = {(T)g.ph[MU][0], -(T)g.ph[MU][1]};
#pragma unroll
            for (int k = 0; k < 6; k++) hs[k] = cmul(eta, hs[k]);
        }
        su3_mul<true>(U, hs, w);
        expand<MU, -SF_, false>(acc, w, sc);
    }
}

// The prefetching variants (PF = 1: the site's eight links; PF = 2: also its
// eight neighbour spinors) issue L2 prefetches for all of them when a thread
// takes its site, before the first hop.  On the F32 hop with 12-real links
// (384 of 576 bytes per site are links, each read once) the link stream then
// keeps up with the copy bandwidth; reading the links from cache instead
// takes a fifth off the time, while reading the neighbour spinors from the
// site's own (coalesced) rows changes nothing.
template <int SP, int GP, int R, int PF>
__device__ __forceinline__ void hop_prefetch(const HopParams& P, const char* in, int p, int h, const int c[4],
                                             int s) {
    if constexpr (PF > 0) {
        const Geom& g = P.g;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            const int L = g.L[mu];
            const int smu = mu == 0 ? 1 : mu == 1 ? g.L[0] : mu == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
            const int hb = (c[mu] == 0 ? s + (L - 1) * smu : s - smu) >> 1;
            prefetch_link<GP, R>(P.gauge, g.stride, p * 4 + mu, h);
            prefetch_link<GP, R>(P.gauge, g.stride, (1 - p) * 4 + mu, hb);
            if constexpr (PF > 1) {
                const int hf = (c[mu] == L - 1 ? s - (L - 1) * smu : s + smu) >> 1;
                prefetch_spinor<SP>(in, g.stride, hf);
                prefetch_spinor<SP>(in, g.stride, hb);
            }
        }
    }
}

// Grid: blockIdx.x = site_block * nrhs + rhs (right-hand sides fastest, so
// the blocks of all right-hand sides of one site tile run back to back and
// share the tile's link loads through L2); blockIdx.y = output parity for
// full-lattice launches.
template <int SP, int GP, int R, bool DAG, int MINB, int PF = 0>
__global__ void __launch_bounds__(256, MINB) hop_kernel(const HopParams P) {
    using SF = SpinorFmt<SP>;
    using T = typename SF::real;
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
    const T a = (T)P.a;
    double nrm = 0.0;
    // The whole block iterates while its tile starts inside the lattice (a
    // block-uniform trip count); this form compiles to faster code than the
    // plain per-thread bound.
    for (int h = sb * blockDim.x + threadIdx.x; h - (int)threadIdx.x < g.Vh; h += nb * blockDim.x) {
        if (h >= g.Vh) continue;
        int c[4], s;
        site_of_half(h, p, g, c, s);
        hop_prefetch<SP, GP, R, PF>(P, in, p, h, c, s);
        cpx<T> acc[12];
        hop_dir<SP, GP, R, DAG, 0, true>(acc, P, in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 1, false>(acc, P, in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 2, false>(acc, P, in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 3, false>(acc, P, in, p, h, c, s);
        if (P.xpay) {
            cpx<T> xv[12];
            SF::load(x, g.stride, h, xv);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                acc[k].re = fma(a, acc[k].re, xv[k].re);
                acc[k].im = fma(a, acc[k].im, xv[k].im);
            }
        } else if (P.a != 1.0) {
#pragma unroll
            for (int k = 0; k < 12; k++) acc[k] = cscale(a, acc[k]);
        }
        if (P.reduce) {
            T n2 = 0;
#pragma unroll
            for (int k = 0; k < 12; k++) n2 += cnorm2(acc[k]);
            nrm += (double)n2;
        }
        if (P.nrhs > 1) SF::template store<true>(out, g.stride, h, acc);
        else SF::store(out, g.stride, h, acc);
    }
    pdl_trigger();
    if (P.reduce) grid_reduce(nrm, P.red, k, nb * gridDim.y, sb + nb * blockIdx.y);
}

// ---------------------------------------------------------------------------
// The same stencil on paired FP32 instructions (sm_100+: FFMA2 / FMUL2 work
// on two floats at once).  Spinors arrive spin-paired (PSpinor); the half
// spinor pairs the two half-spin rows, hr[c] = (h0c.re, h1c.re), so the link
// multiplies both rows in one paired FMA per real term, and the result
// accumulates into the spin-paired accumulator.  Operations and rounding per
// real number are those of the scalar kernel (each paired FMA is two FP32
// FMAs); only the instruction count changes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sw2(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

struct PHalf {
    float2 re[3], im[3];
};

// (1 - S g_mu) psi in paired form (same equations as project()).
template <int MU, int S>
__device__ __forceinline__ void project_p(const PSpinor& q, PHalf& h) {
    constexpr float s = (float)S;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (MU == 0) {  // h0 = p0 - S i p3, h1 = p1 - S i p2
            h.re[c] = fma2(bc2(s), sw2(q.im23[c]), q.re01[c]);
            h.im[c] = fma2(bc2(-s), sw2(q.re23[c]), q.im01[c]);
        } else if (MU == 1) {  // h0 = p0 + S p3, h1 = p1 - S p2
            h.re[c] = fma2(make_float2(s, -s), sw2(q.re23[c]), q.re01[c]);
            h.im[c] = fma2(make_float2(s, -s), sw2(q.im23[c]), q.im01[c]);
        } else if (MU == 2) {  // h0 = p0 - S i p2, h1 = p1 + S i p3
            h.re[c] = fma2(make_float2(s, -s), q.im23[c], q.re01[c]);
            h.im[c] = fma2(make_float2(-s, s), q.re23[c], q.im01[c]);
        } else {  // h0 = p0 - S p2, h1 = p1 - S p3
            h.re[c] = fma2(bc2(-s), q.re23[c], q.re01[c]);
            h.im[c] = fma2(bc2(-s), q.im23[c], q.im01[c]);
        }
    }
}

// (1 - S g_mu) psi of one stored F16 site, projected on packed halves and
// converted to the paired-FP32 half spinor (same equations as project_p).
template <int MU, int S>
__device__ __forceinline__ void project_f16_packed(const uint4 (&d)[3], PHalf& h) {
    // +-1 as F16 bit patterns: 0x3C00 = 1.0, 0xBC00 = -1.0
    constexpr uint32_t P1 = 0x3C00u, M1 = 0xBC00u;
    constexpr uint32_t sp = S > 0 ? P1 : M1;   // +S
    constexpr uint32_t sm = S > 0 ? M1 : P1;   // -S
    auto c2 = [](uint32_t lo, uint32_t hi) {
        const uint32_t u = lo | (hi << 16);
        return *reinterpret_cast<const __half2*>(&u);
    };
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const uint32_t ux = d[c].x, uy = d[c].y, uz = d[c].z, uw = d[c].w;
        const __half2 x = *reinterpret_cast<const __half2*>(&ux);
        const __half2 y = *reinterpret_cast<const __half2*>(&uy);
        const __half2 z = *reinterpret_cast<const __half2*>(&uz);
        const __half2 w = *reinterpret_cast<const __half2*>(&uw);
        __half2 r, i;
        if (MU == 0) {  // h0 = p0 - S i p3, h1 = p1 - S i p2
            r = __hfma2(c2(sp, sp), __lowhigh2highlow(w), x);
            i = __hfma2(c2(sm, sm), __lowhigh2highlow(z), y);
        } else if (MU == 1) {  // h0 = p0 + S p3, h1 = p1 - S p2
            r = __hfma2(c2(sp, sm), __lowhigh2highlow(z), x);
            i = __hfma2(c2(sp, sm), __lowhigh2highlow(w), y);
        } else if (MU == 2) {  // h0 = p0 - S i p2, h1 = p1 + S i p3
            r = __hfma2(c2(sp, sm), w, x);
            i = __hfma2(c2(sm, sp), z, y);
        } else {  // h0 = p0 - S p2, h1 = p1 - S p3
            r = __hfma2(c2(sm, sm), z, x);
            i = __hfma2(c2(sm, sm), w, y);
        }
        h.re[c] = __half22float2(r);
        h.im[c] = __half22float2(i);
    }
}

// w = U h (ADJ = false) or U^dag h (ADJ = true), both half-spin rows at once.
template <bool ADJ>
__device__ __forceinline__ void su3_mul_p(const cpx<float> U[3][3], const PHalf& h, PHalf& w) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float2 wr, wi;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const cpx<float> u = ADJ ? U[k][i] : U[i][k];
            const float ui = ADJ ? -u.im : u.im;  // the adjoint takes conj(U_ki)
            if (k == 0) {
                wr = mul2(bc2(u.re), h.re[0]);
                wi = mul2(bc2(u.re), h.im[0]);
            } else {
                wr = fma2(bc2(u.re), h.re[k], wr);
                wi = fma2(bc2(u.re), h.im[k], wi);
            }
            wr = fma2(bc2(-ui), h.im[k], wr);
            wi = fma2(bc2(ui), h.re[k], wi);
        }
        w.re[i] = wr;
        w.im[i] = wi;
    }
}

// acc (+)= sc * (1 - S g_mu)-image of w (same equations as expand()).
template <int MU, int S, bool FIRST>
__device__ __forceinline__ void expand_p(PSpinor& a, const PHalf& w, float sc) {
    const float t = (float)S * sc;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float2 kr, ki, xr, xi;  // lower pair += kr * xr (re parts), ki * xi (im parts)
        if (MU == 0) {  // (S i w1, S i w0)
            kr = bc2(-t), xr = sw2(w.im[c]);
            ki = bc2(t), xi = sw2(w.re[c]);
        } else if (MU == 1) {  // (-S w1, S w0)
            kr = make_float2(-t, t), xr = sw2(w.re[c]);
            ki = make_float2(-t, t), xi = sw2(w.im[c]);
        } else if (MU == 2) {  // (S i w0, -S i w1)
            kr = make_float2(-t, t), xr = w.im[c];
            ki = make_float2(t, -t), xi = w.re[c];
        } else {  // (-S w0, -S w1)
            kr = bc2(-t), xr = w.re[c];
            ki = bc2(-t), xi = w.im[c];
        }
        if (FIRST) {
            a.re01[c] = mul2(bc2(sc), w.re[c]);
            a.im01[c] = mul2(bc2(sc), w.im[c]);
            a.re23[c] = mul2(kr, xr);
            a.im23[c] = mul2(ki, xi);
        } else {
            a.re01[c] = fma2(bc2(sc), w.re[c], a.re01[c]);
            a.im01[c] = fma2(bc2(sc), w.im[c], a.im01[c]);
            a.re23[c] = fma2(kr, xr, a.re23[c]);
            a.im23[c] = fma2(ki, xi, a.im23[c]);
        }
    }
}

template <int SP, int GP, int R, bool DAG, int MU, bool FIRST>
__device__ __forceinline__ void hop_dir_p(PSpinor& acc, const HopParams& P, const char* in, int p, int h,
                                          const int c[4], int s) {
    using SF = SpinorFmt<SP>;
    using GF = GaugeFmt<GP, R>;
    const Geom& g = P.g;
    const int L = g.L[MU];
    const int smu = MU == 0 ? 1 : MU == 1 ? g.L[0] : MU == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
    constexpr int SF_ = DAG ? -1 : 1;
    {
        const bool wrap = c[MU] == L - 1;
        const int sn = wrap ? s - (L - 1) * smu : s + smu;
        PSpinor q;
        PHalf hh, w;
        cpx<float> U[3][3];
        float sc;
        SF::load_packed(in, g.stride, sn >> 1, q, sc);
        GF::load(P.gauge, g.stride, p * 4 + MU, h, U);
        project_p<MU, SF_>(q, hh);
        if (wrap) {
            const float er = (float)g.ph[MU][0], ei = (float)g.ph[MU][1];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 r = hh.re[k], m = hh.im[k];
                hh.re[k] = fma2(bc2(-ei), m, mul2(bc2(er), r));
                hh.im[k] = fma2(bc2(ei), r, mul2(bc2(er), m));
            }
        }
        su3_mul_p<false>(U, hh, w);
        expand_p<MU, SF_, FIRST>(acc, w, sc);
    }
    {
        const bool wrap = c[MU] == 0;
        const int sn = wrap ? s + (L - 1) * smu : s - smu;
        const int hn = sn >> 1;
        PSpinor q;
        PHalf hh, w;
        cpx<float> U[3][3];
        float sc;
        SF::load_packed(in, g.stride, hn, q, sc);
        GF::load(P.gauge, g.stride, (1 - p) * 4 + MU, hn, U);
        project_p<MU, -SF_>(q, hh);
        if (wrap) {
            const float er = (float)g.ph[MU][0], ei = -(float)g.ph[MU][1];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 r = hh.re[k], m = hh.im[k];
                hh.re[k] = fma2(bc2(-ei), m, mul2(bc2(er), r));
                hh.im[k] = fma2(bc2(ei), r, mul2(bc2(er), m));
            }
        }
        su3_mul_p<true>(U, hh, w);
        expand_p<MU, -SF_, false>(acc, w, sc);
    }
}

template <int SP, int GP, int R, bool DAG, int MINB, int PF = 0>
__global__ void __launch_bounds__(256, MINB) hop_kernel_p(const HopParams P) {
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
    const float a = (float)P.a;
    double nrm = 0.0;
    for (int h = sb * blockDim.x + threadIdx.x; h - (int)threadIdx.x < g.Vh; h += nb * blockDim.x) {
        if (h >= g.Vh) continue;
        int c[4], s;
        site_of_half(h, p, g, c, s);
        hop_prefetch<SP, GP, R, PF>(P, in, p, h, c, s);
        PSpinor acc;
        hop_dir_p<SP, GP, R, DAG, 0, true>(acc, P, in, p, h, c, s);
        hop_dir_p<SP, GP, R, DAG, 1, false>(acc, P, in, p, h, c, s);
        hop_dir_p<SP, GP, R, DAG, 2, false>(acc, P, in, p, h, c, s);
        hop_dir_p<SP, GP, R, DAG, 3, false>(acc, P, in, p, h, c, s);
        if (P.xpay) {
            PSpinor xq;
            float xs;
            SF::load_packed(x, g.stride, h, xq, xs);
            const float2 A = bc2(a), X = bc2(xs);
#pragma unroll
            for (int cc = 0; cc < 3; cc++) {
                acc.re01[cc] = fma2(A, acc.re01[cc], mul2(X, xq.re01[cc]));
                acc.im01[cc] = fma2(A, acc.im01[cc], mul2(X, xq.im01[cc]));
                acc.re23[cc] = fma2(A, acc.re23[cc], mul2(X, xq.re23[cc]));
                acc.im23[cc] = fma2(A, acc.im23[cc], mul2(X, xq.im23[cc]));
            }
        } else if (P.a != 1.0) {
            const float2 A = bc2(a);
#pragma unroll
            for (int cc = 0; cc < 3; cc++) {
                acc.re01[cc] = mul2(A, acc.re01[cc]);
                acc.im01[cc] = mul2(A, acc.im01[cc]);
                acc.re23[cc] = mul2(A, acc.re23[cc]);
                acc.im23[cc] = mul2(A, acc.im23[cc]);
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

// ---------------------------------------------------------------------------
// Register-blocked multi-RHS stencil: one thread computes one output site for
// NB right-hand sides.  Per hop the neighbour index is computed and the link
// loaded and completed once, then applied to the NB neighbour spinors, so the
// link traffic through L1/L2, the 12 -> 18 reconstruction and the index
// arithmetic are shared by NB right-hand sides.  The arithmetic per
// right-hand side is that of hop_kernel_p.  Grid: blockIdx.x = site_block *
// (nrhs / NB) + group.  A group runs unless all its right-hand sides are
// flagged to be skipped; a flagged member is computed but neither stored nor
// reduced, so its output keeps its old value as with the other kernels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void apply_phase_p(PHalf& hh, float er, float ei) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float2 r = hh.re[k], m = hh.im[k];
        hh.re[k] = fma2(bc2(-ei), m, mul2(bc2(er), r));
        hh.im[k] = fma2(bc2(ei), r, mul2(bc2(er), m));
    }
}

// The neighbour's projected half spinor and storage scale: loaded and
// projected in FP32 (HP = false), or (F16, HP = true) projected on the stored
// packed halves and then converted (project_f16_packed).
template <int SP, int MU, int S, bool HP>
__device__ __forceinline__ void load_project(const char* in, int stride, int hn, PHalf& hh, float& sc) {
    using SF = SpinorFmt<SP>;
    if constexpr (HP) {
        uint4 d[3];
        const uint4* b = reinterpret_cast<const uint4*>(in) + hn;
#pragma unroll
        for (int cc = 0; cc < 3; cc++) d[cc] = __ldg(b + (size_t)cc * stride);
        sc = SF::load_scale(in, stride, hn);
        project_f16_packed<MU, S>(d, hh);
    } else {
        PSpinor q;
        SF::load_packed(in, stride, hn, q, sc);
        project_p<MU, S>(q, hh);
    }
}

template <int SP, int GP, int R, bool DAG, int MU, bool FIRST, int NB, bool HP = false>
__device__ __forceinline__ void hop_dir_pm(PSpinor (&acc)[NB], const HopParams& P, const char* in, int p, int h,
                                           const int c[4], int s) {
    using SF = SpinorFmt<SP>;
    using GF = GaugeFmt<GP, R>;
    const Geom& g = P.g;
    const int L = g.L[MU];
    const int smu = MU == 0 ? 1 : MU == 1 ? g.L[0] : MU == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
    constexpr int SF_ = DAG ? -1 : 1;
    {
        const bool wrap = c[MU] == L - 1;
        const int hn = (wrap ? s - (L - 1) * smu : s + smu) >> 1;
        cpx<float> U[3][3];
        GF::load(P.gauge, g.stride, p * 4 + MU, h, U);
#pragma unroll
        for (int r = 0; r < NB; r++) {
            PHalf hh, w;
            float sc;
            load_project<SP, MU, SF_, HP>(in + r * P.in_rstep, g.stride, hn, hh, sc);
            if (wrap) apply_phase_p(hh, (float)g.ph[MU][0], (float)g.ph[MU][1]);
            su3_mul_p<false>(U, hh, w);
            expand_p<MU, SF_, FIRST>(acc[r], w, sc);
        }
    }
    {
        const bool wrap = c[MU] == 0;
        const int hn = (wrap ? s + (L - 1) * smu : s - smu) >> 1;
        cpx<float> U[3][3];
        GF::load(P.gauge, g.stride, (1 - p) * 4 + MU, hn, U);
#pragma unroll
        for (int r = 0; r < NB; r++) {
            PHalf hh, w;
            float sc;
            load_project<SP, MU, -SF_, HP>(in + r * P.in_rstep, g.stride, hn, hh, sc);
            if (wrap) apply_phase_p(hh, (float)g.ph[MU][0], -(float)g.ph[MU][1]);
            su3_mul_p<true>(U, hh, w);
            expand_p<MU, -SF_, false>(acc[r], w, sc);
        }
    }
}

template <int SP, int GP, int R, bool DAG, int MINB, int NB, bool HP = false>
__global__ void __launch_bounds__(256, MINB) hop_kernel_pm(const HopParams P) {
    using SF = SpinorFmt<SP>;
    const int ng = P.nrhs / NB;
    const int grp = blockIdx.x % ng;
    const int sb = blockIdx.x / ng;
    const int nb = gridDim.x / ng;
    const int k0 = grp * NB;
    pdl_wait();
    unsigned act = 0;
#pragma unroll
    for (int r = 0; r < NB; r++)
        if (!P.skip || !__ldcg(P.skip + (size_t)(k0 + r) * P.skip_stride)) act |= 1u << r;
    if (!act) return;
    const int p = P.full ? (int)blockIdx.y : P.out_parity;
    const int pin = 1 - p;
    char* out = P.out + (P.full ? p * P.out_pstep : 0) + k0 * P.out_rstep;
    const char* in = P.in + (P.full ? pin * P.in_pstep : 0) + k0 * P.in_rstep;
    const char* x = P.x ? P.x + (P.full ? p * P.x_pstep : 0) + k0 * P.x_rstep : nullptr;
    const Geom& g = P.g;
    const float a = (float)P.a;
    double nrm[NB];
#pragma unroll
    for (int r = 0; r < NB; r++) nrm[r] = 0.0;
    for (int h = sb * blockDim.x + threadIdx.x; h - (int)threadIdx.x < g.Vh; h += nb * blockDim.x) {
        if (h >= g.Vh) continue;
        int c[4], s;
        site_of_half(h, p, g, c, s);
        PSpinor acc[NB];
        hop_dir_pm<SP, GP, R, DAG, 0, true, NB, HP>(acc, P, in, p, h, c, s);
        hop_dir_pm<SP, GP, R, DAG, 1, false, NB, HP>(acc, P, in, p, h, c, s);
        hop_dir_pm<SP, GP, R, DAG, 2, false, NB, HP>(acc, P, in, p, h, c, s);
        hop_dir_pm<SP, GP, R, DAG, 3, false, NB, HP>(acc, P, in, p, h, c, s);
#pragma unroll
        for (int r = 0; r < NB; r++) {
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
        for (int r = 0; r < NB; r++)
            if (act >> r & 1u) grid_reduce(nrm[r], P.red, k0 + r, nb * gridDim.y, sb + nb * blockIdx.y);
    }
}

// One direction mu of the link-staged multi-RHS kernel: the links come from
// the thread's shared-memory slots (slot j = 2 mu forward, 2 mu + 1
// backward), the neighbour indices and wrap flags were computed once for all
// right-hand sides.  Same arithmetic as hop_dir_p.
template <int SP, int GP, int R, bool DAG, int MU, bool FIRST>
__device__ __forceinline__ void hop_dir_rl(PSpinor& acc, const HopParams& P, const char* in, const int hn[8],
                                           unsigned wrap, const typename GaugeFmt<GP, R>::chunk_t* lsm, int T) {
    using SF = SpinorFmt<SP>;
    using GF = GaugeFmt<GP, R>;
    const Geom& g = P.g;
    constexpr int SF_ = DAG ? -1 : 1;
    {
        PSpinor q;
        PHalf hh, w;
        cpx<float> U[3][3];
        float sc;
        SF::load_packed(in, g.stride, hn[2 * MU], q, sc);
        GF::decode(lsm + (2 * MU) * GF::nchunk * T, T, U);
        project_p<MU, SF_>(q, hh);
        if (wrap >> (2 * MU) & 1u) apply_phase_p(hh, (float)g.ph[MU][0], (float)g.ph[MU][1]);
        su3_mul_p<false>(U, hh, w);
        expand_p<MU, SF_, FIRST>(acc, w, sc);
    }
    {
        PSpinor q;
        PHalf hh, w;
        cpx<float> U[3][3];
        float sc;
        SF::load_packed(in, g.stride, hn[2 * MU + 1], q, sc);
        GF::decode(lsm + (2 * MU + 1) * GF::nchunk * T, T, U);
        project_p<MU, -SF_>(q, hh);
        if (wrap >> (2 * MU + 1) & 1u) apply_phase_p(hh, (float)g.ph[MU][0], -(float)g.ph[MU][1]);
        su3_mul_p<true>(U, hh, w);
        expand_p<MU, -SF_, false>(acc, w, sc);
    }
}

// Multi-RHS hop with the links staged once per site (non-reducing launches):
// a block covers one tile of sites for every right-hand side.  Each thread
// copies its site's eight links (12 reals each, as stored) into its own
// shared-memory slots, laid out [link][chunk][thread] so that a warp's
// accesses are conflict-free,
// computes the neighbour indices and wrap flags once, and then loops over the
// right-hand sides reading only their neighbour spinors from global memory.
// A thread reads only the slots it wrote, so no barrier is needed.  Dynamic
// shared memory: 8 * nchunk * sizeof(chunk_t) bytes per thread.  Staging the
// decoded links instead (nine float2 per link) measured slower: the larger
// slots limit the resident warps (F32 12 RHS: 97.4 against 68.2 us per RHS).
template <int SP, int GP, int R, bool DAG, int MINB>
__global__ void __launch_bounds__(256, MINB) hop_kernel_rl(const HopParams P) {
    using SF = SpinorFmt<SP>;
    using GF = GaugeFmt<GP, R>;
    using CT = typename GF::chunk_t;
    extern __shared__ __align__(16) unsigned char rl_smem[];
    const int T = blockDim.x, t = threadIdx.x;
    const CT* lsm = reinterpret_cast<const CT*>(rl_smem) + t;
    const int sb = blockIdx.x, nb = gridDim.x;
    pdl_wait();
    const int p = P.full ? (int)blockIdx.y : P.out_parity;
    const int pin = 1 - p;
    const Geom& g = P.g;
    const float a = (float)P.a;
    for (int h = sb * T + t; h - t < g.Vh; h += nb * T) {
        if (h >= g.Vh) continue;
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
            CT* dst = reinterpret_cast<CT*>(rl_smem) + t;
#pragma unroll
            for (int j = 0; j < 8; j++)
                GF::load_chunks(P.gauge, g.stride, (j & 1 ? 1 - p : p) * 4 + j / 2, j & 1 ? hn[j] : h,
                                dst + j * GF::nchunk * T, T);
        }
        for (int r = 0; r < P.nrhs; r++) {
            if (P.skip && __ldcg(P.skip + (size_t)r * P.skip_stride)) continue;
            const char* in = P.in + (P.full ? pin * P.in_pstep : 0) + r * P.in_rstep;
            PSpinor A;
            hop_dir_rl<SP, GP, R, DAG, 0, true>(A, P, in, hn, wrap, lsm, T);
            hop_dir_rl<SP, GP, R, DAG, 1, false>(A, P, in, hn, wrap, lsm, T);
            hop_dir_rl<SP, GP, R, DAG, 2, false>(A, P, in, hn, wrap, lsm, T);
            hop_dir_rl<SP, GP, R, DAG, 3, false>(A, P, in, hn, wrap, lsm, T);
            if (P.xpay) {
                const char* x = P.x + (P.full ? p * P.x_pstep : 0) + r * P.x_rstep;
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
            char* out = P.out + (P.full ? p * P.out_pstep : 0) + r * P.out_rstep;
            SF::template store_packed<true>(out, g.stride, h, A);
        }
    }
    pdl_trigger();
}

// One output site of the pipelined F16 / BF16 hop (hop_kernel_pipe, and the
// batch's tile form): the eight hops of site h of parity p, each hop's raw
// data -- the neighbour's three 16-byte chunks and scale, the link's three
// 8-byte chunks -- copied with cp.async into this thread's own shared-memory
// slots D hops ahead (sp [D][3][T], lk [D][3][T], scs [D][T]; T the block
// size, t the thread).  Every copy group is waited for before the function
// returns, so the slots are free for the next site.
template <int SP, bool DAG, int J>
__device__ __forceinline__ void pipe_hop(PSpinor& acc, const uint4 (&d)[3], float sc, const cpx<float> (&U)[3][3],
                                         unsigned wrap, const Geom& g) {
    constexpr int MU = J >> 1;
    constexpr bool FWD = (J & 1) == 0;
    constexpr int SF_ = DAG ? -1 : 1;
    constexpr int S = FWD ? SF_ : -SF_;
    PHalf hh, w;
    if constexpr (SP == P_F16) {
        project_f16_packed<MU, S>(d, hh);
    } else {  // BF16: exact conversion to FP32, projection there
        using LT = LowT<SP>;
        PSpinor q;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            q.re01[c] = LT::to_f2(d[c].x);
            q.im01[c] = LT::to_f2(d[c].y);
            q.re23[c] = LT::to_f2(d[c].z);
            q.im23[c] = LT::to_f2(d[c].w);
        }
        project_p<MU, S>(q, hh);
    }
    if (wrap >> J & 1u) apply_phase_p(hh, (float)g.ph[MU][0], FWD ? (float)g.ph[MU][1] : -(float)g.ph[MU][1]);
    su3_mul_p<!FWD>(U, hh, w);
    expand_p<MU, S, J == 0>(acc, w, sc);
}

template <int SP, bool DAG, int D, int T>
__device__ __forceinline__ void pipe_site(PSpinor& acc, const char* in, const char* gauge, const Geom& g, int p,
                                          int h, uint4* sp, uint2* lk, float* scs, int t) {
    using GF = GaugeFmt<SP, 12>;
    const int pin = 1 - p;
    const float* gscale = reinterpret_cast<const float*>(in + 48LL * g.stride);
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
    // hop j's raw data into slot j % D: the neighbour's chunks and scale,
    // the link of the site (forward) or of the neighbour (backward)
    auto issue = [&](int j) {
        const int slot = j % D;
        const int n = hn[j];
        const uint4* gs = reinterpret_cast<const uint4*>(in) + n;
#pragma unroll
        for (int kk = 0; kk < 3; kk++) __pipeline_memcpy_async(&sp[(slot * 3 + kk) * T + t], gs + (size_t)kk * g.stride, 16);
        __pipeline_memcpy_async(&scs[slot * T + t], gscale + n, 4);
        const int blk = ((j & 1) ? pin : p) * 4 + (j >> 1);
        const uint2* gl = reinterpret_cast<const uint2*>(gauge) + (size_t)blk * 3 * g.stride + ((j & 1) ? n : h);
#pragma unroll
        for (int kk = 0; kk < 3; kk++) __pipeline_memcpy_async(&lk[(slot * 3 + kk) * T + t], gl + (size_t)kk * g.stride, 8);
        __pipeline_commit();
    };
#pragma unroll
    for (int j = 0; j < D; j++) issue(j);
#define WL_PIPE_HOP(J)                                                                                        \
    {                                                                                                         \
        __pipeline_wait_prior(D - 1);                                                                         \
        constexpr int slot = (J) % D;                                                                         \
        uint4 d[3];                                                                                           \
        _Pragma("unroll") for (int kk = 0; kk < 3; kk++) d[kk] = sp[(slot * 3 + kk) * T + t];                 \
        const float sc = scs[slot * T + t];                                                                   \
        cpx<float> U[3][3];                                                                                   \
        GF::decode(&lk[slot * 3 * T + t], T, U);                                                              \
        pipe_hop<SP, DAG, (J)>(acc, d, sc, U, wrap, g);                                                       \
        if ((J) + D < 8) issue((J) + D);                                                                      \
        else __pipeline_commit();                                                                             \
    }
    WL_PIPE_HOP(0) WL_PIPE_HOP(1) WL_PIPE_HOP(2) WL_PIPE_HOP(3)
    WL_PIPE_HOP(4) WL_PIPE_HOP(5) WL_PIPE_HOP(6) WL_PIPE_HOP(7)
#undef WL_PIPE_HOP
}

// Kernel variants: v = 0..5: v % 3 is the register budget (blocks of 256
// threads guaranteed resident per SM: 128 / 85 / 64 registers per thread;
// FP64: 255 / 128 / 85, its operands take two registers each); v >= 3 is the
// paired-FP32 kernel (single and reduced precision only).  v = 6..9: the
// register-blocked multi-RHS kernel with NB = 2, 2, 3, 4 right-hand sides per
// thread and 255, 128, 255, 255 registers (single and reduced precision,
// 12-real links, NB dividing nrhs; NB >= 3 spills at 128 registers).
// v = 10: the link-staged kernel; v = 11: the tensor-core kernel (F16/BF16).
// v = 12..17: the paired kernel with SPT sites per thread (12: SPT 2 at 128
// registers, 13: SPT 2 at 255, 14: SPT 4 at 255; at 85 registers two sites
// spill about 1 KB) and, F16 only, the packed-half projection with one site
// per thread (15, 16, 17: 128, 85, 64 registers).
// v = 18, 19: the register-blocked kernel (NB = 2) with the F16 packed
// projection at 128 and 255 registers (at 85 it spills 1.2 KB).
// v = 20-22: the F16 / BF16 kernel with its neighbour data copied ahead into
// shared memory (cp.async), 2 / 3 / 3 hops ahead at 80 / 80 / 96 registers.
// v = 23-25: the kernels of v = 0 and 3 at 128 registers with L2 prefetches
// of the site's links at its start (23: scalar, 24: paired) and of its links
// and neighbour spinors (25: paired); single and reduced precision.
// v = 26: the t-slab streaming kernel (dslash_slab.cu): tiles of a 3-d slice
// swept along t, the neighbouring input slices staged in shared memory by
// bulk asynchronous copies; one parity, one RHS, non-reducing launches, tiles
// that divide the slice.
// v = 27, 28: the pipelined F16 / BF16 kernel with two right-hand sides per thread
// (one link copy and decode per hop for both), 2 / 3 hops ahead at 128
// registers; even nrhs.
constexpr int kHopVariants = 29;
constexpr int kHopPipe2Variant = 27;     // first two-RHS pipelined variant
constexpr int kHopPrefetchVariant = 23;  // first prefetching variant
constexpr int kHopSlabVariant = 26;      // hop_kernel_slab
constexpr int kHopBaseVariants = 6;
constexpr int kHopStagedVariant = 10;  // hop_kernel_rl (128 registers)
constexpr int kHopMmaVariant = 11;     // hop_kernel_mma (128 registers)
constexpr int kHopSptVariant = 12;     // first hop_kernel_ps variant
constexpr int kHopSptLast = 17;      // last hop_kernel_ps variant
constexpr bool hop_variant_is_pipe(int v) { return v >= 20 && v <= 22; }
constexpr bool hop_variant_is_pipe2(int v) { return v == kHopPipe2Variant || v == kHopPipe2Variant + 1; }
constexpr bool hop_variant_is_pf(int v) { return v >= kHopPrefetchVariant && v <= kHopPrefetchVariant + 2; }
constexpr int hop_variant_pf(int v) { return !hop_variant_is_pf(v) ? 0 : v == kHopPrefetchVariant + 2 ? 2 : 1; }
constexpr bool hop_variant_is_ps(int v) { return (v >= kHopSptVariant && v <= kHopSptLast) || hop_variant_is_pipe(v); }
constexpr int hop_variant_nb(int v) {
    return v == 18 || v == 19 || hop_variant_is_pipe2(v) ? 2
           : v < kHopBaseVariants || v >= kHopStagedVariant ? 1 : v == 6 || v == 7 ? 2 : v == 8 ? 3 : 4;
}
constexpr int hop_variant_spt(int v) { return v == 12 || v == 13 ? 2 : v == 14 ? 4 : 1; }
constexpr bool hop_variant_hproj(int v) { return (v >= 15 && v <= 17) || v == 18 || v == 19; }
// FP64 operands take two registers per real: their budgets start at 255
// registers.
constexpr bool wide_regs(int sp) { return sp == P_F64; }
constexpr bool float_storage(int sp) { return sp == P_F32 || sp == P_F16 || sp == P_BF16; }
constexpr int hop_variant_minb(int v, int sp) {
    return v < kHopBaseVariants ? (wide_regs(sp) ? 1 : 2) + v % 3
           : v == 13 || v == 14 || v == 19 ? 1
           : v == 16 || v == 20 || v == 21 ? 3
           : v == 17 ? 4
           : v == 18 || v == 22 || hop_variant_is_pf(v) || v == kHopSlabVariant || hop_variant_is_pipe2(v) ? 2
           : v >= kHopStagedVariant ? 2
           : v == 7 ? 2 : 1;
}
inline bool hop_variant_valid(int v, Prec sp, int recon, int nrhs) {
    if (v < 0 || v >= kHopVariants) return false;
    if (v < kHopBaseVariants) return true;
    if (hop_variant_is_pf(v)) return float_storage(sp);
    if (v == kHopSlabVariant) return float_storage(sp) && nrhs == 1;
    if (hop_variant_is_pipe2(v)) return (sp == P_F16 || sp == P_BF16) && recon == 12 && nrhs >= 2 && nrhs % 2 == 0;
    if (hop_variant_is_pipe(v)) return (sp == P_F16 || sp == P_BF16) && recon == 12;
    if (hop_variant_is_ps(v)) return hop_variant_hproj(v) ? sp == P_F16 : float_storage(sp);
    if (v == 18 || v == 19) return sp == P_F16 && recon == 12 && nrhs >= 2 && nrhs % 2 == 0;
    if (v == kHopMmaVariant) return (sp == P_F16 || sp == P_BF16) && recon == 12 && nrhs > 1;
    if (v >= kHopStagedVariant) return float_storage(sp) && recon == 12 && nrhs > 1;
    const int nb = hop_variant_nb(v);
    return float_storage(sp) && recon == 12 && nrhs >= nb && nrhs % nb == 0;
}

// The register-blocked kernels (instantiated in dslash_mrhs.cu).
template <int SP, int GP, int R>
void launch_hop_mrhs(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant,
                     cudaStream_t st);
// The tensor-core kernel (dslash_mma.cu; F16 and BF16 storage, 12-real links).
template <int SP>
void launch_hop_mma(const HopParams& P, int block, int site_blocks, int ny, bool dag, cudaStream_t st);
// The t-slab streaming kernel (dslash_slab.cu; F32/F16/BF16, one parity and
// one RHS, non-reducing): hop_slab_fits says whether a block size tiles the
// lattice's 3-d slices; stage_timeouts reads how many of its bounded waits
// have given up since the library was loaded (synchronises the stream).
template <int SP, int GP, int R>
void launch_hop_slab(const HopParams& P, int block, bool dag, cudaStream_t st);
// The pipelined kernels (dslash_pipe.cuh, instantiated in dslash_pipe_f16.cu
// and dslash_pipe_bf16.cu; F16-12 or BF16-12): one right-hand side per thread
// (variants 20-22) and two (27, 28; even nrhs).
template <int SP>
void launch_hop_pipe(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant,
                     cudaStream_t st);
template <int SP>
void launch_hop_pipe2(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant,
                      cudaStream_t st);
extern template void launch_hop_pipe<P_F16>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_pipe<P_BF16>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_pipe2<P_F16>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_pipe2<P_BF16>(const HopParams&, int, int, int, bool, int, cudaStream_t);
bool hop_slab_fits(const Geom& g, int block);
unsigned long long stage_timeouts(cudaStream_t st);
// Sites per thread and the F16 packed projection (dslash_spt.cu; F32/F16/BF16).
template <int SP, int GP, int R>
void launch_hop_ps(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant, cudaStream_t st);

template <int SP, int GP, int R, int V>
void launch_hop_rl_v(const HopParams& P, int block, int site_blocks, int ny, bool dag, cudaStream_t st) {
    constexpr int MINB = hop_variant_minb(V, SP);
    using GF = GaugeFmt<GP, R>;
    constexpr size_t per_thread = (size_t)8 * GF::nchunk * sizeof(typename GF::chunk_t);
    const dim3 grid(site_blocks, ny);
    auto k = dag ? hop_kernel_rl<SP, GP, R, true, MINB> : hop_kernel_rl<SP, GP, R, false, MINB>;
    // the larger dynamic shared memory, once per device and dagger (the
    // attribute is per device)
    static bool opted[64][2] = {};
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    if (!opted[dev][dag]) {
        WL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per_thread * 256)));
        opted[dev][dag] = true;
    }
    launch_dep_smem(k, grid, dim3(block), per_thread * block, st, P);
}

template <int SP, int GP, int R, int V>
void launch_hop_mrhs_v(const HopParams& P, int block, int site_blocks, int ny, bool dag, cudaStream_t st) {
    constexpr int NB = hop_variant_nb(V), MINB = hop_variant_minb(V, SP);
    constexpr bool HP = hop_variant_hproj(V) && SP == P_F16;
    const dim3 grid(site_blocks * (P.nrhs / NB), ny);
    if (dag) launch_dep(hop_kernel_pm<SP, GP, R, true, MINB, NB, HP>, grid, dim3(block), st, P);
    else launch_dep(hop_kernel_pm<SP, GP, R, false, MINB, NB, HP>, grid, dim3(block), st, P);
}

template <int SP, int GP, int R, int V>
void launch_hop_v(const HopParams& P, dim3 grid, int block, bool dag, cudaStream_t st) {
    constexpr int MINB = hop_variant_minb(V, SP), PF = hop_variant_pf(V);
    constexpr bool paired = PF ? V > kHopPrefetchVariant : V >= 3;
    if constexpr (paired && float_storage(SP)) {
        if (dag) launch_dep(hop_kernel_p<SP, GP, R, true, MINB, PF>, grid, dim3(block), st, P);
        else launch_dep(hop_kernel_p<SP, GP, R, false, MINB, PF>, grid, dim3(block), st, P);
    } else {
        if (dag) launch_dep(hop_kernel<SP, GP, R, true, MINB, PF>, grid, dim3(block), st, P);
        else launch_dep(hop_kernel<SP, GP, R, false, MINB, PF>, grid, dim3(block), st, P);
    }
}

// site_blocks: blocks over the half lattice; the grid covers them once per
// right-hand side (or group of right-hand sides).
template <int SP, int GP, int R>
void launch_hop_prec(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant,
                     cudaStream_t st) {
    if (hop_variant_is_ps(variant)) {
        if constexpr (float_storage(SP)) {
            launch_hop_ps<SP, GP, R>(P, block, site_blocks, ny, dag, variant, st);
            return;
        }
        throw Error(7, "the sites-per-thread hop variants need F32/F16/BF16 spinors");
    }
    const dim3 grid(site_blocks * P.nrhs, ny);
    if (variant == kHopSlabVariant) {
        if constexpr (float_storage(SP)) {
            launch_hop_slab<SP, GP, R>(P, block, dag, st);
            return;
        }
        throw Error(7, "the slab hop variant needs F32/F16/BF16 spinors");
    }
    if (hop_variant_is_pipe2(variant)) {
        if constexpr ((SP == P_F16 || SP == P_BF16) && GP == SP && R == 12) {
            launch_hop_pipe2<SP>(P, block, site_blocks, ny, dag, variant, st);
            return;
        }
        throw Error(7, "the two-RHS pipelined hop variants need F16/BF16 spinors and 12-real links");
    }
    if (hop_variant_is_pf(variant)) {
        if constexpr (float_storage(SP)) {
            if (variant == kHopPrefetchVariant) launch_hop_v<SP, GP, R, kHopPrefetchVariant>(P, grid, block, dag, st);
            else if (variant == kHopPrefetchVariant + 1)
                launch_hop_v<SP, GP, R, kHopPrefetchVariant + 1>(P, grid, block, dag, st);
            else launch_hop_v<SP, GP, R, kHopPrefetchVariant + 2>(P, grid, block, dag, st);
            return;
        }
        throw Error(7, "the prefetching hop variants need F32/F16/BF16 spinors");
    }
    if (variant >= kHopBaseVariants) {
        if constexpr (float_storage(SP) && R == 12) {
            launch_hop_mrhs<SP, GP, R>(P, block, site_blocks, ny, dag, variant, st);
            return;
        }
        throw Error(7, "register-blocked hop variant needs F32/F16/BF16 spinors and 12-real links");
    }
    if (wide_regs(SP)) variant %= 3;
    switch (variant) {
        case 1: launch_hop_v<SP, GP, R, 1>(P, grid, block, dag, st); break;
        case 2: launch_hop_v<SP, GP, R, 2>(P, grid, block, dag, st); break;
        case 3: launch_hop_v<SP, GP, R, 3>(P, grid, block, dag, st); break;
        case 4: launch_hop_v<SP, GP, R, 4>(P, grid, block, dag, st); break;
        case 5: launch_hop_v<SP, GP, R, 5>(P, grid, block, dag, st); break;
        default: launch_hop_v<SP, GP, R, 0>(P, grid, block, dag, st); break;
    }
}

// Instantiated in the per-precision translation units.
extern template void launch_hop_prec<P_F64, P_F64, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_prec<P_F64, P_F64, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_prec<P_F32, P_F32, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_prec<P_F32, P_F32, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_prec<P_F16, P_F16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_prec<P_BF16, P_BF16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_prec<P_F16, P_F16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_prec<P_BF16, P_BF16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_ps<P_F32, P_F32, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_ps<P_F32, P_F32, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_ps<P_F16, P_F16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_ps<P_F16, P_F16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_ps<P_BF16, P_BF16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_ps<P_BF16, P_BF16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_mrhs<P_F32, P_F32, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_mrhs<P_F16, P_F16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
extern template void launch_hop_mrhs<P_BF16, P_BF16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);

}  // namespace wl
