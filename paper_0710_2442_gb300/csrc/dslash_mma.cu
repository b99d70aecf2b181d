// dslash_mma.cu -- the multi-RHS hopping term (Sec. 5, Eq. 3, batched over
// right-hand sides) with the link x half-spinor products on the tensor cores:
// mma.sync.m16n8k16 with F16 (or BF16) inputs and FP32 accumulation.  Hop
// kernel variant 11; F16/BF16 storage with 12-real links, any nrhs >= 2.
//
// Mapping.  One warp computes one output site for up to 16 right-hand sides
// (the MMA's M = 16 rows, one per right-hand side).  Per hop the product is
//   W (16 rhs x 12 reals) = H (16 rhs x 12 reals) . B (12 x 12 reals)
// where H holds the projected half spinors (1 -/+ g_mu) psi of the 16
// right-hand sides and B is the real form of the link acting on both half
// spins.  K = 16 holds the 12 reals of H as k = 2c + b (real part of half
// spin b, colour c) and k = 8 + 2c + b (imaginary part); k = 6, 7, 14, 15
// are zero.  The N = 16 outputs are two n-tiles: n-tile a holds W(half spin
// a, colour i) at columns (2i, 2i+1) = (re, im); columns 6, 7 are zero.
//
// With the PTX fragment layouts (lane = 4 g + t), lane (g, t) then holds
//   A: the projected half spin pair of colour t for right-hand sides g and
//      g + 8 -- exactly what one 16-byte chunk (colour t) of the stored
//      spinor gives after one packed-half FMA per register;
//   B: built from ONE link element, U_{g/2, t} (or conj(U_{t, g/2}) for the
//      backward hop);
//   C: W(0, t) and W(1, t) for right-hand sides g and g + 8,
// so each lane accumulates all four spins of colour t for its two
// right-hand sides (the lower spins are fixed by the projector: +-1 or
// +-i times an upper one), applies the neighbour's per-site scale in the
// FP32 accumulation, and at the end stores exactly one 16-byte chunk of the
// output per right-hand side.  Only the per-site maximum of the F16 scale
// needs the other lanes of the quad (two shuffles).
//
// Staging.  A warp takes 32 consecutive sites.  Lane l computes site l's
// neighbour indices and loads its eight links (coalesced), rebuilds row 3,
// multiplies a wrapping hop's link by the boundary phase (the backward hop
// uses (eta U)^dag = eta* U^dag), and writes the nine elements of each link
// to shared memory in the MMA's input type: 8 x 9 words per site, padded to
// 73 words so that both the staging writes and the per-site reads are free
// of bank conflicts.  The warp then walks its sites one by one; the
// neighbour indices come from the staging lane by shuffles.
//
// Rounding.  The projection is one packed-half FMA (rounded once to the
// storage type); the links enter the MMA rounded to it; products and sums
// are FP32.  Emulated on the CPU, this adds 1e-4 (F16) and 8e-4 (BF16) of
// relative L2 error to the 2.5e-4 and 2.0e-3 of the storage formats alone.
//
// Reducing launches (fused |out|^2) do not use this kernel; the dispatcher
// runs the paired-FP32 kernel for them.
#include "dslash_impl.cuh"

namespace wl {

namespace {

constexpr int kSiteWords = 73;  // 8 links x 9 elements + 1 (bank-conflict-free padding)
constexpr int kGroup = 16;      // right-hand sides per warp: the MMA's M

template <int P>
struct MmaT;
template <>
struct MmaT<P_F16> {
    using T2 = __half2;
    static constexpr uint32_t kOne = 0x3C00u;  // 1.0 as a 16-bit pattern
    __device__ static __forceinline__ T2 h2(uint32_t u) { return *reinterpret_cast<T2*>(&u); }
    __device__ static __forceinline__ uint32_t u32(T2 h) { return *reinterpret_cast<uint32_t*>(&h); }
    __device__ static __forceinline__ T2 pack(float a, float b) { return __floats2half2_rn(a, b); }
    __device__ static __forceinline__ float2 unpack(uint32_t u) { return __half22float2(h2(u)); }
    __device__ static __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%10,%10,%10,%10};\n"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
    }
};
template <>
struct MmaT<P_BF16> {
    using T2 = __nv_bfloat162;
    static constexpr uint32_t kOne = 0x3F80u;
    __device__ static __forceinline__ T2 h2(uint32_t u) { return *reinterpret_cast<T2*>(&u); }
    __device__ static __forceinline__ uint32_t u32(T2 h) { return *reinterpret_cast<uint32_t*>(&h); }
    __device__ static __forceinline__ T2 pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
    __device__ static __forceinline__ float2 unpack(uint32_t u) { return __bfloat1622float2(h2(u)); }
    __device__ static __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%10,%10,%10,%10};\n"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
    }
};

// The half2 constant (lo, hi) with lo, hi = +-1 (sign flags: 1 = negative).
template <int P, int NEG_LO, int NEG_HI>
__device__ __forceinline__ typename MmaT<P>::T2 pm_one() {
    constexpr uint32_t one = MmaT<P>::kOne;
    return MmaT<P>::h2((one | (NEG_LO ? 0x8000u : 0u)) | ((one | (NEG_HI ? 0x8000u : 0u)) << 16));
}

// (1 - S g_mu) psi for one colour, packed: the stored chunk holds the half2
// words x = (s0.re, s1.re), y = (s0.im, s1.im), z = (s2.re, s3.re),
// w = (s2.im, s3.im); the result is re = (h0.re, h1.re), im = (h0.im, h1.im)
// (the same equations as project(), one packed FMA per register).

template <int P, int MU, int S>
__device__ __forceinline__ void project_h(const uint4& d, uint32_t& re, uint32_t& im) {
    using M = MmaT<P>;
    using T2 = typename M::T2;
    const T2 x = M::h2(d.x), y = M::h2(d.y), z = M::h2(d.z), w = M::h2(d.w);
    constexpr int N = S < 0;  // "+S" is negative
    constexpr int Q = S > 0;  // "-S" is negative
    T2 r, i;
    if (MU == 0) {  // h0 = p0 - S i p3, h1 = p1 - S i p2
        r = __hfma2(pm_one<P, N, N>(), __lowhigh2highlow(w), x);
        i = __hfma2(pm_one<P, Q, Q>(), __lowhigh2highlow(z), y);
    } else if (MU == 1) {  // h0 = p0 + S p3, h1 = p1 - S p2
        r = __hfma2(pm_one<P, N, Q>(), __lowhigh2highlow(z), x);
        i = __hfma2(pm_one<P, N, Q>(), __lowhigh2highlow(w), y);
    } else if (MU == 2) {  // h0 = p0 - S i p2, h1 = p1 + S i p3
        r = __hfma2(pm_one<P, N, Q>(), w, x);
        i = __hfma2(pm_one<P, Q, N>(), z, y);
    } else {  // h0 = p0 - S p2, h1 = p1 - S p3
        r = __hfma2(pm_one<P, Q, Q>(), z, x);
        i = __hfma2(pm_one<P, Q, Q>(), w, y);
    }
    re = M::u32(r);
    im = M::u32(i);
}

__device__ __forceinline__ float2 f2fma(float s, float2 w, float2 acc) {
    return make_float2(fmaf(s, w.x, acc.x), fmaf(s, w.y, acc.y));
}
// acc + s * (i w)
__device__ __forceinline__ float2 f2fma_i(float s, float2 w, float2 acc) {
    return make_float2(fmaf(-s, w.y, acc.x), fmaf(s, w.x, acc.y));
}

// Raw neighbour data of one hop for the lane's two right-hand-side rows.
struct HopIn {
    uint4 d[2];
    float sc[2];
};

template <int SP>
__device__ __forceinline__ void load_hop(HopIn& in, const char* const (&inr)[2], const bool (&act)[2], int t,
                                         int stride, int hn) {
#pragma unroll
    for (int r = 0; r < 2; r++) {
        in.d[r] = make_uint4(0u, 0u, 0u, 0u);
        in.sc[r] = 0.f;
        if (act[r]) {
            if (t < 3) in.d[r] = __ldg(reinterpret_cast<const uint4*>(inr[r]) + (size_t)t * stride + hn);
            in.sc[r] = __ldg(reinterpret_cast<const float*>(inr[r] + 48LL * stride) + hn);
        }
    }
}

// Hop J (mu = J / 2; J even: forward, odd: backward) into the accumulators.
// bsel: the lane's link element (index into the site's 9 staged words of
// the hop, forward order i*3 + t; the backward hop reads t*3 + i) and
// whether it is used at all (bmask = all ones or zero).
template <int SP, bool DAG, int J>
__device__ __forceinline__ void mma_hop(float2 (&acc)[2][4], const HopIn& in, const uint32_t* ls, int efwd,
                                        int ebwd, bool bim, uint32_t bmask) {
    using M = MmaT<SP>;
    constexpr int MU = J >> 1;
    constexpr bool FWD = (J & 1) == 0;
    constexpr int SF = DAG ? -1 : 1;
    constexpr int S = FWD ? SF : -SF;  // forward (1 - SF g_mu), backward (1 + SF g_mu)
    uint32_t A[4];                     // rows g (re, im) -> A[0], A[2]; rows g + 8 -> A[1], A[3]
    project_h<SP, MU, S>(in.d[0], A[0], A[2]);
    project_h<SP, MU, S>(in.d[1], A[1], A[3]);
    // U'_{i,t}: U_{i,t} forward; conj(U_{t,i}) backward (the staged link is eta U).
    // The B registers hold it as 16-bit patterns: a sign flip is an XOR.
    const uint32_t u = ls[J * 9 + (FWD ? efwd : ebwd)] & bmask;
    const uint32_t ure = u & 0xFFFFu;
    const uint32_t uim = (u >> 16) ^ (FWD ? 0u : (u ? 0x8000u : 0u));
    const uint32_t p0 = bim ? uim : ure;             // coefficient of the real parts of H
    const uint32_t p1 = bim ? ure : (uim ^ (u ? 0x8000u : 0u));  // of the imaginary parts
    __syncwarp();  // converged warp for the aligned MMA
    float c0[4], c1[4];
    M::mma(c0, A, p0, p1);              // W(0, t): rows g (c0[0], c0[1]) and g + 8 (c0[2], c0[3])
    M::mma(c1, A, p0 << 16, p1 << 16);  // W(1, t)
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const float s = in.sc[r];
        const float2 w0 = make_float2(c0[2 * r], c0[2 * r + 1]);
        const float2 w1 = make_float2(c1[2 * r], c1[2 * r + 1]);
        acc[r][0] = f2fma(s, w0, acc[r][0]);
        acc[r][1] = f2fma(s, w1, acc[r][1]);
        const float ss = (float)S * s;
        if (MU == 0) {  // lower = (S i w1, S i w0)
            acc[r][2] = f2fma_i(ss, w1, acc[r][2]);
            acc[r][3] = f2fma_i(ss, w0, acc[r][3]);
        } else if (MU == 1) {  // (-S w1, S w0)
            acc[r][2] = f2fma(-ss, w1, acc[r][2]);
            acc[r][3] = f2fma(ss, w0, acc[r][3]);
        } else if (MU == 2) {  // (S i w0, -S i w1)
            acc[r][2] = f2fma_i(ss, w0, acc[r][2]);
            acc[r][3] = f2fma_i(-ss, w1, acc[r][3]);
        } else {  // (-S w0, -S w1)
            acc[r][2] = f2fma(-ss, w0, acc[r][2]);
            acc[r][3] = f2fma(-ss, w1, acc[r][3]);
        }
    }
}

template <int SP, bool DAG, int MINB>
__global__ void __launch_bounds__(256, MINB) hop_kernel_mma(const HopParams P) {
    using M = MmaT<SP>;
    using LT = LowT<SP>;
    using GF = GaugeFmt<SP, 12>;
    extern __shared__ __align__(16) uint32_t mma_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    uint32_t* lsm = mma_smem + warp * 32 * kSiteWords;
    const int ngrp = (P.nrhs + kGroup - 1) / kGroup;
    const int grp = blockIdx.x % ngrp;
    const int sb = blockIdx.x / ngrp, nb = gridDim.x / ngrp;
    const int k0 = grp * kGroup;
    const int nk = min(kGroup, P.nrhs - k0);
    pdl_wait();
    const int p = P.full ? (int)blockIdx.y : P.out_parity;
    const int pin = 1 - p;
    const Geom& geo = P.g;
    const int stride = geo.stride;
    // the lane's two right-hand-side rows, g and g + 8
    bool act[2];
    const char* inr[2];
    char* outr[2];
    const char* xr[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int row = g + 8 * r, k = k0 + row;
        act[r] = row < nk && !(P.skip && __ldcg(P.skip + (size_t)k * P.skip_stride));
        const int kk = row < nk ? k : k0;
        inr[r] = P.in + (P.full ? pin * P.in_pstep : 0) + kk * P.in_rstep;
        outr[r] = P.out + (P.full ? p * P.out_pstep : 0) + kk * P.out_rstep;
        xr[r] = P.x ? P.x + (P.full ? p * P.x_pstep : 0) + kk * P.x_rstep : nullptr;
    }
    const int bi = g >> 1;              // colour i of the lane's W column pair
    const bool bim = (g & 1) != 0;      // the pair's imaginary column
    const bool bvalid = g < 6 && t < 3;
    const int efwd = bvalid ? bi * 3 + t : 0, ebwd = bvalid ? t * 3 + bi : 0;
    const uint32_t bmask = bvalid ? 0xFFFFFFFFu : 0u;
    const float a = (float)P.a;
    const int ntiles = (geo.Vh + 31) >> 5;

    for (int tile = sb * nwarps + warp; tile < ntiles; tile += nb * nwarps) {
        const int base = tile << 5;
        const int ns = min(32, geo.Vh - base);
        // ---- staging: lane l prepares site base + l
        int hnb[8];
#pragma unroll
        for (int j = 0; j < 8; j++) hnb[j] = 0;
        if (lane < ns) {
            const int h = base + lane;
            int c[4], s;
            site_of_half(h, p, geo, c, s);
            unsigned wrap = 0;
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                const int L = geo.L[mu];
                const int smu = mu == 0 ? 1 : mu == 1 ? geo.L[0] : mu == 2 ? geo.L[0] * geo.L[1]
                                                                            : geo.L[0] * geo.L[1] * geo.L[2];
                const bool wf = c[mu] == L - 1, wb = c[mu] == 0;
                hnb[2 * mu] = (wf ? s - (L - 1) * smu : s + smu) >> 1;
                hnb[2 * mu + 1] = (wb ? s + (L - 1) * smu : s - smu) >> 1;
                wrap |= (unsigned)wf << (2 * mu) | (unsigned)wb << (2 * mu + 1);
            }
            uint32_t* dst = lsm + lane * kSiteWords;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int mu = j >> 1;
                cpx<float> U[3][3];
                GF::load(P.gauge, stride, ((j & 1) ? pin : p) * 4 + mu, (j & 1) ? hnb[j] : h, U);
                if (wrap >> j & 1u) {
                    const cpx<float> eta = {(float)geo.ph[mu][0], (float)geo.ph[mu][1]};
#pragma unroll
                    for (int e = 0; e < 9; e++) U[e / 3][e % 3] = cmul(eta, U[e / 3][e % 3]);
                }
#pragma unroll
                for (int e = 0; e < 9; e++) dst[j * 9 + e] = M::u32(M::pack(U[e / 3][e % 3].re, U[e / 3][e % 3].im));
            }
        }
        __syncwarp();
        // ---- the warp walks its sites
        for (int js = 0; js < ns; js++) {
            const uint32_t* ls = lsm + js * kSiteWords;
            HopIn hin[8];
            load_hop<SP>(hin[0], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[0], js));
            load_hop<SP>(hin[1], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[1], js));
            load_hop<SP>(hin[2], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[2], js));
            load_hop<SP>(hin[3], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[3], js));
            load_hop<SP>(hin[4], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[4], js));
            load_hop<SP>(hin[5], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[5], js));
            load_hop<SP>(hin[6], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[6], js));
            load_hop<SP>(hin[7], inr, act, t, stride, __shfl_sync(0xffffffffu, hnb[7], js));
            float2 acc[2][4];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[r][q] = make_float2(0.f, 0.f);
            mma_hop<SP, DAG, 0>(acc, hin[0], ls, efwd, ebwd, bim, bmask);
            mma_hop<SP, DAG, 1>(acc, hin[1], ls, efwd, ebwd, bim, bmask);
            mma_hop<SP, DAG, 2>(acc, hin[2], ls, efwd, ebwd, bim, bmask);
            mma_hop<SP, DAG, 3>(acc, hin[3], ls, efwd, ebwd, bim, bmask);
            mma_hop<SP, DAG, 4>(acc, hin[4], ls, efwd, ebwd, bim, bmask);
            mma_hop<SP, DAG, 5>(acc, hin[5], ls, efwd, ebwd, bim, bmask);
            mma_hop<SP, DAG, 6>(acc, hin[6], ls, efwd, ebwd, bim, bmask);
            mma_hop<SP, DAG, 7>(acc, hin[7], ls, efwd, ebwd, bim, bmask);
            // ---- epilogue: a D in (+ x), re-quantised with the site's scale
            const int h = base + js;
#pragma unroll
            for (int r = 0; r < 2; r++) {
                float2 v[4];
#pragma unroll
                for (int q = 0; q < 4; q++) v[q] = make_float2(a * acc[r][q].x, a * acc[r][q].y);
                if (P.xpay && act[r] && t < 3) {
                    const uint4 xd = __ldg(reinterpret_cast<const uint4*>(xr[r]) + (size_t)t * stride + h);
                    const float xs = __ldg(reinterpret_cast<const float*>(xr[r] + 48LL * stride) + h);
                    const float2 x01r = LT::to_f2(xd.x), x01i = LT::to_f2(xd.y);
                    const float2 x23r = LT::to_f2(xd.z), x23i = LT::to_f2(xd.w);
                    v[0].x = fmaf(xs, x01r.x, v[0].x), v[0].y = fmaf(xs, x01i.x, v[0].y);
                    v[1].x = fmaf(xs, x01r.y, v[1].x), v[1].y = fmaf(xs, x01i.y, v[1].y);
                    v[2].x = fmaf(xs, x23r.x, v[2].x), v[2].y = fmaf(xs, x23i.x, v[2].y);
                    v[3].x = fmaf(xs, x23r.y, v[3].x), v[3].y = fmaf(xs, x23i.y, v[3].y);
                }
                float m = 0.f;
                if (t < 3) {
#pragma unroll
                    for (int q = 0; q < 4; q++) m = fmaxf(m, fmaxf(fabsf(v[q].x), fabsf(v[q].y)));
                }
                // the site's scale: the largest component over the three colours (lanes t = 0..2)
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
                if (act[r] && t < 3) {
                    const float inv = m > 0.f ? 1.0f / m : 0.f;
                    uint4 o;
                    o.x = LT::from_f2(v[0].x * inv, v[1].x * inv);
                    o.y = LT::from_f2(v[0].y * inv, v[1].y * inv);
                    o.z = LT::from_f2(v[2].x * inv, v[3].x * inv);
                    o.w = LT::from_f2(v[2].y * inv, v[3].y * inv);
                    st_hint<true>(reinterpret_cast<uint4*>(outr[r]) + (size_t)t * stride + h, o);
                    if (t == 0) st_hint<true>(reinterpret_cast<float*>(outr[r] + 48LL * stride) + h, m);
                }
            }
        }
        __syncwarp();  // the next tile's staging overwrites the slots
    }
    pdl_trigger();
}

}  // namespace

template <int SP>
void launch_hop_mma(const HopParams& P, int block, int site_blocks, int ny, bool dag, cudaStream_t st) {
    static_assert(SP == P_F16 || SP == P_BF16, "the tensor-core hop takes F16 or BF16 storage");
    constexpr int MINB = hop_variant_minb(kHopMmaVariant, SP);
    const int ngrp = (P.nrhs + kGroup - 1) / kGroup;
    const dim3 grid(site_blocks * ngrp, ny);
    const size_t smem = (size_t)(block / 32) * 32 * kSiteWords * sizeof(uint32_t);
    auto k = dag ? hop_kernel_mma<SP, true, MINB> : hop_kernel_mma<SP, false, MINB>;
    // opt in to the larger dynamic shared memory, once per device and dagger
    static bool opted[64][2] = {};
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    if (!opted[dev][dag]) {
        WL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(8 * 32 * kSiteWords * sizeof(uint32_t))));
        opted[dev][dag] = true;
    }
    launch_dep_smem(k, grid, dim3(block), smem, st, P);
}

template void launch_hop_mma<P_F16>(const HopParams&, int, int, int, bool, cudaStream_t);
template void launch_hop_mma<P_BF16>(const HopParams&, int, int, int, bool, cudaStream_t);

}  // namespace wl
