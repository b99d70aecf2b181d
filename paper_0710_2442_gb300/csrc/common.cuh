// common.cuh -- device-side building blocks of libwilson_gb300: complex
// arithmetic, lattice geometry, and the site-vectorised structure-of-arrays
// (SoA) storage formats of spinor and gauge fields.
//
// SoA layout.  A field of one parity holds Vh sites.  Its per-site data is
// cut into 16-byte (8-byte for 12-real low-precision links) chunks, and chunk
// c of all sites is one contiguous row:  row c starts at c * stride chunks,
// with stride >= Vh a multiple of 64, so thread i of a warp reads chunk c of
// site i and a warp's request is one coalesced 512-byte line group.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wl {

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// the programmatic-serialization attribute may be scheduled while the
// previous kernel on its stream is still running; pdl_wait() returns once that
// kernel has completed and its memory operations are visible, so a kernel
// calls it before it reads or writes anything an earlier kernel touches.
// pdl_trigger() lets the next such kernel be scheduled once every block of
// this one has called it or exited.  The hop kernels call it when a block has
// finished its sites: calling it at the start, so that the next hop's blocks
// wait resident through the whole launch, gained nothing on the tuned hops
// and slowed a chain of hops sharply whenever a kernel of another stream ran
// alongside (the host-buffer loop with its export on a second stream: 11.9
// against 14.5 TFlop/s).  Both are no-ops for a plain launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3 };

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <class T>
struct cpx {
    T re, im;
};

template <class T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class T>
__device__ __forceinline__ cpx<T> cjmul(cpx<T> a, cpx<T> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc + a * b
template <class T>
__device__ __forceinline__ cpx<T> cfma(cpx<T> a, cpx<T> b, cpx<T> acc) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc + conj(a) * b
template <class T>
__device__ __forceinline__ cpx<T> cjfma(cpx<T> a, cpx<T> b, cpx<T> acc) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}
// i * a
template <class T>
__device__ __forceinline__ cpx<T> ci(cpx<T> a) { return {-a.im, a.re}; }
template <class T>
__device__ __forceinline__ cpx<T> cneg(cpx<T> a) { return {-a.re, -a.im}; }
template <class T>
__device__ __forceinline__ cpx<T> cscale(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
template <class T>
__device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return {a.re, -a.im}; }
template <class T>
__device__ __forceinline__ T cnorm2(cpx<T> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------------------
// lattice geometry
// ---------------------------------------------------------------------------
struct Geom {
    int L[4];          // Lx, Ly, Lz, Lt
    int Vh;            // sites per parity
    int stride;        // SoA row length (chunks) of a parity-field row, >= Vh
    double ph[4][2];   // boundary phases (re, im)
    unsigned int dm[3];  // division by Lx, Ly, Lz: n / L = umulhi(n, dm) >> ds, exact for n < 2^31
    int ds[3];
};

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Round-up division by an invariant integer (Granlund & Montgomery 1994,
// Thm. 4.2, N = 31): with l = ceil(log2 d) and m = floor(2^(31+l) / d) + 1,
// floor(n / d) = (n * m) >> (31 + l) for 0 <= n < 2^31 (d >= 2, so l >= 1).
inline void div_magic(int d, unsigned int& m, int& shift) {
    int l = 0;
    while ((1LL << l) < d) l++;
    m = (unsigned int)((1ULL << (31 + l)) / (unsigned long long)d + 1ULL);
    shift = l - 1;
}

__device__ __forceinline__ int div_by(int n, const Geom& g, int k) {
    return (int)(__umulhi((unsigned int)n, g.dm[k]) >> g.ds[k]);
}

// Coordinates and canonical index of the site with half index h and parity p.
// The canonical index is s = 2h + ((y+z+t+p) & 1) because Lx is even.
__device__ __forceinline__ void site_of_half(int h, int p, const Geom& g, int c[4], int& s) {
    int s0 = 2 * h;
    int r = div_by(s0, g, 0);
    int x0 = s0 - r * g.L[0];
    int r2 = div_by(r, g, 1);
    c[1] = r - r2 * g.L[1];
    c[3] = div_by(r2, g, 2);
    c[2] = r2 - c[3] * g.L[2];
    int odd = (c[1] + c[2] + c[3] + p) & 1;
    c[0] = x0 + odd;
    s = s0 + odd;
}

// Read-only loads go through the non-coherent path (__ldg) by default.  A
// kernel that reads data written earlier in the same launch, possibly by
// another block of its cluster on another SM (the CTA-resident solver),
// instantiates the loads with COH = true: loads from L2 (__ldcg), which the
// other SMs' writes have reached after the cluster barrier.
template <bool COH, class T>
__device__ __forceinline__ T ldro(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// Stores of outputs that are not read again soon (several right-hand sides
// streamed through L2) use the evict-first hint (CS = true), so that they do
// not displace the inputs' neighbour reuse from L2.
template <bool CS, class T>
__device__ __forceinline__ void st_hint(T* p, const T& v) {
    if constexpr (CS) __stcs(p, v);
    else *p = v;
}

// ---------------------------------------------------------------------------
// low-precision helpers
// ---------------------------------------------------------------------------
template <int P>
struct LowT;
template <>
struct LowT<P_F16> {
    using T = __half;
    using T2 = __half2;
    __device__ static __forceinline__ float2 to_f2(uint32_t u) {
        __half2 h = *reinterpret_cast<__half2*>(&u);
        return __half22float2(h);
    }
    __device__ static __forceinline__ uint32_t from_f2(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
};
template <>
struct LowT<P_BF16> {
    using T = __nv_bfloat16;
    using T2 = __nv_bfloat162;
    __device__ static __forceinline__ float2 to_f2(uint32_t u) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
        return __bfloat1622float2(h);
    }
    __device__ static __forceinline__ uint32_t from_f2(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
};

// ---------------------------------------------------------------------------
// spinor storage formats.  v[k], k = spin*3 + colour.
// ---------------------------------------------------------------------------
template <int P>
struct SpinorFmt;

template <>
struct SpinorFmt<P_F64> {
    using real = double;
    static constexpr int nchunk = 12;
    static constexpr int chunk_bytes = 16;
    static constexpr bool scaled = false;
    static __host__ __device__ long long field_bytes(int stride) { return 16LL * 12 * stride; }
    template <bool COH = false>
    __device__ static __forceinline__ void load(const void* base, int stride, int i, cpx<double> v[12]) {
        const double2* b = static_cast<const double2*>(base) + i;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            double2 d = ldro<COH>(b + (size_t)c * stride);
            v[c] = {d.x, d.y};
        }
    }
    // unscaled format: the scale is the constant 1 and folds away
    template <bool COH = false>
    __device__ static __forceinline__ void load_raw(const void* base, int stride, int i, cpx<double> v[12],
                                                    double& s) {
        load<COH>(base, stride, i, v);
        s = 1.0;
    }
    template <bool CS = false>
    __device__ static __forceinline__ void store(void* base, int stride, int i, const cpx<double> v[12]) {
        double2* b = static_cast<double2*>(base) + i;
#pragma unroll
        for (int c = 0; c < 12; c++) st_hint<CS>(b + (size_t)c * stride, make_double2(v[c].re, v[c].im));
    }
};

// Spinors in single and reduced precision are stored spin-paired: for each
// colour c the components of spins (0, 1) and (2, 3) are interleaved as
// (s0.re, s1.re, s0.im, s1.im) and (s2.re, s3.re, s2.im, s3.im), so one
// 8-byte pair is the same real part of two spins.  The paired FP32
// instructions of sm_100+ (FFMA2 etc.) then work on loaded data directly.
//
// PSpinor holds one site that way: re01[c] = (s0c.re, s1c.re), im01[c] =
// (s0c.im, s1c.im), re23[c], im23[c] likewise for spins 2 and 3.
struct PSpinor {
    float2 re01[3], im01[3], re23[3], im23[3];
};

__device__ __forceinline__ void unpack_pairs(const PSpinor& q, cpx<float> v[12]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        v[0 * 3 + c] = {q.re01[c].x, q.im01[c].x};
        v[1 * 3 + c] = {q.re01[c].y, q.im01[c].y};
        v[2 * 3 + c] = {q.re23[c].x, q.im23[c].x};
        v[3 * 3 + c] = {q.re23[c].y, q.im23[c].y};
    }
}

__device__ __forceinline__ void pack_pairs(const cpx<float> v[12], PSpinor& q) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        q.re01[c] = make_float2(v[c].re, v[3 + c].re);
        q.im01[c] = make_float2(v[c].im, v[3 + c].im);
        q.re23[c] = make_float2(v[6 + c].re, v[9 + c].re);
        q.im23[c] = make_float2(v[6 + c].im, v[9 + c].im);
    }
}

// F32: chunk 2c holds colour c, spins 0/1; chunk 2c+1 colour c, spins 2/3.
template <>
struct SpinorFmt<P_F32> {
    using real = float;
    static constexpr int nchunk = 6;
    static constexpr int chunk_bytes = 16;
    static constexpr bool scaled = false;
    static __host__ __device__ long long field_bytes(int stride) { return 16LL * 6 * stride; }
    template <bool COH = false>
    __device__ static __forceinline__ void load_packed(const void* base, int stride, int i, PSpinor& q, float& s) {
        const float4* b = static_cast<const float4*>(base) + i;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 lo = ldro<COH>(b + (size_t)(2 * c) * stride);
            const float4 hi = ldro<COH>(b + (size_t)(2 * c + 1) * stride);
            q.re01[c] = make_float2(lo.x, lo.y);
            q.im01[c] = make_float2(lo.z, lo.w);
            q.re23[c] = make_float2(hi.x, hi.y);
            q.im23[c] = make_float2(hi.z, hi.w);
        }
        s = 1.0f;
    }
    template <bool CS = false>
    __device__ static __forceinline__ void store_packed(void* base, int stride, int i, const PSpinor& q) {
        float4* b = static_cast<float4*>(base) + i;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            st_hint<CS>(b + (size_t)(2 * c) * stride,
                        make_float4(q.re01[c].x, q.re01[c].y, q.im01[c].x, q.im01[c].y));
            st_hint<CS>(b + (size_t)(2 * c + 1) * stride,
                        make_float4(q.re23[c].x, q.re23[c].y, q.im23[c].x, q.im23[c].y));
        }
    }
    template <bool COH = false>
    __device__ static __forceinline__ void load(const void* base, int stride, int i, cpx<float> v[12]) {
        PSpinor q;
        float s;
        load_packed<COH>(base, stride, i, q, s);
        unpack_pairs(q, v);
    }
    template <bool COH = false>
    __device__ static __forceinline__ void load_raw(const void* base, int stride, int i, cpx<float> v[12],
                                                    float& s) {
        load<COH>(base, stride, i, v);
        s = 1.0f;
    }
    template <bool CS = false>
    __device__ static __forceinline__ void store(void* base, int stride, int i, const cpx<float> v[12]) {
        PSpinor q;
        pack_pairs(v, q);
        store_packed<CS>(base, stride, i, q);
    }
};

// 24 low-precision reals in 3 x 16 B chunks (chunk c = colour c: the
// half2 words (s0.re, s1.re), (s0.im, s1.im), (s2.re, s3.re), (s2.im, s3.im)),
// then one FP32 scale per site (a row of stride floats after the 3 chunk
// rows).  value = q * scale, with scale = max |component| of the site, so
// |q| <= 1.
template <int P>
struct SpinorLowFmt {
    using real = float;
    using LT = LowT<P>;
    static constexpr int nchunk = 3;
    static constexpr int chunk_bytes = 16;
    static constexpr bool scaled = true;
    static __host__ __device__ long long field_bytes(int stride) { return 16LL * 3 * stride + 4LL * stride; }
    template <bool COH = false>
    __device__ static __forceinline__ float load_scale(const void* base, int stride, int i) {
        const float* sc = reinterpret_cast<const float*>(static_cast<const char*>(base) + 48LL * stride);
        return ldro<COH>(sc + i);
    }
    // The stored values q (|q| <= 1) and the site's scale separately: the
    // hopping kernels apply the scale in their accumulation FMA for free.
    template <bool COH = false>
    __device__ static __forceinline__ void load_packed(const void* base, int stride, int i, PSpinor& q, float& s) {
        const uint4* b = static_cast<const uint4*>(base) + i;
        s = load_scale<COH>(base, stride, i);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const uint4 d = ldro<COH>(b + (size_t)c * stride);
            q.re01[c] = LT::to_f2(d.x);
            q.im01[c] = LT::to_f2(d.y);
            q.re23[c] = LT::to_f2(d.z);
            q.im23[c] = LT::to_f2(d.w);
        }
    }
    template <bool CS = false>
    __device__ static __forceinline__ void store_packed(void* base, int stride, int i, const PSpinor& q) {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m = fmaxf(m, fmaxf(fmaxf(fabsf(q.re01[c].x), fabsf(q.re01[c].y)), fmaxf(fabsf(q.im01[c].x), fabsf(q.im01[c].y))));
            m = fmaxf(m, fmaxf(fmaxf(fabsf(q.re23[c].x), fabsf(q.re23[c].y)), fmaxf(fabsf(q.im23[c].x), fabsf(q.im23[c].y))));
        }
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        uint4* b = static_cast<uint4*>(base) + i;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            uint4 d;
            d.x = LT::from_f2(q.re01[c].x * inv, q.re01[c].y * inv);
            d.y = LT::from_f2(q.im01[c].x * inv, q.im01[c].y * inv);
            d.z = LT::from_f2(q.re23[c].x * inv, q.re23[c].y * inv);
            d.w = LT::from_f2(q.im23[c].x * inv, q.im23[c].y * inv);
            st_hint<CS>(b + (size_t)c * stride, d);
        }
        float* sc = reinterpret_cast<float*>(static_cast<char*>(base) + 48LL * stride);
        st_hint<CS>(sc + i, m);
    }
    template <bool COH = false>
    __device__ static __forceinline__ void load_raw(const void* base, int stride, int i, cpx<float> v[12],
                                                    float& s) {
        PSpinor q;
        load_packed<COH>(base, stride, i, q, s);
        unpack_pairs(q, v);
    }
    template <bool COH = false>
    __device__ static __forceinline__ void load(const void* base, int stride, int i, cpx<float> v[12]) {
        float s;
        load_raw<COH>(base, stride, i, v, s);
#pragma unroll
        for (int k = 0; k < 12; k++) v[k] = {v[k].re * s, v[k].im * s};
    }
    template <bool CS = false>
    __device__ static __forceinline__ void store(void* base, int stride, int i, const cpx<float> v[12]) {
        PSpinor q;
        pack_pairs(v, q);
        store_packed<CS>(base, stride, i, q);
    }
};
template <>
struct SpinorFmt<P_F16> : SpinorLowFmt<P_F16> {};
template <>
struct SpinorFmt<P_BF16> : SpinorLowFmt<P_BF16> {};

// ---------------------------------------------------------------------------
// gauge storage formats.  One parity-and-direction block holds Vh links;
// block (p, mu) starts at (p*4 + mu) * nchunk rows.  U[i][j] row-major.
// With 12 reals only rows 0 and 1 are stored; row 2 = conj(row0 x row1),
// exact for SU(3).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void recon_row2(cpx<T> U[3][3]) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int a = (j + 1) % 3, b = (j + 2) % 3;
        cpx<T> t = csub(cmul(U[0][a], U[1][b]), cmul(U[0][b], U[1][a]));
        U[2][j] = cconj(t);
    }
}

template <int P, int R>
struct GaugeFmt;

template <>
struct GaugeFmt<P_F64, 18> {
    using real = double;
    static constexpr int nchunk = 9;
    static constexpr int chunk_bytes = 16;
    __device__ static __forceinline__ void load(const void* base, int stride, int blk, int i, cpx<double> U[3][3]) {
        const double2* b = static_cast<const double2*>(base) + (size_t)blk * nchunk * stride + i;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            double2 d = __ldg(b + (size_t)c * stride);
            U[c / 3][c % 3] = {d.x, d.y};
        }
    }
};
template <>
struct GaugeFmt<P_F64, 12> {
    using real = double;
    static constexpr int nchunk = 6;
    static constexpr int chunk_bytes = 16;
    __device__ static __forceinline__ void load(const void* base, int stride, int blk, int i, cpx<double> U[3][3]) {
        const double2* b = static_cast<const double2*>(base) + (size_t)blk * nchunk * stride + i;
#pragma unroll
        for (int c = 0; c < 6; c++) {
            double2 d = __ldg(b + (size_t)c * stride);
            U[c / 3][c % 3] = {d.x, d.y};
        }
        recon_row2(U);
    }
};
template <>
struct GaugeFmt<P_F32, 18> {
    using real = float;
    static constexpr int nchunk = 9;
    static constexpr int chunk_bytes = 8;
    __device__ static __forceinline__ void load(const void* base, int stride, int blk, int i, cpx<float> U[3][3]) {
        const float2* b = static_cast<const float2*>(base) + (size_t)blk * nchunk * stride + i;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            float2 d = __ldg(b + (size_t)c * stride);
            U[c / 3][c % 3] = {d.x, d.y};
        }
    }
};
template <>
struct GaugeFmt<P_F32, 12> {
    using real = float;
    using chunk_t = float4;
    static constexpr int nchunk = 3;
    static constexpr int chunk_bytes = 16;
    // The link's stored chunks, copied to dst[c * dstride] (shared-memory
    // staging), and their decoding: the same arithmetic as load().
    __device__ static __forceinline__ void load_chunks(const void* base, int stride, int blk, int i, chunk_t* dst,
                                                       int dstride) {
        const float4* b = static_cast<const float4*>(base) + (size_t)blk * nchunk * stride + i;
#pragma unroll
        for (int c = 0; c < nchunk; c++) dst[c * dstride] = __ldcs(b + (size_t)c * stride);
    }
    __device__ static __forceinline__ void decode(const chunk_t* src, int sstride, cpx<float> U[3][3]) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 d = src[c * sstride];
            U[(2 * c) / 3][(2 * c) % 3] = {d.x, d.y};
            U[(2 * c + 1) / 3][(2 * c + 1) % 3] = {d.z, d.w};
        }
        recon_row2(U);
    }
    __device__ static __forceinline__ void load(const void* base, int stride, int blk, int i, cpx<float> U[3][3]) {
        const float4* b = static_cast<const float4*>(base) + (size_t)blk * nchunk * stride + i;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float4 d = __ldcs(b + (size_t)c * stride);
            U[(2 * c) / 3][(2 * c) % 3] = {d.x, d.y};
            U[(2 * c + 1) / 3][(2 * c + 1) % 3] = {d.z, d.w};
        }
        recon_row2(U);
    }
};
// 12 low-precision reals in 3 x 8 B chunks (links have |U_ij| <= 1: no scale)
template <int P>
struct GaugeLow12 {
    using real = float;
    using LT = LowT<P>;
    using chunk_t = uint2;
    static constexpr int nchunk = 3;
    static constexpr int chunk_bytes = 8;
    __device__ static __forceinline__ void load_chunks(const void* base, int stride, int blk, int i, chunk_t* dst,
                                                       int dstride) {
        const uint2* b = static_cast<const uint2*>(base) + (size_t)blk * nchunk * stride + i;
#pragma unroll
        for (int c = 0; c < nchunk; c++) dst[c * dstride] = __ldcs(b + (size_t)c * stride);
    }
    __device__ static __forceinline__ void decode(const chunk_t* src, int sstride, cpx<float> U[3][3]) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const uint2 d = src[c * sstride];
            const float2 f0 = LT::to_f2(d.x), f1 = LT::to_f2(d.y);
            U[(2 * c) / 3][(2 * c) % 3] = {f0.x, f0.y};
            U[(2 * c + 1) / 3][(2 * c + 1) % 3] = {f1.x, f1.y};
        }
        recon_row2(U);
    }
    __device__ static __forceinline__ void load(const void* base, int stride, int blk, int i, cpx<float> U[3][3]) {
        const uint2* b = static_cast<const uint2*>(base) + (size_t)blk * nchunk * stride + i;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            uint2 d = __ldcs(b + (size_t)c * stride);
            float2 f0 = LT::to_f2(d.x), f1 = LT::to_f2(d.y);
            U[(2 * c) / 3][(2 * c) % 3] = {f0.x, f0.y};
            U[(2 * c + 1) / 3][(2 * c + 1) % 3] = {f1.x, f1.y};
        }
        recon_row2(U);
    }
};
template <>
struct GaugeFmt<P_F16, 12> : GaugeLow12<P_F16> {};
template <>
struct GaugeFmt<P_BF16, 12> : GaugeLow12<P_BF16> {};

// 18 low-precision reals (no reconstruction arithmetic): two rows of 16 B
// (8 reals each) and one row of 4 B per link, 36 B in all.
template <int P>
struct GaugeLow18 {
    using real = float;
    using LT = LowT<P>;
    static constexpr int nchunk = 3;
    static constexpr int chunk_bytes = 12;  // mean bytes per row (36 B per link)
    __device__ static __forceinline__ void load(const void* base, int stride, int blk, int i, cpx<float> U[3][3]) {
        const char* b = static_cast<const char*>(base) + (size_t)blk * 36 * stride;
        const uint4 d0 = __ldcs(reinterpret_cast<const uint4*>(b) + i);
        const uint4 d1 = __ldcs(reinterpret_cast<const uint4*>(b + 16LL * stride) + i);
        const unsigned int d2 = __ldcs(reinterpret_cast<const unsigned int*>(b + 32LL * stride) + i);
        const unsigned int w[9] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w, d2};
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const float2 f = LT::to_f2(w[k]);
            U[k / 3][k % 3] = {f.x, f.y};
        }
    }
};
template <>
struct GaugeFmt<P_F16, 18> : GaugeLow18<P_F16> {};
template <>
struct GaugeFmt<P_BF16, 18> : GaugeLow18<P_BF16> {};

// L2 prefetches of one link or one spinor of a stored field: a request per
// row of the site's SoA rows, which holds no register and waits for nothing.
// The hop variants that issue them when a thread takes its site start the
// streamed link loads of all eight hops at once (GB300 keeps more of the
// link stream in flight this way than the per-hop loads, which wait for
// registers).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
template <int NR, int RB>
__device__ __forceinline__ void prefetch_rows(const char* b, long long stride, int i) {
#pragma unroll
    for (int r = 0; r < NR; r++) prefetch_l2(b + (long long)r * RB * stride + (long long)i * RB);
}
// Link blk of site i in GaugeFmt<P, R>'s layout (blocks of nchunk rows; the
// 18-real F16/BF16 format has rows of 16, 16 and 4 bytes).
template <int P, int R>
__device__ __forceinline__ void prefetch_link(const void* base, int stride, int blk, int i) {
    using GF = GaugeFmt<P, R>;
    const char* b = static_cast<const char*>(base);
    if constexpr ((P == P_F16 || P == P_BF16) && R == 18) {
        const char* lb = b + (long long)blk * 36 * stride;
        prefetch_rows<2, 16>(lb, stride, i);
        prefetch_l2(lb + 32LL * stride + (long long)i * 4);
    } else {
        prefetch_rows<GF::nchunk, GF::chunk_bytes>(b + (long long)blk * GF::nchunk * GF::chunk_bytes * stride,
                                                   stride, i);
    }
}
// Spinor i in SpinorFmt<P>'s layout (the scale row after the chunks).
template <int P>
__device__ __forceinline__ void prefetch_spinor(const void* base, int stride, int i) {
    using SF = SpinorFmt<P>;
    const char* b = static_cast<const char*>(base);
    prefetch_rows<SF::nchunk, SF::chunk_bytes>(b, stride, i);
    if constexpr (SF::scaled) prefetch_l2(b + (long long)SF::nchunk * SF::chunk_bytes * stride + (long long)i * 4);
}

}  // namespace wl
