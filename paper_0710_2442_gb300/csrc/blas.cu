// blas.cu -- BLAS-1 kernels of the CG solves (the paper's caxpy class of
// kernels, Sec. 4: memory-bound, one pass over each vector), with the FP64
// reductions fused in.  Each kernel checks its right-hand side's "done" flag
// first, so iterations captured after convergence cost one empty launch.
#include "blas.h"

namespace wl {

namespace {

int blas_grid(int Vh, int block, int cap) {
    int b = (Vh + block - 1) / block;
    if (cap > 0 && b > cap) b = cap;
    return b < 1 ? 1 : b;
}

struct RhsIdx {
    int k, sb, nb;
};
__device__ __forceinline__ RhsIdx rhs_index(int nrhs) {
    return RhsIdx{(int)(blockIdx.x % nrhs), (int)(blockIdx.x / nrhs), (int)(gridDim.x / nrhs)};
}

template <class T>
__device__ __forceinline__ T* at(const Vec& v, int k) {
    return reinterpret_cast<T*>(static_cast<char*>(v.p) + k * v.rstep);
}

}  // namespace

// x += alpha p,  s -= alpha q,  [s_low = s],  reduce |s|^2 (FIN_CG_RES)
template <int XP, int PP, bool SLOW>
__global__ void __launch_bounds__(256) cg_xs_kernel(Vec x, Vec p, Vec s, Vec q, Vec s_low, Geom g, int nrhs,
                                                    const CGScalars* sc, RedArgs red) {
    const RhsIdx r = rhs_index(nrhs);
    if (__ldcg(&sc[r.k].done)) return;
    using TX = typename SpinorFmt<XP>::real;
    using TP = typename SpinorFmt<PP>::real;
    const TX alpha = (TX)__ldcg(&sc[r.k].alpha);
    char* X = at<char>(x, r.k);
    char* S = at<char>(s, r.k);
    const char* Pp = at<const char>(p, r.k);
    const char* Q = at<const char>(q, r.k);
    char* SL = SLOW ? at<char>(s_low, r.k) : nullptr;
    double nrm = 0.0;
    for (int h = r.sb * blockDim.x + threadIdx.x; h < g.Vh; h += r.nb * blockDim.x) {
        cpx<TX> xv[12], sv[12];
        cpx<TP> pv[12], qv[12];
        SpinorFmt<XP>::load(X, g.stride, h, xv);
        SpinorFmt<PP>::load(Pp, g.stride, h, pv);
        SpinorFmt<XP>::load(S, g.stride, h, sv);
        SpinorFmt<PP>::load(Q, g.stride, h, qv);
        TX n2 = 0;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            xv[c].re = fma(alpha, (TX)pv[c].re, xv[c].re);
            xv[c].im = fma(alpha, (TX)pv[c].im, xv[c].im);
            sv[c].re = fma(-alpha, (TX)qv[c].re, sv[c].re);
            sv[c].im = fma(-alpha, (TX)qv[c].im, sv[c].im);
            n2 += cnorm2(sv[c]);
        }
        nrm += (double)n2;
        SpinorFmt<XP>::store(X, g.stride, h, xv);
        SpinorFmt<XP>::store(S, g.stride, h, sv);
        if (SLOW) {
            cpx<TP> sl[12];
#pragma unroll
            for (int c = 0; c < 12; c++) sl[c] = {(TP)sv[c].re, (TP)sv[c].im};
            SpinorFmt<PP>::store(SL, g.stride, h, sl);
        }
    }
    grid_reduce(nrm, red, r.k, r.nb, r.sb);
}

// p = r + beta p
template <int PP>
__global__ void __launch_bounds__(256) cg_p_kernel(Vec p, Vec rv, Geom g, int nrhs, const CGScalars* sc) {
    const RhsIdx r = rhs_index(nrhs);
    if (__ldcg(&sc[r.k].done)) return;
    using T = typename SpinorFmt<PP>::real;
    const T beta = (T)__ldcg(&sc[r.k].beta);
    char* P = at<char>(p, r.k);
    const char* R = at<const char>(rv, r.k);
    for (int h = r.sb * blockDim.x + threadIdx.x; h < g.Vh; h += r.nb * blockDim.x) {
        cpx<T> pv[12], rr[12];
        SpinorFmt<PP>::load(P, g.stride, h, pv);
        SpinorFmt<PP>::load(R, g.stride, h, rr);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            pv[c].re = fma(beta, pv[c].re, rr[c].re);
            pv[c].im = fma(beta, pv[c].im, rr[c].im);
        }
        SpinorFmt<PP>::store(P, g.stride, h, pv);
    }
}

// y (YP) += a x (XP)
template <int YP, int XP>
__global__ void __launch_bounds__(256) axpy_kernel(Vec y, Vec x, Geom g, int nrhs, double a) {
    const RhsIdx r = rhs_index(nrhs);
    using TY = typename SpinorFmt<YP>::real;
    using TX = typename SpinorFmt<XP>::real;
    char* Y = at<char>(y, r.k);
    const char* X = at<const char>(x, r.k);
    for (int h = r.sb * blockDim.x + threadIdx.x; h < g.Vh; h += r.nb * blockDim.x) {
        cpx<TY> yv[12];
        cpx<TX> xv[12];
        SpinorFmt<YP>::load(Y, g.stride, h, yv);
        SpinorFmt<XP>::load(X, g.stride, h, xv);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            yv[c].re = fma((TY)a, (TY)xv[c].re, yv[c].re);
            yv[c].im = fma((TY)a, (TY)xv[c].im, yv[c].im);
        }
        SpinorFmt<YP>::store(Y, g.stride, h, yv);
    }
}

// r = b - q, reduce |r|^2   (r, b and the sums FP64; q FP64 or FP32)
template <int QP>
__global__ void __launch_bounds__(256) xmy_norm_kernel(Vec rv, Vec b, Vec q, Geom g, int nrhs, RedArgs red) {
    const RhsIdx r = rhs_index(nrhs);
    using TQ = typename SpinorFmt<QP>::real;
    char* Rr = rv.p ? at<char>(rv, r.k) : nullptr;
    const char* B = at<const char>(b, r.k);
    const char* Q = at<const char>(q, r.k);
    double nrm = 0.0;
    for (int h = r.sb * blockDim.x + threadIdx.x; h < g.Vh; h += r.nb * blockDim.x) {
        cpx<double> bv[12];
        cpx<TQ> qv[12];
        SpinorFmt<P_F64>::load(B, g.stride, h, bv);
        SpinorFmt<QP>::load(Q, g.stride, h, qv);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            bv[c] = csub(bv[c], cpx<double>{(double)qv[c].re, (double)qv[c].im});
            nrm += cnorm2(bv[c]);
        }
        if (Rr) SpinorFmt<P_F64>::store(Rr, g.stride, h, bv);
    }
    grid_reduce(nrm, red, r.k, r.nb, r.sb);
}

template <int P>
__global__ void __launch_bounds__(256) norm_kernel(Vec v, Geom g, int nrhs, RedArgs red) {
    const RhsIdx r = rhs_index(nrhs);
    using T = typename SpinorFmt<P>::real;
    const char* Vp = at<const char>(v, r.k);
    double nrm = 0.0;
    for (int h = r.sb * blockDim.x + threadIdx.x; h < g.Vh; h += r.nb * blockDim.x) {
        cpx<T> vv[12];
        SpinorFmt<P>::load(Vp, g.stride, h, vv);
        T n2 = 0;
#pragma unroll
        for (int c = 0; c < 12; c++) n2 += cnorm2(vv[c]);
        nrm += (double)n2;
    }
    grid_reduce(nrm, red, r.k, r.nb, r.sb);
}

template <int DP, int SP>
__global__ void __launch_bounds__(256) convert_kernel(Vec dst, Vec src, Geom g, int nrhs) {
    const RhsIdx r = rhs_index(nrhs);
    using TS = typename SpinorFmt<SP>::real;
    using TD = typename SpinorFmt<DP>::real;
    char* D = at<char>(dst, r.k);
    const char* S = at<const char>(src, r.k);
    for (int h = r.sb * blockDim.x + threadIdx.x; h < g.Vh; h += r.nb * blockDim.x) {
        cpx<TS> v[12];
        SpinorFmt<SP>::load(S, g.stride, h, v);
        cpx<TD> w[12];
#pragma unroll
        for (int c = 0; c < 12; c++) w[c] = {(TD)v[c].re, (TD)v[c].im};
        SpinorFmt<DP>::store(D, g.stride, h, w);
    }
}

// ---------------------------------------------------------------------------
void cg_xs_update(Prec xp, Prec pp, Vec x, Vec p, Vec s, Vec q, Vec s_low, const Geom& g, int nrhs,
                  const CGScalars* sc, const RedArgs& red, int grid_cap, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, grid_cap) * nrhs;
    WL_REQUIRE(grid / nrhs <= red.slot_cap, "reduction capacity below the grid size");
    if (xp == P_F64 && pp == P_F64)
        cg_xs_kernel<P_F64, P_F64, false><<<grid, block, 0, st>>>(x, p, s, q, s_low, g, nrhs, sc, red);
    else if (xp == P_F32 && pp == P_F32)
        cg_xs_kernel<P_F32, P_F32, false><<<grid, block, 0, st>>>(x, p, s, q, s_low, g, nrhs, sc, red);
    else if (xp == P_F32 && pp == P_F16)
        cg_xs_kernel<P_F32, P_F16, true><<<grid, block, 0, st>>>(x, p, s, q, s_low, g, nrhs, sc, red);
    else if (xp == P_F32 && pp == P_BF16)
        cg_xs_kernel<P_F32, P_BF16, true><<<grid, block, 0, st>>>(x, p, s, q, s_low, g, nrhs, sc, red);
    else throw Error(7, "cg_xs_update: unsupported precision pair");
    WL_LAUNCH_CHECK();
}

void cg_p_update(Prec pp, Vec p, Vec r, const Geom& g, int nrhs, const CGScalars* sc, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, 64 * device_sm_count()) * nrhs;
    switch (pp) {
        case P_F64: cg_p_kernel<P_F64><<<grid, block, 0, st>>>(p, r, g, nrhs, sc); break;
        case P_F32: cg_p_kernel<P_F32><<<grid, block, 0, st>>>(p, r, g, nrhs, sc); break;
        case P_F16: cg_p_kernel<P_F16><<<grid, block, 0, st>>>(p, r, g, nrhs, sc); break;
        case P_BF16: cg_p_kernel<P_BF16><<<grid, block, 0, st>>>(p, r, g, nrhs, sc); break;
    }
    WL_LAUNCH_CHECK();
}

void axpy(Prec yp, Vec y, Prec xp, Vec x, double a, const Geom& g, int nrhs, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, 64 * device_sm_count()) * nrhs;
    if (yp == P_F64 && xp == P_F64) axpy_kernel<P_F64, P_F64><<<grid, block, 0, st>>>(y, x, g, nrhs, a);
    else if (yp == P_F64 && xp == P_F32) axpy_kernel<P_F64, P_F32><<<grid, block, 0, st>>>(y, x, g, nrhs, a);
    else if (yp == P_F32 && xp == P_F32) axpy_kernel<P_F32, P_F32><<<grid, block, 0, st>>>(y, x, g, nrhs, a);
    else throw Error(7, "axpy: unsupported precision pair");
    WL_LAUNCH_CHECK();
}

void xmy_norm(Prec qp, Vec r, Vec b, Vec q, const Geom& g, int nrhs, const RedArgs& red, int grid_cap,
              cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, grid_cap) * nrhs;
    WL_REQUIRE(grid / nrhs <= red.slot_cap, "reduction capacity below the grid size");
    if (qp == P_F64) xmy_norm_kernel<P_F64><<<grid, block, 0, st>>>(r, b, q, g, nrhs, red);
    else if (qp == P_F32) xmy_norm_kernel<P_F32><<<grid, block, 0, st>>>(r, b, q, g, nrhs, red);
    else throw Error(7, "xmy_norm: q must be FP64 or FP32");
    WL_LAUNCH_CHECK();
}

void xmy_norm64(Vec r, Vec b, Vec q, const Geom& g, int nrhs, const RedArgs& red, int grid_cap, cudaStream_t st) {
    xmy_norm(P_F64, r, b, q, g, nrhs, red, grid_cap, st);
}

void norm2(Prec p, Vec v, const Geom& g, int nrhs, const RedArgs& red, int grid_cap, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, grid_cap) * nrhs;
    WL_REQUIRE(grid / nrhs <= red.slot_cap, "reduction capacity below the grid size");
    switch (p) {
        case P_F64: norm_kernel<P_F64><<<grid, block, 0, st>>>(v, g, nrhs, red); break;
        case P_F32: norm_kernel<P_F32><<<grid, block, 0, st>>>(v, g, nrhs, red); break;
        case P_F16: norm_kernel<P_F16><<<grid, block, 0, st>>>(v, g, nrhs, red); break;
        case P_BF16: norm_kernel<P_BF16><<<grid, block, 0, st>>>(v, g, nrhs, red); break;
    }
    WL_LAUNCH_CHECK();
}

template <int DP>
static void convert_from(Prec sp, Vec dst, Vec src, const Geom& g, int nrhs, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, 64 * device_sm_count()) * nrhs;
    switch (sp) {
        case P_F64: convert_kernel<DP, P_F64><<<grid, block, 0, st>>>(dst, src, g, nrhs); break;
        case P_F32: convert_kernel<DP, P_F32><<<grid, block, 0, st>>>(dst, src, g, nrhs); break;
        case P_F16: convert_kernel<DP, P_F16><<<grid, block, 0, st>>>(dst, src, g, nrhs); break;
        case P_BF16: convert_kernel<DP, P_BF16><<<grid, block, 0, st>>>(dst, src, g, nrhs); break;
    }
}

void convert(Prec dp, Vec dst, Prec sp, Vec src, const Geom& g, int nrhs, cudaStream_t st) {
    switch (dp) {
        case P_F64: convert_from<P_F64>(sp, dst, src, g, nrhs, st); break;
        case P_F32: convert_from<P_F32>(sp, dst, src, g, nrhs, st); break;
        case P_F16: convert_from<P_F16>(sp, dst, src, g, nrhs, st); break;
        case P_BF16: convert_from<P_BF16>(sp, dst, src, g, nrhs, st); break;
    }
    WL_LAUNCH_CHECK();
}

}  // namespace wl
