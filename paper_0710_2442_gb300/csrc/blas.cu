// blas.cu -- BLAS-1 kernels of the CG solves (the paper's caxpy class of
// kernels, Sec. 4: memory-bound, one pass over each vector), with the FP64
// reductions fused in.  Each kernel checks the solve's "done" flag first, so
// iterations captured after convergence cost one empty launch each.
#include "blas.h"

namespace wl {

static int blas_grid(int Vh, int block, int cap) {
    int b = (Vh + block - 1) / block;
    if (cap > 0 && b > cap) b = cap;
    return b < 1 ? 1 : b;
}

// x += alpha p,  s -= alpha q,  [s_low = s],  reduce |s|^2 (FIN_CG_RES)
template <int XP, int PP, bool SLOW>
__global__ void __launch_bounds__(256) cg_xs_kernel(char* x, const char* p, char* s, const char* q, char* s_low,
                                                    Geom g, const CGScalars* sc, RedArgs red) {
    if (__ldcg(&sc->done)) return;
    using TX = typename SpinorFmt<XP>::real;
    using TP = typename SpinorFmt<PP>::real;
    const TX alpha = (TX)__ldcg(&sc->alpha);
    double nrm = 0.0;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        cpx<TX> xv[12], sv[12];
        cpx<TP> pv[12], qv[12];
        SpinorFmt<XP>::load(x, g.stride, h, xv);
        SpinorFmt<PP>::load(p, g.stride, h, pv);
        SpinorFmt<XP>::load(s, g.stride, h, sv);
        SpinorFmt<PP>::load(q, g.stride, h, qv);
        TX n2 = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            xv[k].re = fma(alpha, (TX)pv[k].re, xv[k].re);
            xv[k].im = fma(alpha, (TX)pv[k].im, xv[k].im);
            sv[k].re = fma(-alpha, (TX)qv[k].re, sv[k].re);
            sv[k].im = fma(-alpha, (TX)qv[k].im, sv[k].im);
            n2 += cnorm2(sv[k]);
        }
        nrm += (double)n2;
        SpinorFmt<XP>::store(x, g.stride, h, xv);
        SpinorFmt<XP>::store(s, g.stride, h, sv);
        if (SLOW) {
            cpx<TP> sl[12];
#pragma unroll
            for (int k = 0; k < 12; k++) sl[k] = {(TP)sv[k].re, (TP)sv[k].im};
            SpinorFmt<PP>::store(s_low, g.stride, h, sl);
        }
    }
    grid_reduce(nrm, red);
}

// p = r + beta p
template <int PP>
__global__ void __launch_bounds__(256) cg_p_kernel(char* p, const char* r, Geom g, const CGScalars* sc) {
    if (__ldcg(&sc->done)) return;
    using T = typename SpinorFmt<PP>::real;
    const T beta = (T)__ldcg(&sc->beta);
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        cpx<T> pv[12], rv[12];
        SpinorFmt<PP>::load(p, g.stride, h, pv);
        SpinorFmt<PP>::load(r, g.stride, h, rv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            pv[k].re = fma(beta, pv[k].re, rv[k].re);
            pv[k].im = fma(beta, pv[k].im, rv[k].im);
        }
        SpinorFmt<PP>::store(p, g.stride, h, pv);
    }
}

// y (YP) += x (XP)
template <int YP, int XP>
__global__ void __launch_bounds__(256) axpy_kernel(char* y, const char* x, Geom g, double a) {
    using TY = typename SpinorFmt<YP>::real;
    using TX = typename SpinorFmt<XP>::real;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        cpx<TY> yv[12];
        cpx<TX> xv[12];
        SpinorFmt<YP>::load(y, g.stride, h, yv);
        SpinorFmt<XP>::load(x, g.stride, h, xv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            yv[k].re = fma((TY)a, (TY)xv[k].re, yv[k].re);
            yv[k].im = fma((TY)a, (TY)xv[k].im, yv[k].im);
        }
        SpinorFmt<YP>::store(y, g.stride, h, yv);
    }
}

// r = b - q, reduce |r|^2   (all FP64)
__global__ void __launch_bounds__(256) xmy_norm_kernel(char* r, const char* b, const char* q, Geom g, RedArgs red) {
    double nrm = 0.0;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        cpx<double> bv[12], qv[12];
        SpinorFmt<P_F64>::load(b, g.stride, h, bv);
        SpinorFmt<P_F64>::load(q, g.stride, h, qv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            bv[k] = csub(bv[k], qv[k]);
            nrm += cnorm2(bv[k]);
        }
        if (r) SpinorFmt<P_F64>::store(r, g.stride, h, bv);
    }
    grid_reduce(nrm, red);
}

template <int P>
__global__ void __launch_bounds__(256) norm_kernel(const char* v, Geom g, RedArgs red) {
    using T = typename SpinorFmt<P>::real;
    double nrm = 0.0;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        cpx<T> vv[12];
        SpinorFmt<P>::load(v, g.stride, h, vv);
        T n2 = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) n2 += cnorm2(vv[k]);
        nrm += (double)n2;
    }
    grid_reduce(nrm, red);
}

// ---------------------------------------------------------------------------
void cg_xs_update(Prec xp, Prec pp, void* x, const void* p, void* s, const void* q, void* s_low, const Geom& g,
                  const CGScalars* sc, const RedArgs& red, int grid_cap, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, grid_cap);
    char* X = static_cast<char*>(x);
    char* S = static_cast<char*>(s);
    const char* Pp = static_cast<const char*>(p);
    const char* Q = static_cast<const char*>(q);
    char* SL = static_cast<char*>(s_low);
    if (xp == P_F64 && pp == P_F64)
        cg_xs_kernel<P_F64, P_F64, false><<<grid, block, 0, st>>>(X, Pp, S, Q, SL, g, sc, red);
    else if (xp == P_F32 && pp == P_F32)
        cg_xs_kernel<P_F32, P_F32, false><<<grid, block, 0, st>>>(X, Pp, S, Q, SL, g, sc, red);
    else if (xp == P_F32 && pp == P_F16)
        cg_xs_kernel<P_F32, P_F16, true><<<grid, block, 0, st>>>(X, Pp, S, Q, SL, g, sc, red);
    else if (xp == P_F32 && pp == P_BF16)
        cg_xs_kernel<P_F32, P_BF16, true><<<grid, block, 0, st>>>(X, Pp, S, Q, SL, g, sc, red);
    else throw Error(7, "cg_xs_update: unsupported precision pair");
    WL_LAUNCH_CHECK();
}

void cg_p_update(Prec pp, void* p, const void* r, const Geom& g, const CGScalars* sc, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, 64 * device_sm_count());
    char* P = static_cast<char*>(p);
    const char* R = static_cast<const char*>(r);
    switch (pp) {
        case P_F64: cg_p_kernel<P_F64><<<grid, block, 0, st>>>(P, R, g, sc); break;
        case P_F32: cg_p_kernel<P_F32><<<grid, block, 0, st>>>(P, R, g, sc); break;
        case P_F16: cg_p_kernel<P_F16><<<grid, block, 0, st>>>(P, R, g, sc); break;
        case P_BF16: cg_p_kernel<P_BF16><<<grid, block, 0, st>>>(P, R, g, sc); break;
    }
    WL_LAUNCH_CHECK();
}

void axpy(Prec yp, void* y, Prec xp, const void* x, double a, const Geom& g, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, 64 * device_sm_count());
    char* Y = static_cast<char*>(y);
    const char* X = static_cast<const char*>(x);
    if (yp == P_F64 && xp == P_F64) axpy_kernel<P_F64, P_F64><<<grid, block, 0, st>>>(Y, X, g, a);
    else if (yp == P_F64 && xp == P_F32) axpy_kernel<P_F64, P_F32><<<grid, block, 0, st>>>(Y, X, g, a);
    else if (yp == P_F32 && xp == P_F32) axpy_kernel<P_F32, P_F32><<<grid, block, 0, st>>>(Y, X, g, a);
    else throw Error(7, "axpy: unsupported precision pair");
    WL_LAUNCH_CHECK();
}

void xmy_norm64(void* r, const void* b, const void* q, const Geom& g, const RedArgs& red, int grid_cap,
                cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, grid_cap);
    xmy_norm_kernel<<<grid, block, 0, st>>>(static_cast<char*>(r), static_cast<const char*>(b),
                                            static_cast<const char*>(q), g, red);
    WL_LAUNCH_CHECK();
}

void norm2(Prec p, const void* v, const Geom& g, const RedArgs& red, int grid_cap, cudaStream_t st) {
    const int block = 256, grid = blas_grid(g.Vh, block, grid_cap);
    const char* V = static_cast<const char*>(v);
    switch (p) {
        case P_F64: norm_kernel<P_F64><<<grid, block, 0, st>>>(V, g, red); break;
        case P_F32: norm_kernel<P_F32><<<grid, block, 0, st>>>(V, g, red); break;
        case P_F16: norm_kernel<P_F16><<<grid, block, 0, st>>>(V, g, red); break;
        case P_BF16: norm_kernel<P_BF16><<<grid, block, 0, st>>>(V, g, red); break;
    }
    WL_LAUNCH_CHECK();
}

}  // namespace wl
