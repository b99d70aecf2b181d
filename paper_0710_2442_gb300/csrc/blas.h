// blas.h -- launchers of the BLAS-1 kernels used by the CG solves.
//
// Every kernel runs over nrhs right-hand sides at once (grid x = blocks per
// right-hand side x nrhs, right-hand sides fastest); a vector is a parity
// block plus the byte step to the next right-hand side's block.  Scalars
// (alpha, beta, done flags) are per right-hand side in a CGScalars array.
#pragma once

#include "internal.h"

namespace wl {

struct Vec {
    void* p;
    long long rstep;
};
inline Vec vec(const SpinorField& f, int parity) { return Vec{f.block(parity), f.rstep()}; }

// x += alpha p; s -= alpha q; [s_low = s]; |s|^2 -> red (FIN_CG_RES).  alpha
// is read from sc[k] on the device.  x, s in precision xp; p, q, s_low in pp.
void cg_xs_update(Prec xp, Prec pp, Vec x, Vec p, Vec s, Vec q, Vec s_low, const Geom& g, int nrhs,
                  const CGScalars* sc, const RedArgs& red, int grid_cap, cudaStream_t st);

// p = r + beta p (beta read from sc[k]).
void cg_p_update(Prec pp, Vec p, Vec r, const Geom& g, int nrhs, const CGScalars* sc, cudaStream_t st);

// y += a x
void axpy(Prec yp, Vec y, Prec xp, Vec x, double a, const Geom& g, int nrhs, cudaStream_t st);

// r = b - q (FP64; r.p may be null), |b - q|^2 -> red
void xmy_norm64(Vec r, Vec b, Vec q, const Geom& g, int nrhs, const RedArgs& red, int grid_cap, cudaStream_t st);
// the same with q in FP64 or FP32
void xmy_norm(Prec qp, Vec r, Vec b, Vec q, const Geom& g, int nrhs, const RedArgs& red, int grid_cap,
              cudaStream_t st);

// |v|^2 -> red
void norm2(Prec p, Vec v, const Geom& g, int nrhs, const RedArgs& red, int grid_cap, cudaStream_t st);

// dst = src (any precisions), one parity block per right-hand side
void convert(Prec dp, Vec dst, Prec sp, Vec src, const Geom& g, int nrhs, cudaStream_t st);

}  // namespace wl
