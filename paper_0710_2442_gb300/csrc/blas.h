// blas.h -- launchers of the BLAS-1 kernels used by the CG solves.
#pragma once

#include "internal.h"

namespace wl {

// x += alpha p; s -= alpha q; [s_low = s]; |s|^2 -> red (FIN_CG_RES).  alpha
// is read from sc on the device.  x, s in precision xp; p, q, s_low in pp.
void cg_xs_update(Prec xp, Prec pp, void* x, const void* p, void* s, const void* q, void* s_low, const Geom& g,
                  const CGScalars* sc, const RedArgs& red, int grid_cap, cudaStream_t st);

// p = r + beta p (beta read from sc).
void cg_p_update(Prec pp, void* p, const void* r, const Geom& g, const CGScalars* sc, cudaStream_t st);

// y += a x
void axpy(Prec yp, void* y, Prec xp, const void* x, double a, const Geom& g, cudaStream_t st);

// r = b - q (FP64; r may be null), |b - q|^2 -> red
void xmy_norm64(void* r, const void* b, const void* q, const Geom& g, const RedArgs& red, int grid_cap,
                cudaStream_t st);

// |v|^2 -> red
void norm2(Prec p, const void* v, const Geom& g, const RedArgs& red, int grid_cap, cudaStream_t st);

}  // namespace wl
