/*
 * wilson_oracle.c -- plain FP64 CPU oracle for the Wilson hopping term and
 * the even-odd CG solve built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, includes or
 * calls this file.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it (through ctypes, see oracle/__init__.py).
 *
 * What it computes (QCD on the Cell BE, Sec. 5, Eq. 3): for every lattice
 * site x,
 *
 *   psi'_x = sum_{mu=1..4} { (1 - c g_mu) eta_mu(x)  U_{x,mu}        psi_{x+mu}
 *                          + (1 + c g_mu) eta*_mu(x-mu) U^dag_{x-mu,mu} psi_{x-mu} }
 *
 * with c = +1 (the "(1-gamma) forward" convention of the library's C ABI) or
 * c = -1 (Eq. 3 exactly as printed: (1+gamma) forward, (1-gamma) backward).
 * eta_mu(x) is the boundary phase of direction mu when the forward hop from x
 * crosses the lattice boundary (x_mu = L_mu - 1) and 1 otherwise; the backward
 * hop that crosses it (x_mu = 0) takes the complex conjugate.
 *
 * Everything here is the plain definition: the spin projector (1 -/+ g_mu) is
 * applied as a full 4x4 matrix built from the gamma table, the colour matrix
 * as a full 3x3 matrix, one site at a time, in double precision.  No
 * half-spinor projection, no link compression, no blocking.
 *
 * Layouts (canonical, complex numbers stored as (re, im) double pairs):
 *   site index   s = x + Lx*(y + Ly*(z + Lz*t))
 *   spinor       psi[s][spin 0..3][colour 0..2]
 *   gauge        U[s][mu 0..3][row 0..2][col 0..2]     (mu = x, y, z, t)
 *   half field   of parity p = (x+y+z+t) mod 2: site s stored at index s>>1
 *                (needs Lx even, so each pair (2k, 2k+1) holds one site of
 *                each parity)
 *
 * The solve (not in the paper, which only says an iterative solver repeats
 * Eq. 3): conjugate gradients on the normal equations of the even-odd Schur
 * complement, in the residual-tracking form (CGNR; Hestenes & Stiefel 1952,
 * Sec. 10), with the full system's true residual recomputed at the end.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

#define NSPIN 4
#define NCOL 3
#define SPINOR_CPLX (NSPIN * NCOL)   /* 12 complex numbers per site */
#define LINK_CPLX (NCOL * NCOL)      /* 9 complex numbers per link  */

/* ------------------------------------------------------------------------ */
/* DeGrand-Rossi gamma matrices, gamma_1..gamma_4 = x, y, z, t.  Rows are     */
/* the output spin index.                                                    */
/* ------------------------------------------------------------------------ */
static cplx G[5][4][4];
static int g_init = 0;

static void init_gamma(void) {
    if (g_init) return;
    memset(G, 0, sizeof(G));
    const cplx iu = _Complex_I;
    /* gamma_1 */
    G[0][0][3] = iu;  G[0][1][2] = iu;  G[0][2][1] = -iu; G[0][3][0] = -iu;
    /* gamma_2 */
    G[1][0][3] = -1; G[1][1][2] = 1;  G[1][2][1] = 1;  G[1][3][0] = -1;
    /* gamma_3 */
    G[2][0][2] = iu;  G[2][1][3] = -iu; G[2][2][0] = -iu; G[2][3][1] = iu;
    /* gamma_4 */
    G[3][0][2] = 1;  G[3][1][3] = 1;  G[3][2][0] = 1;  G[3][3][1] = 1;
    /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4, by plain matrix products */
    cplx a[4][4], b[4][4];
    memcpy(a, G[0], sizeof(a));
    for (int k = 1; k < 4; k++) {
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) {
                cplx acc = 0;
                for (int l = 0; l < 4; l++) acc += a[i][l] * G[k][l][j];
                b[i][j] = acc;
            }
        memcpy(a, b, sizeof(a));
    }
    memcpy(G[4], a, sizeof(a));
    g_init = 1;
}

/* Export a gamma matrix (mu = 0..3 for gamma_1..gamma_4, 4 for gamma_5) as
 * 16 complex numbers, row-major. */
void oracle_gamma(int mu, double *out) {
    init_gamma();
    if (mu < 0 || mu > 4) return;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            out[2 * (4 * i + j)] = creal(G[mu][i][j]);
            out[2 * (4 * i + j) + 1] = cimag(G[mu][i][j]);
        }
}

/* ------------------------------------------------------------------------ */
/* threads                                                                   */
/* ------------------------------------------------------------------------ */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* lattice geometry                                                          */
/* ------------------------------------------------------------------------ */
static long volume(const int *L) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(long s, const int *L, int c[4]) {
    for (int mu = 0; mu < 4; mu++) {
        c[mu] = (int)(s % L[mu]);
        s /= L[mu];
    }
}

static long index_of(const int c[4], const int *L) {
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

static int dims_ok(const int *L) {
    for (int mu = 0; mu < 4; mu++)
        if (L[mu] < 1) return 0;
    return 1;
}

static int eo_dims_ok(const int *L) {
    for (int mu = 0; mu < 4; mu++)
        if (L[mu] < 2 || (L[mu] & 1)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* the hopping term, Eq. 3, one site                                         */
/* ------------------------------------------------------------------------ */

/* out[a][col] += eta * P[a][b] * M[col][k] * in[b][k], where
 * P = 1 - sgn*gamma_mu and M = U or U^dagger, all as full matrices. */
static void hop_term(cplx *acc, const cplx *psi, const cplx *U, int mu, int sgn,
                     int dagger, cplx eta) {
    cplx P[4][4];
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) P[a][b] = (a == b ? 1.0 : 0.0) - sgn * G[mu][a][b];
    cplx M[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[i][j] = dagger ? conj(U[3 * j + i]) : U[3 * i + j];
    /* spin projection first: w = P psi */
    cplx w[4][3];
    for (int a = 0; a < 4; a++)
        for (int k = 0; k < 3; k++) {
            cplx v = 0;
            for (int b = 0; b < 4; b++) v += P[a][b] * psi[3 * b + k];
            w[a][k] = v;
        }
    /* then colour: acc += eta * M w */
    for (int a = 0; a < 4; a++)
        for (int i = 0; i < 3; i++) {
            cplx v = 0;
            for (int k = 0; k < 3; k++) v += M[i][k] * w[a][k];
            acc[3 * a + i] += eta * v;
        }
}

/* psi'_x for one site x (coordinates c).  conv = +1: (1-g) forward,
 * conv = -1: (1+g) forward (Eq. 3 as printed). */
static void dslash_site(cplx *out, const cplx *U, const cplx *in, const int *L,
                        const cplx *phase, int conv, const int c[4]) {
    cplx acc[SPINOR_CPLX];
    for (int k = 0; k < SPINOR_CPLX; k++) acc[k] = 0;
    long s = index_of(c, L);
    for (int mu = 0; mu < 4; mu++) {
        int cf[4] = {c[0], c[1], c[2], c[3]};
        int cb[4] = {c[0], c[1], c[2], c[3]};
        cf[mu] = (c[mu] + 1) % L[mu];
        cb[mu] = (c[mu] - 1 + L[mu]) % L[mu];
        long sf = index_of(cf, L), sb = index_of(cb, L);
        cplx eta_f = (c[mu] == L[mu] - 1) ? phase[mu] : 1.0;
        cplx eta_b = (c[mu] == 0) ? conj(phase[mu]) : 1.0;
        /* forward: (1 - conv g_mu) eta U_{x,mu} psi_{x+mu} */
        hop_term(acc, in + SPINOR_CPLX * sf, U + LINK_CPLX * (4 * s + mu), mu, conv, 0, eta_f);
        /* backward: (1 + conv g_mu) eta* U^dag_{x-mu,mu} psi_{x-mu} */
        hop_term(acc, in + SPINOR_CPLX * sb, U + LINK_CPLX * (4 * sb + mu), mu, -conv, 1, eta_b);
    }
    for (int k = 0; k < SPINOR_CPLX; k++) out[k] = acc[k];
}

static void load_phases(cplx ph[4], const double *phases) {
    for (int mu = 0; mu < 4; mu++) ph[mu] = phases[2 * mu] + _Complex_I * phases[2 * mu + 1];
}

/* Full-lattice hopping term D_h.  out, in: V spinors; gauge: 4V links.
 * out must not alias in.  Returns 0, or -1 on bad arguments. */
int oracle_dslash(double *out, const double *gauge, const double *in, const int *dims,
                  const double *phases, int conv) {
    init_gamma();
    if (!dims_ok(dims) || (conv != 1 && conv != -1) || out == in) return -1;
    cplx ph[4];
    load_phases(ph, phases);
    const long V = volume(dims);
    cplx *o = (cplx *)out;
    const cplx *U = (const cplx *)gauge, *p = (const cplx *)in;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(s, dims, c);
        dslash_site(o + SPINOR_CPLX * s, U, p, dims, ph, conv, c);
    }
    return 0;
}

/* Full Wilson operator M = 1 - kappa D_h (conv = +1). */
int oracle_wilson_m(double *out, const double *gauge, const double *in, const int *dims,
                    const double *phases, double kappa) {
    int rc = oracle_dslash(out, gauge, in, dims, phases, 1);
    if (rc) return rc;
    const long n = 2 * SPINOR_CPLX * volume(dims);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) out[i] = in[i] - kappa * out[i];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* even-odd blocks, by their definition: D_{p,1-p} = P_p D_h P_{1-p}         */
/* ------------------------------------------------------------------------ */

/* Scatter a half field of parity par into a zeroed full field. */
static void embed(cplx *full, const cplx *half, const int *L, int par) {
    const long V = volume(L);
    memset(full, 0, sizeof(cplx) * SPINOR_CPLX * V);
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(s, L, c);
        if (parity_of(c) == par) memcpy(full + SPINOR_CPLX * s, half + SPINOR_CPLX * (s >> 1), sizeof(cplx) * SPINOR_CPLX);
    }
}

/* Gather the sites of parity par of a full field. */
static void extract(cplx *half, const cplx *full, const int *L, int par) {
    const long V = volume(L);
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(s, L, c);
        if (parity_of(c) == par) memcpy(half + SPINOR_CPLX * (s >> 1), full + SPINOR_CPLX * s, sizeof(cplx) * SPINOR_CPLX);
    }
}

/* out (parity out_parity, V/2 sites) = [D_h applied to in (parity 1-out_parity)]
 * restricted to out_parity.  All extents must be even. */
int oracle_dslash_eo(double *out, const double *gauge, const double *in, const int *dims,
                     const double *phases, int out_parity, int conv) {
    if (!eo_dims_ok(dims) || (out_parity != 0 && out_parity != 1)) return -1;
    const long V = volume(dims);
    cplx *a = (cplx *)malloc(sizeof(cplx) * SPINOR_CPLX * V);
    cplx *b = (cplx *)malloc(sizeof(cplx) * SPINOR_CPLX * V);
    if (!a || !b) { free(a); free(b); return -2; }
    embed(a, (const cplx *)in, dims, 1 - out_parity);
    int rc = oracle_dslash((double *)b, gauge, (const double *)a, dims, phases, conv);
    if (!rc) extract((cplx *)out, b, dims, out_parity);
    free(a);
    free(b);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Schur complement on parity p: Mhat = 1 - kappa^2 D_{p,1-p} D_{1-p,p}.      */
/* Its adjoint is gamma_5 Mhat gamma_5 (gamma_5-hermiticity of D_h).         */
/* ------------------------------------------------------------------------ */
static void apply_gamma5(cplx *v, long nsites) {
    init_gamma();
    for (long s = 0; s < nsites; s++) {
        cplx w[SPINOR_CPLX];
        for (int a = 0; a < 4; a++)
            for (int k = 0; k < 3; k++) {
                cplx acc = 0;
                for (int b = 0; b < 4; b++) acc += G[4][a][b] * v[SPINOR_CPLX * s + 3 * b + k];
                w[3 * a + k] = acc;
            }
        memcpy(v + SPINOR_CPLX * s, w, sizeof(w));
    }
}

int oracle_schur(double *out, const double *gauge, const double *in, const int *dims,
                 const double *phases, double kappa, int parity, int dagger) {
    if (!eo_dims_ok(dims) || (parity != 0 && parity != 1)) return -1;
    const long Vh = volume(dims) / 2;
    const long n = SPINOR_CPLX * Vh;
    cplx *src = (cplx *)malloc(sizeof(cplx) * n);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
    cplx *res = (cplx *)malloc(sizeof(cplx) * n);
    if (!src || !tmp || !res) { free(src); free(tmp); free(res); return -2; }
    memcpy(src, in, sizeof(cplx) * n);
    if (dagger) apply_gamma5(src, Vh);
    int rc = oracle_dslash_eo((double *)tmp, gauge, (const double *)src, dims, phases, 1 - parity, 1);
    if (!rc) rc = oracle_dslash_eo((double *)res, gauge, (const double *)tmp, dims, phases, parity, 1);
    if (!rc) {
        for (long i = 0; i < n; i++) res[i] = src[i] - kappa * kappa * res[i];
        if (dagger) apply_gamma5(res, Vh);
        memcpy(out, res, sizeof(cplx) * n);
    }
    free(src);
    free(tmp);
    free(res);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* CG on the normal equations of the even Schur complement                   */
/* ------------------------------------------------------------------------ */
static double norm2(const cplx *v, long n) {
    double acc = 0;
    for (long i = 0; i < n; i++) acc += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return acc;
}

/* Solves M x = b (full lattice, M = 1 - kappa D_h) through the even Schur
 * complement:
 *   bhat_e = b_e + kappa D_eo b_o
 *   Mhat x_e = bhat_e        by CGNR:  Mhat^dag Mhat x_e = Mhat^dag bhat_e
 *   x_o = b_o + kappa D_oe x_e
 * The iteration tracks the Schur residual s = bhat_e - Mhat x_e, which equals
 * the even part of the full residual b - M x (its odd part is zero when x_o is
 * reconstructed exactly).  It stops when |s| <= tol |b|, confirms that with
 * a recomputed s, and restarts from the recomputed s if the recursion drifted.
 *
 * info[0] = iterations, info[1] = Mhat applications; out_resid[0] = true
 * relative residual |b - M x| / |b| recomputed with the full operator.
 * Returns 0 on convergence, 1 if maxiter was reached, <0 on bad arguments. */
int oracle_cg(double *x, const double *gauge, const double *b, const int *dims,
              const double *phases, double kappa, double tol, int maxiter, int *info,
              double *out_resid) {
    if (!eo_dims_ok(dims)) return -1;
    const long V = volume(dims), Vh = V / 2;
    const long n = SPINOR_CPLX * Vh;
    cplx *be = malloc(sizeof(cplx) * n), *bo = malloc(sizeof(cplx) * n);
    cplx *bh = malloc(sizeof(cplx) * n), *xe = malloc(sizeof(cplx) * n);
    cplx *s = malloc(sizeof(cplx) * n), *r = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *q = malloc(sizeof(cplx) * n);
    cplx *full = malloc(sizeof(cplx) * SPINOR_CPLX * V);
    int rc = 0, iters = 0, napp = 0;
    if (!be || !bo || !bh || !xe || !s || !r || !p || !q || !full) { rc = -2; goto done; }

    extract(be, (const cplx *)b, dims, 0);
    extract(bo, (const cplx *)b, dims, 1);
    /* bhat_e = b_e + kappa D_eo b_o */
    if ((rc = oracle_dslash_eo((double *)bh, gauge, (const double *)bo, dims, phases, 0, 1))) goto done;
    for (long i = 0; i < n; i++) bh[i] = be[i] + kappa * bh[i];

    const double bnorm = sqrt(norm2((const cplx *)b, SPINOR_CPLX * V));
    const double target = tol * bnorm;
    for (long i = 0; i < n; i++) xe[i] = 0;
    memcpy(s, bh, sizeof(cplx) * n);

    int restart = 1;
    double gam = 0;
    while (1) {
        if (restart) {
            /* r = Mhat^dag s, p = r */
            if ((rc = oracle_schur((double *)r, gauge, (const double *)s, dims, phases, kappa, 0, 1))) goto done;
            napp++;
            memcpy(p, r, sizeof(cplx) * n);
            gam = norm2(r, n);
            restart = 0;
        }
        if (sqrt(norm2(s, n)) <= target) {
            /* confirm with the true Schur residual */
            if ((rc = oracle_schur((double *)q, gauge, (const double *)xe, dims, phases, kappa, 0, 0))) goto done;
            napp++;
            for (long i = 0; i < n; i++) s[i] = bh[i] - q[i];
            if (sqrt(norm2(s, n)) <= target) break;
            restart = 1;
            continue;
        }
        if (iters >= maxiter) { rc = 1; break; }
        /* q = Mhat p, alpha = |r|^2 / |q|^2 */
        if ((rc = oracle_schur((double *)q, gauge, (const double *)p, dims, phases, kappa, 0, 0))) goto done;
        napp++;
        const double alpha = gam / norm2(q, n);
        for (long i = 0; i < n; i++) {
            xe[i] += alpha * p[i];
            s[i] -= alpha * q[i];
        }
        /* r = Mhat^dag s, beta = |r_new|^2 / |r_old|^2, p = r + beta p */
        if ((rc = oracle_schur((double *)r, gauge, (const double *)s, dims, phases, kappa, 0, 1))) goto done;
        napp++;
        const double gnew = norm2(r, n);
        const double beta = gnew / gam;
        gam = gnew;
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        iters++;
    }
    {
        int rc2;
        /* x_o = b_o + kappa D_oe x_e */
        if ((rc2 = oracle_dslash_eo((double *)q, gauge, (const double *)xe, dims, phases, 1, 1))) { rc = rc2; goto done; }
        for (long i = 0; i < n; i++) q[i] = bo[i] + kappa * q[i];
        embed(full, xe, dims, 0);
        /* add the odd sites */
        for (long st = 0; st < V; st++) {
            int c[4];
            coords_of(st, dims, c);
            if (parity_of(c) == 1) memcpy(full + SPINOR_CPLX * st, q + SPINOR_CPLX * (st >> 1), sizeof(cplx) * SPINOR_CPLX);
        }
        memcpy(x, full, sizeof(cplx) * SPINOR_CPLX * V);
        /* true residual of the full system */
        cplx *mx = malloc(sizeof(cplx) * SPINOR_CPLX * V);
        if (!mx) { rc = -2; goto done; }
        if ((rc2 = oracle_wilson_m((double *)mx, gauge, x, dims, phases, kappa))) { free(mx); rc = rc2; goto done; }
        double rr = 0;
        const cplx *bb = (const cplx *)b;
        for (long i = 0; i < SPINOR_CPLX * V; i++) {
            cplx d = bb[i] - mx[i];
            rr += creal(d) * creal(d) + cimag(d) * cimag(d);
        }
        free(mx);
        if (out_resid) out_resid[0] = bnorm > 0 ? sqrt(rr) / bnorm : sqrt(rr);
    }
done:
    if (info) { info[0] = iters; info[1] = napp; }
    free(be); free(bo); free(bh); free(xe); free(s); free(r); free(p); free(q); free(full);
    return rc;
}
