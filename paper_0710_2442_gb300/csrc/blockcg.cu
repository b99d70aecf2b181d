// blockcg.cu -- block CG over several right-hand sides (O'Leary, "The block
// conjugate gradient algorithm and related methods", 1980), in the form that
// carries an orthonormal basis of the block residual (Dubrulle, "Retooling
// the method of block conjugate gradients", 2001).  It is the inner solver of
// the FP64 defect correction in solver.cu when the caller asks for it; the
// paper's own statement (Sec. 5) only requires that the solver repeat Eq. 3.
//
// On the normal equations A E = R0 (A = Mhat^dag Mhat, nb columns), with the
// block residual written as R = Q C (Q orthonormal, C nb x nb):
//   Q C = R0                      (QR, by Cholesky QR done twice)
//   S = Q
//   repeat
//     Z  = A S                    (four half-lattice hops per column)
//     xi = (S^H Z)^-1
//     E += S (xi C)
//     Q' psi = Q - Z xi           (QR by Cholesky QR; psi upper triangular)
//     S  = Q' + S psi^H
//     C  = psi C
// Column j's normal residual is |C e_j|.  The search directions of all
// columns span one shared Krylov space, so each column converges in fewer
// iterations than alone; the price per iteration is the nb x nb Gram
// matrices and block updates below.  A block that loses rank (a Cholesky
// pivot that is not positive) stops with status 3 and the caller falls back
// to independent CGs.
//
// Kernels:  bgram (nb x nb Gram matrix of two blocks, FP64 across threads and
// blocks, deterministic); bsmall (one CTA: Cholesky factors, triangular
// inverses and the coefficient matrices, FP64); bqupd (Q -= Z xi); bupd
// (E += S xi C; Q = Q psi^-1; S = Q + S psi^H).  Each block kernel maps one
// thread to one (site, column) pair; the columns of a site sit in one CTA,
// which makes the in-place updates safe with one barrier between reads and
// writes.  Everything stays on the device; the host reads one flag per chunk
// of captured iterations.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "blockcg.h"
#include "solver.h"

namespace wl {

struct BCGState {
    cpx<double> G[kBlockMax * kBlockMax];     // result of the last Gram launch
    cpx<double> xi[kBlockMax * kBlockMax];
    cpx<double> C[kBlockMax * kBlockMax];
    cpx<double> E[kBlockMax * kBlockMax];     // xi C: coefficients of the E update
    cpx<double> Pinv[kBlockMax * kBlockMax];  // psi^-1: coefficients of the Q update
    cpx<double> PsiH[kBlockMax * kBlockMax];  // psi^H: coefficients of the S update
    cpx<double> Cprev[kBlockMax * kBlockMax]; // C at the end of the previous run (reliable restart)
    double cn0[kBlockMax];                    // |C e_j| at the start
    double cn[kBlockMax];                     // |C e_j| now
    double delta[kBlockMax];                  // stop when every cn_j <= delta_j cn0_j
    double rank_tol;                          // smallest sin^2 between a column and the others
    int idx[kBlockMax];                       // field (right-hand side) of block column j
    int nb;
    int iter, maxiter;
    int done;  // 0 running, 1 reduced by delta, 2 iteration cap, 3 breakdown, 4 NaN/Inf
    int halt;  // 1: the block kernels do nothing (set by the gate after done, or at once on 3/4)
    int final; // 1: the run ends with this iteration: its update moves X only, and S, Q, C stay
               //    those of the last step (a reliable restart continues from them)
    int nr;
    int* skip;  // nr hop skip flags: all set once done
};

namespace {

constexpr int kBThreads = 128;
constexpr double kRelPsiMax = 8.0;  // largest |psi_ij| a reliable restart accepts
using cd = cpx<double>;
constexpr int LD = kBlockMax;
enum BMode { BM_INIT = 0, BM_INIT2 = 1, BM_XI = 2, BM_QR = 3, BM_SAVE = 4, BM_REL = 5 };
// update kernel flags: X += S E;  Q = Q Pinv;  S = Q (+ S PsiH)
enum UFlag { UF_X = 1, UF_Q = 2, UF_SSET = 4, UF_SADD = 8 };
constexpr int UP_INIT = UF_Q | UF_SSET;                 // Cholesky QR step of a fresh start
constexpr int UP_INIT_KEEP = UF_Q;                      // the same, keeping S (reliable restart)
constexpr int UP_REL = UF_SSET | UF_SADD;               // S = Q + S psi^H (reliable restart)
constexpr int UP_ITER = UF_X | UF_Q | UF_SSET | UF_SADD;  // one block CG step

template <class T>
__device__ __forceinline__ T* col(const Vec& v, int k) {
    return reinterpret_cast<T*>(static_cast<char*>(v.p) + (long long)k * v.rstep);
}

// ---------------------------------------------------------------------------
// Chunked access to one column's site data: chunk k of site h holds C complex
// components (FP64: 12 chunks of 1, F32: 6 of 2, F16/BF16: 3 of 4 with the
// site's scale applied).  The Gram sum runs over all components, so their
// order inside a site does not matter as long as both operands use it.
// ---------------------------------------------------------------------------
template <int P>
struct Chunks;
template <>
struct Chunks<P_F64> {
    static constexpr int N = 12, C = 1;
    using T = double;
    __device__ static __forceinline__ T scale(const char*, int, int) { return 1.0; }
    __device__ static __forceinline__ void load(const char* base, int stride, int h, int k, T, cpx<T>* v) {
        const double2 d = __ldg(reinterpret_cast<const double2*>(base) + (size_t)k * stride + h);
        v[0] = {d.x, d.y};
    }
};
template <>
struct Chunks<P_F32> {
    static constexpr int N = 6, C = 2;
    using T = float;
    __device__ static __forceinline__ T scale(const char*, int, int) { return 1.f; }
    __device__ static __forceinline__ void load(const char* base, int stride, int h, int k, T, cpx<T>* v) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(base) + (size_t)k * stride + h);
        v[0] = {f.x, f.z};  // (s0.re, s1.re, s0.im, s1.im)
        v[1] = {f.y, f.w};
    }
};
template <int P>
struct ChunksLow {
    static constexpr int N = 3, C = 4;
    using T = float;
    __device__ static __forceinline__ T scale(const char* base, int stride, int h) {
        return __ldg(reinterpret_cast<const float*>(base + 48LL * stride) + h);
    }
    __device__ static __forceinline__ void load(const char* base, int stride, int h, int k, T s, cpx<T>* v) {
        const uint4 d = __ldg(reinterpret_cast<const uint4*>(base) + (size_t)k * stride + h);
        const float2 r01 = LowT<P>::to_f2(d.x), i01 = LowT<P>::to_f2(d.y);
        const float2 r23 = LowT<P>::to_f2(d.z), i23 = LowT<P>::to_f2(d.w);
        v[0] = {r01.x * s, i01.x * s};
        v[1] = {r01.y * s, i01.y * s};
        v[2] = {r23.x * s, i23.x * s};
        v[3] = {r23.y * s, i23.y * s};
    }
};
template <>
struct Chunks<P_F16> : ChunksLow<P_F16> {};
template <>
struct Chunks<P_BF16> : ChunksLow<P_BF16> {};

// ---------------------------------------------------------------------------
// G = A^H B over the nb active columns: G_ij = sum over sites and the 12
// spin-colour components of conj(A_i) B_j, for Gram matrices that are
// Hermitian (A = B) or used through their Hermitian part (S^H A S): only the
// upper triangle of TB x TB tiles is computed and the lower one mirrored.
// Thread (tile, site) keeps a TB x TB block of accumulators (FP32 for FP32 /
// F16 / BF16 data, FP64 for FP64 data) and streams its 2 TB columns chunk by
// chunk; one warp (32 consecutive sites, coalesced loads) per tile.  The sums
// over threads and blocks run in FP64 in a fixed order (warp shuffles, then
// the block's warps, then the last block over all blocks' partials).
// ---------------------------------------------------------------------------
constexpr int kGramSites = 32;  // sites per tile and block iteration: one warp

template <int P, int TB>
__global__ void __launch_bounds__(TB == 6 ? 6 * kGramSites : 10 * kGramSites) bgram_kernel(Vec A, Vec B, Geom g, BCGState* st, double* partials,
                                                   unsigned int* counter) {
    if (__ldcg(&st->halt)) return;
    using CH = Chunks<P>;
    using T = typename CH::T;
    constexpr int C = CH::C;
    __shared__ int s_idx[kBlockMax];
    __shared__ cd s_warp[10][TB * TB];  // one row per warp = tile (at most 10 tiles)
    __shared__ int s_last;
    const int nb = st->nb;
    if (threadIdx.x < kBlockMax) s_idx[threadIdx.x] = threadIdx.x < nb ? st->idx[threadIdx.x] : 0;
    __syncthreads();
    const int nt = (nb + TB - 1) / TB;
    const int tile = threadIdx.x / kGramSites, sub = threadIdx.x % kGramSites;
    int ti = 0, tj = 0;
    for (int t = tile, r = 0; r < nt; r++) {  // tile -> (ti, tj), ti <= tj
        if (t < nt - r) {
            ti = r;
            tj = r + t;
            break;
        }
        t -= nt - r;
    }
    const char* pa[TB];
    const char* pb[TB];
#pragma unroll
    for (int r = 0; r < TB; r++) {
        const int ia = min(ti * TB + r, nb - 1), ib = min(tj * TB + r, nb - 1);
        pa[r] = col<const char>(A, s_idx[ia]);
        pb[r] = col<const char>(B, s_idx[ib]);
    }
    cpx<T> acc[TB][TB];
#pragma unroll
    for (int r = 0; r < TB; r++)
#pragma unroll
        for (int q = 0; q < TB; q++) acc[r][q] = {(T)0, (T)0};
    for (int h = blockIdx.x * kGramSites + sub; h < g.Vh; h += gridDim.x * kGramSites) {
        T sa[TB], sb[TB];
#pragma unroll
        for (int r = 0; r < TB; r++) {
            sa[r] = CH::scale(pa[r], g.stride, h);
            sb[r] = CH::scale(pb[r], g.stride, h);
        }
#pragma unroll 1
        for (int k = 0; k < CH::N; k++) {
            cpx<T> a[TB][C], b[TB][C];
#pragma unroll
            for (int r = 0; r < TB; r++) {
                CH::load(pa[r], g.stride, h, k, sa[r], a[r]);
                CH::load(pb[r], g.stride, h, k, sb[r], b[r]);
            }
#pragma unroll
            for (int r = 0; r < TB; r++)
#pragma unroll
                for (int q = 0; q < TB; q++)
#pragma unroll
                    for (int c = 0; c < C; c++) acc[r][q] = cjfma(a[r][c], b[q][c], acc[r][q]);
        }
    }
    // columns past nb were clamped to column nb - 1 above: their entries are dropped below
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < TB; r++)
#pragma unroll
        for (int q = 0; q < TB; q++) {
            const double re = warp_sum((double)acc[r][q].re), im = warp_sum((double)acc[r][q].im);
            if (lane == 0) s_warp[warp][r * TB + q] = {re, im};
        }
    __syncthreads();
    // per-block partial: the full NBM x NBM layout (kBlockMax), upper tiles only
    double* part = partials + (size_t)blockIdx.x * kBlockMax * kBlockMax * 2;
    const int ntiles = nt * (nt + 1) / 2;
    for (int t = threadIdx.x; t < ntiles * TB * TB; t += blockDim.x) {
        const int tl = t / (TB * TB), e = t % (TB * TB);
        int a0 = 0, b0 = 0;
        for (int u = tl, r = 0; r < nt; r++) {
            if (u < nt - r) {
                a0 = r;
                b0 = r + u;
                break;
            }
            u -= nt - r;
        }
        const int i = a0 * TB + e / TB, j = b0 * TB + e % TB;
        if (i >= nb || j >= nb) continue;
        part[2 * (i * kBlockMax + j)] = s_warp[tl][e].re;
        part[2 * (i * kBlockMax + j) + 1] = s_warp[tl][e].im;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        const bool upper = i / TB <= j / TB;  // (i, j) lies in a computed tile
        const int ii = upper ? i : j, jj = upper ? j : i;
        double re = 0.0, im = 0.0;
        for (unsigned int b = 0; b < gridDim.x; b++) {
            const double* pp = partials + ((size_t)b * kBlockMax * kBlockMax + ii * kBlockMax + jj) * 2;
            re += __ldcg(pp);
            im += __ldcg(pp + 1);
        }
        st->G[i * kBlockMax + j] = upper ? cd{re, im} : cd{re, -im};
    }
    if (threadIdx.x == 0) {
        *counter = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// nb x nb FP64 linear algebra in one CTA (matrices row-major, leading
// dimension kBlockMax, in shared memory).  All threads call every function.
// ---------------------------------------------------------------------------

// a (Hermitian) -> its upper Cholesky factor R with a = R^H R, zero below
// the diagonal.  Returns (in every thread) 1, or -1 if an entry is not
// finite, or 0 if a pivot is not above rel_tol times the original diagonal
// entry (the block lost rank): the pivot over the
// diagonal entry is sin^2 of the angle between column k and the span of the
// columns before it, so this detects a (numerically) rank-deficient block
// whatever the columns' scales.
__device__ int chol_upper(cd* a, int n, double rel_tol) {
    __shared__ int ok;
    __shared__ double diag[LD];
    if (threadIdx.x == 0) ok = 1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) diag[k] = a[k * LD + k].re;
    __syncthreads();
    for (int k = 0; k < n; k++) {
        if (threadIdx.x == 0) {
            const double d = a[k * LD + k].re;
            if (!isfinite(d) || !isfinite(diag[k])) ok = ok == 1 ? -1 : ok;  // NaN / Inf
            else if (!(d > rel_tol * diag[k]) || !(d > 0.0)) ok = ok == 1 ? 0 : ok;  // lost rank
            a[k * LD + k] = {ok ? sqrt(d) : 1.0, 0.0};
        }
        __syncthreads();
        const double inv = 1.0 / a[k * LD + k].re;
        for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) a[k * LD + j] = cscale(inv, a[k * LD + j]);
        __syncthreads();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t / n, j = t % n;
            if (i > k && j >= i) a[i * LD + j] = csub(a[i * LD + j], cjmul(a[k * LD + i], a[k * LD + j]));
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        if (i > j) a[i * LD + j] = {0.0, 0.0};
    }
    __syncthreads();
    const int res = ok;
    __syncthreads();
    return res;
}

// x = r^-1 for upper-triangular r (one thread per column).
__device__ void triu_inv(const cd* r, cd* x, int n) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        for (int i = 0; i < n; i++) x[i * LD + j] = {0.0, 0.0};
        x[j * LD + j] = {1.0 / r[j * LD + j].re, 0.0};
        for (int i = j - 1; i >= 0; i--) {
            cd s = {0.0, 0.0};
            for (int k = i + 1; k <= j; k++) s = cfma(r[i * LD + k], x[k * LD + j], s);
            x[i * LD + j] = cscale(-1.0 / r[i * LD + i].re, s);
        }
    }
    __syncthreads();
}

// c = a b (adj_b: c = a b^H).  c must not alias a or b.
__device__ void matmul(const cd* a, const cd* b, cd* c, int n, bool adj_b) {
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        cd s = {0.0, 0.0};
        for (int k = 0; k < n; k++) s = adj_b ? cfma(a[i * LD + k], cconj(b[j * LD + k]), s)
                                              : cfma(a[i * LD + k], b[k * LD + j], s);
        c[i * LD + j] = s;
    }
    __syncthreads();
}

__device__ void copy_mat(const cd* a, cd* b, int n) {
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) b[(t / n) * LD + t % n] = a[(t / n) * LD + t % n];
    __syncthreads();
}

// |C e_j| for every column, and whether they are all finite.
__device__ bool col_norms(const cd* c, double* out, int n) {
    __shared__ int finite;
    if (threadIdx.x == 0) finite = 1;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += cnorm2(c[i * LD + j]);
        out[j] = sqrt(s);
        if (!isfinite(s)) finite = 0;
    }
    __syncthreads();
    const bool res = finite != 0;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(256) bsmall_kernel(BCGState* st, int mode) {
    if (st->halt) return;
    __shared__ cd a[LD * LD], b[LD * LD], c[LD * LD];
    const int n = st->nb;
    if (mode == BM_SAVE) {
        copy_mat(st->C, st->Cprev, n);
        return;
    }
    if (mode == BM_REL) {
        // psi = C_new Cprev^-1 (both upper triangular): S = Q + S psi^H continues the
        // previous run's directions with the recomputed residual (for one column this
        // is p = r + (|r|^2 / |r_old|^2) p)
        copy_mat(st->Cprev, a, n);
        triu_inv(a, b, n);
        copy_mat(st->C, a, n);
        matmul(a, b, c, n, false);
        // Accepted only while psi stays modest, as it does when the recomputed residual
        // continues the previous one; an ill-conditioned Cprev (columns reduced very
        // unevenly in reduced precision) would blow the directions up, and a plain
        // restart (S = Q) is taken instead.
        __shared__ int good;
        if (threadIdx.x == 0) good = 1;
        __syncthreads();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const cd v = c[(t / n) * LD + t % n];
            if (!(fabs(v.re) <= kRelPsiMax) || !(fabs(v.im) <= kRelPsiMax)) good = 0;
        }
        __syncthreads();
        const bool ok = good != 0;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t / n, j = t % n;
            st->PsiH[i * LD + j] = ok ? cconj(c[j * LD + i]) : cd{0.0, 0.0};
        }
        return;
    }
    copy_mat(st->G, a, n);
    auto fail = [&](int why) {
        if (threadIdx.x == 0) {
            st->done = why;
            st->halt = 1;
        }
        for (int k = threadIdx.x; k < st->nr; k += blockDim.x) st->skip[k] = 1;
    };
    if (mode == BM_XI) {
        // symmetrise S^H Z (Hermitian in exact arithmetic), then xi = L^-1 L^-H
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t / n, j = t % n;
            if (i < j) {
                const cd u = a[i * LD + j], l = a[j * LD + i];
                const cd m = {0.5 * (u.re + l.re), 0.5 * (u.im - l.im)};
                a[i * LD + j] = m;
                a[j * LD + i] = cconj(m);
            } else if (i == j) {
                a[i * LD + i].im = 0.0;
            }
        }
        __syncthreads();
        if (const int ch = chol_upper(a, n, st->rank_tol); ch != 1) return fail(ch < 0 ? 4 : 3);
        triu_inv(a, b, n);         // b = L^-1
        matmul(b, b, c, n, true);  // c = L^-1 L^-H = (S^H Z)^-1
        copy_mat(c, st->xi, n);
        copy_mat(st->C, a, n);
        matmul(c, a, b, n, false);  // E = xi C
        copy_mat(b, st->E, n);
        return;
    }
    // BM_INIT, BM_INIT2, BM_QR: Cholesky QR factor psi of the Gram matrix in a
    if (const int ch = chol_upper(a, n, st->rank_tol); ch != 1) return fail(ch < 0 ? 4 : 3);
    triu_inv(a, b, n);
    if (mode == BM_INIT) {
        copy_mat(b, st->Pinv, n);
        copy_mat(a, st->C, n);
        return;
    }
    copy_mat(b, st->Pinv, n);
    copy_mat(st->C, b, n);
    matmul(a, b, c, n, false);  // psi C
    __shared__ double cn[LD];
    if (!col_norms(c, cn, n)) return fail(4);
    if (mode == BM_INIT2) {
        copy_mat(c, st->C, n);
        for (int j = threadIdx.x; j < n; j += blockDim.x) st->cn0[j] = st->cn[j] = cn[j];
        return;
    }
    // BM_QR: convergence test on the new residual coefficients
    __shared__ int s_done;
    if (threadIdx.x == 0) {
        bool reduced = true;
        for (int j = 0; j < n; j++) {
            st->cn[j] = cn[j];
            reduced = reduced && cn[j] <= st->delta[j] * st->cn0[j];
        }
        const int it = st->iter + 1;
        st->iter = it;
        s_done = reduced ? 1 : it >= st->maxiter ? 2 : 0;
        if (s_done) {
            st->done = s_done;
            st->final = 1;
        }
    }
    __syncthreads();
    if (s_done) {
        for (int k = threadIdx.x; k < st->nr; k += blockDim.x) st->skip[k] = 1;
        return;  // C, Q and S stay those of the last step
    }
    copy_mat(c, st->C, n);
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        st->PsiH[i * LD + j] = cconj(a[j * LD + i]);
    }
}

// Start of an iteration: once the previous iteration finished the block,
// every block kernel of this and later iterations does nothing.
__global__ void bgate_kernel(BCGState* st) {
    if (st->done) st->halt = 1;
}

// ---------------------------------------------------------------------------
// Q_j -= sum_i Z_i xi_ij   (Q in precision PQ, Z in PZ)
// ---------------------------------------------------------------------------
template <int PQ, int PZ, int NBM>
__global__ void __launch_bounds__(kBThreads) bqupd_kernel(Vec Q, Vec Z, Geom g, BCGState* st) {
    if (__ldcg(&st->halt)) return;
    using TQ = typename SpinorFmt<PQ>::real;
    using TZ = typename SpinorFmt<PZ>::real;
    constexpr int SPB = kBThreads / NBM;
    __shared__ int s_idx[NBM];
    __shared__ cpx<TQ> s_xi[NBM][NBM];
    const int nb = st->nb;
    for (int t = threadIdx.x; t < NBM * NBM; t += blockDim.x) {
        const int i = t / NBM, j = t % NBM;
        const cd v = (i < nb && j < nb) ? st->xi[i * kBlockMax + j] : cd{0.0, 0.0};
        s_xi[i][j] = {(TQ)v.re, (TQ)v.im};
    }
    if (threadIdx.x < NBM) s_idx[threadIdx.x] = threadIdx.x < nb ? st->idx[threadIdx.x] : 0;
    __syncthreads();
    const int j = threadIdx.x % NBM, sub = threadIdx.x / NBM;
    if (sub >= SPB || j >= nb) return;
    char* Qj = col<char>(Q, s_idx[j]);
    for (int h = blockIdx.x * SPB + sub; h < g.Vh; h += gridDim.x * SPB) {
        cpx<TQ> qv[12];
        SpinorFmt<PQ>::load(Qj, g.stride, h, qv);
#pragma unroll
        for (int i = 0; i < NBM; i++) {
            if (i < nb) {
                cpx<TZ> zv[12];
                SpinorFmt<PZ>::load(col<const char>(Z, s_idx[i]), g.stride, h, zv);
                const cpx<TQ> m = cneg(s_xi[i][j]);
#pragma unroll
                for (int c = 0; c < 12; c++) qv[c] = cfma(cpx<TQ>{(TQ)zv[c].re, (TQ)zv[c].im}, m, qv[c]);
            }
        }
        SpinorFmt<PQ>::store(Qj, g.stride, h, qv);
    }
}

// ---------------------------------------------------------------------------
// One pass over the block, by flags:
//   UF_X:  X_j += sum_i S_i E_ij
//   UF_Q:  Q_j  = sum_i Q_i Pinv_ij        (else Q_j is read as it is)
//   UF_SSET: S_j = Q_j (the new Q_j), plus sum_i S_i PsiH_ij with UF_SADD
// (Q, X in precision PX; S in PS.)  In the final iteration of a run only X
// moves.  Reads of a site's columns all happen before the CTA's barrier,
// writes after it.
// ---------------------------------------------------------------------------
template <int PX, int PS, int NBM>
__global__ void __launch_bounds__(kBThreads) bupd_kernel(Vec Q, Vec S, Vec X, Geom g, BCGState* st, int flags) {
    if (__ldcg(&st->halt)) return;
    if (flags == UP_ITER && __ldcg(&st->final)) flags = UF_X;
    const bool fx = flags & UF_X, fq = flags & UF_Q, fset = flags & UF_SSET, fadd = flags & UF_SADD;
    using TX = typename SpinorFmt<PX>::real;
    using TS = typename SpinorFmt<PS>::real;
    constexpr int SPB = kBThreads / NBM;
    __shared__ int s_idx[NBM];
    __shared__ cpx<TX> s_p[NBM][NBM], s_e[NBM][NBM], s_h[NBM][NBM];
    const int nb = st->nb;
    for (int t = threadIdx.x; t < NBM * NBM; t += blockDim.x) {
        const int i = t / NBM, j = t % NBM;
        const bool in = i < nb && j < nb;
        const cd p = in && fq ? st->Pinv[i * kBlockMax + j] : cd{0.0, 0.0};
        const cd e = in && fx ? st->E[i * kBlockMax + j] : cd{0.0, 0.0};
        const cd hh = in && fadd ? st->PsiH[i * kBlockMax + j] : cd{0.0, 0.0};
        s_p[i][j] = {(TX)p.re, (TX)p.im};
        s_e[i][j] = {(TX)e.re, (TX)e.im};
        s_h[i][j] = {(TX)hh.re, (TX)hh.im};
    }
    if (threadIdx.x < NBM) s_idx[threadIdx.x] = threadIdx.x < nb ? st->idx[threadIdx.x] : 0;
    __syncthreads();
    const int j = threadIdx.x % NBM, sub = threadIdx.x / NBM;
    const bool act = sub < SPB && j < nb;
    const int col_j = s_idx[j];
    // block-uniform trip count: every thread reaches every barrier
    for (int h0 = blockIdx.x * SPB; h0 < g.Vh; h0 += gridDim.x * SPB) {
        const int h = h0 + sub;
        const bool on = act && h < g.Vh;
        cpx<TX> qn[12], sn[12], xn[12];
        if (on) {
#pragma unroll
            for (int c = 0; c < 12; c++) qn[c] = sn[c] = {(TX)0, (TX)0};
            if (fx) SpinorFmt<PX>::load(col<const char>(X, col_j), g.stride, h, xn);
            if (!fq && fset) SpinorFmt<PX>::load(col<const char>(Q, col_j), g.stride, h, qn);
#pragma unroll
            for (int i = 0; i < NBM; i++) {
                if (i < nb) {
                    if (fq) {
                        cpx<TX> qi[12];
                        SpinorFmt<PX>::load(col<const char>(Q, s_idx[i]), g.stride, h, qi);
                        const cpx<TX> p = s_p[i][j];
#pragma unroll
                        for (int c = 0; c < 12; c++) qn[c] = cfma(qi[c], p, qn[c]);
                    }
                    if (fx || fadd) {
                        cpx<TS> si[12];
                        SpinorFmt<PS>::load(col<const char>(S, s_idx[i]), g.stride, h, si);
                        const cpx<TX> e = s_e[i][j], hh = s_h[i][j];
#pragma unroll
                        for (int c = 0; c < 12; c++) {
                            const cpx<TX> v = {(TX)si[c].re, (TX)si[c].im};
                            xn[c] = cfma(v, e, xn[c]);
                            sn[c] = cfma(v, hh, sn[c]);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (on) {
            if (fq) SpinorFmt<PX>::store(col<char>(Q, col_j), g.stride, h, qn);
            if (fset) {
                cpx<TS> so[12];
#pragma unroll
                for (int c = 0; c < 12; c++) {
                    const cpx<TX> v = cadd(qn[c], sn[c]);
                    so[c] = {(TS)v.re, (TS)v.im};
                }
                SpinorFmt<PS>::store(col<char>(S, col_j), g.stride, h, so);
            }
            if (fx) SpinorFmt<PX>::store(col<char>(X, col_j), g.stride, h, xn);
        }
    }
}

// Precision dispatch: a Gram matrix of two blocks of one precision, and the
// (accumulation, inner) pairs of the updates.
template <class F>
void with_same(Prec p, F&& f) {
    using std::integral_constant;
    switch (p) {
        case P_F64: f(integral_constant<int, P_F64>{}); break;
        case P_F32: f(integral_constant<int, P_F32>{}); break;
        case P_F16: f(integral_constant<int, P_F16>{}); break;
        case P_BF16: f(integral_constant<int, P_BF16>{}); break;
    }
}

template <class F>
void with_xi(Prec xp, Prec ip, F&& f) {
    using std::integral_constant;
    if (xp == P_F64 && ip == P_F64) f(integral_constant<int, P_F64>{}, integral_constant<int, P_F64>{});
    else if (xp == P_F32 && ip == P_F32) f(integral_constant<int, P_F32>{}, integral_constant<int, P_F32>{});
    else if (xp == P_F32 && ip == P_F16) f(integral_constant<int, P_F32>{}, integral_constant<int, P_F16>{});
    else if (xp == P_F32 && ip == P_BF16) f(integral_constant<int, P_F32>{}, integral_constant<int, P_BF16>{});
    else throw Error(7, "block CG: unsupported precision pair");
}

template <class F>
void with_nbm(int nbm, F&& f) {
    switch (nbm) {
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 12: f(std::integral_constant<int, 12>{}); break;
        default: f(std::integral_constant<int, 16>{}); break;
    }
}

}  // namespace

BlockInner::BlockInner(Prec ip, Prec xp, const Geom& g, int nrhs) : ip_(ip), xp_(xp), g_(g), nr_(nrhs) {
    WL_REQUIRE(nrhs >= 1 && nrhs <= kBlockMax, "block CG takes at most 16 right-hand sides");
    nbm_ = nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : nrhs <= 12 ? 12 : 16;
    const int spb = kBThreads / nbm_;
    grid_ = std::max(1, std::min((g.Vh + spb - 1) / spb, 4 * device_sm_count()));
    q_.alloc(xp, 0, nrhs, g);
    state_.alloc(sizeof(BCGState));
    partials_.alloc(sizeof(double) * 2 * (size_t)kBlockMax * kBlockMax * grid_);
    counter_.alloc(sizeof(unsigned int));
    skip_.alloc(sizeof(int) * nrhs);
    WL_CUDA(cudaMemset(counter_.p, 0, sizeof(unsigned int)));
    WL_CUDA(cudaMemset(state_.p, 0, sizeof(BCGState)));
}

BlockInner::~BlockInner() {
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
}

void BlockInner::gram(Prec p, Vec a, Vec b, cudaStream_t st) {
    BCGState* s = state_.as<BCGState>();
    double* part = partials_.as<double>();
    unsigned int* cnt = counter_.as<unsigned int>();
    // tiles of 6 columns (4 in FP64: its accumulators take twice the registers);
    // one warp per upper tile: at most 6 (10 in FP64) warps
    const int tb = p == P_F64 ? 4 : 6;
    const int nt = (nr_ + tb - 1) / tb, threads = kGramSites * nt * (nt + 1) / 2;
    with_same(p, [&](auto A) {
        constexpr int PA = decltype(A)::value;
        bgram_kernel<PA, PA == P_F64 ? 4 : 6><<<grid_, threads, 0, st>>>(a, b, g_, s, part, cnt);
    });
    WL_LAUNCH_CHECK();
}

void BlockInner::small(int mode, cudaStream_t st) {
    bsmall_kernel<<<1, 256, 0, st>>>(state_.as<BCGState>(), mode);
    WL_LAUNCH_CHECK();
}

void BlockInner::update(int mode, Vec S, Vec X, cudaStream_t st) {
    with_nbm(nbm_, [&](auto N) {
        with_xi(xp_, ip_, [&](auto A, auto B) {
            bupd_kernel<decltype(A)::value, decltype(B)::value, decltype(N)::value>
                <<<grid_, kBThreads, 0, st>>>(vec(q_, 0), S, X, g_, state_.as<BCGState>(), mode);
        });
    });
    WL_LAUNCH_CHECK();
}

void BlockInner::iteration(const GaugeField& glo, double kappa, Vec S, Vec W, Vec Z, Vec T, Vec X, cudaStream_t st) {
    BCGState* s = state_.as<BCGState>();
    bgate_kernel<<<1, 1, 0, st>>>(s);
    WL_LAUNCH_CHECK();
    const int* skip = skip_.as<int>();
    schur_apply(glo, ip_, W, S, T, nr_, kappa, 0, nullptr, skip, 1, 0, st);  // W = Mhat S
    schur_apply(glo, ip_, Z, W, T, nr_, kappa, 1, nullptr, skip, 1, 0, st);  // Z = Mhat^dag W
    gram(ip_, S, Z, st);                                                      // S^H Z
    small(BM_XI, st);
    with_nbm(nbm_, [&](auto N) {
        with_xi(xp_, ip_, [&](auto A, auto B) {
            bqupd_kernel<decltype(A)::value, decltype(B)::value, decltype(N)::value>
                <<<grid_, kBThreads, 0, st>>>(vec(q_, 0), Z, g_, s);
        });
    });
    WL_LAUNCH_CHECK();
    gram(xp_, vec(q_, 0), vec(q_, 0), st);  // (Q - Z xi)^H (Q - Z xi)
    small(BM_QR, st);
    update(UP_ITER, S, X, st);
}

BlockInner::Result BlockInner::run(const GaugeField& glo, double kappa, Vec s_in, Vec S, Vec W, Vec Z, Vec T, Vec X,
                                   const std::vector<int>& finished, const std::vector<double>& delta,
                                   int maxiter, int chunk, bool use_graph, bool reliable, cudaStream_t st) {
    NvtxRange nvtx("block cg");
    // host-side state: the active columns
    BCGState h;
    std::memset(&h, 0, sizeof(h));
    std::vector<int> skip(nr_, 1);
    for (int k = 0; k < nr_; k++)
        if (!finished[k]) {
            h.idx[h.nb++] = k;
            skip[k] = 0;
        }
    Result res;
    if (h.nb == 0) return res;
    const std::vector<int> active(h.idx, h.idx + h.nb);
    const bool rel = reliable && prev_ok_ && active == prev_active_;
    for (int j = 0; j < h.nb; j++) h.delta[j] = delta[h.idx[j]];
    h.rank_tol = xp_ == P_F64 ? 1e-12 : 1e-6;
    h.maxiter = std::max(1, maxiter);
    h.nr = nr_;
    h.skip = skip_.as<int>();
    BCGState* d = state_.as<BCGState>();
    // only the header fields change; the matrices are recomputed below
    const size_t off = offsetof(BCGState, cn0);
    WL_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(d) + off, reinterpret_cast<char*>(&h) + off,
                            sizeof(BCGState) - off, cudaMemcpyHostToDevice, st));
    WL_CUDA(cudaMemcpyAsync(skip_.p, skip.data(), sizeof(int) * nr_, cudaMemcpyHostToDevice, st));
    for (int k = 0; k < nr_; k++) WL_CUDA(cudaMemsetAsync(static_cast<char*>(X.p) + k * X.rstep, 0,
                                                          q_.pbytes, st));

    // R0 = Mhat^dag s (into Z), Q = R0 in xp, then Cholesky QR twice: Q C = R0; then
    // S = Q (fresh start) or S = Q + S psi^H with psi = C Cprev^-1 (reliable restart:
    // the previous run's directions continue with the recomputed residual)
    if (rel) small(BM_SAVE, st);
    schur_apply(glo, ip_, Z, s_in, T, nr_, kappa, 1, nullptr, skip_.as<int>(), 1, 0, st);
    convert(xp_, vec(q_, 0), ip_, Z, g_, nr_, st);
    gram(xp_, vec(q_, 0), vec(q_, 0), st);
    small(BM_INIT, st);
    update(rel ? UP_INIT_KEEP : UP_INIT, S, X, st);
    gram(xp_, vec(q_, 0), vec(q_, 0), st);
    small(BM_INIT2, st);
    update(rel ? UP_INIT_KEEP : UP_INIT, S, X, st);
    if (rel) {
        small(BM_REL, st);
        update(UP_REL, S, X, st);
    }

    if (use_graph && !exec_) {
        WL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            for (int k = 0; k < chunk; k++) iteration(glo, kappa, S, W, Z, T, X, st);
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(st, &junk);
            if (junk) cudaGraphDestroy(junk);
            throw;
        }
        WL_CUDA(cudaStreamEndCapture(st, &graph_));
        WL_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
    }
    int flags[2] = {0, 0};
    while (true) {
        if (exec_) WL_CUDA(cudaGraphLaunch(exec_, st));
        else for (int k = 0; k < chunk; k++) iteration(glo, kappa, S, W, Z, T, X, st);
        WL_CUDA(cudaMemcpyAsync(flags, &d->iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));  // iter, maxiter
        int done = 0;
        WL_CUDA(cudaMemcpyAsync(&done, &d->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        WL_CUDA(cudaStreamSynchronize(st));
        if (done) {
            res.iterations = flags[0];
            res.status = done >= 3 ? done : 0;
            prev_ok_ = res.status == 0;
            prev_active_ = active;
            if (const char* e = std::getenv("WILSON_BLOCK_VERBOSE"))
                if (std::atoi(e)) std::fprintf(stderr, "[wilson] block cg: %d columns, %d iterations, end %d\n",
                                               h.nb, flags[0], done);
            break;
        }
    }
    return res;
}

}  // namespace wl
