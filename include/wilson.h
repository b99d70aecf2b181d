/*
 * wilson.h -- C ABI of libwilson_gb300: the Wilson-Dirac hopping term, its
 * even-odd (checkerboard) form and CG solves built on it, on one GB300 GPU.
 *
 * The operator (QCD on the Cell BE, Sec. 5, Eq. 3), in the convention this
 * library uses ("(1-gamma) forward"):
 *
 *   (D_h psi)_x = sum_{mu=1..4} [ (1 - g_mu) eta_mu(x)      U_{x,mu}         psi_{x+mu}
 *                               + (1 + g_mu) eta*_mu(x-mu)  U^dag_{x-mu,mu}  psi_{x-mu} ]
 *
 * Eq. 3 as printed in the paper puts (1 + g_mu) on the forward hop; the two
 * are related by D_printed = g_5 D_h g_5.  g_mu are the DeGrand-Rossi gamma
 * matrices (g_5 = diag(1,1,-1,-1)); mu = 1..4 are x, y, z, t.  eta_mu(x) is
 * the boundary phase of direction mu when the forward hop from x wraps from
 * x_mu = L_mu - 1 to 0; the backward hop that wraps takes its conjugate.
 * The Wilson matrix is M = 1 - kappa D_h.
 *
 * Even-odd form: with parity p = (x+y+z+t) mod 2, D_h couples only opposite
 * parities; D_{p,1-p} is the block from parity 1-p to parity p.  The Schur
 * complement on parity p is Mhat_p = 1 - kappa^2 D_{p,1-p} D_{1-p,p}, and
 * Mhat_p^dag = g_5 Mhat_p g_5.
 *
 * Canonical field layout (all "canon" pointers): complex numbers as
 * interleaved (re, im) doubles,
 *   spinor  [site][spin 0..3][colour 0..2]             24 doubles per site
 *   gauge   [site][mu 0..3][row 0..2][col 0..2]         72 doubles per site
 *   site    s = x + Lx*(y + Ly*(z + Lz*t))
 *   half (parity-p) field: the sites of parity p, site s stored at s >> 1
 *   (Vh = V/2 entries; needs even extents).
 *
 * Conventions of every entry point:
 *   - returns a wilson_status; never throws; wilson_last_error() gives a
 *     thread-local message for the last failure on the calling thread;
 *   - the caller owns every field pointer it passes; the library owns the
 *     handles it creates and its internal workspace;
 *   - "stream" is a cudaStream_t (NULL = legacy default stream); operator
 *     calls are asynchronous on it; solves synchronise it before returning;
 *   - validation: all extents >= 2 and even, V < 2^31, non-null pointers,
 *     finite kappa, |phase| = 1 within 1e-12.  Violations give WILSON_ERR_ARG
 *     and launch nothing.
 *
 * There is no CPU fallback: every call runs on the current CUDA device and
 * returns WILSON_ERR_CUDA if there is none.
 *
 * Environment (none is needed; they serve measurement and tests):
 *   WILSON_TUNE=0                 no autotuning: default launch configurations
 *   WILSON_TUNE_CACHE=path        load tuning decisions from path, append new ones
 *   WILSON_TUNE_VERBOSE=1         report tuning candidates and decisions on stderr
 *   WILSON_HOP_VARIANT=v          pin the hop kernel variant (0..28) of every launch;
 *                                 a variant that does not fit a launch runs variant 3
 *   WILSON_HOP_BLOCK=n            block size with WILSON_HOP_VARIANT (64, 128, 256)
 *   WILSON_TEST_STAGE_TIMEOUT=1   failure-detection test only: the t-slab hop's
 *                                 staged slices never complete, so its bounded
 *                                 waits give up (NaN outputs, counted by
 *                                 wilson_stage_timeouts)
 *   WILSON_PDL=0                  hops without programmatic dependent launch (read
 *                                 once per process)
 *   WILSON_BATCH_SMALL_VH=n       batched solves: lattices with at most n sites per
 *                                 parity run on the on-chip solver
 *   WILSON_BATCH_SMALL_CLUSTER=1  one CTA per small lattice instead of a cluster of four
 *   WILSON_BATCH_CLASSES=n        at most n lattice-size classes (default 4)
 *   WILSON_BATCH_PRIORITY=0       no graph-node priorities between the classes
 *   WILSON_BATCH_GRID_PER_SM=n    n blocks per SM for the tile-walking kernels
 *                                 (default: one block per tile)
 *   WILSON_BATCH_HOP=v:b          batched solves: the inner hop's kernel variant and
 *                                 block instead of the tuned one (0-5 with 64, 128 or
 *                                 256 threads; for F16 and BF16 also 22, the
 *                                 pipelined stencil, with 64 or 128)
 *   WILSON_BATCH_TILE=n           batch tile size (128, 256 or 512 sites) instead of
 *                                 the autotuned one
 *   WILSON_BATCH_HOST_LOOP=1      host-replayed graphs instead of device-side loops
 *   WILSON_BATCH_MAX_LOOP=n       lower the batch loop's iteration cap
 *   WILSON_BATCH_BUDGET_MS=t      lower the batch loop's wall-clock budget (60 s)
 *   WILSON_BLOCK_VERBOSE=1        report each block-CG run on stderr
 */
#ifndef WILSON_GB300_H
#define WILSON_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WILSON_OK = 0,
    WILSON_ERR_ARG = 1,         /* invalid argument; nothing was launched        */
    WILSON_ERR_CUDA = 2,        /* a CUDA call failed                            */
    WILSON_ERR_OOM = 3,         /* device allocation failed                      */
    WILSON_ERR_NOCONV = 4,      /* solve stopped at maxiter / max_restarts       */
    WILSON_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out            */
    WILSON_ERR_NUMERIC = 6,     /* NaN or Inf met in a reduction                 */
    WILSON_ERR_UNSUPPORTED = 7  /* valid but not implemented combination         */
} wilson_status;

typedef enum { WILSON_F64 = 0, WILSON_F32 = 1, WILSON_F16 = 2, WILSON_BF16 = 3 } wilson_prec;

typedef enum {
    WILSON_OP_HOP = 0,        /* D_h (full field) or D_{p,1-p} (half field)                  */
    WILSON_OP_M = 1,          /* M = 1 - kappa D_h; full fields only                          */
    WILSON_OP_SCHUR = 2,      /* Mhat_p = 1 - kappa^2 D_{p,1-p} D_{1-p,p}; half fields only   */
    WILSON_OP_SCHUR_DAG = 3   /* Mhat_p^dag = g_5 Mhat_p g_5; half fields only                */
} wilson_op;

typedef enum { WILSON_EVEN = 0, WILSON_ODD = 1, WILSON_FULL = 2 } wilson_subset;

typedef struct {
    int dims[4];            /* Lx, Ly, Lz, Lt (t = the 4-direction)                      */
    double bc_phase[4][2];  /* (re, im) boundary phase per direction; periodic x,y,z and */
                            /* antiperiodic t is {1,0},{1,0},{1,0},{-1,0}                 */
} wilson_lattice;

/* ---------------------------------------------------------------------- */
/* Stateless calls on canonical complex128 device fields (Sec. 5, Eq. 3).  */
/* Computed in FP64 with 18-real links.  Each call packs its inputs into   */
/* workspace taken from a per-device memory pool of the library with       */
/* stream-ordered allocation on the caller's stream (the pool keeps its    */
/* memory, so only the first call of a size grows it).  The calls do not   */
/* synchronise, except that the first call for a new lattice, operator    */
/* and dagger flag times the kernel's launch configurations (autotuning)   */
/* and so synchronises the stream once; WILSON_TUNE=0 turns that off.      */
/* ---------------------------------------------------------------------- */

/* out = D_h in (op = HOP) or M in (op = M), full lattice.
 * out, in: V spinors (canonical, device); gauge: 4V links (canonical, device).
 * out must not overlap in. */
int wilson_dslash(double* out, const double* gauge, const double* in, const wilson_lattice* L,
                  double kappa, int op, void* stream);

/* Half-lattice form.  op = HOP: out (parity out_parity) = D_{p,1-p} in (parity 1-p).
 * op = SCHUR / SCHUR_DAG: out and in are both parity out_parity.
 * out, in: V/2 spinors (canonical half fields, device). */
int wilson_dslash_eo(double* out, const double* gauge, const double* in, const wilson_lattice* L,
                     int out_parity, double kappa, int op, void* stream);

/* ---------------------------------------------------------------------- */
/* Solver (not in the paper, which only notes that an iterative solver     */
/* repeats Eq. 3): CG on the normal equations of the even Schur complement */
/*   bhat_e = b_e + kappa D_eo b_o;  Mhat^dag Mhat x_e = Mhat^dag bhat_e;   */
/*   x_o = b_o + kappa D_oe x_e,                                           */
/* stopped when the true relative residual |b - M x| / |b| <= tol,          */
/* recomputed in FP64 on the GPU.  With inner = F32/F16/BF16 the CG runs in */
/* that storage precision (FP32 arithmetic) inside an FP64 defect          */
/* correction; with inner = F64 it is plain FP64 CG.  A correction whose    */
/* expected residual (the last one times the inner reduction) is above      */
/* 1e-4 |bhat| (and tol < 1e-7) computes it with FP32 fields and links      */
/* (error about 1e-7 |Mhat| |x|); every other residual, and every          */
/* convergence decision, is FP64.                                          */
/* ---------------------------------------------------------------------- */
typedef struct {
    int inner;              /* wilson_prec of the inner CG (F64 = plain FP64 CG)            */
    int recon;              /* link storage of the inner operator: 12 or 18 reals           */
    double tol;             /* target true relative residual, e.g. 1e-10                    */
    int maxiter;            /* cap on inner CG iterations over the whole solve              */
    int max_restarts;       /* cap on FP64 outer corrections                                */
    double delta;           /* inner reduction per outer correction; 0 = default per inner
                               precision: F32 1e-4, F16 0.02, BF16 0.1 (FP64: none).  An
                               inner solve also stops after 1000 iterations, and the next
                               FP64 correction continues it.                                */
    int use_initial_guess;  /* 1: x holds the initial guess on entry                        */
    int reliable;           /* 1: reliable updates (keep the CG direction), 0: restart CG   */
    int block_cg;           /* wilson_cg_solve_multi with 2..16 right-hand sides: 1 = one
                               block CG over all of them (O'Leary 1980, in Dubrulle's 2001
                               form with an orthonormal residual basis) inside the FP64
                               correction, instead of independent CGs in lockstep; 0 (default)
                               = independent CGs.  Ignored for a single right-hand side.    */
} wilson_solver_params;

typedef struct {
    int status;               /* wilson_status of the solve                          */
    int outer_iters;          /* FP64 corrections (residual recomputations)          */
    int inner_iters;          /* CG iterations in total                              */
    int hop_applications;     /* half-lattice hopping-term applications, all precisions */
    double true_rel_resid;    /* |b - M x| / |b|, FP64, recomputed at the end       */
    double seconds;           /* wall time of the solve (device-synchronised)        */
    double inner_seconds;     /* device time of the inner CG iterations (CUDA events
                                 around their replays; 0 for block CG and batches)  */
    int outer_f32;            /* corrections whose residual was computed in FP32     */
} wilson_solve_stats;

/* Default parameters for an inner precision (tol 1e-10). */
wilson_solver_params wilson_solver_defaults(int inner);

/* x, b: V spinors (canonical, device); gauge: 4V links (canonical, device).
 * Returns WILSON_OK, or WILSON_ERR_NOCONV with x holding the last iterate
 * (maxiter or max_restarts spent, or an FP64 residual grown 1000-fold past
 * the smallest one of the solve: a diverging inner solve). */
int wilson_cg_solve(double* x, const double* gauge, const double* b, const wilson_lattice* L,
                    double kappa, const wilson_solver_params* p, wilson_solve_stats* st, void* stream);

/* Several right-hand sides sharing one gauge field, solved as independent
 * CGs in lockstep (each launch covers all of them; a finished one is
 * skipped).  x, b: nrhs canonical full fields back to back (device);
 * st: nrhs entries (outer_iters, hop_applications and seconds are shared).
 * Returns WILSON_OK only if every right-hand side converged. */
int wilson_cg_solve_multi(double* x, const double* gauge, const double* b, int nrhs, const wilson_lattice* L,
                          double kappa, const wilson_solver_params* p, wilson_solve_stats* st, void* stream);

/* Many independent solves on lattices of different sizes, each with its
 * own links, kappa and source, in ONE CUDA graph launch (Sec. 5 sets the
 * lattice sizes that fit each memory level; here every size shares one GPU).
 * Every problem runs the same CGNR + FP64-correction state machine as
 * wilson_cg_solve.  Problems with at most 4096 sites per parity are each
 * solved by one thread block that keeps the whole solve on its SM.  The
 * others are grouped by lattice size into at most four classes; each class
 * has its own device-side loop (a conditional graph node) over a tile table
 * of its problems, FP64 corrections and reduced-precision CG steps of
 * different problems running as parallel graph branches, and the kernels of
 * smaller classes are scheduled ahead of larger ones (graph node priority),
 * so every class finishes at its own pace.  Inner precision F32, F16 or BF16
 * (links with 12 reals).  st[i].seconds is problem i's completion time
 * measured on the device from the start of the batch; each loop stops after
 * an iteration cap or a wall-clock budget (60 s) even if some problem is
 * unfinished (WILSON_ERR_TIMEOUT for those).  Returns WILSON_OK if every
 * problem converged, else WILSON_ERR_NUMERIC if any problem met a
 * non-finite value, else the first non-OK status over the problems. */
typedef struct {
    wilson_lattice L;
    double kappa;
    const double* gauge;  /* 4V links, canonical, device                                  */
    const double* b;      /* V spinors, canonical, device                                 */
    double* x;            /* V spinors, canonical, device: solution (initial guess if set) */
} wilson_problem;

typedef struct {
    double seconds;         /* host wall time of the call (set-up, solve, read-back)      */
    double device_seconds;  /* device time from the batch's start to its end               */
    int iterations;         /* loop iterations of the longest class loop (one CG step or FP64
                               correction per problem and iteration)                        */
    int graph_launches;     /* 1 when the loop runs on the device                          */
    int device_loop;        /* 1: conditional-node loop; 0: host-replayed graph chunks     */
    int timed_out;          /* 1: the iteration cap or wall-clock budget ended the loop    */
    int tiles;              /* tiles over the problems the class loops solve (each class's
                               tile size, 128, 256 or 512 sites, is autotuned)              */
} wilson_batch_info;

int wilson_batch_solve(int n, const wilson_problem* probs, const wilson_solver_params* p, wilson_solve_stats* st,
                       wilson_batch_info* info, void* stream);

/* ---------------------------------------------------------------------- */
/* Handles: prepared fields for repeated (timed) applications.             */
/* A gauge handle holds the links in the site-vectorised structure-of-     */
/* arrays layout of one precision with 12 (two rows; the third rebuilt as  */
/* the conjugate cross product, SU(3) only) or 18 reals per link (every    */
/* precision supports both).  A spinor                                      */
/* handle holds one subset (even, odd or full) of nrhs fields in one       */
/* precision; F16/BF16 spinors carry one FP32 scale per site and rhs.      */
/* ---------------------------------------------------------------------- */
typedef struct wilson_gauge_s wilson_gauge;
typedef struct wilson_spinor_s wilson_spinor;

/* The link field U_{x,mu} of Eq. 3 (Sec. 5: 18 words per link, of which
 * the 12-real form stores 12).  canon: 4V links, canonical complex128, host
 * or device memory; prec: wilson_prec; recon: 12 or 18.  The handle owns
 * its device copy; canon may be freed on return (the call synchronises the
 * stream).  WILSON_ERR_ARG for invalid arguments, WILSON_ERR_OOM when the
 * device copy cannot be allocated. */
int wilson_gauge_create(wilson_gauge** g, const double* canon, const wilson_lattice* L, int prec,
                        int recon, void* stream);
/* Frees the handle's device memory; NULL is accepted. */
int wilson_gauge_destroy(wilson_gauge* g);

/* Storage for nrhs spinor fields psi_x of Eq. 3 (Sec. 5: 24 words per
 * site) on one subset (wilson_subset: even, odd or full lattice), in one
 * precision.  The contents are undefined until imported or written by an
 * operator.  WILSON_ERR_ARG for invalid arguments, WILSON_ERR_OOM when the
 * fields cannot be allocated. */
int wilson_spinor_create(wilson_spinor** s, const wilson_lattice* L, int subset, int nrhs, int prec);
/* Frees the handle's device memory; NULL is accepted. */
int wilson_spinor_destroy(wilson_spinor* s);
/* Bytes of device memory the handle holds. */
long long wilson_spinor_bytes(const wilson_spinor* s);

/* Conversion between the canonical spinor layout and the handle's storage
 * (the fields psi of Eq. 3, Sec. 5).  F16/BF16 storage quantises each
 * site to max|component| * q with |q| <= 1 on import.
 * canon: nrhs fields back to back, each V (full) or V/2 (half) canonical
 * spinors; host or device memory.  Device and page-locked (pinned) host
 * memory: asynchronous and ordered on the stream, like cudaMemcpyAsync (an
 * import's source must stay unchanged, and an export's destination unread,
 * until the stream has been synchronized); host copies run on the library's
 * own copy streams through its workspace, so that they overlap kernels
 * already queued on the stream.  Pageable host memory: staged, and the call
 * returns when it is done. */
int wilson_spinor_import(wilson_spinor* s, const double* canon, void* stream);
int wilson_spinor_export(const wilson_spinor* s, double* canon, void* stream);

/* Apply an operator to prepared fields of matching lattice and precision
 * (links stored in the spinors' precision, 12 or 18 reals): the hopping
 * term of Eq. 3 (Sec. 5) and the operators built from it.
 *   HOP:  full -> full (D_h) or parity 1-p -> parity p (D_{p,1-p})
 *   M:    full -> full
 *   SCHUR, SCHUR_DAG: parity p -> parity p (the intermediate field of the
 *         other parity is allocated once and kept with the gauge handle)
 * All nrhs fields are applied in one launch per hop, right-hand sides of a
 * site tile back to back so that they share the tile's link loads; out must
 * not be in.  Asynchronous and ordered on the stream.  Outside stream capture
 * each hop is launched with programmatic dependent launch: its blocks may be
 * scheduled while the previous kernel on the stream drains, but they touch
 * no memory before that kernel has completed, so stream order holds for
 * every earlier operation.  The environment variable WILSON_PDL=0 launches
 * plainly. */
int wilson_dslash_h(wilson_spinor* out, const wilson_gauge* g, const wilson_spinor* in, double kappa,
                    int op, void* stream);

/* ---------------------------------------------------------------------- */
/* Domain decomposition along t (Sec. 5: the lattice split over SPEs and   */
/* Cell nodes, whose external communication T_ext ships projected half     */
/* spinors, 12 reals per boundary site and face; Table 1).  A sub-lattice  */
/* of Lr consecutive t-slices (Lr even, so local parity = global parity)   */
/* is an ordinary handle lattice {Lx, Ly, Lz, Lr} with the lattice's       */
/* boundary phases; its half fields are the contiguous global half-site    */
/* range [t0 Vs/2, (t0 + Lr) Vs/2), Vs = Lx Ly Lz.  One application of      */
/* D_{p,1-p} on every sub-lattice is: wilson_dd_pack on each, move each     */
/* send_prev buffer to the previous sub-lattice's recv_next and each        */
/* send_next buffer to the next one's recv_prev (cyclically; a device copy  */
/* on one GPU, NCCL send/recv or a peer copy between GPUs), then            */
/* wilson_dd_hop on each.  F64 or F32 fields, one right-hand side.          */
/* ---------------------------------------------------------------------- */

/* Bytes of one face buffer of a sub-lattice (96 B per face site for F64,
 * 48 B for F32, over Vs/2 face sites rounded up to 64); -1 on invalid
 * arguments (wilson_last_error() says why). */
long long wilson_dd_halo_bytes(const wilson_lattice* L, int prec);

/* Fills the two face buffers (device memory, wilson_dd_halo_bytes each)
 * from the input field in (parity 1-p) of this sub-lattice:
 *   send_prev: (1 - g_4) psi on the first t-slice (the previous sub-lattice's
 *              forward t-hop), or (1 + g_4) psi with dagger = 1;
 *   send_next: U^dag_{y,4} (1 + g_4) psi(y) on the last t-slice (the next
 *              sub-lattice's backward t-hop; the link lives here), or with
 *              (1 - g_4) for dagger = 1.
 * dagger = 1 applies the hop of g_5 D g_5.  Asynchronous on the stream. */
int wilson_dd_pack(void* send_prev, void* send_next, const wilson_gauge* g, const wilson_spinor* in,
                   int dagger, void* stream);

/* Parts of the sub-lattice hop (the part argument of wilson_dd_hop). */
typedef enum {
    WILSON_DD_ALL = 0,       /* every site                                                  */
    WILSON_DD_INTERIOR = 1,  /* t-slices 1 .. Lr-2: needs no face buffer, so it can run while  */
                             /* the buffers are still being exchanged                          */
    WILSON_DD_FACES = 2      /* t-slices 0 and Lr-1 (the sites whose t-hops cross a face)    */
} wilson_dd_part;

/* out (parity p) = D_{p,1-p} in on this sub-lattice (or on one part of its
 * sites: INTERIOR and FACES together are ALL), the t-hops across its two
 * faces taken from recv_next (the next sub-lattice's send_prev) and
 * recv_prev (the previous one's send_next); INTERIOR reads neither (they
 * may be NULL).  t_first / t_last: the sub-lattice holds the lattice's
 * first / last t-slice, so that the boundary phase of t (g's lattice)
 * applies on that face.  A single sub-lattice (t_first = t_last = 1, its
 * own buffers) is the undecomposed operator.  The first ALL call of a
 * lattice times its launch configurations (synchronising once); the
 * parts use that choice.  Asynchronous on the stream. */
int wilson_dd_hop(wilson_spinor* out, const wilson_gauge* g, const wilson_spinor* in, const void* recv_next,
                  const void* recv_prev, int dagger, int t_first, int t_last, int part, void* stream);

/* ---------------------------------------------------------------------- */
/* No-allocation variant (the paper has no counterpart; this is a service  */
/* of the library).  For callers that cannot let a library allocate device */
/* memory: hosts whose memory manager owns the whole device (a framework's */
/* caching allocator, a fixed arena sized to the card), and loops that     */
/* must never block in an allocator or see a pool grow.                    */
/* ---------------------------------------------------------------------- */
#define WILSON_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Same arguments, result and precision (FP64, 18-real links) as
 * wilson_dslash_eo, but the packed fields live in one fixed device array of
 * WILSON_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading the library
 * holds until exit; nothing is allocated or freed.  Fits lattices with
 * V/2 up to about 19,000 sites (8^4, 12^4, 8^3 x 32, 12^3 x 22); larger ones
 * return WILSON_ERR_ARG before any work.  The first call in a CUDA context
 * resolves the array's device address in that context (cudaGetSymbolAddress)
 * and caches it under the context's unique ID.  The call never times launch
 * configurations: it uses the one an earlier wilson_dslash_eo call on the
 * same lattice and operator chose (or the WILSON_TUNE_CACHE file holds), else
 * a fixed default; it neither allocates nor synchronises and is
 * asynchronous on the stream.  All calls on a device share the array (it
 * keeps the last call's contents; nothing in it needs clearing): calls whose
 * GPU work overlaps race on it and must be serialised by the caller. */
int wilson_dslash_eo_noalloc(double* out, const double* gauge, const double* in, const wilson_lattice* L,
                             int out_parity, double kappa, int op, void* stream);

/* ---------------------------------------------------------------------- */
/* Measurement: the device's peak FP rate (Sec. 3: T_peak is the time the  */
/* FP operations take at the machine's peak FP throughput, and the         */
/* efficiency of Eq. 2's model is T_peak over the execution time).         */
/* ---------------------------------------------------------------------- */
typedef enum {
    WILSON_PROBE_FMA_F64 = 0,    /* FP64 fused multiply-add                        */
    WILSON_PROBE_FMA_F32 = 1,    /* FP32 fused multiply-add                        */
    WILSON_PROBE_FMA_F32X2 = 2   /* paired FP32 fused multiply-add (two lanes each) */
} wilson_probe_kind;

/* Measures the current device's peak rate of one kind of FMA: a kernel of
 * independent FMA chains on every SM at full occupancy, timed with CUDA
 * events on the stream (best of three launches of about 50-100 ms each).
 * *gflops: 2 flops per FMA (per lane).  Allocates a small result buffer and
 * synchronises the stream.  WILSON_ERR_ARG for an unknown kind. */
int wilson_probe_fma_peak(int kind, double* gflops, void* stream);

/* The memory-access pattern of the even-odd hop with the arithmetic taken
 * out (Sec. 5, after Table 1: the paper benchmarked the access pattern of
 * Eq. 3 and compared its time with the model's memory time T_mem).  A kernel
 * makes exactly the DRAM accesses of wilson_dslash_h(out, g, in, 0,
 * WILSON_OP_HOP): for each site of out's parity p it reads the eight
 * neighbours' spinors of in (parity 1 - p, periodic wrap) and the eight links,
 * and writes the site's rows of out; each loaded word is folded into an
 * integer checksum, which is stored in place of the spinor, so out's contents
 * afterwards are NOT a spinor field.  One RHS; in and out of the gauge's
 * lattice and precision, of opposite parities.  Times reps back-to-back
 * launches at each block size of 64, 128 and 256 threads and each of four
 * register budgets with CUDA events on the stream (after three warm-up
 * launches) and returns the best mean time per launch in *seconds.  Synchronises the stream; allocates nothing.
 * WILSON_ERR_ARG for mismatched handles or reps outside [1, 100000]. */
int wilson_probe_hop_access(wilson_spinor* out, const wilson_gauge* g, const wilson_spinor* in, int reps,
                            double* seconds, void* stream);

/* Failure detection: *count = how many bounded waits in the library's
 * kernels have given up since the library was loaded in this process (the
 * t-slab hop waits for its staged slices with an iteration limit of about a
 * second; a wait that runs out stores NaN at its site, ends that block's
 * sweep and returns, so a solver reports WILSON_ERR_NUMERIC).  A healthy run
 * reads 0.  Synchronises the stream. */
int wilson_stage_timeouts(unsigned long long* count, void* stream);

/* ---------------------------------------------------------------------- */
/* Errors and version                                                      */
/* ---------------------------------------------------------------------- */
const char* wilson_last_error(void);
int wilson_version(void);   /* major*10000 + minor*100 + patch */

#ifdef __cplusplus
}
#endif
#endif /* WILSON_GB300_H */
