/*
 * lqcd.h -- C ABI of the GB300 (sm_103a) staggered-fermion hot path.
 *
 * Operations (arXiv:1701.00426, Bonati et al.):
 *   D_eo / D_oe   the even/odd blocks of the staggered operator,
 *                 M = m I + [[0, D_oe], [D_eo, 0]], D_oe^dag = -D_eo
 *                 (Sec. 2.2, Eq. diracblock);
 *   A             the even-site normal operator m^2 - D_eo D_oe
 *                 (Sec. 2.2, Eq. lineqeo);
 *   multi-shift   (A + sigma_i) x_i = b for all poles sigma_i at once, one
 *                 operator application per iteration (Sec. 2.2, Eq. shlineq).
 *
 * Conventions shared by every call:
 *   - Lattice sides N0..N3 are even and >= 2 (Sec. 4.1: all sides even).
 *     Time is direction 3.
 *   - Operator normalisation, staggered phases and boundary:
 *       (D psi)(n) = 1/2 sum_mu [ s_mu(n) U_mu(n) psi(n+mu)
 *                                 - s_mu(n-mu) U_mu(n-mu)^dag psi(n-mu) ],
 *       s_mu(n) = eta_mu(n) * (-1 if mu == 3 and n3 == N3-1 else 1),
 *       eta_0 = 1, eta_mu(n) = (-1)^(n0 + ... + n_{mu-1}).
 *     The phases are computed from coordinates; links are stored raw.
 *   - Host gauge field ("canonical links"): complex128 interleaved (re, im),
 *     [4][V][3][3], U_mu(x)[row][col] at lexicographic index
 *     lex = x0 + N0 (x1 + N1 (x2 + N2 x3)).  Links must be SU(3) (unitary,
 *     det 1) when 12-real storage is used; every entry must satisfy
 *     |re|, |im| < 2^60.
 *   - Host half-lattice field ("canonical spinor"): complex128 interleaved,
 *     [Vh][3] (Vh = V/2) on the sites of one parity, site order given by the
 *     half index idxh = lex / 2 (Sec. 4.1, Eq. lexicographic_eo).
 *   - Device half-lattice field ("device spinor"): the three colour
 *     components stored as three consecutive arrays (structure of arrays,
 *     like the paper's vec3_soa): element (idxh, c) at offset c*Vh + idxh.
 *     The element type is complex128 (double2) for FP64 calls and complex64
 *     (float2) for FP32 / FP16 calls.  Device buffers are allocated and owned
 *     by the caller and must stay valid until the call's stream has finished.
 *   - Host buffers are always owned by the caller; the library copies.
 *   - Every call returns an lqcd_status; nothing throws across this ABI.  On
 *     failure lqcd_last_error() describes the cause (thread-local string).
 *   - A context is not thread-safe: one thread at a time per context.
 *   - A context lives on the device that was current at lqcd_create.  Every
 *     call that takes a context makes that device current for the call and
 *     restores the calling thread's current device before it returns, so a
 *     context may be driven from any thread.  The contexts of one packed
 *     solve must share a device.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lqcd_status {
    LQCD_OK = 0,
    LQCD_EINVAL = -1,     /* bad argument (sizes, pointers, odd sides, ...) */
    LQCD_ENOMEM = -2,     /* device or host allocation failed, or over budget */
    LQCD_ENOCONV = -3,    /* max_iter reached; best x and info still written */
    LQCD_ENAN = -4,       /* NaN/Inf met in a reduction */
    LQCD_EBUSY = -5,      /* server queue full */
    LQCD_ENOTREADY = -6,  /* request not finished yet */
    LQCD_ETIMEOUT = -7,   /* a bounded device wait gave up */
    LQCD_ECUDA = -8,      /* CUDA runtime error */
    LQCD_ESTATE = -9      /* call out of order (e.g. no links uploaded) */
} lqcd_status;

/* Arithmetic of a D_eo application or of a solver's inner iterations. */
typedef enum lqcd_prec {
    LQCD_PREC_FP64 = 0,         /* FP64 storage; products/sums in double-float
                                   on the FP32 pipes, result within 1e-13 */
    LQCD_PREC_FP32 = 1,         /* FP32 links and spinors, FP32 arithmetic */
    LQCD_PREC_FP16 = 2,         /* FP16 links, FP32 spinors and arithmetic */
    LQCD_PREC_FP64_NATIVE = 3   /* IEEE FP64 storage and native DFMA */
} lqcd_prec;

typedef struct lqcd_ctx lqcd_ctx;

/* Solver options. */
typedef struct lqcd_opts {
    int prec;              /* lqcd_prec of the inner iterations (default FP64) */
    int recon;             /* link storage for FP32/FP16 hops: 18 or 12 reals
                              (12: third row rebuilt as conj(r0 x r1), Sec. 2.3) */
    double delta_reliable; /* mixed precision: reliable update when the low-
                              precision residual falls below delta times the
                              residual at the last update (default 0.1) */
    int max_iter;          /* iteration cap per solve (default 20000) */
    int check_every;       /* iterations between host convergence checks (default 32) */
    double fp64_until;     /* mixed precision with FP32 links: the multi-shift
                              iteration runs in FP64 (double-float) until
                              ||r|| <= fp64_until * ||b||, then in FP32 with
                              reliable updates (0 = FP32 from the start; must
                              be in [0, 1); default 3e-4).  Rounding of the FP32
                              phase enters the shifted systems in proportion to
                              the residual at the switch, so a later switch
                              leaves less for the per-shift refinement.
                              Ignored by FP64 and FP16 solves. */
    int staged;            /* FP64 (double-float) D_eo kernels of the solver
                              and of lqcd_deo_apply: 1 = links streamed into
                              shared memory by bulk asynchronous copies
                              (default; needs a second, tile-ordered copy of
                              the FP64 links, 2 x 1152 B per even site),
                              0 = per-thread loads from the structure-of-
                              arrays links only.  Both give bitwise
                              identical results.  Takes effect at the next
                              lqcd_links_upload (the staged copy is built
                              there) and at the next solve. */
    int pdl;               /* 1 = the kernels of consecutive solver iterations
                              are launched with programmatic dependent launch:
                              a kernel starts, and streams what does not
                              depend on its predecessor, while that kernel
                              drains; 0 = plain stream order (default: on a
                              32^4 FP64 solve PDL measured 1 % slower).  Both
                              give bitwise identical results. */
} lqcd_opts;

#define LQCD_MAX_SHIFTS 32

/* Per-solve report. */
typedef struct lqcd_solve_info {
    int iters;                        /* iterations of the (outer) solve */
    int n_shift;
    int reliable_updates;             /* mixed precision: FP64 residual refreshes */
    int refine_iters;                 /* iterations spent in per-shift refinement */
    int shift_iters[LQCD_MAX_SHIFTS]; /* iteration at which each shift stopped */
    double true_resid[LQCD_MAX_SHIFTS]; /* ||(A+sigma_i) x_i - b|| / ||b|| in FP64 */
    double secs;                      /* wall time of the call */
    double bytes_moved;               /* algorithmic device bytes of the solve */
    int status;                       /* lqcd_status of the solve */
    int kernel_launches;              /* library kernels launched by the call */
} lqcd_solve_info;

/* Fill *opts with the defaults listed above. */
void lqcd_default_opts(lqcd_opts *opts);

/* Last error message of the calling thread ("" if none). */
const char *lqcd_last_error(void);

/* Host-side fault injection for tests of the error paths: the k-th device
 * allocation from now (k >= 1) fails as an out-of-memory cudaMalloc would,
 * and the call that made it returns LQCD_ENOMEM; k <= 0 disarms.  Process
 * wide.  A failed lqcd_links_upload leaves the context without links
 * (LQCD_ESTATE until the next successful upload). */
void lqcd_inject_alloc_failure(long k);

/* Bounds-checked builds (liblqcd_checked.so, compiled with
 * -DLQCD_CHECK_BOUNDS): every neighbour and link index a kernel computes is
 * compared with its array extent; an index out of range is replaced by an
 * in-range one and recorded.  This call synchronises the device, writes the
 * OR of the recorded error bits since the last call to *word (0: no index
 * was ever out of range) and clears them.  In the default build it writes 0
 * and returns LQCD_ESTATE. */
int lqcd_bounds_errors(unsigned *word);

/* Measured FMA issue rates of the current device, for rooflines of the
 * arithmetic-bound kernels: every thread of 8 blocks per SM runs 8
 * independent FMA chains (a = a m + c); *fp64_fma_per_s and *fp32_fma_per_s
 * receive the best of five timed launches (CUDA events), in FMA per second
 * (one FMA = 2 flop).  Synchronous, on the default stream. */
int lqcd_measure_fma_rates(double *fp64_fma_per_s, double *fp32_fma_per_s);

/* ABI version (major*10000 + minor*100 + patch). */
int lqcd_version(void);

/* ---------------------------------------------------------------- context */

/* Create a context for an N0 x N1 x N2 x N3 lattice on the current CUDA
 * device.  dims: 4 even sides >= 2 (Sec. 4.1); opts may be NULL (defaults).
 * The context owns its CUDA stream and every device allocation it makes.
 * Returns LQCD_EINVAL for odd/small sides, LQCD_ECUDA / LQCD_ENOMEM on CUDA
 * failures. */
int lqcd_create(const int dims[4], const lqcd_opts *opts, lqcd_ctx **ctx);

/* Free every device and host resource of ctx (NULL is ignored). */
void lqcd_destroy(lqcd_ctx *ctx);

/* Replace the solver options of ctx (validated; LQCD_EINVAL if invalid). */
int lqcd_set_opts(lqcd_ctx *ctx, const lqcd_opts *opts);

/* Device bytes held by ctx (links, workspaces). */
size_t lqcd_device_bytes(const lqcd_ctx *ctx);

/* ------------------------------------------------------------------ links */

/* Upload a gauge field in the canonical host layout (n_doubles must equal
 * 4*V*18).  The library copies it and derives every device storage format
 * (FP64 18-real, FP32 18/12-real, FP16 12-real) on the device; host and
 * device copies of the stored links only move at this call, as in the
 * paper's update-device step (Sec. 4.1).  Synchronous.  LQCD_EINVAL for a
 * wrong size or an entry out of range. */
int lqcd_links_upload(lqcd_ctx *ctx, const double *links, size_t n_doubles);

/* Copy the FP64 links back to the host in the canonical layout. */
int lqcd_links_download(lqcd_ctx *ctx, double *links, size_t n_doubles);

/* ------------------------------------------------------------------- D_eo */

/* out = D_eo in (out_parity 0: odd input, even output) or out = D_oe in
 * (out_parity 1: even input, odd output), Eq. (diracblock), in FP64.
 * where = 0: in/out are host canonical spinors ([Vh][3] complex128);
 *            the call is synchronous.
 * where = 1: in/out are device spinors (complex128 structure of arrays);
 *            the call is asynchronous on `stream` (cudaStream_t, NULL = the
 *            context's stream).
 * in and out must not overlap.  LQCD_ESTATE before lqcd_links_upload. */
int lqcd_deo_apply(lqcd_ctx *ctx, int out_parity, const void *in, void *out,
                   int where, void *stream);

/* Same operation as lqcd_deo_apply with host buffers (where = 0), for
 * callers that cannot allocate device memory -- for example a process whose
 * device memory is handed out by another framework's pool allocator, or a
 * loop that cannot pay for the device-wide synchronisation of cudaMalloc and
 * cudaFree.  The paper has no counterpart of this call.
 * It allocates nothing: the host input and output are staged through a
 * fixed array inside the library (a device global of 3 x 3 x 131072
 * complex128 = 18.9 MB), which every device that loads the library holds
 * until the process exits.  in / out: host canonical spinors ([Vh][3]
 * complex128), as for lqcd_deo_apply.  Lattices with V/2 > 131072 sites are
 * rejected with LQCD_EINVAL.  The first call in a CUDA context of a device
 * looks up the array's device address (with the context's device current)
 * and keeps it with that CUDA context's identifier; after a device reset the
 * next call looks it up again.  Make the first call before capturing work on
 * any stream.  Every call uses the same array and leaves its contents
 * behind, so calls that overlap on the GPU (from several threads, contexts
 * or streams at once) race.  Synchronous, on the context's stream. */
int lqcd_deo_apply_host_noalloc(lqcd_ctx *ctx, int out_parity, const double *in, double *out);

/* Same operator in a chosen arithmetic on device spinors (asynchronous):
 *   prec LQCD_PREC_FP64: complex128 spinors, recon 18 or 12 (12: the first
 *     two rows of each link are streamed, 96 of 144 bytes, and the third row
 *     is rebuilt in double-float arithmetic, Sec. 2.3; within 1e-13 for
 *     SU(3) links);
 *   prec LQCD_PREC_FP64_NATIVE: complex128 spinors, recon 18;
 *   prec LQCD_PREC_FP32: complex64 spinors, recon 18 or 12;
 *   prec LQCD_PREC_FP16: complex64 spinors, FP16 links, recon 12. */
int lqcd_deo_apply_ex(lqcd_ctx *ctx, int out_parity, int prec, int recon,
                      const void *in, void *out, void *stream);

/* D_eo / D_oe with FP16 links (12 reals, Sec. 2.3) and FP16 spinors with a
 * per-site FP32 norm, FP32 arithmetic (the half-precision storage variant
 * with block-scaled spinors; 224 algorithmic bytes per output site).  Device
 * spinors: `in` / `out` are half2 [3][Vh] (re, im per colour, structure of
 * arrays as the other device spinors), `in_norm` / `out_norm` float [Vh]; the
 * value of colour c at half index k is norm[k] * half2[c][k].  Each output
 * site's norm is the largest |re|, |im| of its three result colours (0 for a
 * zero site) and its halves are the result over that norm, rounded to
 * nearest.  Relative error of a few 2^-11 (links, inputs and outputs each
 * rounded to FP16).  Asynchronous on `stream` (NULL = the context's stream).
 * in and out (and their norms) must not overlap. */
int lqcd_deo_apply_h16(lqcd_ctx *ctx, int out_parity, const void *in, const float *in_norm, void *out,
                       float *out_norm, void *stream);

/* Environment variables read by the autotuners:
 *   LQCD_TUNE_CACHE=<file>  the stand-alone D_eo's launch choices are read
 *                           from and appended to this file (lines
 *                           "deo2 v<variant> <N0>x<N1>x<N2>x<N3> <code>"),
 *                           so that later processes skip the timing, or a
 *                           test fixes a variant;
 *   LQCD_MRHS_R=<R>         the multi-RHS D_eo uses R fields per thread
 *                           (1, 2, 4, 8 or 16, when R divides n_rhs) instead
 *                           of timing the choices;
 *   LQCD_PERSIST_REDUCTIONS=0  the solver iterations compute r -= alpha q,
 *                           ||r||^2 (every precision) and, in FP32 and FP16,
 *                           q = A p, <p, q> with one block per tile instead
 *                           of a grid of resident blocks that walk the tiles
 *                           (read once per process and device).
 * Every choice gives results within the documented tolerances; the
 * multi-RHS choices and the two forms of the reductions give identical
 * bits. */

/* Launch configuration the autotuner chose for lqcd_deo_apply_ex(prec,
 * recon) on this context's lattice (the first such call times the candidates,
 * each after emptying L2, and keeps the fastest for the process): *code =
 * kind * 1024 + threads per block, kind 0 = one thread per site, 1 / 2 / 4 =
 * 2 / 4 / 8 threads per site (the directions, or for 8 the half-hops, split
 * over adjacent lanes), 3 = the staged persistent FP64 kernel, 5 = FP32 /
 * FP16 with the direction loop unrolled; 0 before the first call.  LQCD_EINVAL for a (prec, recon) pair without a kernel. */
int lqcd_deo_tuned_config(const lqcd_ctx *ctx, int prec, int recon, int *code);

/* Multi-right-hand-side D_eo/D_oe in FP32: each link is loaded once for all
 * n_rhs (1..16) fields.  Device layout of in/out: complex64 [3][Vh][n_rhs]
 * (colour-major, then site, right-hand side fastest).  recon 18 or 12.
 * With in and out 16-byte aligned, the kernel may read and write two fields
 * per access (the fields per thread are picked by timing on the first call);
 * any alignment of complex64 is accepted.  Asynchronous on `stream`. */
int lqcd_deo_apply_mrhs(lqcd_ctx *ctx, int out_parity, int n_rhs, int recon,
                        const void *in, void *out, void *stream);

/* Batch layouts of lqcd_deo_apply_mrhs_layout. */
#define LQCD_MRHS_SITE_MAJOR 0   /* complex64 [3][Vh][n_rhs]: the fields of a site contiguous */
#define LQCD_MRHS_FIELD_MAJOR 1  /* complex64 [3][n_rhs][Vh]: the sites of a field contiguous */

/* lqcd_deo_apply_mrhs with the batch layout chosen by the caller
 * (LQCD_MRHS_SITE_MAJOR is lqcd_deo_apply_mrhs).  In the field-major layout
 * neighbouring threads read neighbouring sites of one field, so every
 * spinor access is a contiguous run across the warp; each thread still
 * applies a link it loads once to several fields.  Same bits as the
 * single-field operator in either layout.  LQCD_EINVAL for another layout
 * value.  Asynchronous on `stream`. */
int lqcd_deo_apply_mrhs_layout(lqcd_ctx *ctx, int out_parity, int n_rhs, int recon, int layout,
                               const void *in, void *out, void *stream);

/* ----------------------------------------------------------------- solver */

/* Multi-shift CG for (A + shifts[i]) x_i = b, A = m^2 - D_eo D_oe on even
 * sites (Eqs. lineqeo, shlineq).  b: host canonical spinor ([Vh][3]
 * complex128); x: host array [n_shift][Vh][3] complex128 written by the
 * call.  shifts >= 0 in any order, 1 <= n_shift <= LQCD_MAX_SHIFTS;
 * tol: target of the FP64 true residual ||(A+sigma_i)x_i - b||/||b|| for
 * every shift (> 0).  The arithmetic of the inner iterations follows the
 * context's opts.prec; the true residual and the solution are always FP64.
 * info may be NULL.  Synchronous.  LQCD_ENOCONV when max_iter is reached
 * (x and info still hold the best result). */
int lqcd_mscg_solve(lqcd_ctx *ctx, double mass, const double *shifts, int n_shift,
                    double tol, const double *b, double *x, lqcd_solve_info *info);

/* Same on device spinors: b is a complex128 device spinor, x a device array
 * of n_shift complex128 device spinors (shift-major).  Runs on `stream`
 * (NULL = context stream) and returns when the solve has finished. */
int lqcd_mscg_solve_dev(lqcd_ctx *ctx, double mass, const double *shifts, int n_shift,
                        double tol, const void *b, void *x, lqcd_solve_info *info,
                        void *stream);

/* Rational function of A applied to a source, the step of the RHMC that
 * replaces the root of the fermion matrix (Sec. 2.2, Eq. rooting, with the
 * poles of Eq. shlineq; heatbath and actions of Algorithm 1, steps 3, 4, 6):
 *   y = a0 b + sum_i a[i] (A + shifts[i])^{-1} b,   A = m^2 - D_eo D_oe,
 * and, if action != NULL, *action = Re <b, y> (the pseudofermion action
 * b^dag r(A) b).  a[i]: real coefficient of the pole shifts[i] (n_shift of
 * each, 1..LQCD_MAX_SHIFTS; shifts >= 0; a0 and a[i] finite, any sign).
 * One multi-shift solve to the FP64 true residual tol for every pole (as
 * lqcd_mscg_solve; the per-pole residuals are in info), then a device
 * epilogue forms y and the action in FP64 without moving the shifted
 * solutions off the GPU; the error of y is at most
 * tol ||b|| sum_i |a[i]| / (lambda_min + shifts[i]).  The shifted solutions
 * live in a device scratch array of the context (n_shift x 48 B per even
 * site), kept for later calls.  b, y: host canonical spinors ([Vh][3]
 * complex128).  Synchronous.  LQCD_ENOCONV at max_iter (y, action and info
 * still written); LQCD_EINVAL for a non-finite coefficient. */
int lqcd_rational_apply(lqcd_ctx *ctx, double mass, double a0, const double *a,
                        const double *shifts, int n_shift, double tol, const double *b,
                        double *y, double *action, lqcd_solve_info *info);

/* Same on device spinors (complex128 structure of arrays, as
 * lqcd_mscg_solve_dev).  b is read and y written on the context's stream
 * after `stream` (NULL = context stream) has been synchronised; returns when
 * y and the action are complete. */
int lqcd_rational_apply_dev(lqcd_ctx *ctx, double mass, double a0, const double *a,
                            const double *shifts, int n_shift, double tol, const void *b,
                            void *y, double *action, lqcd_solve_info *info, void *stream);

/* Batched single-shift CG for n_rhs sources sharing the gauge field:
 * (A + sigma) x_k = b_k, k < n_rhs (1..16).  Inner iterations use the FP32
 * multi-right-hand-side D_eo (each link loaded once per application for all
 * sources) with FP64 reliable updates; the solution and the true residual are
 * FP64.  b: host [n_rhs][Vh][3] complex128, x: same shape.  info: array of
 * n_rhs reports (or NULL).  Synchronous. */
int lqcd_cg_solve_mrhs(lqcd_ctx *ctx, double mass, double sigma, int n_rhs, double tol,
                       const double *b, double *x, lqcd_solve_info *info);

/* Packed multi-lattice solve: one multi-shift solve per context, all
 * contexts (different lattice sizes allowed) advanced together, every
 * kernel of an iteration launched once over a work list spanning all
 * lattices.  Arguments are arrays of length n (one entry per context; x[i]
 * is the host output of context i).  Each result is identical to the one
 * the context would get alone.  Synchronous. */
int lqcd_mscg_solve_packed(lqcd_ctx *const *ctxs, int n, const double *mass,
                           const double *const *shifts, const int *n_shift,
                           const double *tol, const double *const *b,
                           double *const *x, lqcd_solve_info *info);

/* Diagnostics: run up to `iters` iterations of the multi-shift iteration of
 * lqcd_mscg_solve (same kernels, same precision as opts.prec, same stopping
 * rule for tol, so shifts drop out as in a solve) on the device source b
 * (complex128 device spinor), launching the four kernels of an iteration
 * one by one with CUDA events between them on the context's stream.
 * ms_out[0..3] receive the average device time (ms) over the iterations
 * that ran of
 *   0: t = D_oe p            1: q = (m^2+sigma) p - D_eo t and <p,q>
 *   2: r -= alpha q, ||r||^2  3: x_i += alpha_i p_i, p_i = zeta_i r + beta_i p_i
 * and *n_active_avg the mean number of shifts updated by kernel 3.
 * Synchronous. */
int lqcd_profile_iteration(lqcd_ctx *ctx, double mass, const double *shifts, int n_shift,
                           double tol, const void *b, int iters, double ms_out[4],
                           double *n_active_avg);

/* ------------------------------------------------- gauge molecular dynamics */

/* The gauge part of the molecular dynamics step (Sec. 4.2, Algorithm 2: the
 * gauge cycle; Table md-norm), for the tree-level Symanzik improved action
 * (Sec. 2.1), read as
 *   S_g = -(beta/3) sum_x [ c0 sum_{mu<nu} Re Tr P_{mu nu}(x)
 *                         + c1 sum_{mu!=nu} Re Tr R_{mu nu}(x) ],
 *   c0 = 5/3, c1 = -1/12, P the plaquette, R the 2x1 rectangle (two links
 *   along mu), every loop once;
 * momenta H_mu(x) Hermitian and traceless, links moving as U -> exp(i e H) U,
 * kinetic term (1/2) sum Tr H^2, so the force F_mu(x) (Hermitian, traceless)
 * is the derivative of S_g along those motions and the momenta move as
 * H -> H - e F.  The context keeps the momenta on the device.  prec:
 *   LQCD_PREC_FP64: FP64 links and momenta, SU(3) products in double-float
 *     arithmetic on the FP32 pipes (~48-bit products; GB300 issues FP32 64
 *     times faster than FP64);
 *   LQCD_PREC_FP64_NATIVE: the same with native FP64 (DFMA) arithmetic;
 *   LQCD_PREC_FP32: FP32 arithmetic on FP32 copies of links and momenta
 *     (Algorithm 1, step 5: "possibly in single precision"); the copies are
 *     made when the precision changes, and the FP32 links become the FP64
 *     links again before any D_eo or solve.
 * All calls are synchronous. */

/* Momenta in the canonical host layout [4][V][3][3] complex128 (n_doubles =
 * 4*V*18), Hermitian and traceless to 1e-12 relative (else LQCD_EINVAL). */
int lqcd_mom_upload(lqcd_ctx *ctx, const double *H, size_t n_doubles);
int lqcd_mom_download(lqcd_ctx *ctx, double *H, size_t n_doubles);

/* H <- H - eps F(U) on every link. */
int lqcd_gauge_mom_update(lqcd_ctx *ctx, int prec, double beta, double eps);

/* U <- exp(i eps H) U on every link (the exponential of the traceless
 * Hermitian momentum to rounding). */
int lqcd_gauge_link_update(lqcd_ctx *ctx, int prec, double eps);

/* n_steps times: the momentum update, then the link update, each with eps
 * (the unit that Table md-norm times per site); n_steps >= 0. */
int lqcd_gauge_md_steps(lqcd_ctx *ctx, int prec, double beta, double eps, int n_steps);

/* Fermion force of the rational pseudofermion action (Sec. 2.2: Eq. rooting
 * with the rational function of Eq. shlineq; the fermion force steps of
 * Algorithm 2): S_f = phi^dag r(A) phi, r(A) = a0 + sum_i a[i] (A + shifts[i])^{-1},
 * A = m^2 - D_eo D_oe.  Solves (A + shifts[i]) x_i = phi to the FP64 true
 * residual tol for every pole (as lqcd_rational_apply), forms y_i = D_oe x_i,
 * and updates the context's momenta H <- H - eps F_f with the Hermitian
 * traceless force F_f_mu(n) = traceless part of (i s_mu(n)/2) c sum_i a_i
 * (W_i - W_i^dag), W_i = U_mu(n) y_i(n+mu) x_i(n)^dag for even n (c = +1),
 * U_mu(n) x_i(n+mu) y_i(n)^dag for odd n (c = -1), s_mu(n) the staggered
 * sign of the link with the antiperiodic time boundary: the derivative of
 * S_f along U -> exp(i e X) U is sum Tr(X F_f).  phi: host canonical even
 * spinor ([Vh][3] complex128); *action (may be NULL) receives S_f.  The
 * force is computed in native FP64 from the FP64 links; momenta must have
 * been uploaded.  While the links are stout-smeared (lqcd_stout_smear) the
 * action is that of the smeared links and the force is chained back to the
 * thin links (as lqcd_stout_force) before the update: the momenta belong to
 * the thin links.  Synchronous.  LQCD_ENOCONV at max_iter (the update is
 * still applied). */
int lqcd_fermion_force_update(lqcd_ctx *ctx, double mass, double a0, const double *a,
                              const double *shifts, int n_shift, double tol, const double *phi,
                              double eps, double *action, lqcd_solve_info *info);

/* *S = S_g(U) of the current links (sums in FP64 in a fixed order). */
int lqcd_gauge_action(lqcd_ctx *ctx, int prec, double beta, double *S);

/* *K = (1/2) sum Tr H^2 of the current momenta. */
int lqcd_mom_energy(lqcd_ctx *ctx, int prec, double *K);

/* ----------------------------------------------------------------- serving */

typedef struct lqcd_server lqcd_server;

/* Server statistics (latencies in seconds, measured submit -> finished). */
typedef struct lqcd_serve_stats {
    uint64_t submitted, completed, rejected;
    int active_slots, queued;
    size_t hbm_in_use, hbm_budget;
    double p50_latency, p99_latency, mean_latency;
    double solves_per_sec;   /* completed / (last completion - first submit) */
    uint64_t ticks;          /* packed iteration launches issued */
} lqcd_serve_stats;

/* Create a continuous-batching solve server on the current device.
 * hbm_budget_bytes caps the device memory of resident fields plus active
 * requests; max_slots caps concurrently active requests (1..64); max_queue
 * caps requests waiting for admission.  A scheduler thread owned by the
 * server admits requests when slots and memory free up and advances every
 * active request by one iteration per packed launch. */
int lqcd_serve_create(size_t hbm_budget_bytes, int max_slots, int max_queue,
                      lqcd_server **srv);

/* Register a resident gauge field (canonical host links, copied).
 * *field_id receives its handle.  LQCD_ENOMEM if it does not fit. */
int lqcd_serve_register_field(lqcd_server *srv, const int dims[4], const double *links,
                              size_t n_doubles, int *field_id);

/* Queue one multi-shift solve on a registered field (b: host canonical
 * spinor, copied at submit).  *ticket identifies it.  LQCD_EBUSY when the
 * queue is full; LQCD_ENOMEM if the request can never fit the budget. */
int lqcd_serve_submit(lqcd_server *srv, int field_id, double mass, const double *shifts,
                      int n_shift, double tol, const double *b, uint64_t *ticket);

/* Options of the requests submitted after this call, and of every field's
 * context: prec LQCD_PREC_FP64 (default) or LQCD_PREC_FP32 (mixed precision:
 * double-float iterations down to fp64_until, then FP32 iterations with FP64
 * reliable updates and per-shift refinement; recon selects the FP32 link
 * format).  A mixed request reserves its FP32 and refinement workspaces in
 * the HBM budget as well.  LQCD_EINVAL for invalid options or another prec;
 * LQCD_EBUSY while requests are queued or running.  No counterpart in the
 * paper (serving is outside its scope). */
int lqcd_serve_set_opts(lqcd_server *srv, const lqcd_opts *opts);

/* LQCD_ENOTREADY until the request has finished; then copies x
 * ([n_shift][Vh][3] complex128) and info, and forgets the ticket. */
int lqcd_serve_poll(lqcd_server *srv, uint64_t ticket, double *x, lqcd_solve_info *info);

/* Block until every submitted request has finished (timeout_s <= 0: no
 * limit); LQCD_ETIMEOUT when the limit passes first. */
int lqcd_serve_drain(lqcd_server *srv, double timeout_s);

int lqcd_serve_stats_get(lqcd_server *srv, lqcd_serve_stats *stats);

/* Stop the scheduler, free every resource.  Unpolled results are dropped. */
void lqcd_serve_destroy(lqcd_server *srv);

/* Failure-detection self-test of the bounded device waits.  Every wait of the
 * staged kernels (a consumer for a stage of links, the producer for a free
 * stage) gives up after a time limit, records the stall, and the call
 * returns LQCD_ETIMEOUT with the context still usable.  This call runs one
 * block of the staged layout whose stage is never filled, with the wait
 * limited to limit_s seconds (0 < limit_s <= 10), and returns what such a
 * stall returns: LQCD_ETIMEOUT.  No fault, no hang; the context stays
 * usable.  Synchronous. */
int lqcd_selftest_stage_wait(lqcd_ctx *ctx, double limit_s);

/* ---------------------------------------------------------------- stout smearing
 * Stout smearing of the fermion links (Sec. 2.1: stout-improved staggered
 * action, Ref. Morningstar:2003gk; Sec. 2.2: a few stout levels).  One level
 * maps every link to U' = exp(iQ) U with
 *   C_mu(x) = rho sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
 *                                 + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ],
 *   Omega = C U^dag,  Q = (i/2)(Omega^dag - Omega) - (i/6) Tr(Omega^dag - Omega).
 * Native FP64. */

/* Smear the context's links n_levels times (1..8) with weight rho >= 0.  The
 * smeared links become the links of every later D_eo, solve, rational
 * application, fermion force and lqcd_links_download; levels 0 .. n-1 (level
 * 0 = the links before smearing) stay on the device for the force chain
 * (n_levels x 1152 B per even site).  LQCD_ESTATE without links or when
 * already smeared.  Synchronous. */
int lqcd_stout_smear(lqcd_ctx *ctx, double rho, int n_levels);

/* Put the links from before lqcd_stout_smear back (no-op when not smeared).
 * The gauge MD updates (lqcd_gauge_mom_update, lqcd_gauge_link_update,
 * lqcd_gauge_md_steps) move the thin links and return LQCD_ESTATE while the
 * links are smeared.  lqcd_links_upload also ends the smearing. */
int lqcd_stout_restore(lqcd_ctx *ctx);

/* Force on the thin links from a force on the smeared links: F_smeared and
 * F_thin are host [4][V][3][3] complex128 (n_doubles = 4*V*18), Hermitian
 * and traceless (else LQCD_EINVAL), with d/de S(exp(i e X) U') = sum Tr(X F)
 * for the smeared links U'; F_thin is the same for the thin links U of the
 * smearing, chained through every level: with Sigma' = -i U'^dag F_smeared,
 * Gamma = the derivative of exp at iQ in the direction U Sigma', L its
 * traceless anti-Hermitian part, the gradient G of each link collects
 * Sigma' exp(iQ) - C^dag L and rho times the staple products that carry
 * U^dag L of the links whose C contains it, and F = traceless part of
 * (i/2)(U G - G^dag U^dag).  LQCD_ESTATE when not smeared.  Synchronous. */
int lqcd_stout_force(lqcd_ctx *ctx, const double *F_smeared, double *F_thin, size_t n_doubles);

/* ------------------------------------------------- domain decomposition
 * The lattice split into slabs of time slices over ranks, one context per
 * rank (the distribution over several GPUs that Sec. 6 names as the next
 * step).  Rank r of `world` owns global time slices [t0, t0 + nt), nt =
 * N3 / world (even, >= 2), t0 = r nt.  Its context holds an extended slab of
 * nt + 4 slices (two ghost slices on each side); a rank's field is a device
 * spinor of that slab ([3][Vh_ext] complex128, Vh_ext = N0 N1 N2 (nt + 4) / 2)
 * whose owned sites are the half-index range [lo, hi) = [2 h, (2 + nt) h),
 * h = N0 N1 N2 / 2, in the global half-index order of those slices.  The
 * hops of the owned sites read one ghost slice on each side, [lo - h, lo)
 * and [hi, hi + h): the top owned slice of rank r - 1 and the bottom owned
 * slice of rank r + 1 (periodic in the rank). */

/* Shard context of rank `rank` of `world` for the global N0 x N1 x N2 x N3
 * lattice, on the current device.  LQCD_EINVAL unless N3 / world is even and
 * >= 2.  A shard context is an ordinary context of its extended slab for
 * every other call (which then treats the slab as a periodic lattice of its
 * own); the calls below are the sharded operations. */
int lqcd_shard_create(const int dims[4], int world, int rank, const lqcd_opts *opts, lqcd_ctx **ctx);

/* info[0..5] = t0, nt, Vh_ext, h, lo, hi (see above).  LQCD_EINVAL for a
 * context that is not a shard. */
int lqcd_shard_geometry(const lqcd_ctx *ctx, long info[6]);

/* Upload the links of the rank's extended slab from the GLOBAL canonical
 * field (4*V*18 doubles, V the global volume; copied, periodic in time);
 * the time links of global slice N3 - 1 carry the antiperiodic sign.
 * Synchronous. */
int lqcd_shard_links_upload(lqcd_ctx *ctx, const double *links, size_t n_doubles);

/* out = D_eo in (out_parity 0) or D_oe in (out_parity 1) at the rank's owned
 * sites, in FP64 (double-float arithmetic, as lqcd_deo_apply), from a device
 * spinor `in` of the extended slab whose ghost slices hold the neighbours'
 * faces (lqcd_shard_exchange, or the caller's own transport).  Only the
 * owned sites of `out` are written.  Asynchronous on `stream` (NULL = the
 * context's stream). */
int lqcd_shard_deo_apply(lqcd_ctx *ctx, int out_parity, const void *in, void *out, void *stream);

/* Fill the ghost slices of every rank's field when all `world` ranks live in
 * this process: ctxs[r] is rank r (n == world), fields[r] its device spinor
 * of the extended slab.  Each face is one 2-D device copy (three colour rows)
 * into the receiving rank's own memory, ordered after all work queued so far
 * on every rank's stream and before any work queued after the call.
 * Contexts on different devices are allowed (peer copies). */
int lqcd_shard_exchange(lqcd_ctx *const *ctxs, int n, void *const *fields);

/* CG for (A + sigma) x = b, A = m^2 - D_eo D_oe (Eq. lineqeo), with the
 * sharded operator over the n = world ranks ctxs[0..n-1] of this process:
 * two face exchanges per iteration, and the FP64 reductions summed per rank
 * in a fixed block order, then over ranks in rank order, so that every rank
 * uses the same scalars.  b, x: GLOBAL host canonical even spinors ([Vh][3]
 * complex128); each rank reads and writes its owned slices.  Iterates to
 * tol / 2 and accepts an FP64 true residual <= tol (recomputed with the
 * sharded operator; up to three restarts).  info (may be NULL): iterations
 * and true_resid[0].  Synchronous.  LQCD_ENOCONV at opts.max_iter. */
int lqcd_shard_cg_solve(lqcd_ctx *const *ctxs, int n, double mass, double sigma, double tol, const double *b,
                        double *x, lqcd_solve_info *info);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
