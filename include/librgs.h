/*
 * librgs -- randomized Gram-Schmidt (RGS) and RGS-GMRES on one NVIDIA GB300 GPU.
 *
 * Method: L. Balabanov and L. Grigori, "Randomized Gram-Schmidt process with
 * application to GMRES" (arXiv 2011.05090).  Every entry point below cites the
 * section, algorithm or equation whose operation it performs.
 *
 * Conventions shared by all entry points
 *  - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *  - Array arguments are device pointers owned by the caller unless a function
 *    says otherwise; the library never frees them.  rgs_qr additionally accepts
 *    host pointers (pinned or pageable) and stages them through device memory.
 *  - Work is issued on the stream bound to the handle (rgs_create /
 *    rgs_set_stream).  Functions that return device-computed status (breakdown,
 *    convergence, timeouts) synchronise that stream before returning.
 *  - Errors are reported by return value, never by aborting; a human-readable
 *    message for the last error on a handle is available from rgs_last_error.
 *  - Workspaces (sketch tables, Householder factors, partial sketches) belong
 *    to the handle or to the object that needs them and are freed with it.
 *  - Random sketches are drawn from Philox4x32-10 (Salmon et al., SC'11) with
 *    key = (seed mod 2^32, seed div 2^32) and these counter streams:
 *      Gaussian entry (l, c): counter (c, l>>1, 0, 0); Box-Muller on the two
 *        53-bit midpoint uniforms of words (x0,x1) and (x2,x3); cosine for even
 *        l, sine for odd l; scaled by 1/sqrt(k).
 *      SRHT sign of column c: bit (c mod 128) of the words at (c>>7, 0, 0, 1).
 *      SRHT sample: the k indices c < s with the smallest (x0*2^32+x1, c) at
 *        counter (c, 0, 0, 2), in ascending order.
 */
#ifndef LIBRGS_H
#define LIBRGS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RGS_API __attribute__((visibility("default")))
#else
#define RGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RGS_OK = 0,
    RGS_ERR_INVALID_ARG = 1,     /* shape, pointer, alignment or option rejected */
    RGS_ERR_CUDA = 2,            /* a CUDA runtime call failed */
    RGS_ERR_ALLOC = 3,           /* device or host allocation failed */
    RGS_ERR_BREAKDOWN = 4,       /* r_ii <= 16 u ||p_i||: column i depends on the previous ones */
    RGS_ERR_NOT_CONVERGED = 5,   /* solver stopped at max_cycles above the tolerance; x is the last iterate */
    RGS_ERR_TIMEOUT = 6,         /* a device-side grid barrier gave up waiting */
    RGS_ERR_NONFINITE = 7,       /* NaN or Inf met in a sketched norm */
    RGS_ERR_NOT_IMPLEMENTED = 8,
    RGS_ERR_CERT_FAILED = 9,     /* rgs_certify_embedding: omega_bar >= 1, no embedding certificate */
    RGS_ERR_CALLBACK = 10        /* a caller's preconditioner callback returned nonzero */
} rgs_status;

typedef enum { RGS_F64 = 0, RGS_F32 = 1, RGS_BF16 = 2 } rgs_dtype;

typedef enum { RGS_SKETCH_GAUSSIAN = 0, RGS_SKETCH_SRHT = 1 } rgs_sketch_kind;

typedef struct rgs_context* rgs_handle;
typedef struct rgs_sketch_obj* rgs_sketch;
typedef struct rgs_arnoldi_obj* rgs_arnoldi;

/* Library handle on the current CUDA device.  stream: a cudaStream_t, or NULL
 * for the default stream.  Returns RGS_ERR_CUDA if no device is usable. */
RGS_API rgs_status rgs_create(rgs_handle* out, void* stream);
RGS_API rgs_status rgs_destroy(rgs_handle h);
RGS_API rgs_status rgs_set_stream(rgs_handle h, void* stream);
/* Clock-cycle budget of every device-side wait of the handle's kernels (grid and team barriers;
 * no counterpart in the paper).  A wait that runs past it records RGS_ERR_TIMEOUT, every CTA of
 * the launch leaves at its next barrier, later launches of the call do nothing, and the call
 * returns RGS_ERR_TIMEOUT; the next call on the handle starts afresh.  cycles <= 0 restores the
 * default of 4e9 cycles (about two seconds at GB300's clock).  A tiny budget makes the
 * timeout path run on purpose (used by the tests); the setting persists until changed. */
RGS_API rgs_status rgs_set_wait_budget(rgs_handle h, int64_t cycles);
RGS_API const char* rgs_status_string(rgs_status s);
RGS_API const char* rgs_last_error(rgs_handle h);

/* ---------------------------------------------------------------- sketches
 * Sec. 2.1: Theta (k x n) is either Gaussian with N(0, 1/k) entries or the
 * partial SRHT -- the first n columns of (1/sqrt(k)) P H_s D with s the power of
 * two n <= s < 2n, D random signs, H_s the +-1 Walsh-Hadamard matrix and P a
 * uniform sample of k rows.  Both are fully determined by (kind, n, k, seed).
 * Requires 1 <= k; SRHT requires k <= s; Gaussian stores Theta in device memory
 * (8 k n bytes).  The object holds device tables until rgs_sketch_destroy, which
 * does not use the handle (objects may be destroyed in any order). */
RGS_API rgs_status rgs_sketch_create(rgs_handle h, rgs_sketch_kind kind, int64_t n, int32_t k,
                             uint64_t seed, rgs_sketch* out);
RGS_API rgs_status rgs_sketch_destroy(rgs_sketch s);

/* Y (k x ncols, ldy >= k) = Theta X (n x ncols, ldx >= n), FP64, device pointers (host memory
 * is rejected with RGS_ERR_INVALID_ARG).  The sketch of Alg. 2 step 1 / step 4 applied to a block
 * of vectors; any number of columns (launched in groups of at most 65535). */
RGS_API rgs_status rgs_sketch_apply(rgs_handle h, rgs_sketch s, int32_t ncols, const double* X, int64_t ldx,
                            double* Y, int64_t ldy);

/* Y = Theta X exactly like rgs_sketch_apply, but without allocating device memory during the
 * call, for callers that cannot allow an allocation there: cudaMalloc synchronises the device
 * (a stall inside a latency-critical loop), and an application whose framework allocator holds
 * nearly all free device memory would see it fail.  The paper has no counterpart: this is an
 * interface variant of rgs_sketch_apply.
 *  - The partial sketches live in a fixed device array of RGS_NOALLOC_SCRATCH_BYTES (8 MiB).
 *    rgs_create loads it on the handle's device and looks up its address there, so the 8 MiB
 *    are reserved when the handle is created (the CUDA runtime may load a library's device
 *    code lazily) and stay reserved until the process exits.  Calls make no further
 *    reservation on a device that has a handle.
 *  - Requires k * ncols <= RGS_NOALLOC_SCRATCH_BYTES / 8; larger calls return
 *    RGS_ERR_INVALID_ARG (split the columns).  More than 65535 columns are processed in
 *    launches of at most 65535 columns each, one after another on the stream.
 *  - X and Y must be device pointers (host memory is rejected with RGS_ERR_INVALID_ARG) on
 *    the handle's device, which must be current.
 *  - Every call shares the array: calls whose work overlaps on the GPU (other streams or
 *    host threads) race and must be serialised by the caller.
 *  - Calls no cudaMalloc / cudaFree; work is queued on the handle's stream. */
#define RGS_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
RGS_API rgs_status rgs_sketch_apply_noalloc(rgs_handle h, rgs_sketch s, int32_t ncols, const double* X,
                                            int64_t ldx, double* Y, int64_t ldy);

/* ---------------------------------------------------------------- RGS QR
 * Alg. 2: given W (n x m, FP64) and Theta with m <= k, computes Q (n x m) and
 * the upper-triangular R (m x m, FP64, positive diagonal) with W = Q R and
 * Theta Q orthonormal.  Step 2 uses a Householder QR of S_{i-1} (Sec. 5),
 * step 3 runs in the storage precision qtype (FP64, or FP32 accumulation for
 * RGS_F32 / RGS_BF16 storage: the working precision u_crs), steps 1, 2, 4-8 in
 * a fine precision u_fine: FP64 for FP64 storage.  With FP32 / BF16 storage the
 * SRHT's Walsh-Hadamard sums and the least-squares steps 2, 5, 6 use double-float
 * arithmetic (a value is hi + lo in two FP32 words: about 2^-48 relative error
 * per operation, against 2^-24 for u_crs; GB300's FP64 rate is 1/64 of its FP32
 * rate), squared norms and every returned value stay FP64; RGS_QR_FP64_FINE makes
 * all of it FP64 in every storage mode.
 *   Q      n x m in qtype, ldq >= n.  If qscale is non-NULL, Q receives the
 *          unnormalised q'_i and qscale[i] = 1/r_ii (FP64), so the basis is
 *          Q diag(qscale) exactly (the Step 7 division is never rounded to
 *          qtype).  If qscale is NULL, Q is scaled in place at the end.
 *   R      m x m, ldr >= m (strictly lower part set to 0).
 *   S      optional (NULL): k x m, lds >= k, receives S = Theta Q (FP64).
 *   flags  RGS_QR_NO_CERTIFICATES: skip step 8; RGS_QR_TIMINGS: per-phase event timings;
 *          RGS_QR_FP64_FINE (= RGS_FP64_FINE): FP64 transform sums and least squares in every
 *          storage mode; RGS_FP64_LS: FP64 least squares, double-float transform sums;
 *          RGS_FP32_FINE: everything in FP32 (the unique-precision comparison run of Sec. 5.1);
 *          RGS_LS_RICHARDSON: step 2 by two Richardson sweeps on the normal equations.
 *   info   optional host struct: step-8 certificates and breakdown column.
 * W, Q, R, S, qscale may be all device or all host pointers.  Returns
 * RGS_ERR_BREAKDOWN (info->breakdown_col set) if some r_ii vanishes. */
#define RGS_QR_NO_CERTIFICATES 1
#define RGS_QR_TIMINGS 2         /* bit 1: time each phase with CUDA events (fills the *_ms fields) */
#define RGS_FP64_FINE 4          /* bit 2: fine precision u_fine = FP64 for every storage type: the SRHT's
                                    transform sums, the products with A (Arnoldi) and the least-squares
                                    steps 2, 5, 6 (and Givens) in FP64 (rgs_qr, rgs_arnoldi_create,
                                    rgmres_opts.flags) */
#define RGS_FP64_LS 8            /* bit 3: the sketched least-squares steps 2, 5, 6 (and the Givens
                                    rotations of GMRES) in FP64 for every storage type, while the SRHT
                                    transform sums and the products with A of FP32 / BF16 bases stay in
                                    double-float (about 2^-48, finer than FP32 accumulation) */
#define RGS_FP32_FINE 16         /* bit 4, rgs_qr only: the unique-precision setting of Sec. 5.1 (u_fine =
                                    u_crs = FP32): FP32 transform sums, FP32 least squares and FP32
                                    squared norms; needs an FP32 / BF16 basis and an SRHT sketch */
#define RGS_LS_RICHARDSON 32     /* bit 5, rgs_qr only: step 2 by the normal equations S^T S x = S^T p with
                                    two Richardson sweeps from x = 0 (the alternative of Sec. 2.3) instead
                                    of Householder; needs FP64 least squares (an FP64 basis, RGS_FP64_LS or
                                    RGS_FP64_FINE).  Accurate only while S stays close to orthonormal. */
#define RGS_QR_FP64_FINE RGS_FP64_FINE
#define RGS_QR_FP64_SKETCH RGS_FP64_FINE
typedef struct {
    double delta;          /* Delta_m  = ||I - S^T S||_F            (Alg. 2 step 8) */
    double delta_tilde;    /* Delta~_m = ||P - S R||_F / ||P||_F    (Alg. 2 step 8) */
    int32_t breakdown_col; /* -1, or the column at which r_ii vanished */
    int32_t launches;      /* kernels this call launched */
    double sketch_ms;      /* step 1 for all columns (P = Theta W), with RGS_QR_TIMINGS */
    double update_ms;      /* fused steps 3-4 over all columns, with RGS_QR_TIMINGS */
    double ls_ms;          /* steps 2, 5, 6 over all columns, with RGS_QR_TIMINGS */
} rgs_qr_info;

RGS_API rgs_status rgs_qr(rgs_handle h, rgs_sketch s, int64_t n, int32_t m, const double* W, int64_t ldw,
                  void* Q, rgs_dtype qtype, int64_t ldq, double* qscale, double* R, int64_t ldr,
                  double* S, int64_t lds, int32_t flags, rgs_qr_info* info);

/* ---------------------------------------------------------------- embedding certificate
 * Sec. 3.2, Prop. cert01: an a posteriori certificate that Theta is an omega_bar-embedding for
 * range(V) (V n x m), from the sketches V^Theta = Theta V and V^Phi = Phi V, with Phi a second
 * sketch drawn independently of V and Theta (for instance the same kind and size, another seed):
 *     omega_bar = max(1 - (1 - eps_star) s_min^2, (1 + eps_star) s_max^2 - 1),
 * s the singular values of V^Theta X with V^Phi X orthonormal.  It holds with probability at
 * least 1 - delta* when Phi is an (eps_star, delta*, 1) oblivious embedding.  Everything is
 * FP64 on the GPU: Phi V (and Theta V when not given), the Gram matrices G_Phi and G_Theta, the
 * Cholesky factor L of G_Phi, C = L^{-1} G_Theta L^{-T} (eigenvalues s^2), Lanczos with full
 * (two-pass) reorthogonalisation on C until its extreme Ritz values settle (at most m steps),
 * and multisection with Sturm counts on the Lanczos tridiagonal matrix.
 *   V       device, n x m in vtype, ld ldv; column j multiplied by vscale[j] if vscale != NULL
 *           (pass rgs_qr's Q' and qscale to certify the basis Q).
 *   VTheta  NULL (Theta V is computed), or Theta V on the device, k x m FP64, ld ldvt (rgs_qr's S).
 *   out     host double[3]: omega_bar, s_min, s_max.
 * Requires 1 <= m <= min(1024, k of theta, k of phi), phi->n == theta->n == n.  Returns
 * RGS_ERR_CERT_FAILED when omega_bar >= 1 (out is filled), RGS_ERR_NONFINITE when G_Phi is not
 * numerically positive definite.  Synchronises the handle's stream; allocates workspace on the
 * handle (about 8 (kmax + 4 m) m bytes and one chunk of FP64 columns). */
RGS_API rgs_status rgs_certify_embedding(rgs_handle h, rgs_sketch theta, rgs_sketch phi, int64_t n, int32_t m,
                                         const void* V, rgs_dtype vtype, int64_t ldv, const double* vscale,
                                         const double* VTheta, int64_t ldvt, double eps_star, double* out);

/* ---------------------------------------------------------------- sparse operator */
typedef struct {
    int64_t n;              /* rows = columns */
    int64_t nnz;
    const int32_t* rowptr;  /* n + 1 entries, device */
    const int32_t* colind;  /* nnz entries, device, ascending within a row */
    const double* val;      /* nnz entries, device */
} rgs_csr;

/* ---------------------------------------------------------------- RGS-Arnoldi
 * Alg. 3: builds Q_j (Theta-orthonormal Krylov basis) and R_j one column at a
 * time; H_j = R_j(1:j, 2:j) (Sec. 4.1).  The object owns the basis (n x mmax in
 * qtype, stored as q'_i with scale 1/r_ii), S, R, the Householder factors of S
 * and a work vector.  The least-squares steps run in FP64 for an FP64 basis and
 * in double-float arithmetic (about 2^-48) for FP32 / BF16 bases, as in rgs_qr; with
 * flags = RGS_FP64_LS they run in FP64 for every basis type, and with RGS_FP64_FINE the SRHT
 * transform sums and the products with A do too (flags: 0, RGS_FP64_LS or RGS_FP64_FINE).
 *   rgs_arnoldi_start: iteration 1 with w_1 (device FP64, n).
 *   rgs_arnoldi_step:  next iteration with w_i = A q_{i-1} (A given, FP64 SpMV),
 *                      or with the caller's w (device FP64) when A is NULL.
 *   rgs_arnoldi_get:   number of columns, and copies of R (ncols x ncols, ldr)
 *                      and qscale (ncols) to host memory; Q stays in the object
 *                      and rgs_arnoldi_basis returns its device pointer and ld.
 * A step after a breakdown returns RGS_ERR_BREAKDOWN (happy breakdown in
 * GMRES terms). */
RGS_API rgs_status rgs_arnoldi_create(rgs_handle h, rgs_sketch s, int64_t n, int32_t mmax, rgs_dtype qtype,
                              int32_t flags, rgs_arnoldi* out);
RGS_API rgs_status rgs_arnoldi_destroy(rgs_arnoldi a);
RGS_API rgs_status rgs_arnoldi_start(rgs_handle h, rgs_arnoldi a, const double* w1);
RGS_API rgs_status rgs_arnoldi_step(rgs_handle h, rgs_arnoldi a, const rgs_csr* A, const double* w);
RGS_API rgs_status rgs_arnoldi_get(rgs_handle h, rgs_arnoldi a, int32_t* ncols, double* R_host, int64_t ldr,
                           double* qscale_host);
RGS_API rgs_status rgs_arnoldi_basis(rgs_arnoldi a, void** Q, int64_t* ldq);

/* ---------------------------------------------------------------- GMRES
 * rgmres_solve: restarted randomized GMRES (Sec. 4.2, Eq. hls) on A x = b with
 * the RGS-Arnoldi basis; in each cycle y = argmin ||H z - r_11 e_1|| by Givens
 * rotations in FP64, x += Q y, and the true residual b - A x is recomputed in
 * FP64 (restarting is not in the paper, which runs one cycle).  A cycle that
 * leaves ||b - A x|| without a relative decrease of 2^-10 draws a new Theta (same
 * kind, n and k; the r-th with seed + r * 0x9E3779B97F4A7C15 mod 2^64) for the
 * following cycles (rgmres_info.sketch_refreshes).  With an SRHT sketch the
 * products with A read it in SELL-32 form, built once per call (rgmres_info.sell).
 * cgs2_gmres_solve: the same restarted GMRES with an l2-orthonormal FP64 basis
 * built by CGS2 (projector (I - Q Q^T)^2, Sec. 1.2): the comparator.
 * b, x: device FP64 (x holds x0 on entry, the solution on exit).
 * Returns RGS_OK on convergence, RGS_ERR_NOT_CONVERGED otherwise. */
typedef struct {
    int32_t restart;        /* Arnoldi steps (products with A) per cycle */
    int32_t max_cycles;
    double rtol;            /* stop when ||b - A x|| <= rtol ||b|| */
    double inner_factor;    /* cycle ends when the Givens residual <= inner_factor * rtol * ||Theta b||;
                               a cycle that ended so but left ||b - A x|| > rtol ||b|| multiplies
                               this threshold by inner_factor * rtol ||b|| / ||b - A x|| for the
                               cycles after it */
    rgs_dtype qtype;        /* basis storage (RGS only) */
    int32_t fixed_steps;    /* 1: always run `restart` steps per cycle */
    int32_t flags;          /* 0, RGS_FP64_LS (FP64 least squares and Givens) or RGS_FP64_FINE (also
                               FP64 sketch sums and products with A) for FP32 / BF16 bases (RGS only) */
} rgmres_opts;

typedef struct {
    int32_t cycles;
    int32_t total_steps;
    int32_t converged;
    int32_t status;
    double rel_residual;    /* final ||b - A x|| / ||b|| in FP64 */
    double* history;        /* optional host array (max_cycles + 1): residual after each cycle */
    int32_t fallback_cycle; /* cycle at which the preconditioner was switched off, or -1 */
    int32_t sell;           /* 1: the products with A read it in SELL-32 form (slices of 32 rows,
                               entry-major; built once per solve when the SRHT sketch is used and
                               the padding stays within nnz / 4; RGS_SELL=0 in the environment
                               keeps CSR), 0: CSR.  The two give bit-identical results. */
    int32_t sketch_refreshes; /* rgmres_solve: cycles after which Theta was redrawn because the cycle
                                 had not reduced ||b - A x|| by a relative 2^-10 (the r-th redraw
                                 uses seed + r * 0x9E3779B97F4A7C15 mod 2^64; restarting, and so
                                 this rule, is outside the paper, which runs one cycle) */
    int32_t reserved;
} rgmres_info;

/* y = A x in FP64 (device arrays of A->n entries, no aliasing), stream-ordered.  The product
 * that Alg. 3 applies to each basis vector, exported for callers that form right-hand sides
 * b = A y or residuals themselves. */
RGS_API rgs_status rgs_csr_matvec(rgs_handle h, const rgs_csr* A, const double* x, double* y);
/* r = b - A x in FP64 (device arrays of A->n entries; r must not alias x): the restart residual of
 * Sec. 4.2's restarted solver, exported for callers that harvest residuals.  rnorm: NULL, or a host
 * double receiving ||r|| (then the stream is synchronised). */
RGS_API rgs_status rgs_csr_residual(rgs_handle h, const rgs_csr* A, const double* x, const double* b, double* r,
                                    double* rnorm);

RGS_API rgs_status rgmres_solve(rgs_handle h, rgs_sketch s, const rgs_csr* A, const double* b, double* x,
                        const rgmres_opts* opts, rgmres_info* info);
RGS_API rgs_status cgs2_gmres_solve(rgs_handle h, const rgs_csr* A, const double* b, double* x,
                            const rgmres_opts* opts, rgmres_info* info);

/* ---------------------------------------------------------------- preconditioning
 * Right preconditioning follows Sec. 5.3: GMRES runs on A M and returns x = x0 + M (Q y).
 * rgmres_set_preconditioner selects it for the following rgmres_solve calls on the handle:
 *   RGS_PRECOND_NONE         -- none (the default);
 *   RGS_PRECOND_JACOBI       -- M = diag(A)^{-1} (linear; A D^{-1} is formed once per solve);
 *   RGS_PRECOND_LEARNED_CONV -- M(r) = rms(r) net(r / rms(r), log kappa) with rms(r) = ||r|| / sqrt(n),
 *                               a trained rgs_convnet on
 *                               the H x W grid of the unknowns; nonlinear, so flexible = 1 is
 *                               required and the solver keeps z_j = M(q_j) (flexible GMRES,
 *                               x = x0 + Z y).  params points to an rgs_learned_precond.
 *   RGS_PRECOND_CALLBACK     -- the caller's M (an incomplete factorisation, say: Sec. 5.3 uses
 *                               ILU(0)); params points to an rgs_callback_precond.  The solver calls
 *                               apply(user, n, v, vtype, z, ztype, stream) from the calling thread
 *                               between its launches; apply enqueues z = M(v) on stream (the
 *                               handle's cudaStream_t) and returns 0, or nonzero to end the solve
 *                               with RGS_ERR_CALLBACK.  v (read only) and z are device vectors of n
 *                               entries, z never overlapping v; vtype is the basis storage type
 *                               (RGS_F64 for the vector Q y below), ztype is RGS_F64 for an FP64
 *                               basis and RGS_F32 otherwise.  flexible = 1 keeps every z_j = M(q_j)
 *                               (n (restart + 1) entries of ztype; x = x0 + Z y; any M); flexible =
 *                               0 is for a linear M: one z per step and x = x0 + M (Q y) after each
 *                               cycle.  nonlinear = 1 puts M under the fallback rule below.
 * With the learned preconditioner set (or a callback with nonlinear = 1), a restart whose true
 * residual is not below (1 - 2^-10) times the previous one switches the rest of the solve to the
 * unpreconditioned method (rgmres_info.fallback_cycle); Jacobi is never switched off.
 * The handle keeps the pointers in params (not copies): keep them valid while solving. */
typedef enum {
    RGS_PRECOND_NONE = 0,
    RGS_PRECOND_JACOBI = 1,
    RGS_PRECOND_LEARNED_CONV = 2,
    RGS_PRECOND_CALLBACK = 3
} rgs_precond_kind;
typedef struct rgs_convnet_obj* rgs_convnet;
typedef struct {
    rgs_convnet net;
    const double* logkappa;   /* device, H x W (row-major, x fastest): second input channel */
} rgs_learned_precond;
typedef int32_t (*rgs_precond_apply_fn)(void* user, int64_t n, const void* v, int32_t vtype, void* z,
                                        int32_t ztype, void* stream);
typedef struct {
    rgs_precond_apply_fn apply;
    void* user;               /* passed through unchanged */
    int32_t nonlinear;        /* 1: the fallback rule applies to M */
    int32_t reserved;         /* 0 */
} rgs_callback_precond;
RGS_API rgs_status rgmres_set_preconditioner(rgs_handle h, rgs_precond_kind kind, const void* params,
                                             int32_t flexible);

/* ---------------------------------------------------------------- learned preconditioner network
 * Six 3x3 convolutions (zero padding) with channels 2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 and
 * ReLU between layers, on a batch of H x W grids (H a multiple of 8, W of 16).  Weights are
 * BF16 copies of FP32 master parameters; products run on the tensor cores with FP32
 * accumulation; activations are BF16.  Parameters are flat FP32: for each layer l the weights
 * W_l[c_out][c_in][3][3] then the biases b_l[c_out] (rgs_convnet_num_params() in all).
 *   in:     batch x 2 x H x W FP32 (device): channel 0 the residual scaled to unit root mean
 *           square, channel 1 log kappa.
 *   out:    batch x H x W FP32 (device).
 *   target: batch x H x W FP32 (device).
 *   stencil: NULL, or batch x 5 x H x W FP32 (device): the 5-point operator A_b of each sample,
 *           coefficients of row (y, x) for (y, x) itself, (y, x-1), (y, x+1), (y-1, x), (y+1, x)
 *           (entries that reach outside the grid are ignored).
 * Loss: mean_b ||F_b - t_b||^2 / ||t_b||^2 with F_b = out_b, or F_b = A_b out_b when stencil is
 * given (the residual-norm loss: with t_b = r_b it measures ||A_b (out_b - A_b^{-1} r_b)||, the
 * quantity a right preconditioner has to make small).
 * rgs_convnet_train_step: forward, loss, backward and one Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8) on the batch; rgs_convnet_loss_grad: loss and the FP32 gradient (host) without
 * updating.  max_batch bounds the batch of every call (it sizes the saved activations). */
RGS_API int64_t rgs_convnet_num_params(void);
/* The network's input for one grid (device arrays; n = H W points): out[0:n] = r / rms(r),
 * out[n:2n] = log kappa, FP32, with rms(r) = ||r|| / sqrt(n) summed in FP64 (rms 0 gives a zero
 * channel).  The same scaling the preconditioner applies inside flexible RGMRES. */
RGS_API rgs_status rgs_convnet_input(rgs_handle h, int64_t n, const double* r, const double* logkappa, float* out);
/* out (device, 5 x H x W FP32): the 5-point stencil of A (n = H W, x fastest) in the loss's layout
 * (centre, west, east, north, south coefficients of each row; repeated entries add).  Returns
 * RGS_ERR_INVALID_ARG if an entry lies at another offset.  Synchronises the stream. */
RGS_API rgs_status rgs_csr_to_stencil(rgs_handle h, const rgs_csr* A, int32_t H, int32_t W, float* out);
/* rgs_convnet_create: weights drawn U(-1/sqrt(9 c_in), 1/sqrt(9 c_in)) from Philox (key = seed,
 * counter (parameter index, 0, 0, 8)), biases 0. */
RGS_API rgs_status rgs_convnet_create(rgs_handle h, int32_t height, int32_t width, int32_t max_batch, uint64_t seed,
                                      rgs_convnet* out);
RGS_API rgs_status rgs_convnet_destroy(rgs_convnet net);
RGS_API rgs_status rgs_convnet_get_params(rgs_handle h, rgs_convnet net, float* host, int64_t count);
RGS_API rgs_status rgs_convnet_set_params(rgs_handle h, rgs_convnet net, const float* host, int64_t count);
RGS_API rgs_status rgs_convnet_forward(rgs_handle h, rgs_convnet net, int32_t batch, const float* in, float* out);
RGS_API rgs_status rgs_convnet_loss_grad(rgs_handle h, rgs_convnet net, int32_t batch, const float* in,
                                         const float* target, const float* stencil, double* loss,
                                         float* grad_host);
RGS_API rgs_status rgs_convnet_train_step(rgs_handle h, rgs_convnet net, int32_t batch, const float* in,
                                          const float* target, const float* stencil, float lr, double* loss);

/* ---------------------------------------------------------------- batched solves
 * rgmres_solve_batched solves nbatch independent systems A_b x_b = b_b with restarted RGMRES in
 * one persistent cooperative kernel (issued through a CUDA graph): the grid is split into
 * teams of CTAs, each team runs the whole solve of its instance(s) with team-local barriers
 * (bounded waits; RGS_ERR_TIMEOUT), so no host round trip happens between cycles.
 * Sketch: Gaussian, Theta_b = G[0:k_b, 0:n_b] / sqrt(k_b) with G the N(0,1) draws of the
 * Gaussian sketch layout above for sketch_seed, rounded to bfloat16 (one shared matrix for the
 * whole batch); products with it accumulate in double-float.  The sketched least-squares
 * problem (step 2 of Alg. 2) is solved in FP64 through a CGS2 QR factorisation of S; Givens
 * rotations and the restart residual b - A x are FP64.
 *   A, b, x, opts, info: host arrays of nbatch entries; A[i] holds device CSR arrays, b[i] and
 *   x[i] device FP64 vectors (x[i]: initial guess in, solution out).  info may be NULL;
 *   info[i].history, if set, is a host array of max_cycles + 1 entries.
 *   opts[i]: restart in [1, 127], restart + 1 <= k <= 192, one qtype (RGS_F64 or RGS_F32) for
 *   the whole batch.
 * Returns RGS_OK when the launch completed; per-instance results (RGS_OK,
 * RGS_ERR_NOT_CONVERGED, RGS_ERR_NONFINITE, ...) are in info[i].status. */
typedef struct {
    int32_t restart;
    int32_t k;
    int32_t max_cycles;
    int32_t qtype;
    double rtol;
    double inner_factor;
    int32_t fixed_steps;
    int32_t reserved;
} rgmres_batch_opts;

RGS_API rgs_status rgmres_solve_batched(rgs_handle h, int32_t nbatch, const rgs_csr* A, const double* const* b,
                                        double* const* x, const rgmres_batch_opts* opts, uint64_t sketch_seed,
                                        rgmres_info* info);

/* ---------------------------------------------------------------- launch tuning
 * Tunable launch shapes of the handle (no counterpart in the paper; every choice computes the
 * same quantities, only the grouping of partial sums changes):
 *   upd_blocks_per_sm    CTAs per SM of the fused update / sketch pass of steps 3-4 (1..4); it is
 *                        also the number of partial sketches per SM that step 2 reduces.
 *   batch_blocks_per_sm  CTAs per SM of the batched solver's persistent grid (0 = occupancy limit).
 *   batch_min_team_work  rows x (k + restart) per CTA below which a batched instance gets no
 *                        further CTA for its team.
 *   ls_blocks            CTAs of the cooperative least-squares kernel (0: one per SM).
 *   batch_rows_per_thread  rows per thread of the batched kernel (2 or 4): a tile shape, one
 *                        compiled kernel per value.
 * rgs_autotune_update times the update pass of an n-row basis of ncols columns (s->n rows, SRHT s)
 * for upd_blocks_per_sm in 2..4 and keeps the fastest; ms (optional, 3 entries) receives the
 * mean launch times.  rgs_autotune_batched times `cycles` fixed cycles of the given batch for
 * batch_rows_per_thread in {4, 2} x batch_blocks_per_sm in {occupancy limit, one less} x
 * batch_min_team_work in {2^17, 2^19, 2^21} and keeps the fastest; ms (optional, 12 entries, in
 * that nesting order) receives the times (0 for a candidate that was not run).  Both leave the choice on the handle and
 * copy it to out (optional). */
typedef struct {
    int32_t upd_blocks_per_sm;
    int32_t batch_blocks_per_sm;
    double batch_min_team_work;
    int32_t ls_blocks;            /* CTAs of the least-squares kernel of step 2 (0: one per SM) */
    int32_t batch_rows_per_thread;  /* rows per thread (2 or 4; 0 = 4) of the batched kernel's streaming
                                       phases and of its tensor-core sketch tile: two kernel builds */
} rgs_tuning;
RGS_API rgs_status rgs_get_tuning(rgs_handle h, rgs_tuning* out);
RGS_API rgs_status rgs_set_tuning(rgs_handle h, const rgs_tuning* t);
RGS_API rgs_status rgs_autotune_update(rgs_handle h, rgs_sketch s, int32_t ncols, rgs_dtype qtype, rgs_tuning* out,
                                       float* ms);
RGS_API rgs_status rgs_autotune_batched(rgs_handle h, int32_t nbatch, const rgs_csr* A, const double* const* b,
                                        const rgmres_batch_opts* opts, uint64_t sketch_seed, int32_t cycles,
                                        rgs_tuning* out, float* ms);

#ifdef __cplusplus
}
#endif

#endif /* LIBRGS_H */
