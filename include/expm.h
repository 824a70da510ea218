/*
 * expm.h -- C interface of the GB300 partial-fraction matrix-exponential library.
 *
 * Method (Hecht, Kaber, Perrin, Plagne, Salomon, "Parallel approximation of the
 * exponential of Hermitian matrices"): exp(z) is approximated by the (0,n) Pade
 * approximant R_n(z) = 1/exp_n(-z) (Sec. 2.2), whose partial-fraction form is
 *     R_n(z) = sum_k a_k / (z + theta_k)                     (Prop. 2.1, eq. yoyo)
 * with theta_k the roots of the truncated Taylor series exp_n (Sec. 2.1) and
 *     a_k = -n! / prod_{j != k} (theta_k - theta_j)           (eq. yoyo2).
 * For a Hermitian A and a block of vectors V,
 *     exp(tA) V ~ e^c R_n(tA - cI) V = e^c sum_k a_k (tA - cI + theta_k I)^{-1} V
 * (eqs. ExpoMatRat and expAx; the shift c of Remark 3.2): n independent shifted
 * solves and a residue-weighted sum.  For real A and real V only one member of
 * each conjugate pair is solved and the sum is 2 Re(...) (Remark 5.1).
 *
 * Conventions used throughout this header
 * ---------------------------------------
 * Poles and weights.  The interface carries the POLES lambda_k = -theta_k of R_n
 *   and the WEIGHTS w_k = a_k, so that R_n(z) = sum_k w_k / (z - lambda_k) and
 *   each solve is (tA - cI - lambda_k I) X_k = V.  Arrays of complex numbers are
 *   interleaved (re, im) doubles; an array "of n complex" holds 2n doubles.
 *   Conjugate pairs must be adjacent: lambda_{2l+1} = conj(lambda_{2l}) and
 *   w_{2l+1} = conj(w_{2l}).  The degree n is even (Sec. 2.2 assumes it; an odd
 *   n has a real root, and A - lambda I could then be singular).
 * Layout.  Matrices are row-major; ld* are leading dimensions in ELEMENTS.
 *   Complex data is interleaved re/im (layout-compatible with C99 double
 *   complex, std::complex<double> and torch.complex128).
 * Memory.  Every data pointer may be device memory or host memory; the library
 *   tells them apart with cudaPointerGetAttributes.  Device pointers are used in
 *   place and the call is asynchronous on opts->stream (it returns after
 *   enqueueing; outputs are ready when the stream reaches that point).  If any
 *   data pointer is host memory the call stages it through device workspace owned
 *   by the plan, copies the result back and synchronises opts->stream before it
 *   returns.  The caller owns all data buffers; they must stay valid until the
 *   call's work on the stream is complete.
 * Errors.  Every function returns an expm_status; nothing else is reported and no
 *   exception or device trap crosses the interface.  On EXPM_EINVAL nothing is
 *   enqueued.  EXPM_ECUDA means a CUDA runtime call failed; the message of the
 *   last failure is available from expm_last_error().
 * Threads.  A plan is not thread safe: use one plan per host thread (plans are
 *   cheap).  Each plan belongs to the CUDA device that was current at creation.
 */
#ifndef EXPM_H
#define EXPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum expm_status {
    EXPM_OK = 0,
    EXPM_EINVAL = 1,     /* invalid argument (size, stride, degree, pairing, ...)   */
    EXPM_ENOMEM = 2,     /* device workspace could not be allocated / over budget  */
    EXPM_EGROWTH = 3,    /* pivot growth of an unpivoted LU exceeded opts.growth_max */
    EXPM_ENOCONV = 4,    /* iterative refinement did not reach opts.tol            */
    EXPM_ETIMEOUT = 5,   /* a bounded device-side wait gave up                     */
    EXPM_EAGAIN = 6,     /* server / queue: full, or request still pending         */
    EXPM_ECUDA = 7,      /* a CUDA runtime call failed                             */
    EXPM_ENOTFOUND = 8,  /* server / queue: unknown or released ticket, unknown id */
    EXPM_ENOTSUP = 9     /* combination of options not implemented                 */
} expm_status;

typedef enum expm_precision {
    EXPM_FP64 = 0,        /* binary64 arithmetic throughout                         */
    EXPM_MIXED_F32X2 = 1, /* tridiagonal: float-float (pairs of binary32, ~48-bit
                             significand) on the FP32 pipe; dense: as EXPM_MIXED_FP32 */
    EXPM_MIXED_FP32 = 2,  /* dense: binary32 LU + binary64-residual refinement;
                             tridiagonal: binary32 factors and solves + refinement
                             with float-float residuals (FP32 pipe only)            */
    EXPM_MIXED_TF32X3 = 3, /* dense: LU trailing updates on the tensor cores with a
                              3-term TF32 split, + binary64-residual refinement     */
    EXPM_MIXED_BF16X3 = 4  /* dense: LU trailing updates on the tensor cores with a
                              3-part bf16 split (six products), + binary64-residual
                              refinement                                            */
} expm_precision;

typedef struct expm_opts {
    int prec;           /* expm_precision                                          */
    double tol;         /* refinement target: max_k ||R_k||_F / ((||A||_F + |lambda_k|) ||X_k||_F);
                           default 1e-14                                            */
    int max_refine;     /* refinement sweep cap (default 6)                         */
    double t;           /* time factor t of exp(tA)V (default 1)                    */
    double shift_c;     /* shift c of Remark 3.2: result = e^c R_n(tA - cI) V (default 0) */
    double growth_max;  /* allowed growth max|U|/max|A - lambda I| of the unpivoted LU
                           (dense paths; default 1e6)                              */
    void *stream;       /* cudaStream_t to enqueue on (NULL = legacy default stream) */
    int flags;          /* 0, or EXPM_FLAG_SKIP_FINAL_RESIDUAL (see below)          */
} expm_opts;

/* EXPM_MIXED_FP32 tridiagonal path only: do not form the residual after the last
 * correction pass.  Saves one residual evaluation per call; info.resid_rel_max then
 * reports the residual before the last pass and EXPM_ENOCONV is never returned. */
#define EXPM_FLAG_SKIP_FINAL_RESIDUAL 1

typedef struct expm_info {
    int refine_iters_max;   /* largest number of refinement sweeps any pole used   */
    double growth_max_seen; /* largest LU growth factor seen (dense paths)          */
    double resid_rel_max;   /* largest final relative residual (mixed dense paths)  */
    int status_worst;       /* worst per-pole expm_status                           */
} expm_info;

typedef struct expm_plan_s *expm_plan;

/* Fill *opts with the defaults listed above.  Never fails for a non-NULL opts. */
void expm_opts_default(expm_opts *opts);

/* Human-readable name of a status code (static string). */
const char *expm_status_string(expm_status s);

/* Message of the most recent EXPM_ECUDA / EXPM_EINVAL in this thread ("" if none). */
const char *expm_last_error(void);

/*
 * expm_coeffs -- poles and weights of R_n for degree n (host only, no GPU use).
 * Sec. 2.1 (roots theta_k of exp_n) and Prop. 2.1 eq. yoyo2 (a_k), computed in
 * double-double arithmetic (Aberth-Ehrlich iteration polished by Newton steps,
 * residues by the product formula the paper keeps in Sec. 4) and rounded once to
 * binary64, as the paper's Fig. 4.1 caption recommends (>= 32 digits, then 16).
 *   degree        even, 2 <= degree <= 64
 *   poles_ri      out, 2*degree doubles: lambda_k = -theta_k interleaved (re, im)
 *   residues_ri   out, 2*degree doubles: w_k = a_k interleaved (re, im)
 * Order: conjugate pairs adjacent, pairs by Re(theta) ascending, Im(theta) > 0
 * member first.  Returns EXPM_EINVAL for an odd/out-of-range degree or NULL
 * outputs.
 */
expm_status expm_coeffs(int degree, double *poles_ri, double *residues_ri);

/*
 * expm_plan_create -- validate pole data and make it resident on the current device.
 *   poles_ri, residues_ri   host arrays of `degree` complex (see conventions)
 *   degree                  even, 2 <= degree <= 64
 *   out                     receives the plan (owned by the caller; release it
 *                           with expm_plan_destroy)
 * Checks: finite values, adjacent conjugate pairs (relative 1e-12), and
 * R_n(0) = -sum_k w_k/lambda_k = 1 within 1e-8 (Sec. 2.2, R_n(0) = 1).
 * Returns EXPM_EINVAL on failed checks, EXPM_ENOMEM / EXPM_ECUDA on device errors.
 */
expm_status expm_plan_create(const double *poles_ri, const double *residues_ri, int degree,
                             expm_plan *out);

/* Release a plan and its device workspace (synchronises the device). NULL is OK. */
expm_status expm_plan_destroy(expm_plan plan);

/*
 * expm_apply_tridiag -- Y = e^c R_n(tT - cI) V for a Hermitian tridiagonal T.
 * Eq. expAx with one shifted tridiagonal solve per pole (pole-batched, Sec. 3),
 * the 2 Re halving of Remark 5.1 when T and V are real, and the residue sum.
 *   N             rows, N >= 1
 *   d             N doubles: diagonal of T (real)
 *   e             N-1 off-diagonal entries T_{i,i+1} (T_{i+1,i} = conj(e_i)):
 *                 doubles if e_is_complex == 0, else N-1 complex
 *   V             N x r right-hand sides, row-major, ld = r; real doubles if
 *                 v_is_complex == 0, else complex
 *   r             number of right-hand sides, 1 <= r <= 1024
 *   Y             N x r output, row-major; complex when V or e is complex, else real.
 *                 Must not overlap V, d or e.
 *   opts          precision EXPM_FP64, EXPM_MIXED_F32X2 or EXPM_MIXED_FP32; t, shift_c,
 *                 stream; for EXPM_MIXED_FP32 also tol, max_refine and flags
 *   info          optional (may be NULL).  EXPM_FP64 / EXPM_MIXED_F32X2: not used
 *                 (zeroed).  EXPM_MIXED_FP32: when info is given the call waits for
 *                 the result and reports refine_iters_max (correction passes applied)
 *                 and resid_rel_max (the last residual formed, see below); without
 *                 info the call stays asynchronous and reports nothing.
 * EXPM_MIXED_FP32 (binary32 + refinement): the shifted matrices are factored and
 * solved in binary32; pass 0 solves with V, and each of at most max_refine further
 * passes solves with the residual r = V - (tT - cI + theta I) X of the running
 * solution X and adds the correction.  Residuals are formed in float-float from
 * the binary64 entries.  The passes stop once every system meets
 *   ||r_s||_F <= tol (beta + |theta_s|) ||X_s||_F,  beta = max_i |d'_i| + |e'_{i-1}| + |e'_i|
 * (d' = t d - c, e' = t e: beta bounds ||tT - cI||_2).  EXPM_ENOCONV (with info)
 * when the residual after the last pass still exceeds tol.  Scratch: about
 * 16 S N + 8 S r' N (max_refine >= 1) + 8 S r' N (max_refine >= 2) bytes, S = degree/2
 * rounded up to a power of two, r' = real columns.  Not available in
 * expm_apply_tridiag_noalloc.
 * Method: the rows are split into blocks separated by single separator rows;
 * each block is factored (unpivoted LU; (A - lambda I) scaled by a unit complex
 * number has a positive-definite Hermitian part when Im lambda != 0, so no pivot
 * is needed), the separators solve a reduced tridiagonal system by cyclic
 * reduction, and the blocks are then solved and summed with their weights.
 * Complex e (a general Hermitian T): D = diag(phi), phi_0 = 1, phi_{i+1} = phi_i
 * conj(e_i)/|e_i|, is unitary and D^H T D is real symmetric with off-diagonal |e|;
 * since every resolvent satisfies (tT - cI + theta I)^{-1} = D (tD^H T D - cI +
 * theta I)^{-1} D^H, the call forms phi (a parallel prefix product), solves the real
 * problem on D^H V and multiplies row i of the result by phi_i.  Extra device scratch:
 * 24 N + 16 N r bytes; Y is complex.
 * Returns EXPM_EINVAL for bad sizes.
 */
expm_status expm_apply_tridiag(expm_plan plan, int64_t N, const double *d, const void *e,
                               int e_is_complex, const void *V, int r, int v_is_complex,
                               void *Y, const expm_opts *opts, expm_info *info);

/*
 * expm_apply_tridiag_noalloc -- expm_apply_tridiag for callers that must not allocate.
 * The paper has no counterpart: this is a deployment variant of the same computation.
 * Who needs it: callers that cannot let the library call cudaMalloc/cudaFree, for
 * example a serving process whose device memory is reserved at start-up by another
 * framework's caching allocator, or a latency-critical loop in which an allocation
 * (which may synchronise the device and take unbounded time) is not acceptable.
 * It runs the same kernels as expm_apply_tridiag, with their scratch in a fixed array
 * of EXPM_NOALLOC_SCRATCH_BYTES bytes that the library holds in device memory on
 * every GPU that loads it, until the process exits.  The call allocates nothing and
 * enqueues asynchronously on opts->stream.
 *   Arguments and result: as expm_apply_tridiag, except that d, e, V and Y must be
 *   device memory (host buffers would need staging memory: EXPM_EINVAL).
 *   Size limit: a problem whose scratch exceeds EXPM_NOALLOC_SCRATCH_BYTES is
 *   rejected with EXPM_EINVAL and a message giving the bytes needed (about
 *   N * (400 + 136 r) bytes for degree 16 and r >= 2 real right-hand sides, so N up
 *   to about 22,000 for r = 8; complex e counts its right-hand sides as complex and
 *   adds 24 N + 16 N r bytes for |e|, the phases and D^H V).
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and caches it.  With CUDA's lazy
 *   module loading (the default) that first lookup is also when the library's module,
 *   and with it the fixed array, is loaded onto the device: the first call may
 *   allocate device memory and synchronise.  Callers that need no allocation at all
 *   should make one warm-up call at start-up, outside any stream capture and any
 *   latency-critical loop; later calls allocate nothing.  The cached address belongs
 *   to the device's current context: after cudaDeviceReset in the same process the
 *   library must not be used on that device again (the cache is not refreshed).
 *   Sharing: all calls on a device share the one array and it keeps whatever the last
 *   call left in it (every kernel writes the scratch it later reads; nothing needs to
 *   start at zero).  Calls whose work overlaps on the GPU -- different streams, or
 *   different host threads -- race on the array: serialise them.
 */
#define EXPM_NOALLOC_SCRATCH_BYTES (32u << 20)
expm_status expm_apply_tridiag_noalloc(expm_plan plan, int64_t N, const double *d, const void *e,
                                       int e_is_complex, const void *V, int r, int v_is_complex, void *Y,
                                       const expm_opts *opts, expm_info *info);

/*
 * expm_apply_dense -- Y = e^c R_n(tA - cI) V for a dense Hermitian A.
 * Eq. expAx with one shifted dense solve per pole: unpivoted blocked LU of
 * tA - cI + theta I per conjugate pole pair (Sec. 3), triangular solves, and the
 * residue-weighted sum.  Real symmetric A with real V solves one pole of each pair
 * and takes 2 Re(...) (Remark 5.1); complex Hermitian A solves both poles of a pair
 * with one factorization, since tA - cI + conj(theta) I = (tA - cI + theta I)^H.
 *   n             order of A, n >= 1
 *   A             n x n, row-major, leading dimension lda >= n (elements); real
 *                 doubles if a_is_complex == 0, else complex.  Only Hermitian A is
 *                 supported; the full matrix is read (no symmetry is exploited).
 *   V             n x k right-hand sides, leading dimension ldv >= k; real if
 *                 v_is_complex == 0, else complex
 *   k             1 <= k <= 4096
 *   Y             n x k output, leading dimension ldy >= k; complex when A or V is
 *                 complex, else real.  Must not overlap A or V.
 *   opts          prec: EXPM_FP64 (binary64 throughout), EXPM_MIXED_FP32 /
 *                 EXPM_MIXED_F32X2 (binary32 factorization on the CUDA cores) or
 *                 EXPM_MIXED_TF32X3 / EXPM_MIXED_BF16X3 (binary32 factorization whose
 *                 trailing updates run on the tensor cores: tcgen05 kind::tf32 with the
 *                 3xTF32 split, or kind::f16 with each value split into three bf16
 *                 parts and the six products of order <= 2), each
 *                 followed by iterative refinement with binary64-accurate residuals until
 *                 ||R_k||_F <= tol (||tA||_F + |theta_k - c|) ||X_k||_F, at most
 *                 max_refine sweeps); growth_max bounds max|U| / max|tA - cI + theta I|.
 *   info          optional: refinement sweeps, worst relative residual, worst growth.
 * Device workspace (held by the plan, grown on demand): the factors, n^2 complex per
 * pole pair (binary64, or binary32 in the mixed modes); for k > 8 also the inverses of
 * the factors' 128-row diagonal panels (the triangular solves multiply by them), about
 * 3 n min(n, 128) complex per pair; the solutions (and, mixed, residuals and corrections)
 * n k complex per solved pole; the tensor-core modes' split operands.
 * The call synchronises opts->stream before returning (it reads back the growth
 * factors and, in mixed precision, the residual norms).  Returns EXPM_EGROWTH if a
 * growth factor exceeds growth_max, EXPM_ENOCONV if refinement did not reach tol
 * (Y is written in both cases), EXPM_ETIMEOUT if a bounded wait inside a tensor-core
 * kernel gave up (about one second without progress; Y is not valid), EXPM_EINVAL for
 * bad sizes.
 */
expm_status expm_apply_dense(expm_plan plan, int n, const void *A, int lda, int a_is_complex, const void *V,
                             int ldv, int k, int v_is_complex, void *Y, int ldy, const expm_opts *opts,
                             expm_info *info);

/*
 * expm_apply_dense_full -- the full matrix Y = e^c R_n(tA - cI) (eq. ExpoMatRat: R_n(A) =
 * sum_k a_k (A + theta_k I)^{-1}), the approximation of exp(tA) itself.
 * Equivalent to expm_apply_dense with V = I; the per-pair LUs are formed once and the
 * identity passes through the solve part in blocks of 512 columns.
 *   n, A, lda, a_is_complex   as expm_apply_dense
 *   Y             n x n row-major, leading dimension ldy >= n (elements); real for
 *                 real symmetric A (Remark 5.1), interleaved complex for complex A
 *   opts, info    as expm_apply_dense (info over all column blocks)
 * A and Y may be host or device memory (host buffers are staged; the call then
 * synchronises).  Returns as expm_apply_dense.
 */
expm_status expm_apply_dense_full(expm_plan plan, int n, const void *A, int lda, int a_is_complex, void *Y, int ldy,
                                  const expm_opts *opts, expm_info *info);

/*
 * expm_apply_dense_reduced -- Y = e^c R_n(tA - cI) V for a dense Hermitian A through a
 * unitary reduction to real symmetric tridiagonal form: A = Q T Q^H by Householder
 * reflectors (each mapping the column below the diagonal to a real multiple of e_1, so
 * T is real), then Y = Q [e^c R_n(tT - cI) (Q^H V)] (Remark 3.1: R_n commutes with the
 * similarity) with the pole-batched tridiagonal path.  The reduction costs about
 * (8/3) n^3 complex multiply-adds once, whatever the degree, against n/2 LUs for
 * expm_apply_dense.  No counterpart in the paper's experiments (it is named there as a
 * way to use tridiagonal solvers for dense Hermitian A).
 *   n, A, lda, a_is_complex, V, ldv, k, v_is_complex, Y, ldy   as expm_apply_dense, with
 *                 n <= 12000, 1 <= k <= 1024; A, V and Y must be device memory (A is not modified:
 *                 the reduction works on a copy)
 *   opts          t, shift_c, stream; prec selects the tridiagonal solves (EXPM_FP64,
 *                 EXPM_MIXED_F32X2 or EXPM_MIXED_FP32 with tol / max_refine / flags as in
 *                 expm_apply_tridiag); the reduction and the reflector products are
 *                 binary64 in every case
 *   info          as expm_apply_tridiag for the tridiagonal solves
 * Asynchronous on opts->stream (except the refinement report of EXPM_MIXED_FP32 with
 * info, as in expm_apply_tridiag).
 */
expm_status expm_apply_dense_reduced(expm_plan plan, int n, const void *A, int lda, int a_is_complex, const void *V,
                                     int ldv, int k, int v_is_complex, void *Y, int ldy, const expm_opts *opts,
                                     expm_info *info);

/*
 * expm_apply_laplacian2d -- Y = e^c R_n(tA - cI) V for the separable operator of the 2D
 * finite-difference Laplacian (the paper's second workload, Sec. 5):
 *     A = I_y (x) T_x + T_y (x) I_x,  T_x = tridiag(ax, bx, ax) (dx points),
 *                                     T_y = tridiag(ay, by, ay) (dy points),
 * unknown (ix, iy) at row iy * dx + ix.  T_y is diagonalised by the orthonormal DST-I S,
 * so A = (S (x) I)[(+)_j (T_x + mu_j I)](S (x) I) with mu_j = by + 2 ay cos((j+1) pi/(dy+1)),
 * and (Remark 3.1) Y = (S (x) I) e^c R_n(tB - cI) (S (x) I) V with B block-diagonal
 * tridiagonal: the pole-batched tridiagonal path on dx * dy rows between two products
 * with S along y.  With EXPM_FP64 the products are binary64; with the mixed precisions
 * (and an even number dx r (1 + v_is_complex) of real columns) they are the
 * binary64-accurate slice products on the bf16 tensor cores used by the dense
 * refinement (error a few 2^-48 of the row and column scales).
 *   V, Y          device memory, (dx dy) x r row-major, real or complex (v_is_complex);
 *                 1 <= r <= 512, dx * dy <= 2^28
 *   opts, info    as expm_apply_tridiag (its precisions select the tridiagonal solves)
 * Returns EXPM_ETIMEOUT if a bounded wait inside a tensor-core product gave up (Y is then
 * not valid).  Asynchronous on opts->stream with EXPM_FP64; with the tensor-core products
 * the call synchronises the stream once at the end to read their status.
 */
expm_status expm_apply_laplacian2d(expm_plan plan, int dx, int dy, double ax, double bx, double ay, double by,
                                   const void *V, int r, int v_is_complex, void *Y, const expm_opts *opts,
                                   expm_info *info);

/*
 * expm_apply_batched -- Y_i = e^c R_n(tA_i - cI) V_i for `count` independent dense
 * Hermitian problems of uneven sizes (eq. expAx per instance, Sec. 3).
 *   count            number of instances (0 is a no-op)
 *   n[i], k[i]       order of A_i and number of right-hand sides (1 <= k[i] <= 4096);
 *                    host arrays
 *   A[i]             n[i] x n[i], row-major, leading dimension n[i]; real symmetric
 *                    (a_is_complex == 0) or complex Hermitian, device memory
 *   V[i], Y[i]       n[i] x k[i], row-major, leading dimension k[i], device memory;
 *                    V complex iff v_is_complex (complex V needs complex A); Y complex
 *                    iff A or V is complex
 *   opts             as expm_apply_dense (precision, refinement, growth limit, stream);
 *                    EXPM_MIXED_TF32X3 / EXPM_MIXED_BF16X3 run the LU's trailing updates
 *                    on the tensor cores for buckets of padded order above 256 (binary32
 *                    LU on the FP32 pipe below), refined as EXPM_MIXED_FP32
 *   per_instance     optional host array of `count` expm_info, filled per instance
 * Method: instances are grouped by size into buckets and zero-padded to the bucket's
 * order (exact: the padded part of tA - cI + theta I is the diagonal (theta - c) I);
 * each bucket is one batch of (instance, pole pair) units for the dense kernels
 * (unpivoted LU, triangular solves, refinement, residue sum).  The call
 * synchronises opts->stream.  Returns EXPM_EGROWTH / EXPM_ENOCONV if any instance
 * failed the growth or refinement test (all Y_i are written; per_instance says
 * which), EXPM_ENOTSUP for complex V with real A, EXPM_ETIMEOUT if a bounded wait in a
 * tensor-core update gave up.
 */
expm_status expm_apply_batched(expm_plan plan, int count, const int *n, const void *const *A, int a_is_complex,
                               const void *const *V, const int *k, int v_is_complex, void *const *Y,
                               const expm_opts *opts, expm_info *per_instance);

/*
 * Captured batched evaluation (no counterpart in the paper: a launch pattern around
 * eq. expAx for many instances).  expm_batched_capture records the whole of an
 * expm_apply_batched call -- per size bucket the padding gather, the per-pair LUs, the
 * refinement with its stopping test decided on the device (every sweep is recorded
 * and skips itself once all instances of the bucket have converged), the residue sums
 * and the scatter -- into one CUDA graph over the given buffers; expm_batched_replay
 * then evaluates the batch again with a single graph launch, reading whatever A_i and
 * V_i hold at that time and writing Y_i.
 *   count, n, A, a_is_complex, V, k, v_is_complex, Y, opts   as expm_apply_batched,
 *                 except 1 <= k[i] <= 8 and every padded order must fit the fused
 *                 narrow triangular solve (n[i] up to about 1500 for k = 1); the
 *                 pointer arrays are read during the call only
 *   scheme        padded orders of the size buckets: 0 (multiples of 32 up to 128, then
 *                 steps of about a quarter; the expm_apply_batched default), 1 (all
 *                 multiples of 32), 2 (powers of two and midpoints), or -1: capture all
 *                 three, time two launches of each and keep the fastest (autotuning);
 *                 with -1 every bucket factorised on the FP32 pipe (EXPM_MIXED_FP32,
 *                 and the mixed tensor-core precisions below order 257) first times its
 *                 factorization with 128 x 64 and 64 x 64 trailing-update tiles and
 *                 keeps the faster shape
 *   out           the graph; it owns its device memory (workspace, staging copies of
 *                 the padded instances, pointer tables, per-instance results)
 * The call runs the evaluation once outside the capture (so Y holds a result on return)
 * and synchronises.  EXPM_EINVAL for bad arguments, EXPM_ENOMEM when the graph memory
 * cannot be allocated, EXPM_ECUDA when the capture fails.
 *   expm_batched_replay      enqueues the graph on stream; with per_instance (host
 *                 array of count entries) the call waits and reports each instance as
 *                 expm_apply_batched does, returning EXPM_EGROWTH / EXPM_ENOCONV /
 *                 EXPM_ETIMEOUT likewise.  A single instance small enough for the
 *                 one-launch kernel of expm_apply_dense is captured as that launch.
 *   expm_batched_graph_info  chosen scheme, number of launch groups (bucket chunks),
 *                 device bytes, and the timed ms per scheme (-1 where not timed).
 *   expm_batched_graph_buckets  per launch group i < max of the chosen graph: padded
 *                 order[i], instances ninst[i], trailing-update tile[i] (0: 128 x 64,
 *                 1: 64 x 64) and the timed factorization ms with each (ms_tile0[i],
 *                 ms_tile1[i]; -1 where not timed).  Any output pointer may be NULL
 *                 (host arrays of max entries).  Returns the number of launch groups
 *                 (0 for a captured one-launch small instance), -1 for a NULL graph.
 */
typedef struct expm_batch_graph_s *expm_batch_graph;
expm_status expm_batched_capture(expm_plan plan, int count, const int *n, const void *const *A, int a_is_complex,
                                 const void *const *V, const int *k, int v_is_complex, void *const *Y,
                                 const expm_opts *opts, int scheme, expm_batch_graph *out);
expm_status expm_batched_replay(expm_batch_graph graph, void *stream, expm_info *per_instance);
expm_status expm_batched_graph_info(expm_batch_graph graph, int *scheme, int *launch_groups, size_t *device_bytes,
                                    double ms_per_scheme[3]);
int expm_batched_graph_buckets(expm_batch_graph graph, int max, int *order, int *ninst, int *tile, double *ms_tile0,
                              double *ms_tile1);
expm_status expm_batched_graph_destroy(expm_batch_graph graph);

/*
 * Request server (no counterpart in the paper: a serving pattern around eq. expAx).
 * Operators are registered once and copied into server-owned device memory; requests
 * bring device buffers V (n x k, row-major, ld k; real or complex) and Y and are
 * executed asynchronously by `max_inflight` worker threads, each on its own CUDA
 * stream, as soon as a worker and enough of the HBM budget are free (continuous
 * batching: work of requests admitted at different times overlaps on the device).
 * Factorizations (tridiagonal block LUs and spikes; dense per-pair LUs) are cached per
 * (operator, plan, precision class, t, c), counted in the budget and evicted least
 * recently used; a request whose factorization is cached runs only its solve part.
 * Plans are told apart by an id that is never reused (a plan destroyed and another
 * created at the same address do not share factors); a factorization whose build
 * failed is dropped once unused, so the next request rebuilds it.  A worker thread that
 * has stopped between requests is restarted by the next submit or poll.
 * Each result depends only on its own inputs (deterministic kernels, no reduction
 * across requests), so it is the same alone and in the mix.
 *
 *   expm_server_create     hbm_budget_bytes: bound on solve scratch + cached factors
 *                          (operator copies are not counted); 1 <= max_inflight <= 64.
 *                          Uses the CUDA device current at creation.
 *   expm_server_register_op  desc: EXPM_OP_TRIDIAG (d, e, e_is_complex as in
 *                          expm_apply_tridiag; for complex e the phases phi and |e|
 *                          are formed once here and each request solves on D^H V,
 *                          with 16 n k more bytes of solve scratch) or EXPM_OP_DENSE
 *                          (A, lda, a_is_complex); the data may be host or device
 *                          memory and is copied.
 *   expm_server_submit     V and Y device memory (EXPM_EINVAL otherwise), valid until
 *                          poll reports the request finished, as is the plan; 1 <= k <= 64;
 *                          opts as for the matching apply call
 *                          (opts->stream is ignored).  EXPM_EAGAIN when the queue is
 *                          full, EXPM_ENOMEM when one request exceeds the whole budget,
 *                          EXPM_ENOTFOUND for an unknown operator.
 *   expm_server_poll       EXPM_EAGAIN while pending; otherwise the request's final
 *                          status, its info and timestamps ts = {submit, admit, start,
 *                          done} in seconds since server creation; the ticket is then
 *                          released (a second poll returns EXPM_ENOTFOUND).
 *   expm_server_destroy    drops queued requests, waits for running ones, frees all.
 */
typedef struct expm_server_s *expm_server;
enum { EXPM_OP_TRIDIAG = 1, EXPM_OP_DENSE = 2 };
typedef struct expm_op_desc {
    int kind;          /* EXPM_OP_TRIDIAG or EXPM_OP_DENSE             */
    int64_t n;         /* rows (tridiagonal N or dense order n)        */
    const double *d;   /* tridiagonal: diagonal (n doubles)            */
    const void *e;     /* tridiagonal: off-diagonal (n-1 entries)      */
    int e_is_complex;  /* tridiagonal: e complex (Hermitian T; Y complex) */
    const void *A;     /* dense: n x n, row-major                      */
    int lda;           /* dense: leading dimension (elements)          */
    int a_is_complex;  /* dense: complex Hermitian if nonzero          */
} expm_op_desc;

expm_status expm_server_create(size_t hbm_budget_bytes, int max_inflight, expm_server *out);
expm_status expm_server_register_op(expm_server server, const expm_op_desc *desc, uint64_t *op_id);
expm_status expm_server_submit(expm_server server, uint64_t op_id, const expm_plan plan, const void *V, int k,
                               int v_is_complex, void *Y, const expm_opts *opts, uint64_t *ticket);
expm_status expm_server_poll(expm_server server, uint64_t ticket, expm_info *info, double ts[4]);
expm_status expm_server_destroy(expm_server server);
/*   expm_server_set_queue_limit  at most max_queue requests wait for admission (default
 *                          2^16, 1 <= max_queue <= 2^20); a submit beyond it returns
 *                          EXPM_EAGAIN and queues nothing (the caller retries later). */
expm_status expm_server_set_queue_limit(expm_server server, int max_queue);

/*
 * Device-fed work queue of small dense evaluations (no counterpart in the paper: a
 * serving pattern around eq. expAx for problems too small to amortise a kernel launch).
 * Each request is Y = e^c R_n(tA - cI) V for one dense Hermitian A of order n <= 64,
 * evaluated as expm_apply_dense's one-launch small path does (the same device code,
 * compiled into another kernel: results agree with that call to rounding, and identical
 * requests give identical results).  Instead of a launch per request, a
 * persistent kernel of thread-block clusters (one cluster per request in flight, one CTA
 * per solved system) takes requests from a ring of `capacity` slots in mapped host
 * memory: submit writes a slot and publishes it, a cluster claims it, evaluates it and
 * publishes its completion, and poll reads that completion.  Every device-side wait is
 * bounded: when no request arrives for idle_ms the kernel exits with the exit status
 * EXPM_ETIMEOUT (expm_queue_state); the next submit or poll that finds it finished
 * launches it again, so no request is lost, and results only need polling to advance.
 *   expm_queue_create   plan (its poles and weights are copied: the plan may be destroyed
 *                       afterwards); a_is_complex: A complex Hermitian, else real
 *                       symmetric; k right-hand sides per request, complex iff
 *                       v_is_complex (real A with complex V solves 2k real columns);
 *                       at most 4 solved columns and 16 solved systems (degree/2 for
 *                       real A, degree for complex A); opts: precision (EXPM_FP64, or any
 *                       mixed precision: the binary32 inverse with binary64-residual
 *                       refinement), tol, max_refine, growth_max (t, shift_c and stream
 *                       are per request / unused); capacity 1..65536 slots; max_clusters
 *                       requests in flight at most (0: as many clusters as fit on the
 *                       device at once); idle_ms in (0, 600000]
 *   expm_queue_submit   n <= 64; A (n x n, ld lda), V and Y (n x k, ld ldv / ldy),
 *                       row-major, device memory that stays valid until the request is
 *                       polled complete; whatever writes A and V must have completed
 *                       before the call (the kernel may read them at once: it does not
 *                       follow stream order); t and shift_c of this request.  *ticket
 *                       identifies it.  EXPM_EAGAIN when `capacity` submitted requests
 *                       have not yet been polled complete (nothing is queued).
 *   expm_queue_poll     EXPM_EAGAIN while pending; then the request's status (EXPM_OK,
 *                       EXPM_EGROWTH, EXPM_ENOCONV as expm_apply_dense, Y written in all
 *                       three) with info filled, and the ticket is released (a second
 *                       poll returns EXPM_ENOTFOUND).
 *   expm_queue_state    running: the consumer kernel is on the device; last_exit:
 *                       EXPM_ETIMEOUT when its last run ended on an idle wait, else
 *                       EXPM_OK; launches: kernel launches so far; clusters: requests in
 *                       flight at most.
 *   expm_queue_destroy  sets the stop flag (clusters leave after the request they are
 *                       evaluating), waits for the kernel and frees everything; requests
 *                       not yet claimed are dropped.
 * The consumer kernel runs on the queue's own stream; a device-wide synchronisation
 * (cudaDeviceSynchronize, or a framework call that does one) waits for it, that is until
 * it has been idle for idle_ms: synchronise streams instead while a queue is live.
 */
typedef struct expm_queue_s *expm_queue;
expm_status expm_queue_create(expm_plan plan, int a_is_complex, int k, int v_is_complex, const expm_opts *opts,
                              int capacity, int max_clusters, double idle_ms, expm_queue *out);
expm_status expm_queue_submit(expm_queue queue, int n, const void *A, int lda, const void *V, int ldv, void *Y,
                              int ldy, double t, double shift_c, uint64_t *ticket);
expm_status expm_queue_poll(expm_queue queue, uint64_t ticket, expm_info *info);
expm_status expm_queue_state(expm_queue queue, int *running, int *last_exit, uint64_t *launches, int *clusters);
expm_status expm_queue_destroy(expm_queue queue);

/*
 * Measurement hooks (no counterpart in the paper).  When enabled on a plan, every
 * kernel launch made through that plan is bracketed by CUDA events recorded on the
 * launch stream; expm_profile_read synchronises on the recorded events and returns,
 * per kernel name, the number of launches and their summed device time since the
 * last reset.  Off by default; enabling it adds two event records per launch.
 *   expm_profile_enable   on = 1 enables, 0 disables; both reset the counters
 *   expm_profile_read     idx-th kernel seen (0-based, in first-launch order);
 *                         *name points to a static string.  EXPM_ENOTFOUND when
 *                         idx is past the last kernel.
 */
expm_status expm_profile_enable(expm_plan plan, int on);
expm_status expm_profile_read(expm_plan plan, int idx, const char **name, int64_t *launches,
                              double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* EXPM_H */
