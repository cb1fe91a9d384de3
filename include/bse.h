/*
 * bse.h -- C ABI of the GB300 (sm_103a) iterative Bethe-Salpeter eigensolver.
 *
 * The library computes the lowest excitation eigenpairs of the dense BSE
 * problem in both forms treated by the paper:
 *
 *   Tamm-Dancoff (TDA): A x = lambda x, A Hermitian N x N
 *       (the C = 0 case, Sec. 1 after Eq. 3);
 *   pseudo-Hermitian (PH): H z = omega z with
 *       H = [[A, B], [-conj(B), -conj(A)]]  (Eq. 1, optical case of Sec. 1:
 *       R = A Hermitian, C = B complex symmetric, anti-resonant block conj(A)),
 *       right eigenvectors z = (X; Y) normalised to z^H Omega z = 1 with
 *       Omega = diag(I, -I) (Eq. 2).
 *
 * The PH solve is a structure-preserving thick-restart Lanczos on the folded
 * operator (Sec. 2.2.1): it never forms the 2N x 2N matrix and works only with
 * the stored blocks A and B.  Every arithmetic step runs in CUDA kernels of
 * this library; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Complex matrices are interleaved (re, im) pairs, row-major, full N x N
 *     storage.  Only the upper triangle (i <= j) of A and B is read: A is taken
 *     as Hermitian (its diagonal's imaginary part is ignored) and B as
 *     symmetric.
 *   - Vectors and blocks of vectors are column-major with leading dimension N
 *     (TDA) or 2N (stacked PH vectors (X; Y)), complex, in the handle's dtype.
 *   - Every function returns a bse_status; no exception or abort crosses the
 *     ABI.  On an error the handle stays valid unless stated otherwise.
 *   - All device work of one handle runs on the CUDA stream given at creation;
 *     functions that return host data synchronise that stream.  A handle must
 *     not be used from two threads at once.
 */
#ifndef BSE_H_
#define BSE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bse_handle bse_handle;

typedef enum bse_status {
  BSE_OK = 0,
  BSE_EINVAL = 1,     /* invalid argument (size, pointer, enum, nev > N, ...)  */
  BSE_ENOMEM = 2,     /* device or host allocation failed                       */
  BSE_ENOTPD = 3,     /* M of Eq. 2 not positive definite (negative K-norm or   */
                      /* non-positive Ritz value omega^2 met by the iteration)  */
  BSE_ENOCONV = 4,    /* fewer than nev pairs passed the FP64 residual test;   */
                      /* every computed pair is still returned                */
  BSE_ETIMEOUT = 5,   /* a device-side iteration limit expired                  */
  BSE_ECUDA = 6,      /* a CUDA runtime call failed                             */
  BSE_ESTATE = 7,     /* call out of order (e.g. backward before a solve)       */
  BSE_ENOTFINITE = 8  /* NaN or Inf met in the Lanczos coefficients             */
} bse_status;

typedef enum bse_form { BSE_TDA = 0, BSE_PH = 1 } bse_form;

typedef enum bse_dtype {
  /* complex64 storage of A, B and of the Krylov basis; FP32 products;
     FP64 projected eigenproblem, Ritz coefficients, final residuals and
     Rayleigh-quotient refinement (the mixed-precision path) */
  BSE_C64 = 0,
  /* complex128 storage; FP64 products (the FP64 path) */
  BSE_C128 = 1,
  /* complex64 input and storage of A and B (half the bytes of BSE_C128);
     FP64 Krylov basis; the Lanczos products in double-FP32 arithmetic on
     the complex64 tiles (each stored value is exact in FP32), so the
     folded iteration is not limited by FP32 rounding -- the small tiles
     (tile_tau) with rounded A + B, A - B and fixed-point-grid sums; the
     Gram-Schmidt passes and the restart in double-FP32 on FP32 shadows of
     the basis (about 2^-44 relative); FP64 projected problem, residuals and
     Rayleigh quotients.  Eigenvectors are returned as complex64. */
  BSE_C64_MIXED = 2,
  /* complex128 input and storage, FP64 Krylov basis, projected problem and
     final residuals; the streaming Lanczos products in double-FP32
     arithmetic (error-free transformations on the FP32 pipes, 2^-48
     relative per term) on a split copy of the packed tiles.  Needs twice
     the packed storage of BSE_C128. */
  BSE_C128_DF = 3
} bse_dtype;

typedef enum bse_where { BSE_HOST = 0, BSE_DEVICE = 1 } bse_where;

typedef enum bse_which { BSE_LOWEST = 0 } bse_which;

/* Operators for bse_apply (all ignore the lower triangles of A and B). */
typedef enum bse_op {
  BSE_OP_A = 0,       /* Y = A X                                  (N rows)  */
  BSE_OP_MPLUS = 1,   /* Y = A X + B conj(X)   (real-linear half) (N rows)  */
  BSE_OP_MMINUS = 2,  /* Y = A X - B conj(X)                      (N rows)  */
  BSE_OP_H = 3        /* Y = H X, X and Y stacked (X1; X2), 2N rows         */
} bse_op;

/* Structure-preserving Lanczos variants for BSE_PH handles (Sec. 2.2.1 lists
   three variations of a structure-preserving thick-restart Lanczos).  All
   build the Krylov space of H from an even start vector (u; conj(u)), work
   only with the top halves of the basis (the lower blocks are implicit), use
   two structured products per step and return the same eigenpairs; they
   differ in the recurrence, its inner product and the projected problem:
     SHAO       the folded recurrence on M- M+ (M+- u = A u +- B conj(u)) in
                the inner product Re(x^H M+ y); projected matrix of omega^2
                (arrowhead + tridiagonal), solved by bisection and inverse
                iteration; omega recovered at the end;
     GRUNING    the Lanczos recurrence of H itself in the M inner product of
                Eq. 2, alternating even and odd vectors (two bases, two
                Gram-Schmidt passes per step); projected matrix with zero
                diagonal whose eigenvalues are +-omega directly;
     PROJECTED  the folded recurrence, with the projected problem written as
                a small BSE matrix [[A_k, B_k], [-B_k, -A_k]] (A_k, B_k real
                symmetric) and solved at every restart by the dense
                structure-preserving method of Sec. 2.1.1 on the GPU.
   TDA handles run the plain Hermitian Lanczos recurrence for every value. */
typedef enum bse_variant {
  BSE_VARIANT_SHAO = 0,
  BSE_VARIANT_GRUNING = 1,
  BSE_VARIANT_PROJECTED = 2
} bse_variant;

/* Solver options.  Zero-initialise and set what you need; zero fields take
   the defaults given in brackets. */
typedef struct bse_solve_opts {
  int ncv;            /* Krylov subspace size m [max(2 nev, nev + 32)];
                         raised to nev + 1, then capped at the smallest N
                         of the handle (and at 1024)                          */
  int maxit;          /* limit on Krylov steps [20000]                        */
  uint64_t seed;      /* start vector seed [12345]                            */
  const void* v0;     /* optional device start vector: N complex values in
                         the Krylov-basis precision (complex64 for BSE_C64,
                         complex128 for the other dtypes); single-problem
                         handles only; NULL = counter-based random start      */
  double lock_tol;    /* Ritz-estimate tolerance used for locking, relative
                         to the Ritz value [tol / 4]                          */
  int stream_launches; /* 0: the Krylov steps of a restart cycle are replayed
                         as CUDA graphs of 1, 2, 4, ... steps, captured once
                         per handle and subspace size -- or, for a single
                         problem of N <= 6144 on the folded (Shao) or TDA
                         recurrence with BSE_C128 or BSE_C64, run as one
                         persistent cooperative launch per restart cycle
                         (phases separated by a bounded grid barrier; the
                         same results bit for bit); 1: every kernel is
                         launched on the stream one by one; 2: graphs, never
                         the persistent launch [0]                            */
  double tile_tau;    /* BSE_C64_MIXED with B only: a packed tile whose bound
                         on |A + B|, |A - B| (per component) is at most
                         tile_tau times the largest tile bound of its problem
                         is "coarse": its U = A + s B, V = A - s B are rounded
                         to FP32 (a fixed perturbation of <= 2^-24 |U| per
                         entry) and its products accumulated on a fixed-point
                         grid (about 2^-35 of the tile's scale); the others
                         get exact double-FP32 products.  Negative: every
                         tile exact.  [min(2^-7, tol 2^24 / (16 sqrt(N)))].
                         If a solve with coarse tiles leaves a pair above tol
                         on the FP64 residual check before maxit, it is
                         repeated with every tile exact (retried_exact).      */
  int variant;        /* bse_variant; values outside it: BSE_EINVAL [SHAO]    */
} bse_solve_opts;

/* Per-solve counters, filled by bse_get_stats after a solve. */
typedef struct bse_stats {
  int64_t steps;         /* Krylov steps (one new basis vector each)          */
  int64_t passes;        /* structured products over the stored A (and B)     */
  int64_t restarts;      /* thick restarts                                    */
  int nconv;             /* converged eigenpairs                              */
  double max_residual;   /* max FP64 relative residual of returned pairs      */
  double ms_total;       /* device time of the last solve (CUDA events)       */
  double ms_product;     /* device time inside the structured products        */
  int64_t launches;      /* CUDA kernels launched by the last solve           */
  int shape_ctas_per_sm; /* launch shape the product tuner chose: CTAs per SM
                            (0 = as many as fit, -1 = one CTA per tile)       */
  int shape_strided;     /* 1: each CTA takes every grid-th tile job; 0: a
                            contiguous run                                    */
  int tuned;             /* 1 once the shape was chosen by timing (bse_solve
                            times the candidates on its own first products)   */
  int64_t tiles_fine;    /* packed tiles per product on the exact path        */
  int64_t tiles_coarse;  /* mixed path: tiles with rounded U, V (tile_tau)    */
  int retried_exact;     /* 1 if the last solve was repeated with every tile
                            exact after its FP64 residual check failed        */
} bse_stats;

/* Human-readable message for a status code (static storage). */
const char* bse_strerror(int status);

/*
 * bse_create -- copy and repack A (and B) into the library's device storage.
 *
 *   N       order of A and B, 1 <= N <= 2^31 - 1
 *   A, B    full N x N row-major complex matrices in the precision of dtype
 *           (complex64 for BSE_C64/BSE_C64_MIXED, complex128 for BSE_C128),
 *           on the host or the device as `where` says.  B is ignored for
 *           BSE_TDA and may be NULL there; it is required for BSE_PH.
 *   form    BSE_TDA or BSE_PH
 *   stream  cudaStream_t (NULL = legacy default stream)
 *   out     receives the handle
 *
 * Ownership: the library copies A and B into packed upper-triangle tiles in
 * its own device memory (about N^2 * elem_size bytes for A and B together;
 * BSE_C64_MIXED pseudo-Hermitian handles also keep fl(A + B) and fl(A - B)
 * in the same layout, twice that; BSE_C128_DF keeps a split copy, three times);
 * the caller may free its buffers as soon as the call returns.  The handle
 * owns all its device memory and releases it in bse_destroy.
 * Paper: the redistribution of Sec. 2.1.2 / 2.2.2 from the application's
 * layout into the solver's layout, here onto one GPU.
 */
int bse_create(int64_t N, const void* A, const void* B, int form, int dtype,
               int where, void* stream, bse_handle** out);

/*
 * bse_create_batched -- one handle for `count` independent problems of
 * uneven orders N[i] (same form and dtype), solved together by
 * bse_solve_batched in lock-step launches.  A[i], B[i] as in bse_create.
 */
int bse_create_batched(int count, const int64_t* N, const void* const* A,
                       const void* const* B, int form, int dtype, int where,
                       void* stream, bse_handle** out);

/*
 * bse_solve -- lowest `nev` eigenpairs (BSE_LOWEST: smallest positive omega
 * for PH, smallest lambda for TDA, ascending).
 *
 *   tol        relative residual target ||H z - omega z|| <= tol |omega| ||z||
 *              (TDA: ||A x - lambda x|| <= tol |lambda| ||x||), e.g. 1e-12
 *              for BSE_C128 and 1e-6 for BSE_C64
 *   eval_out   host array of nev doubles (eigenvalues, FP64 Rayleigh
 *              quotients of the returned vectors)
 *   evec_out   device array or NULL: TDA N x nev, PH 2N x nev (stacked
 *              (X; Y), Omega-normalised), column-major, handle dtype
 *   nconv_out  host int or NULL: number of converged pairs
 *
 * The eigenvectors stay in the handle for bse_backward.  Method: the
 * structure-preserving thick-restart Lanczos of Sec. 2.2.1 (spectrum folding
 * for PH), eigenvector recovery and the partner relations of Eq. 7.
 *
 * Convergence: the iteration locks a pair once its Ritz estimate is below
 * lock_tol; after the recovery every returned pair gets an FP64 residual
 * ||H z - rho z|| / (|rho| ||z||) with the FP64 Rayleigh quotient rho
 * (bse_get_residuals), and only pairs whose residual is <= tol count in
 * *nconv_out.  Returns BSE_ENOCONV if fewer than nev pairs pass that test
 * (maxit reached, or storage/product rounding above tol, e.g. BSE_C64 with a
 * tol near its FP32 floor); eval_out and evec_out still receive every pair
 * that was computed (NaN eigenvalues beyond them).  BSE_EINVAL unless
 * 1 <= nev <= N.
 */
int bse_solve(bse_handle* h, int nev, double tol, int which, double* eval_out,
              void* evec_out, int* nconv_out);

/* bse_solve with options (opts may be NULL). */
int bse_solve_ex(bse_handle* h, int nev, double tol, int which,
                 const bse_solve_opts* opts, double* eval_out, void* evec_out,
                 int* nconv_out);

/*
 * bse_solve_batched -- solve every problem of a batched handle.
 *   eval_out   host, count * nev doubles (problem-major)
 *   evec_out   host array of `count` device pointers (each as in bse_solve)
 *              or NULL
 *   nconv_out  host, count ints, or NULL
 */
int bse_solve_batched(bse_handle* h, int nev, double tol, int which,
                      const bse_solve_opts* opts, double* eval_out,
                      void* const* evec_out, int* nconv_out);

/*
 * bse_backward -- Hellmann-Feynman adjoint of the last solve.
 *
 * Given g = dL/dlambda (nev doubles, host or device as `where` says),
 * writes the full N x N gradients (row-major, handle dtype, device memory):
 *   TDA: dA = X diag(g) X^H
 *   PH : dA = X diag(g) X^H + conj(Y diag(g) Y^H)      (Hermitian)
 *        dB = X diag(g) Y^H + (X diag(g) Y^H)^T         (symmetric)
 * from d omega = z^H Omega dH z with the left eigenvector Omega z (Eq. 7).
 * Convention (PyTorch's): dL = Re<dA, E_A> + Re<dB, E_B> for Hermitian E_A
 * and symmetric E_B, <G, E> = sum conj(G_ij) E_ij.  dB must be NULL for TDA.
 * Degenerate eigenvalues need a loss symmetric over each degenerate group.
 * Returns BSE_ESTATE if no solve has completed on h.
 */
int bse_backward(bse_handle* h, const double* dL_dlambda, int where, void* dA,
                 void* dB);

/* Implementation choice for bse_backward_ex. */
typedef enum bse_impl {
  BSE_IMPL_AUTO = 0,          /* tensor cores for complex64 outputs, else CUDA cores */
  BSE_IMPL_CUDA_CORES = 1,    /* SIMT FMA kernel (FP64 for complex128, FP32 for complex64) */
  BSE_IMPL_TENSOR_CORES = 2   /* tcgen05 3xTF32 rank-2k update; complex64 outputs only */
} bse_impl;

/* bse_backward with an explicit implementation (impl from bse_impl).  The
   tensor-core path computes dA, dB as real GEMMs of the stacked eigenvector
   panels with TF32 hi/lo splits (about FP32 accuracy) and FP32 accumulation
   in tensor memory; it returns BSE_EINVAL for complex128 handles and
   BSE_ETIMEOUT if a bounded device-side wait expired. */
int bse_backward_ex(bse_handle* h, const double* dL_dlambda, int where, void* dA,
                    void* dB, int impl);

/*
 * bse_apply -- one structured product on device blocks of k columns.
 *   X, Y   device, column-major, handle dtype; N rows (BSE_OP_A/MPLUS/MMINUS)
 *          or 2N rows (BSE_OP_H); X and Y must not overlap.
 * Each stored tile of A and B is read once per call and serves both block
 * rows (A = A^H, B = B^T).  Only for single-problem handles.
 */
int bse_apply(bse_handle* h, int op, int k, const void* X, void* Y);

/*
 * bse_solve_dense -- the nev lowest positive eigenpairs of a single-problem
 * pseudo-Hermitian handle by dense, structure-preserving diagonalisation
 * (Sec. 2.1.1, Eqs. 4-6: M_r of Eq. 5, its Cholesky factor L, the real
 * skew-symmetric W = L^T J L, Householder reduction of W to skew-tridiagonal
 * form, bisection and inverse iteration on the equivalent real symmetric
 * tridiagonal matrix, back-transformation and z = Q L^{-T} q).  The direct
 * method of the paper for the regime where a large share of the spectrum is
 * wanted; O(N^3) work, FP64 throughout whatever the storage dtype.
 *   tol        a pair counts in *nconv_out if its FP64 relative residual is
 *              <= tol (as in bse_solve; e.g. 1e-10)
 *   eval_out   host, nev doubles (FP64 Rayleigh quotients, ascending)
 *   evec_out   device or NULL: 2N x nev, column-major, handle dtype,
 *              Omega-normalised
 * Allocates about 2 (2N)^2 doubles of scratch for the call.  BSE_ENOTPD if
 * M_r is not positive definite, BSE_ENOCONV if fewer than nev pairs pass
 * the residual test, BSE_EINVAL for TDA or batched handles.  The
 * eigenvectors stay in the handle for bse_backward.
 */
int bse_solve_dense(bse_handle* h, int nev, double tol, double* eval_out, void* evec_out, int* nconv_out);

/*
 * bse_apply_mixed -- the mixed path's Lanczos product on one vector:
 *   y = A x + B conj(x)   (op BSE_OP_MPLUS)
 *   y = A x - B conj(x)   (op BSE_OP_MMINUS)
 * for a BSE_C64_MIXED pseudo-Hermitian handle, with x and y device arrays of
 * N complex128 values (the precision of that path's Krylov basis).  Tiles are
 * split into exact and coarse ones as in a solve (bse_solve_opts.tile_tau):
 * tile_tau > 0 sets the threshold, tile_tau < 0 makes every tile exact, 0
 * takes the default of a solve at tol = 1e-6.  bse_get_stats then reports
 * tiles_fine / tiles_coarse.  Same real form of Eq. 5 as the solver's
 * product; BSE_EINVAL for other handles or ops.
 */
int bse_apply_mixed(bse_handle* h, int op, double tile_tau, const void* X, void* Y);

/*
 * bse_apply_noalloc -- one structured product that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library call cudaMalloc -- a process whose device memory is
 * all reserved up front by its own pool allocator, or a latency-bound loop in
 * which a cudaMalloc (it may synchronise the device) is not acceptable.  It
 * needs no handle and reads the caller's matrices directly:
 *
 *   y = A x                (op BSE_OP_A)
 *   y = A x + B conj(x)    (op BSE_OP_MPLUS)
 *   y = A x - B conj(x)    (op BSE_OP_MMINUS)
 *
 *   N       1 <= N <= BSE_NOALLOC_MAX_N (4096); larger N returns BSE_EINVAL
 *   A, B    device, full N x N row-major, complex64 (dtype BSE_C64, FP32
 *           products) or complex128 (BSE_C128, FP64 products); only the upper
 *           triangles are read (A Hermitian, B symmetric); B may be NULL for
 *           BSE_OP_A.  Other dtypes return BSE_EINVAL.
 *   x, y    device, N complex entries each, same dtype; must not overlap
 *   stream  cudaStream_t (NULL = legacy default stream); the call is
 *           asynchronous on it
 *
 * Its only scratch is a fixed 2 MiB array in the library's device image
 * (every GPU that loads the library holds it until the process exits).  The
 * first call on a device looks up that array's address with the device
 * current and caches it for the process; make that first call before any
 * stream capture, and do not use this entry point across cudaDeviceReset.
 * All calls share the array: calls that overlap on the GPU (other streams or
 * threads) race.  Returns BSE_EINVAL for bad arguments, BSE_ECUDA if a launch
 * fails or a CUDA error from earlier work is pending (that error is left for
 * the caller to read).
 */
#define BSE_NOALLOC_MAX_N 4096
int bse_apply_noalloc(int64_t N, const void* A, const void* B, int dtype, int op,
                      const void* x, void* y, void* stream);

/*
 * bse_haydock -- optical absorption spectrum by the Lanczos-Haydock
 * recurrence (Sec. 2.2: the iterative route that gives the spectrum from
 * Lanczos coefficients and continued fractions, without eigenpairs).
 *
 * With z = omega + i eta the response is
 *   TDA: F(z) = d^H (z - A)^{-1} d,
 *   PH:  F(z) = D^H Omega (z - H)^{-1} D,  D = (d; sign conj(d)),
 * and spectrum_out[i] = -Im F(omega[i] + i eta) / pi (>= 0 for omega > 0).
 * TDA runs m steps of the three-term Lanczos recurrence on A from d/|d| and
 * returns |d|^2 CF(z); PH runs it on the folded operator M+ M- (sign = -1)
 * or M- M+ (sign = +1), self-adjoint in <x, y> = Re(x^H M-/+ y), and returns
 * 2 <d, d> CF(z^2), with M+ u = A u + B conj(u), M- w = A w - B conj(w).
 * There is no re-orthogonalisation: the recurrence is the method, and its
 * continued fraction converges to F as m grows (for m of order 2N it agrees
 * with the dense resolvent to rounding).  Each step costs one (TDA) or two
 * (PH) structured products; the steps replay as a CUDA graph.
 *
 *   d             N complex128 values (host or device, per `where`),
 *                 whatever the handle's dtype
 *   m             Lanczos steps, 1 <= m <= 10^6 (fewer if the Krylov space
 *                 becomes invariant: *steps_out says how many)
 *   sign          -1 or +1 (PH only; ignored for TDA)
 *   nw, omega     host array of nw >= 1 real frequencies
 *   eta           broadening, > 0
 *   spectrum_out  host, nw doubles
 *   response_out  host, 2 nw doubles (Re F, Im F interleaved) or NULL
 *   coef_out      host, 2 m + 1 doubles or NULL: alpha_0..alpha_{m-1},
 *                 beta_0..beta_{m-1} (beta_j couples steps j and j+1; zero
 *                 beyond *steps_out), then <d, d>
 *   steps_out     host int or NULL
 * Single-problem handles only.  The library allocates and frees its own
 * scratch (6 vectors of N).  BSE_EINVAL for bad arguments, BSE_ENOTPD if
 * <d, d> (|d|^2, or Re(d^H M-/+ d)) is not positive, BSE_ECUDA on CUDA
 * errors.  bse_get_stats afterwards reports steps, passes, time, launches.
 */
int bse_haydock(bse_handle* h, const void* d, int where, int m, int sign,
                int nw, const double* omega, double eta, double* spectrum_out,
                double* response_out, double* coef_out, int* steps_out);

/*
 * bse_selftest_bounded_wait -- exercise the failure path of the device-side
 * waits (no handle needed).  Every wait of this library's kernels on an
 * mbarrier (tensor-core pipelines) polls a bounded number of times; on expiry
 * the kernel records an error, releases what it holds and returns, and the
 * call reports BSE_ETIMEOUT, leaving the CUDA context usable.  This launches
 * one such wait on the current device: arrive = 0 waits on a barrier that
 * nothing completes (*expired = 1 after about 10^6 polls), arrive = 1 completes
 * it first (*expired = 0).  Returns BSE_EINVAL for bad arguments, BSE_ECUDA on
 * a CUDA error.  The paper has no counterpart; it is a test of this build.
 */
int bse_selftest_bounded_wait(int arrive, int* expired);

/* FP64 relative residuals ||H z - rho z|| / (|rho| ||z||) of the pairs the
   last solve returned for problem `problem` (0 for single-problem handles), in
   output order: res_out[c] for c < n (NaN beyond the computed pairs).
   BSE_ESTATE before the first solve, BSE_EINVAL for bad arguments. */
int bse_get_residuals(const bse_handle* h, int problem, double* res_out, int n);

/*
 * bse_measure_fp64_peak -- FP64 FMA throughput of the current device, for the
 * roofline of the FP64 path (whose structured product is bound by the FP64
 * pipe on this GPU).  One launch of `iters` iterations of 8 independent FMA
 * chains per thread on every SM, timed with CUDA events after a warm-up;
 * *tflops_out = 2 x FMAs / time.  The paper has no counterpart.  Allocates a
 * small output buffer; BSE_EINVAL for iters outside [1, 2^24].
 */
int bse_measure_fp64_peak(int iters, double* tflops_out, double* ms_out);

/* Counters of the last solve or spectrum (single-problem handles; for
   batched handles the sums over problems). */
int bse_get_stats(const bse_handle* h, bse_stats* out);

/* Release every resource of the handle (synchronises its stream). */
int bse_destroy(bse_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* BSE_H_ */
