// Internal declarations shared by the translation units of libbse.
//
// Storage layout in HBM (one problem):
//   * A and B as packed upper-triangle tiles of TS x TS complex elements,
//     tile (I, J), I <= J, in row-major order over the triangle, each tile
//     row-major; diagonal tiles hold both halves (Hermitian / symmetric
//     completion); rows and columns beyond N are zero.
//   * vectors as Npad = nT * TS complex entries (zero padded); blocks of
//     vectors column-major with leading dimension Npad.
//   * the Lanczos basis V and its image P = M+ V (PH) as Npad x (ncv + 1),
//     columns [0, ncv] the Krylov basis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bse {

constexpr int TS = 128;            // tile edge of the packed storage
constexpr int PROD_THREADS = 256;  // 16 x 16 threads per tile
constexpr int ROWBLK = 2048;       // rows per CTA in the tall-skinny reductions
constexpr int MAXM = 1024;         // largest Krylov subspace supported

// ---------------------------------------------------------------- complex
template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

__host__ __device__ inline double2 mk(double x, double y) { return make_double2(x, y); }
__host__ __device__ inline float2 mk(float x, float y) { return make_float2(x, y); }

template <typename T> __host__ __device__ inline T czero();
template <> __host__ __device__ inline float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ inline double2 czero<double2>() { return make_double2(0.0, 0.0); }

// y += a * x
__host__ __device__ inline void cfma(double2& y, double2 a, double2 x) {
  y.x = fma(a.x, x.x, y.x); y.x = fma(-a.y, x.y, y.x);
  y.y = fma(a.x, x.y, y.y); y.y = fma(a.y, x.x, y.y);
}
__host__ __device__ inline void cfma(float2& y, float2 a, float2 x) {
  y.x = fmaf(a.x, x.x, y.x); y.x = fmaf(-a.y, x.y, y.x);
  y.y = fmaf(a.x, x.y, y.y); y.y = fmaf(a.y, x.x, y.y);
}
// y += conj(a) * x
__host__ __device__ inline void cfmac(double2& y, double2 a, double2 x) {
  y.x = fma(a.x, x.x, y.x); y.x = fma(a.y, x.y, y.x);
  y.y = fma(a.x, x.y, y.y); y.y = fma(-a.y, x.x, y.y);
}
__host__ __device__ inline void cfmac(float2& y, float2 a, float2 x) {
  y.x = fmaf(a.x, x.x, y.x); y.x = fmaf(a.y, x.y, y.x);
  y.y = fmaf(a.x, x.y, y.y); y.y = fmaf(-a.y, x.x, y.y);
}
template <typename T> __host__ __device__ inline T conjc(T a) { a.y = -a.y; return a; }
template <typename T> __host__ __device__ inline T cadd(T a, T b) { a.x += b.x; a.y += b.y; return a; }
template <typename T> __host__ __device__ inline T csub(T a, T b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T, typename R> __host__ __device__ inline T cscale(T a, R s) { a.x *= s; a.y *= s; return a; }

struct alignas(32) D4 { double x, y, z, w; };

// FP64 complex -> {re_hi, im_hi, re_lo, im_lo}: hi = fl32(v), lo = fl32(v - hi) (48 bits of v)
__host__ __device__ inline float4 dsplit(double2 v) {
  const float xh = (float)v.x, yh = (float)v.y;
  return make_float4(xh, yh, (float)(v.x - (double)xh), (float)(v.y - (double)yh));
}

template <typename To, typename From> __host__ __device__ inline To ccvt(From a) {
  To r; r.x = a.x; r.y = a.y; return r;
}

// ---------------------------------------------------------------- state
enum Status : int {
  ST_OK = 0, ST_NOTPD = 3, ST_NOCONV = 4, ST_TIMEOUT = 5, ST_NOTFINITE = 8,
};

// Dynamic Krylov state of one problem, device resident.
struct KState {
  int k;        // locked Ritz vectors: columns [0, k)
  int l;        // kept (locked + arrow) vectors: columns [0, l)
  int j;        // index of the newest basis vector
  int m;        // ncv
  int nev;
  int status;   // Status
  int done;     // 1 when k >= nev (or stopped)
  int breakdown;
  // pending restart decision (written by k_lock_decide, consumed by restart kernels)
  int r_k0, r_nl, r_nkeep, r_pkeep;
  int r_go;     // 1 between a restart decision and its commit (active problems only)
  long long steps, passes, restarts, maxit;
  double tol, lock_tol;
  double beta_last;   // beta_{m-1}: coupling of the last vector to V[:, m]
  double theta_scale; // max |theta| over the kept vectors [k, l) (scale of the breakdown test)
};

// Structure-preserving Lanczos variants of the pseudo-Hermitian iteration
// (Sec. 2.2.1 names three): VAR_SHAO, the folded recurrence on M- M+ in the
// M+ inner product; VAR_GRUNING, the Lanczos recurrence of H itself in the
// M inner product (even and odd basis vectors, projected matrix with a zero
// diagonal, eigenvalues +-omega); VAR_PROJECTED, the folded recurrence with
// the projected problem written as a small BSE matrix and solved by the
// dense structure-preserving method of Sec. 2.1.1.
enum Variant : int { VAR_SHAO = 0, VAR_GRUNING = 1, VAR_PROJECTED = 2 };

// Static description of one problem (device resident, read-only in kernels).
struct Prob {
  int64_t N;
  int nT;
  int64_t Npad;       // nT * TS
  int ph;             // 1 for the pseudo-Hermitian form
  int ncv;
  int ncol;           // stride of the CGS partial sums and coefficients: 2 ncv + 1
                      // (PH: ncv + 1 K-inner products and ncv + 1 twin coefficients)
  const void* A;      // packed tiles
  const void* B;      // packed tiles (PH) or null
  void* V;            // Npad x (ncv + 1)
  void* P;            // Npad x (ncv + 1) (PH)
  void* V2;           // Npad x ncv restart scratch
  void* P2;
  void* w;            // Npad work vectors
  void* pw;
  void* part;         // product partials nT * nT * TS * KMAXP (compute type)
  double* cpart;      // CGS / norm partials: nrb * ncol complex
  double* coef;       // 2 * ncol complex (pass 1, pass 2)
  double* theta;      // [ncv + 1] Ritz values of kept vectors
  double* barrow;     // [ncv + 1] arrow couplings
  double* alpha;      // [ncv + 1]
  double* beta;       // [ncv + 1] beta[t] couples t and t+1
  double* ritz;       // [ncv] Ritz values of the active block
  double* rest;       // [ncv] Ritz estimates
  double* S;          // ncv x ncv, column-major, ld ncv
  int nrb;            // row blocks of the tall-skinny reductions
  KState* st;
  // complex128 path with double-FP32 products: the packed tiles split into
  // (hi, lo) float pairs, float4 {re_hi, im_hi, re_lo, im_lo} per element
  const void* Ahl;
  const void* Bhl;
  // complex64 PH handles on the mixed path: per tile, an upper bound on every
  // |U|, |V| component (U, V = A +- B), indexed like the packed tiles
  const float* tmax;
  const void* UV;     // mixed PH path: per packed element {U_re, V_re, U_im, V_im}, U = fl(A + B),
                      // V = fl(A - B) (float4, laid out like the packed tiles)
  void* xs;           // mixed PH path: the pre-split vector of a product, Npad x 16 B
  float* xmax;        // ... and the max |hi part| of each 128-entry chunk [nT]
  int variant;        // Variant (PH handles; TDA runs the plain Lanczos recurrence)
  // VAR_GRUNING: the odd basis W (tops of the odd vectors (w; -conj(w))), Npad x ncv,
  // its image Z = M- W, their restart scratch, the projected tree of H (jw: four arrays
  // of jwld entries -- leaf values, leaf couplings, hub/tail diagonal, tail couplings --
  // then its Ritz vectors, jwld x ncv), and the odd-side Ritz coefficients S2 (ncv x ncv)
  void* W;
  void* Z;
  void* W2;
  void* Z2;
  double* jw;
  int jwld;           // 2 ncv + 2
  double* S2;
  // mixed PH path: double-FP32 shadows {re_hi, im_hi, re_lo, im_lo} of the FP64 basis V, P
  // (Npad x (ncv + 1)) and of the work vector w, kept in step with them, so that the
  // Gram-Schmidt passes run on the FP32 pipes (null elsewhere)
  float4* Vs;
  float4* Ps;
  float4* ws;
};

// Jobs of the tiled product: problem, tile row I, tile column J, tile index.
struct TileJob { int prob, I, J, t; };

// Product modes (which vectors feed the product and where the result goes).
enum ProdMode : int {
  PM_STEP_MMINUS = 0,  // w  = A p_j - B conj(p_j)    (PH step, first pass)
  PM_STEP_MPLUS = 1,   // pw = A w + B conj(w)         (PH step, second pass)
  PM_STEP_A = 2,       // w  = A v_j                   (TDA step)
  PM_START_MPLUS = 3,  // pw = A w + B conj(w) at start / new-vector time
  PM_GENERIC = 4,      // Y = A XA + sB B XB, explicit blocks (K columns)
  PM_STEP_MMINUS_W = 5,  // pw = A w - B conj(w)      (Gruning step, odd half)
};

struct GenericIO {     // explicit operands for PM_GENERIC (single problem)
  const void* xa; const void* xb;  // Npad x K blocks (compute type) ; xb may be null -> conj(xa)
  int ldx;
  double sB;           // sign of the B term (0 disables it)
  void* y; int ldy;    // output (compute type) Npad x K
};

// Kernel launches issued by this process (reported per solve in bse_stats).
inline long long& launch_counter() {
  static long long c = 0;
  return c;
}
inline void count_launch(int n = 1) { launch_counter() += n; }

// ---------------------------------------------------------------- launchers
// packing (k_product.cu): tiles (I, J >= I) of block row I from TS rows
template <typename TIn, typename TSt>
void launch_pack_row(const TIn* rows, int64_t N, int nT, int I, int herm, TSt* dst, cudaStream_t s);

// Launch shape of the streaming product, chosen per handle by measurement
// (bse_api.cu): CTAs per SM (0 = as many as fit, -1 = one CTA per tile) and
// the walk of a CTA over the job list (0 = one contiguous run, 1 = every
// gridDim.x-th job, which keeps the load even when some problems of a batch
// have finished and their jobs are skipped).
struct ProdShape {
  int ctas_per_sm;
  int strided;
};

// complex128 PH storage: tiles of A and B become P = A + B and Q = A - B (k_product.cu)
void launch_pq_combine(double2* a, double2* b, int64_t n, cudaStream_t s);
// packing of device-resident full matrices in one launch (k_product.cu)
template <typename TIn, typename TSt>
void launch_pack_all(const TIn* src, int64_t N, int nT, int herm, TSt* dst, cudaStream_t s);
void launch_pack_pq(const double2* A, const double2* B, int64_t N, int nT, double2* P, double2* Q, cudaStream_t s);

// products (k_product.cu); ST = storage complex type, R = compute real type
template <typename ST, typename R>
void launch_product(const Prob* dprobs, const TileJob* jobs, int njobs, int nprob, int maxnT,
                    int mode, int K, const GenericIO* io_host, bool hasB, ProdShape shape, cudaStream_t s);
// resident CTAs per SM of the tile kernel launch_product / launch_product_df would use
template <typename ST, typename R>
int product_occupancy(bool hasB);
int product_df_occupancy(bool hasB, bool split);
// grid of the tile kernels for a shape, given their occupancy
int product_grid(int occ, ProdShape shape, int njobs);
template <typename ST, typename R>
void launch_rowblock(const Prob* dprobs, int prob, int nT, const void* xa, const void* xb, int ldx,
                     double sB, void* y, int ldy, int K, bool hasB, cudaStream_t s);
// complex128 products in double-FP32 arithmetic on the split tiles (k_product.cu)
// split = true: float4 split complex128 tiles; false: complex64 tiles (exact in FP32)
void launch_product_df(const Prob* dprobs, const TileJob* jobs, int njobs, int nprob, int maxnT,
                       int mode, const GenericIO* io_host, bool hasB, bool split, ProdShape shape,
                       cudaStream_t s);
void launch_split_tiles(const double2* packed, int64_t nelem, float4* split, cudaStream_t s);
// mixed path (complex64 PH tiles, FP64 vectors): exact double-FP32 products on the
// "fine" tiles (k_prod_tiles_df2), fixed-point-grid accumulation with rounded U, V on
// the "coarse" ones (k_prod_tiles_mx), then the FP64 reduction (k_product_df.cu)
void launch_product_mixed(const Prob* dprobs, const TileJob* fine, int nfine, const TileJob* coarse, int ncoarse,
                          int nprob, int maxnT, int mode, const GenericIO* io_host, ProdShape shape, int* err,
                          cudaStream_t s);
int product_mx_occupancy();
// {U_re, V_re, U_im, V_im} records of U = fl(A + B), V = fl(A - B) (k_product_df.cu)
void launch_uv_pack(const float2* A, const float2* B, int64_t nelem, float4* uv, cudaStream_t s);
// per-tile bound max(|A_re| + |B_re|, |A_im| + |B_im|) of complex64 tiles (k_product_df.cu)
void launch_tile_bound(const float2* A, const float2* B, int64_t ntiles, float* out, cudaStream_t s);
// sums the float4 (hi, lo) partial-sum slots of the double-FP32 kernels in FP64 (k_product.cu)
void launch_prod_reduce_d(const Prob* dprobs, int nprob, int maxnT, int mode, GenericIO io, cudaStream_t s);

// bounded-wait self-test (k_adjoint_tc.cu): 0 on success, -1 on a CUDA error
int selftest_bounded_wait(int arrive, int* expired_host);

// Lanczos-Haydock spectrum (k_haydock.cu); device-resident recurrence state
struct HdState {
  int j;        // current step
  int m;        // step limit
  int done;     // the Krylov space became invariant (or <d, d>_K was not positive)
  int nsteps;   // valid coefficients: alpha[0, nsteps), beta[0, nsteps - 1)
  double n2;    // <d, d>_K (TDA: |d|^2)
};
int haydock_partials();   // length of the partial-sum array of launch_hd_dot
template <typename ST>
void launch_hd_dot(const ST* x, const ST* y, int64_t n, double* partial, cudaStream_t s);
void launch_hd_scalar(HdState* st, const double* partial, double* alpha, double* beta, int which, cudaStream_t s);
template <typename ST>
void launch_hd_axpy(const HdState* st, const double* alpha, const double* beta, const ST* w, const ST* q,
                    const ST* qprev, ST* r, int64_t n, cudaStream_t s);
template <typename ST>
void launch_hd_scale(const HdState* st, const double* beta, const ST* r, const ST* pr, ST* q, ST* qprev, ST* p,
                     int64_t n, int init, cudaStream_t s);
template <typename ST>
void launch_hd_load(const double2* d, int64_t N, int64_t Npad, ST* x, cudaStream_t s);
void launch_hd_cf(const HdState* st, const double* alpha, const double* beta, int nw, const double* omega,
                  double eta, int ph, double* out, cudaStream_t s);

// tensor-core adjoint for complex64 outputs (k_adjoint_tc.cu); tiles128 lists
// the 128 x 128 output tiles (I <= J).  Returns 0, 1 (device wait expired), -1 (CUDA error).
size_t adjoint_tc_panel_bytes(int64_t N, int k, int ph);
int launch_adjoint_tc(const double2* Z, int64_t ldz, int64_t Npad, int64_t N, int k, const double* g, int ph,
                      const int2* tiles128, int64_t ntiles, float* panels, int* derr, float2* dA, float2* dB,
                      cudaStream_t s);

// persistent Krylov steps for one small problem (k_persist.cu): up to `steps` steps of the
// folded (ph) or TDA recurrence in one cooperative launch whose phases meet at a bounded grid
// barrier.  Returns 0 (launched), 1 (not available: no cooperative launch; the caller uses the
// per-phase kernels) or -1 (CUDA error).  A barrier wait that expires sets gb->err.
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};
template <typename ST, typename R>
int launch_steps_persist(const Prob* dprobs, const TileJob* jobs, int njobs, bool ph, int steps, GridBar* gb,
                         cudaStream_t s);

// dense structure-preserving diagonalisation (k_dense.cu): the nev lowest positive omega of
// problem 0 of a PH handle and their right eigenvectors in Z (ld 2 Npad); returns 0, 1 (M_r not
// positive definite) or -1 (CUDA error); `work` holds dense_scratch_doubles(N, nev) doubles
size_t dense_scratch_doubles(int64_t N, int nev);
int dense_shao(const Prob* dprobs, int64_t N, int64_t Npad, bool tiles64, bool pq, int nev, double* work,
               int* dflag, double2* Z, double* lam_out, cudaStream_t s);

// Krylov kernels (k_krylov.cu); launch_restart's df: the restart GEMM of an FP64 basis in
// double-FP32 arithmetic (the mixed path).  `half` selects the vectors of a Gram-Schmidt pass or a
// normalisation: 0 the folded (or TDA) step, 1 the odd half of a Gruning step (against W
// and the twins i V), 2 its even half and its fresh vectors (against V and the twins i W)
template <typename ST>
void launch_step_cgs(const Prob* dprobs, int nprob, int ph, int maxnrb, int64_t maxNpad,
                     int ncol, int pass, int half, bool dfs, cudaStream_t s);
template <typename ST>
void launch_step_normalize(const Prob* dprobs, int nprob, int ph, int maxnrb, int64_t maxNpad,
                           int start, int half, cudaStream_t s);
template <typename ST>
void launch_start_vector(const Prob* dprobs, int nprob, int64_t maxNpad, uint64_t seed,
                         const void* v0, cudaStream_t s);
template <typename ST>
void launch_restart(const Prob* dprobs, int nprob, int ph, int64_t maxNpad, int ncv, bool gruning, bool df,
                    cudaStream_t s);

// projected eigenproblem (k_ritz.cu); gruning: the tree of H's projection instead of the
// folded one
void launch_ritz(const Prob* dprobs, int nprob, int ncv, bool gruning, cudaStream_t s);
void launch_lock_decide_form(const Prob* dprobs, int nprob, int ph, cudaStream_t s);
// VAR_PROJECTED (k_dense.cu): the active projected problem of problem iprob as the BSE
// matrix [[A_k, B_k], [-B_k, -A_k]] of order 2 n, solved by the dense structure-preserving
// method; writes ritz, S and rest like launch_ritz.  n = m - k and nw = the wanted count,
// as the host read them from the Krylov state.  Returns 0, 1 (not positive definite) or
// -1 (CUDA error); `work` holds dense_scratch_doubles(n, nw) + projected_scratch_doubles(n, nw).
size_t projected_scratch_doubles(int n, int nw);
int projected_ritz(const Prob* dprobs, int iprob, int n, int nw, double* work, int* dflag, cudaStream_t s);

// post-processing (k_post.cu); Z is FP64, ld 2 Npad (PH) or Npad (TDA)
template <typename ST>
void launch_recover(const Prob* dprobs, int iprob, int ph, int64_t Npad, int64_t N, int nev,
                    double2* Z, int ldz, cudaStream_t s);
void launch_colnormalize(double2* Z, int64_t ldz, int64_t Npad, int k, int ph, double* part,
                         int nrb, cudaStream_t s);
void launch_prepare_hz2(const double2* Z, int64_t ldz, int64_t Npad, int k, double2* XA,
                        double2* XB, cudaStream_t s);
void launch_residuals2(const double2* Z, int64_t ldz, const double2* U, int64_t Npad, int k,
                       int ph, D4* part, int nrb, double* rho, double* znorm2, double* res,
                       cudaStream_t s);
template <typename ST>
void launch_store_vectors2(const double2* Z, int64_t ldz, int64_t Npad, int64_t N, int ph, int k,
                           const int* perm, ST* out, int64_t ldo, cudaStream_t s);
template <typename ST, typename R>
void launch_adjoint2(const double2* Z, int64_t ldz, int64_t Npad, int64_t N, int k,
                     const double* g, int ph, const int2* tiles, int64_t ntiles, ST* dA, ST* dB,
                     cudaStream_t s);

}  // namespace bse
