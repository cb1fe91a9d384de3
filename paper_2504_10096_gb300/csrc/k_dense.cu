// Dense structure-preserving diagonalisation of the pseudo-Hermitian BSE
// matrix on the GPU (the direct method of Sec. 2.1.1, Eqs. 4-6), in FP64.
//
// With Q and the real skew-symmetric J of Eq. 4, Q^H H Q = -i J M_r, where
//     M_r = [[Re(A + B), Im(A - B)], [-Im(A + B), Re(A - B)]]     (Eq. 5)
// is real symmetric and positive definite when M of Eq. 2 is.  With the
// Cholesky factor M_r = L L^T, W = L^T J L is real skew-symmetric and -iW is
// Hermitian with the eigenvalues +-omega of H (Eq. 6).  The steps, all in
// this file and all FP64 on the CUDA cores (GB300's FP64 tensor rate is far
// below its FP64 FMA rate, so no tensor-core path is used):
//   1. assemble M_r (order n = 2N, column-major) from the handle's packed tiles;
//   2. blocked right-looking Cholesky (64-column panels: diagonal block in one
//      CTA, panel solve, trailing symmetric rank-64 update);
//   3. W = L_top^T L_bot - L_bot^T L_top (J swaps the two halves of L's rows);
//   4. Householder reduction of W to skew-tridiagonal form: the reflector
//      H = I - tau v v^T of column k turns the trailing block into
//      W + tau (v p^T - p v^T), p = W v (v^T W v = 0 for skew W);
//   5. -iT (T skew-tridiagonal, sub-diagonal e) is unitarily similar, through
//      a diagonal phase matrix D, to the real symmetric tridiagonal S with zero
//      diagonal and off-diagonals |e_k|: the wanted eigenvalues (indices N ...
//      N + nev - 1 of S's ascending spectrum) by bisection with Sturm counts,
//      their eigenvectors by inverse iteration;
//   6. back-transformation q = H_0 ... H_{n-3} D s, then y = L^{-T} q and
//      z = Q y, which the caller Omega-normalises (Eq. 7 gives the partners).
#include <algorithm>
#include <cmath>

#include "../../include/bse.h"
#include "bse_internal.cuh"

namespace bse {
namespace {

constexpr int DNB = 64;        // Cholesky panel width and GEMM tile edge

// (A_ij, B_ij) from the packed upper-triangle tiles of problem p (any i, j < N):
// complex128 PH tiles hold P = A + B, Q = A - B; complex64 tiles hold A, B
template <typename ST>
__device__ __forceinline__ void dn_ab(const Prob& p, int64_t i, int64_t j, bool pq, double2& a, double2& b) {
  const bool up = i <= j;
  const int64_t r = up ? i : j, c = up ? j : i;
  const int I = (int)(r / TS), J = (int)(c / TS);
  const int64_t t = (int64_t)I * p.nT - (int64_t)I * (I - 1) / 2 + (J - I);
  int rr = (int)(r % TS), cc = (int)(c % TS);
  if (!up && I == J) {           // diagonal tiles hold both halves: read (i, j) itself
    rr = (int)(i % TS);
    cc = (int)(j % TS);
  }
  const int64_t e = t * (TS * TS) + (int64_t)rr * TS + cc;
  double2 x = ccvt<double2>(((const ST*)p.A)[e]), y = ccvt<double2>(((const ST*)p.B)[e]);
  if (pq) {
    a = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
    b = make_double2(0.5 * (x.x - y.x), 0.5 * (x.y - y.y));
  } else {
    a = x;
    b = y;
  }
  if (!up && I != J) a = conjc(a);   // lower triangle: A Hermitian, B symmetric
}

// 1. M_r (n x n, column-major, leading dimension ld); grid (ceil(n/32), ceil(n/8)), 32 x 8
template <typename ST>
__global__ void k_dn_assemble(const Prob* __restrict__ probs, int pq, double* __restrict__ M, int64_t ld) {
  const Prob& p = probs[0];
  const int64_t N = p.N, n = 2 * N;
  const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n) return;
  const bool ti = i >= N, tj = j >= N;
  double2 a, b;
  dn_ab<ST>(p, ti ? i - N : i, tj ? j - N : j, pq != 0, a, b);
  double v;
  if (!ti && !tj) v = a.x + b.x;          // Re(A + B)
  else if (!ti && tj) v = a.y - b.y;      // Im(A - B)
  else if (ti && !tj) v = -(a.y + b.y);   // -Im(A + B)
  else v = a.x - b.x;                     // Re(A - B)
  M[j * ld + i] = v;
}

// 2a. Cholesky of the diagonal block at k0 (kb <= 64 columns) in one CTA
__global__ void __launch_bounds__(256) k_dn_potrf(double* __restrict__ M, int64_t ld, int64_t k0, int kb,
                                                  int* __restrict__ notpd) {
  __shared__ double a[DNB][DNB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += 256) {
    const int r = e % kb, c = e / kb;
    a[r][c] = M[(k0 + c) * ld + k0 + r];
  }
  __syncthreads();
  for (int c = 0; c < kb; ++c) {
    if (tid == 0) {
      double d = a[c][c];
      if (!(d > 0.0)) {            // M_r not positive definite: flag it, keep the numbers finite
        atomicExch(notpd, 1);
        d = 1.0;
      }
      a[c][c] = sqrt(d);
    }
    __syncthreads();
    const double inv = 1.0 / a[c][c];
    for (int r = c + 1 + tid; r < kb; r += 256) a[r][c] *= inv;
    __syncthreads();
    for (int e = tid; e < (kb - c - 1) * (kb - c - 1); e += 256) {
      const int r = c + 1 + e % (kb - c - 1), q = c + 1 + e / (kb - c - 1);
      if (r >= q) a[r][q] -= a[r][c] * a[q][c];
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += 256) {
    const int r = e % kb, c = e / kb;
    if (r >= c) M[(k0 + c) * ld + k0 + r] = a[r][c];
  }
}

// 2b. panel below the diagonal block: rows r >= k0 + kb solve x L11^T = a; one thread per row
__global__ void __launch_bounds__(128) k_dn_trsm(double* __restrict__ M, int64_t ld, int64_t n, int64_t k0, int kb) {
  __shared__ double l[DNB][DNB + 1];
  for (int e = threadIdx.x; e < kb * kb; e += 128) {
    const int r = e % kb, c = e / kb;
    l[r][c] = r >= c ? M[(k0 + c) * ld + k0 + r] : 0.0;
  }
  __syncthreads();
  const int64_t row = k0 + kb + (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (row >= n) return;
  double x[DNB];
#pragma unroll
  for (int c = 0; c < DNB; ++c)
    if (c < kb) x[c] = M[(k0 + c) * ld + row];
#pragma unroll
  for (int c = 0; c < DNB; ++c) {
    if (c < kb) {
      double s = x[c];
#pragma unroll
      for (int q = 0; q < DNB; ++q)
        if (q < c) s -= x[q] * l[c][q];
      x[c] = s / l[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < DNB; ++c)
    if (c < kb) M[(k0 + c) * ld + row] = x[c];
}

// C (m x m' block of an n x n column-major matrix) op= sum_q A(i, q) B(j, q) over kk
// columns: 64 x 64 output tiles, 256 threads x (4 x 4), K staged 16 at a time.
// mode 0: trailing Cholesky update C -= L21 L21^T on the lower triangle (tiles i >= j);
// mode 1: G = A^T B with A, B row blocks (W step): C[i][j] = sum_k A[k][i] B[k][j].
template <int MODE>
__global__ void __launch_bounds__(256) k_dn_gemm(double* __restrict__ C, int64_t ldc, const double* __restrict__ Am,
                                                 const double* __restrict__ Bm, int64_t lda, int64_t m, int64_t kk,
                                                 int64_t off) {
  __shared__ double sa[16][DNB + 1], sb[16][DNB + 1];
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (MODE == 0 && bi < bj) return;                 // lower triangle only
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  const int64_t i0 = (int64_t)bi * DNB, j0 = (int64_t)bj * DNB;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int64_t q0 = 0; q0 < kk; q0 += 16) {
    __syncthreads();
    for (int e = tid; e < 16 * DNB; e += 256) {
      const int r = e % DNB, q = e / DNB;
      const int64_t gi = i0 + r, gj = j0 + r, gq = q0 + q;
      if (MODE == 0) {   // A(i, q) = L21[i][q] = M[(off + q) * lda + off + i] style, passed as column-major panel
        sa[q][r] = (gi < m && gq < kk) ? Am[gq * lda + gi] : 0.0;
        sb[q][r] = (gj < m && gq < kk) ? Bm[gq * lda + gj] : 0.0;
      } else {           // A(i, q) = Atop[q][i]: row q of the top block, column i
        sa[q][r] = (gi < m && gq < kk) ? Am[gi * lda + gq] : 0.0;
        sb[q][r] = (gj < m && gq < kk) ? Bm[gj * lda + gq] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      double av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = sa[q][tr + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) bv[v] = sb[q][tc + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t gi = i0 + tr + 16 * u, gj = j0 + tc + 16 * v;
      if (gi >= m || gj >= m) continue;
      if (MODE == 0) {
        if (gi >= gj) C[(off + gj) * ldc + off + gi] -= acc[u][v];
      } else {
        C[gj * ldc + gi] = acc[u][v];
      }
    }
}

// W = G - G^T, elementwise (column-major); the upper triangle of G is read before either
// element of a pair is written because each thread owns one unordered pair (i > j)
__global__ void k_dn_skew(double* __restrict__ W, int64_t ld, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n || i < j) return;
  if (i == j) { W[j * ld + i] = 0.0; return; }
  const double gij = W[j * ld + i], gji = W[i * ld + j];
  W[j * ld + i] = gij - gji;
  W[i * ld + j] = gji - gij;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < nw; ++q) t += red[q];
  return t;
}

// 4a. reflector of column k: x = W[k+1:, k]; beta = -sign(x0) |x|; v = x / (x0 - beta), v0 = 1,
// tau = (beta - x0) / beta (tau = 0 when x below x0 is zero).  Stores e_k = beta in E[k], tau in
// T[k], v (with v0 = 1) in V[k+1:] of a work column.  One CTA.
__global__ void __launch_bounds__(1024) k_dn_house(const double* __restrict__ W, int64_t ld, int64_t n, int64_t k,
                                                   double* __restrict__ E, double* __restrict__ T,
                                                   double* __restrict__ V) {
  __shared__ double red[32];
  const double* x = W + k * ld;
  double s = 0.0;
  for (int64_t r = k + 2 + threadIdx.x; r < n; r += blockDim.x) s += x[r] * x[r];
  const double sig = block_sum(s, red);
  const double x0 = x[k + 1];
  double beta, tau, scale;
  if (sig == 0.0) {
    beta = x0;
    tau = 0.0;
    scale = 0.0;
  } else {
    const double nrm = sqrt(x0 * x0 + sig);
    beta = x0 >= 0.0 ? -nrm : nrm;
    tau = (beta - x0) / beta;
    scale = 1.0 / (x0 - beta);
  }
  for (int64_t r = k + 1 + threadIdx.x; r < n; r += blockDim.x) V[r] = r == k + 1 ? 1.0 : x[r] * scale;
  if (threadIdx.x == 0) {
    E[k] = beta;
    T[k] = tau;
  }
}

// 4b. p = W22 v over the trailing block rows/columns [k+1, n): one thread per row, columns
// in chunks of 32 staged in shared memory
__global__ void __launch_bounds__(256) k_dn_skew_mv(const double* __restrict__ W, int64_t ld, int64_t n, int64_t k,
                                                    const double* __restrict__ V, double* __restrict__ Pv) {
  __shared__ double sv[256];
  const int64_t i = k + 1 + (int64_t)blockIdx.x * 256 + threadIdx.x;
  double acc = 0.0;
  for (int64_t j0 = k + 1; j0 < n; j0 += 256) {
    __syncthreads();
    const int64_t jj = j0 + threadIdx.x;
    sv[threadIdx.x] = jj < n ? V[jj] : 0.0;
    __syncthreads();
    if (i < n) {
      const int64_t jn = min((int64_t)256, n - j0);
      const double* col = W + j0 * ld + i;
#pragma unroll 4
      for (int64_t q = 0; q < jn; ++q) acc = fma(col[q * ld], sv[q], acc);
    }
  }
  if (i < n) Pv[i] = acc;
}

// 4c. W22 += tau (v p^T - p v^T); also stores v below the sub-diagonal of column k (the
// reflector, for the back-transformation) and sets W[k+1][k] = beta
__global__ void k_dn_skew_r2(double* __restrict__ W, int64_t ld, int64_t n, int64_t k, const double* __restrict__ V,
                             const double* __restrict__ Pv, const double* __restrict__ T) {
  const int64_t i = k + 1 + (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t j = k + 1 + (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n) return;
  const double tau = T[k];
  W[j * ld + i] += tau * (V[i] * Pv[j] - Pv[i] * V[j]);
}

__global__ void k_dn_store_v(double* __restrict__ W, int64_t ld, int64_t n, int64_t k, const double* __restrict__ V,
                             const double* __restrict__ E) {
  const int64_t r = k + 1 + (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (r >= n) return;
  W[k * ld + r] = r == k + 1 ? E[k] : V[r];
}

// 5a. Sturm count of S - sigma I, S symmetric tridiagonal with zero diagonal and
// off-diagonals |e_k| (k < n - 1): number of eigenvalues below sigma
__device__ int dn_sturm(const double* __restrict__ e, int64_t n, double sigma, double pivmin) {
  int cnt = 0;
  double q = -sigma;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int64_t t = 1; t < n; ++t) {
    q = -sigma - e[t - 1] * e[t - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// one warp per wanted eigenvalue (index idx0 + blockIdx.x of the ascending spectrum)
__global__ void __launch_bounds__(32) k_dn_bisect(const double* __restrict__ e, int64_t n,
                                                  const double* __restrict__ bound_p, int64_t idx0,
                                                  double* __restrict__ lam) {
  const int64_t idx = idx0 + blockIdx.x;
  const int lane = threadIdx.x;
  const double bound = *bound_p;
  double lo = -bound, hi = bound;
  const double pivmin = 1e-290 * fmax(1.0, bound * bound);
  const double eps = 2.220446049250313e-16;
  for (int it = 0; it < 100; ++it) {
    const double width = hi - lo;
    if (width <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;
    const double sig = lo + width * (double)(lane + 1) / 33.0;
    const int c = dn_sturm(e, n, sig, pivmin);
    const unsigned mask = __ballot_sync(0xffffffffu, c > idx);
    if (mask == 0u) {
      lo = __shfl_sync(0xffffffffu, sig, 31);
    } else {
      const int L = __ffs(mask) - 1;
      const double sL = __shfl_sync(0xffffffffu, sig, L);
      const double sLm = __shfl_sync(0xffffffffu, sig, L > 0 ? L - 1 : 0);
      if (L > 0) lo = sLm;
      hi = sL;
    }
  }
  if (lane == 0) lam[blockIdx.x] = 0.5 * (lo + hi);
}

__device__ __forceinline__ uint64_t dn_mix(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// 5b. inverse iteration for the eigenvectors of S, one thread per cluster of close eigenvalues
// (Gram-Schmidt inside a cluster); GEPP of S - lambda I in per-vector scratch (5 n doubles):
// vectors s_c (n doubles each, unit 2-norm) go to Sv[c * n ...]
__global__ void k_dn_inverse(const double* __restrict__ e, int64_t n, int nev, const double* __restrict__ lam,
                             const double* __restrict__ bound_p, double* __restrict__ scratch,
                             double* __restrict__ Sv) {
  const int c0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (c0 >= nev) return;
  const double bound = *bound_p;
  const double eps = 2.220446049250313e-16;
  const double ctol = 1e-7 * bound;
  if (c0 > 0 && lam[c0] - lam[c0 - 1] < ctol) return;     // not a cluster leader
  int c1 = c0 + 1;
  while (c1 < nev && lam[c1] - lam[c1 - 1] < ctol) ++c1;
  double* d = scratch + (int64_t)c0 * 5 * n;
  double* du = d + n;
  double* du2 = du + n;
  double* dl = du2 + n;
  double* pv = dl + n;                                     // pivots as doubles (0 / 1)
  const double pivmin = eps * fmax(bound, 1e-300);
  double lprev = -1e300;
  for (int c = c0; c < c1; ++c) {
    double lm = lam[c];
    if (c > c0 && lm - lprev < 10.0 * eps * bound) lm = lprev + 10.0 * eps * bound;
    lprev = lm;
    for (int64_t t = 0; t < n; ++t) {
      d[t] = -lm;
      du[t] = t + 1 < n ? fabs(e[t]) : 0.0;
      dl[t] = du[t];
      du2[t] = 0.0;
    }
    for (int64_t t = 0; t + 1 < n; ++t) {
      if (fabs(d[t]) >= fabs(dl[t])) {
        pv[t] = 0.0;
        if (d[t] == 0.0) d[t] = pivmin;
        const double f = dl[t] / d[t];
        dl[t] = f;
        d[t + 1] -= f * du[t];
      } else {
        pv[t] = 1.0;
        const double f = d[t] / dl[t];
        d[t] = dl[t];
        dl[t] = f;
        const double tmp = du[t];
        du[t] = d[t + 1];
        d[t + 1] = tmp - f * d[t + 1];
        if (t + 2 < n) {
          du2[t] = du[t + 1];
          du[t + 1] = -f * du[t + 1];
        }
      }
    }
    if (fabs(d[n - 1]) < pivmin) d[n - 1] = pivmin;
    double* x = Sv + (int64_t)c * n;
    for (int64_t t = 0; t < n; ++t)
      x[t] = (double)(dn_mix((uint64_t)(c + 1) * 0x100000001b3ull + (uint64_t)t) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    for (int it = 0; it < 4; ++it) {
      for (int rep = 0; rep < 2; ++rep)
        for (int q = c0; q < c; ++q) {
          const double* sq = Sv + (int64_t)q * n;
          double dot = 0.0;
          for (int64_t t = 0; t < n; ++t) dot += sq[t] * x[t];
          for (int64_t t = 0; t < n; ++t) x[t] -= dot * sq[t];
        }
      double nr = 0.0;
      for (int64_t t = 0; t < n; ++t) nr += x[t] * x[t];
      const double inv = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
      for (int64_t t = 0; t < n; ++t) x[t] *= inv;
      if (it == 3) break;
      for (int64_t t = 0; t + 1 < n; ++t) {          // forward: L
        if (pv[t] == 0.0) {
          x[t + 1] -= dl[t] * x[t];
        } else {
          const double tmp = x[t];
          x[t] = x[t + 1];
          x[t + 1] = tmp - dl[t] * x[t];
        }
      }
      x[n - 1] /= d[n - 1];                           // backward: U
      if (n > 1) x[n - 2] = (x[n - 2] - du[n - 2] * x[n - 1]) / d[n - 2];
      for (int64_t t = n - 3; t >= 0; --t) x[t] = (x[t] - du[t] * x[t + 1] - du2[t] * x[t + 2]) / d[t];
    }
  }
}

// zero the upper triangle of the Cholesky factor (the M_r values left there)
__global__ void k_dn_zero_upper(double* __restrict__ M, int64_t ld, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (i < n && j < n && i < j) M[j * ld + i] = 0.0;
}

// the last sub-diagonal entry of T needs no reflector
__global__ void k_dn_store_last(const double* __restrict__ W, int64_t ld, int64_t n, double* __restrict__ E,
                                double* __restrict__ T) {
  E[n - 2] = W[(n - 2) * ld + n - 1];
  T[n - 2] = 0.0;
}

// Gershgorin bound of S: 2 max |e| (and a tiny floor), one CTA
__global__ void __launch_bounds__(1024) k_dn_bound(const double* __restrict__ E, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t t = threadIdx.x; t + 1 < n; t += blockDim.x) m = fmax(m, fabs(E[t]));
#pragma unroll
  for (int k = 16; k >= 1; k >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, k));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, red[q]);
    *out = 2.0 * t * (1.0 + 1e-14) + 1e-300;
  }
}

// 6. one CTA per eigenvector: q = H_0 ... H_{n-3} D s (D: the phases that make -iT real, so q is
// complex), then y = L^{-T} q, then z = Q y into Z (FP64 complex, ld 2 Npad: X rows then Y rows)
__global__ void __launch_bounds__(256) k_dn_back(const double* __restrict__ Wv, const double* __restrict__ L,
                                                 int64_t ld, int64_t n, const double* __restrict__ E,
                                                 const double* __restrict__ T, const double* __restrict__ Sv,
                                                 double2* __restrict__ qbuf, int64_t Npad, double2* __restrict__ Z) {
  __shared__ double red[8];
  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t N = n / 2;
  double2* q = qbuf + (int64_t)c * n;
  const double* s = Sv + (int64_t)c * n;
  // D: d_0 = 1, d_{k+1} = d_k (-i) sign(e_k); the phase is i^(-k) times a sign, so it is
  // tracked as an index mod 4 and a sign (sequential, one thread)
  if (tid == 0) {
    int ph = 0;
    double sg = 1.0;
    for (int64_t t = 0; t < n; ++t) {
      const double v = s[t] * sg;
      const double2 dv = (ph == 0) ? make_double2(v, 0.0)
                       : (ph == 1) ? make_double2(0.0, -v)
                       : (ph == 2) ? make_double2(-v, 0.0)
                                   : make_double2(0.0, v);       // v (-i)^ph
      q[t] = dv;
      if (t + 1 < n) {
        ph = (ph + 1) & 3;
        if (E[t] < 0.0) sg = -sg;
      }
    }
  }
  __syncthreads();
  for (int64_t k = n - 3; k >= 0; --k) {              // q <- H_k q on rows k+1 ... n-1
    const double tau = T[k];
    if (tau == 0.0) continue;                          // uniform: T is read by every thread
    const double* v = Wv + k * ld;                     // v_{k+1} = 1 (stored as beta), v_r below
    double sr = 0.0, si = 0.0;
    for (int64_t r = k + 1 + tid; r < n; r += 256) {
      const double vr = r == k + 1 ? 1.0 : v[r];
      sr += vr * q[r].x;
      si += vr * q[r].y;
    }
    sr = block_sum(sr, red);
    si = block_sum(si, red);
    for (int64_t r = k + 1 + tid; r < n; r += 256) {
      const double vr = r == k + 1 ? 1.0 : v[r];
      q[r].x -= tau * vr * sr;
      q[r].y -= tau * vr * si;
    }
    __syncthreads();
  }
  // y = L^{-T} q: for i = n-1 ... 0, y_i = (q_i - sum_{j > i} L[j][i] y_j) / L[i][i] (in place)
  for (int64_t i = n - 1; i >= 0; --i) {
    const double* col = L + i * ld;
    double sr = 0.0, si = 0.0;
    for (int64_t j = i + 1 + tid; j < n; j += 256) {
      sr += col[j] * q[j].x;
      si += col[j] * q[j].y;
    }
    sr = block_sum(sr, red);
    si = block_sum(si, red);
    if (tid == 0) {
      const double inv = 1.0 / col[i];
      q[i] = make_double2((q[i].x - sr) * inv, (q[i].y - si) * inv);
    }
    __syncthreads();
  }
  // z = Q y, Q = (1/sqrt 2) [[I, -iI], [I, iI]]: X = (y1 - i y2) / sqrt 2, Y = (y1 + i y2) / sqrt 2
  const double r2 = 0.70710678118654752440;
  double2* z = Z + (int64_t)c * 2 * Npad;
  for (int64_t r = tid; r < Npad; r += 256) {
    double2 X = make_double2(0.0, 0.0), Y = make_double2(0.0, 0.0);
    if (r < N) {
      const double2 a = q[r], b = q[N + r];
      X = make_double2((a.x + b.y) * r2, (a.y - b.x) * r2);
      Y = make_double2((a.x - b.y) * r2, (a.y + b.x) * r2);
    }
    z[r] = X;
    z[Npad + r] = Y;
  }
}

}  // namespace

// scratch of dense_shao in doubles: M_r / L and W (ld x n each), the reflector work
// vectors, the eigenvector scratch of the inverse iteration, and the complex q vectors
size_t dense_scratch_doubles(int64_t N, int nev) {
  const int64_t n = 2 * N;
  const int64_t ld = (n + 31) / 32 * 32;
  // ten sub-buffers, each rounded up to 32 doubles
  return (size_t)(2 * ld * n + 4 * n + (int64_t)nev * (5 * n + n + 2 * n) + nev + 8 + 10 * 32);
}

// Steps 2-6 on an assembled M_r (step 1 is `assemble(M, ld)`): the nev lowest positive omega
// (device, *lam_dev) and their right eigenvectors (unnormalised) in Z (ld 2 Npad).  Returns 0,
// 1 (M_r not positive definite) or -1 (CUDA error); the stream is synchronised.
template <typename Assemble>
int dense_run(int64_t N, int64_t Npad, int nev, double* work, int* dflag, double2* Z, double** lam_dev,
              Assemble assemble, cudaStream_t s) {
  const int64_t n = 2 * N;
  const int64_t ld = (n + 31) / 32 * 32;
  // sub-buffers start on 256-byte boundaries (q is read and written as double2)
  size_t off = 0;
  auto take = [&](int64_t count) {
    double* p = work + off;
    off += (size_t)((count + 31) / 32 * 32);
    return p;
  };
  double* M = take(ld * n);         // M_r, then L (lower)
  double* W = take(ld * n);         // G, then W, then the reduced form with the reflectors
  double* E = take(n);              // sub-diagonal of T
  double* T = take(n);              // reflector scalars
  double* V = take(n);              // current reflector
  double* Pv = take(n);             // W22 v
  double* lam = take(nev + 8);      // wanted eigenvalues of S, then the bound of S
  double* inv = take((int64_t)nev * 5 * n);   // inverse-iteration scratch, 5 n per vector
  double* Sv = take((int64_t)nev * n);
  double2* qb = reinterpret_cast<double2*>(take((int64_t)nev * 2 * n));
  *lam_dev = lam;
  if (cudaMemsetAsync(dflag, 0, sizeof(int), s) != cudaSuccess) return -1;
  // 1.
  const dim3 g2((unsigned)((n + 31) / 32), (unsigned)((n + 7) / 8)), b2(32, 8);
  assemble(M, ld);
  // 2. Cholesky
  for (int64_t k0 = 0; k0 < n; k0 += DNB) {
    const int kb = (int)std::min<int64_t>(DNB, n - k0);
    count_launch();
    k_dn_potrf<<<1, 256, 0, s>>>(M, ld, k0, kb, dflag);
    const int64_t rest = n - k0 - kb;
    if (rest > 0) {
      count_launch(2);
      k_dn_trsm<<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(M, ld, n, k0, kb);
      const unsigned nt = (unsigned)((rest + DNB - 1) / DNB);
      // A = B = the panel L21, rows k0 + kb ..., columns k0 ... k0 + kb (column-major, ld)
      const double* panel = M + k0 * ld + k0 + kb;
      k_dn_gemm<0><<<dim3(nt, nt), 256, 0, s>>>(M, ld, panel, panel, ld, rest, kb, k0 + kb);
    }
  }
  count_launch();
  k_dn_zero_upper<<<g2, b2, 0, s>>>(M, ld, n);
  // 3. G = L_top^T L_bot (rows 0..N-1 and N..2N-1 of L, all n columns), then W = G - G^T.
  // In mode 1 the kernel reads A(i, q) = Am[i * lda + q]: column i of L, row q of the block
  count_launch(2);
  const unsigned ng = (unsigned)((n + DNB - 1) / DNB);
  k_dn_gemm<1><<<dim3(ng, ng), 256, 0, s>>>(W, ld, M, M + N, ld, n, N, 0);
  k_dn_skew<<<g2, b2, 0, s>>>(W, ld, n);
  // 4. skew-tridiagonalisation
  for (int64_t k = 0; k + 2 < n; ++k) {
    const int64_t m = n - k - 1;
    count_launch(4);
    k_dn_house<<<1, 1024, 0, s>>>(W, ld, n, k, E, T, V);
    k_dn_skew_mv<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(W, ld, n, k, V, Pv);
    k_dn_skew_r2<<<dim3((unsigned)((m + 31) / 32), (unsigned)((m + 7) / 8)), dim3(32, 8), 0, s>>>(W, ld, n, k, V, Pv,
                                                                                                  T);
    k_dn_store_v<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(W, ld, n, k, V, E);
  }
  // the last sub-diagonal entry needs no reflector
  if (n >= 2) {
    count_launch();
    k_dn_store_last<<<1, 1, 0, s>>>(W, ld, n, E, T);
  }
  // 5. eigenvalues N ... N + nev - 1 of S and their eigenvectors
  count_launch(3);
  k_dn_bound<<<1, 1024, 0, s>>>(E, n, lam + nev);
  k_dn_bisect<<<nev, 32, 0, s>>>(E, n, lam + nev, N, lam);
  k_dn_inverse<<<(nev + 31) / 32, 32, 0, s>>>(E, n, nev, lam, lam + nev, inv, Sv);
  // 6.
  count_launch();
  k_dn_back<<<nev, 256, 0, s>>>(W, M, ld, n, E, T, Sv, qb, Npad, Z);
  int h = 0;
  if (cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1;
  return h ? 1 : 0;
}

namespace {

// ---------------------------------------------------------------- projected BSE variant
// The folded recurrence builds V (M+-orthonormal) and P = M+ V, and H maps the even vectors
// e_j = (v_j; conj(v_j)) to the odd ones o_j = (p_j; -conj(p_j)) and o_j to sum_i e_i T_ij
// (T the projected M- M+).  In the basis x_j = e_j + o_j, y_j = e_j - o_j, which the
// swap-and-conjugate symmetry of H maps onto each other, H's projection is the BSE matrix
// [[A_k, B_k], [-B_k, -A_k]] of Eq. 1 with the real symmetric blocks A_k = (T + I) / 2 and
// B_k = (I - T) / 2; its M_r (Eq. 5) is diag(I, T), positive definite.  The dense
// structure-preserving method solves it (its omega are the singular values of T's Cholesky
// factor, computed without squaring), and an eigenvector (a; b) is the Ritz vector
// x a + y b = e (a + b) + o (a - b): the folded coefficients are a + b.

// M_r = diag(I, T_active) of problem ip (column-major, ld); grid as k_dn_assemble
__global__ void k_pj_assemble(const Prob* __restrict__ probs, int ip, double* __restrict__ M, int64_t ld) {
  const Prob& p = probs[ip];
  const KState* st = p.st;
  const int k = st->k, l = st->l, m = st->m, h = l - k;
  const int64_t na = m - k, n = 2 * na;
  const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n) return;
  double v = 0.0;
  if (i < na || j < na) {
    v = i == j ? 1.0 : 0.0;
  } else {
    const int64_t a = i - na, b = j - na;
    const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
    if (a == b) v = a < h ? p.theta[k + a] : p.alpha[l + (a - h)];
    else if (hi == h && lo < h) v = p.barrow[k + lo];
    else if (lo >= h && hi == lo + 1) v = p.beta[l + (lo - h)];
  }
  M[j * ld + i] = v;
}

// folded Ritz data from the small problem's eigenvectors: one CTA per wanted pair
__global__ void __launch_bounds__(256) k_pj_coef(const Prob* __restrict__ probs, int ip, int64_t na,
                                                 const double2* __restrict__ Zs, const double* __restrict__ lam) {
  __shared__ double red[8];
  __shared__ double sv[8];
  __shared__ int si[8];
  const Prob& p = probs[ip];
  const KState* st = p.st;
  const int i = blockIdx.x, tid = threadIdx.x;
  const double2* z = Zs + (int64_t)i * 2 * na;
  // the entry of largest modulus of c~ = a + b fixes the common phase (lowest index on ties)
  double best = -1.0;
  int bi = 0;
  for (int64_t t = tid; t < na; t += 256) {
    const double2 c = cadd(z[t], z[na + t]);
    const double a2 = c.x * c.x + c.y * c.y;
    if (a2 > best) { best = a2; bi = (int)t; }
  }
  for (int o = 16; o >= 1; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((tid & 31) == 0) { sv[tid >> 5] = best; si[tid >> 5] = bi; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < 8; ++w)
      if (sv[w] > sv[0] || (sv[w] == sv[0] && si[w] < si[0])) { sv[0] = sv[w]; si[0] = si[w]; }
  }
  __syncthreads();
  const double2 cm = cadd(z[si[0]], z[na + si[0]]);
  const double cmn = sqrt(cm.x * cm.x + cm.y * cm.y);
  const double2 ph = cmn > 0.0 ? make_double2(cm.x / cmn, -cm.y / cmn) : make_double2(1.0, 0.0);  // conj phase
  double* S = p.S + (int64_t)i * p.ncv;
  double nr = 0.0;
  for (int64_t t = tid; t < na; t += 256) {
    const double2 c = cadd(z[t], z[na + t]);
    const double v = c.x * ph.x - c.y * ph.y;   // Re(c e^{-i phi})
    S[t] = v;
    nr += v * v;
  }
  nr = block_sum(nr, red);
  const double inv = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
  for (int64_t t = tid; t < na; t += 256) S[t] *= inv;
  __syncthreads();
  if (tid == 0) {
    p.ritz[i] = lam[i] * lam[i];
    p.rest[i] = fabs(p.beta[st->m - 1] * S[na - 1]);
  }
}

__global__ void k_pj_fail(const Prob* __restrict__ probs, int ip) {
  KState* st = probs[ip].st;
  if (threadIdx.x == 0 && st->status == ST_OK) st->status = ST_NOTPD;
}

}  // namespace

// Dense diagonalisation of problem 0 of a PH handle: the nev lowest positive omega and
// their right eigenvectors (unnormalised) in Z (ld 2 Npad).  Returns 0, 1 (M_r not positive
// definite) or -1 (CUDA error).  `work` holds dense_scratch_doubles(N, nev) doubles.
int dense_shao(const Prob* dprobs, int64_t N, int64_t Npad, bool tiles64, bool pq, int nev, double* work,
               int* dflag, double2* Z, double* lam_out, cudaStream_t s) {
  const int64_t n = 2 * N;
  const dim3 g2((unsigned)((n + 31) / 32), (unsigned)((n + 7) / 8)), b2(32, 8);
  double* lam = nullptr;
  const int rc = dense_run(N, Npad, nev, work, dflag, Z, &lam, [&](double* M, int64_t ld) {
    count_launch();
    if (tiles64) k_dn_assemble<float2><<<g2, b2, 0, s>>>(dprobs, pq ? 1 : 0, M, ld);
    else k_dn_assemble<double2><<<g2, b2, 0, s>>>(dprobs, pq ? 1 : 0, M, ld);
  }, s);
  if (rc) return rc;
  if (lam_out && (cudaMemcpyAsync(lam_out, lam, sizeof(double) * nev, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                  cudaStreamSynchronize(s) != cudaSuccess))
    return -1;
  return 0;
}

size_t projected_scratch_doubles(int n, int nw) { return (size_t)4 * n * nw + 64; }

int projected_ritz(const Prob* dprobs, int iprob, int n, int nw, double* work, int* dflag, cudaStream_t s) {
  if (n < 1 || nw < 1) return 0;
  const int64_t n2 = 2 * (int64_t)n;
  const dim3 g2((unsigned)((n2 + 31) / 32), (unsigned)((n2 + 7) / 8)), b2(32, 8);
  const size_t dsz = (dense_scratch_doubles(n, nw) + 31) / 32 * 32;
  double2* Zs = reinterpret_cast<double2*>(work + dsz);
  double* lam = nullptr;
  const int rc = dense_run(n, n, nw, work, dflag, Zs, &lam, [&](double* M, int64_t ld) {
    count_launch();
    k_pj_assemble<<<g2, b2, 0, s>>>(dprobs, iprob, M, ld);
  }, s);
  if (rc < 0) return rc;
  count_launch();
  if (rc == 1) {
    k_pj_fail<<<1, 32, 0, s>>>(dprobs, iprob);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
  }
  k_pj_coef<<<nw, 256, 0, s>>>(dprobs, iprob, n, Zs, lam);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}


}  // namespace bse
