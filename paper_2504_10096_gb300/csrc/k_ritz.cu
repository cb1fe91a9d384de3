// Projected eigenproblem and restart decision of the thick-restart Lanczos
// iteration (Sec. 2.2.1: the problem is projected onto a small structured
// problem; a thick restart keeps Ritz vectors without destroying structure).
//
// After a restart the projected matrix of the active (unlocked) block is
//     [ diag(theta_kept)   b          0   ]
//     [ b^T                alpha_l   beta ]
//     [ 0                  beta      tridiagonal ...]
// i.e. an arrowhead glued to a tridiagonal: its graph is a star (the kept
// Ritz vectors) attached to a path (the new Lanczos vectors).  Gaussian
// elimination from the leaves of that tree has no fill-in, so
//   * the inertia of T - sigma I (a Sturm count) costs O(n): used for
//     multisection of every wanted eigenvalue, one warp per eigenvalue;
//   * (T - lambda I) x = r costs O(n): used for inverse iteration, one warp
//     per cluster of close eigenvalues, Gram-Schmidt inside a cluster.
// Everything is FP64.
//
// Gruning variant: the projected matrix is H's own, the symmetric matrix with
// zero diagonal that couples u_j -- w_j (alpha_j) and w_j -- u_{j+1} (beta_j);
// after a restart each kept Ritz pair (u~_i, w~_i) is coupled by sigma_i and
// w~_i to the hub u_l by rho_i.  Rotating each kept pair to (u~ +- w~)/sqrt 2
// gives leaves +sigma_i and -sigma_i with couplings +-rho_i / sqrt 2 to the hub,
// followed by the path u_l, w_l, u_{l+1}, ..., w_{m-1}: the same star-plus-path
// tree, of order 2 (m - k), whose spectrum is +-sigma.  The wanted values are
// the indices m - k, m - k + 1, ... of its ascending spectrum (bisection as
// above), and each eigenvector splits into even-side (V) and odd-side (W)
// coefficients of norm 1 / sqrt 2 each.
#include "bse_internal.cuh"

namespace bse {

struct TV {        // view of the active projected matrix of one problem
  const double* d; // leaves' diagonal (theta[k..l))
  const double* b; // leaves' couplings to the hub (barrow[k..l))
  int h;           // number of leaves
  const double* a; // hub and tail diagonal (alpha[l..m))
  const double* e; // tail off-diagonal: e[t] couples a[t] and a[t+1]
  int n;           // order = h + (m - l)
};

__device__ __forceinline__ bool is_gk(const Prob& p) { return p.ph && p.variant == VAR_GRUNING; }

__device__ __forceinline__ TV make_tv(const Prob& p, const KState* st) {
  TV t;
  if (is_gk(p)) {
    const int ld = p.jwld;
    t.d = p.jw;
    t.b = p.jw + ld;
    t.h = 2 * (st->l - st->k);
    t.a = p.jw + 2 * ld;
    t.e = p.jw + 3 * ld;
    t.n = 2 * (st->m - st->k);
    return t;
  }
  t.d = p.theta + st->k;
  t.b = p.barrow + st->k;
  t.h = st->l - st->k;
  t.a = p.alpha + st->l;
  t.e = p.beta + st->l;
  t.n = st->m - st->k;
  return t;
}

// column i of the projected problem's Ritz vectors (the tree's, on the Gruning path)
__device__ __forceinline__ double* ritz_vec(const Prob& p, int i) {
  return is_gk(p) ? p.jw + 4 * (int64_t)p.jwld + (int64_t)i * p.jwld : p.S + (int64_t)i * p.ncv;
}

// Gruning path: the tree arrays of the active block (one thread per problem)
__global__ void k_gk_form(const Prob* __restrict__ probs, int nprob) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= nprob) return;
  const Prob& p = probs[ip];
  const KState* st = p.st;
  if (st->done || st->status != ST_OK) return;
  const int k = st->k, l = st->l, m = st->m, h = l - k, ld = p.jwld;
  double* d = p.jw;
  double* b = p.jw + ld;
  double* a = p.jw + 2 * ld;
  double* e = p.jw + 3 * ld;
  const double r2 = 0.70710678118654752440;
  for (int i = 0; i < h; ++i) {
    d[i] = p.theta[k + i];
    d[h + i] = -p.theta[k + i];
    b[i] = p.barrow[k + i] * r2;
    b[h + i] = -p.barrow[k + i] * r2;
  }
  for (int t = 0; t < 2 * (m - l); ++t) a[t] = 0.0;
  for (int t = 0; t < m - l; ++t) {
    e[2 * t] = p.alpha[l + t];
    if (t + 1 < m - l) e[2 * t + 1] = p.beta[l + t];
  }
}

__device__ __forceinline__ int nwanted(const KState* st) {
  const int n = st->m - st->k;
  const int w = st->r_pkeep - st->k;
  return w < n ? w : n;
}

// number of eigenvalues < sigma (LDL^T pivots of T - sigma I, leaves first)
__host__ __device__ int sturm_count(const TV& T, double sigma, double pivmin) {
  int cnt = 0;
  double s = 0.0;
  for (int i = 0; i < T.h; ++i) {
    double di = T.d[i] - sigma;
    if (fabs(di) < pivmin) di = -pivmin;
    cnt += di < 0.0;
    s += T.b[i] * T.b[i] / di;
  }
  double q = T.a[0] - sigma - s;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  const int q_n = T.n - T.h;
  for (int t = 1; t < q_n; ++t) {
    q = T.a[t] - sigma - T.e[t - 1] * T.e[t - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

__device__ void gersh(const TV& T, double& lo, double& hi, double& tnorm, int lane) {
  double glo = 1e300, ghi = -1e300, sb = 0.0, mx = 0.0;
  for (int i = lane; i < T.h; i += 32) {
    glo = fmin(glo, T.d[i] - fabs(T.b[i]));
    ghi = fmax(ghi, T.d[i] + fabs(T.b[i]));
    sb += fabs(T.b[i]);
  }
  const int q_n = T.n - T.h;
  for (int t = lane; t < q_n; t += 32) {
    double r = (t > 0 ? fabs(T.e[t - 1]) : 0.0) + (t + 1 < q_n ? fabs(T.e[t]) : 0.0);
    if (t == 0) r += 0.0;  // the leaves' couplings are added below
    glo = fmin(glo, T.a[t] - r);
    ghi = fmax(ghi, T.a[t] + r);
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, m));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, m));
    sb += __shfl_xor_sync(0xffffffffu, sb, m);
  }
  // hub row also carries sum |b_i|
  const double r0 = sb + (q_n > 1 ? fabs(T.e[0]) : 0.0);
  glo = fmin(glo, T.a[0] - r0);
  ghi = fmax(ghi, T.a[0] + r0);
  mx = fmax(fabs(glo), fabs(ghi));
  const double pad = 2.2e-16 * 8.0 * mx + 1e-300;
  lo = glo - pad;
  hi = ghi + pad;
  tnorm = mx;
}

// one warp per wanted eigenvalue; grid (ncv, nprob), block 32
__global__ void __launch_bounds__(32) k_ritz_values(const Prob* __restrict__ probs) {
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (st->done || st->status != ST_OK) return;
  const int i = blockIdx.x;
  if (i >= nwanted(st)) return;
  const TV T = make_tv(p, st);
  const int idx = is_gk(p) ? (st->m - st->k) + i : i;   // position in the ascending spectrum
  const int lane = threadIdx.x;
  double lo, hi, tnorm;
  gersh(T, lo, hi, tnorm, lane);
  const double pivmin = 1e-290 * fmax(1.0, tnorm * tnorm);
  const double eps = 2.220446049250313e-16;
  for (int it = 0; it < 100; ++it) {
    const double width = hi - lo;
    if (width <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;
    const double sig = lo + width * (double)(lane + 1) / 33.0;
    const int c = sturm_count(T, sig, pivmin);
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
  if (lane == 0) p.ritz[i] = 0.5 * (lo + hi);
}

// ---------------------------------------------------------------- inverse iteration
struct Fact {      // factorisation of T - lambda I (shared memory, n entries each)
  double* invd;    // 1 / delta_i for the leaves
  double* dl;      // tail GEPP: multipliers
  double* d;       // tail GEPP: U diagonal
  double* du;      // tail GEPP: U first super-diagonal
  double* du2;     // tail GEPP: U second super-diagonal
  unsigned char* piv;
};

// Factor T - lambda I: leaves eliminated into the hub, then Gaussian
// elimination with partial pivoting on the tridiagonal hub+tail block.
__host__ __device__ void factor_tree(const TV& T, double lam, double pivmin, Fact& F) {
  double s = 0.0;
  for (int i = 0; i < T.h; ++i) {
    double di = T.d[i] - lam;
    if (fabs(di) < pivmin) di = (di < 0.0 ? -pivmin : pivmin);
    F.invd[i] = 1.0 / di;
    s += T.b[i] * T.b[i] * F.invd[i];
  }
  const int q = T.n - T.h;
  for (int t = 0; t < q; ++t) {
    F.d[t] = T.a[t] - lam - (t == 0 ? s : 0.0);
    if (t + 1 < q) { F.du[t] = T.e[t]; F.dl[t] = T.e[t]; }
    F.du2[t] = 0.0;
  }
  for (int t = 0; t + 1 < q; ++t) {
    if (fabs(F.d[t]) >= fabs(F.dl[t])) {
      F.piv[t] = 0;
      if (F.d[t] == 0.0) F.d[t] = pivmin;
      const double f = F.dl[t] / F.d[t];
      F.dl[t] = f;
      F.d[t + 1] -= f * F.du[t];
    } else {
      F.piv[t] = 1;
      const double f = F.d[t] / F.dl[t];
      F.d[t] = F.dl[t];
      F.dl[t] = f;
      const double tmp = F.du[t];
      F.du[t] = F.d[t + 1];
      F.d[t + 1] = tmp - f * F.d[t + 1];
      if (t + 2 < q) {
        F.du2[t] = F.du[t + 1];
        F.du[t + 1] = -f * F.du[t + 1];
      }
    }
  }
  if (q > 0 && F.d[q - 1] == 0.0) F.d[q - 1] = pivmin;
}

// Solve (T - lambda I) x = r in place (x holds r on entry), x has n entries.
__host__ __device__ void solve_tree(const TV& T, const Fact& F, double* x) {
  const int h = T.h, q = T.n - T.h;
  double* y = x + h;   // hub + tail part
  double s = 0.0;
  for (int i = 0; i < h; ++i) s += T.b[i] * x[i] * F.invd[i];
  y[0] -= s;
  for (int t = 0; t + 1 < q; ++t) {
    if (F.piv[t] == 0) {
      y[t + 1] -= F.dl[t] * y[t];
    } else {
      const double tmp = y[t];
      y[t] = y[t + 1];
      y[t + 1] = tmp - F.dl[t] * y[t];
    }
  }
  y[q - 1] /= F.d[q - 1];
  if (q > 1) y[q - 2] = (y[q - 2] - F.du[q - 2] * y[q - 1]) / F.d[q - 2];
  for (int t = q - 3; t >= 0; --t) y[t] = (y[t] - F.du[t] * y[t + 1] - F.du2[t] * y[t + 2]) / F.d[t];
  const double xh = y[0];
  for (int i = 0; i < h; ++i) x[i] = (x[i] - T.b[i] * xh) * F.invd[i];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// one warp per cluster leader; grid (ncv, nprob), block 32, dynamic smem.
__global__ void __launch_bounds__(32) k_ritz_vectors(const Prob* __restrict__ probs) {
  extern __shared__ double sm[];
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (st->done || st->status != ST_OK) return;
  const int nw = nwanted(st);
  const int i0 = blockIdx.x;
  if (i0 >= nw) return;
  const TV T = make_tv(p, st);
  const int n = T.n, lane = threadIdx.x;
  double lo, hi, tnorm;
  gersh(T, lo, hi, tnorm, lane);
  const double eps = 2.220446049250313e-16;
  const double ctol = 1e-7 * tnorm;             // cluster threshold
  const double* rz = p.ritz;
  if (i0 > 0 && rz[i0] - rz[i0 - 1] < ctol) return;   // not a cluster leader
  int i1 = i0 + 1;
  while (i1 < nw && rz[i1] - rz[i1 - 1] < ctol) ++i1;
  const int M = is_gk(p) ? p.jwld : p.ncv;    // scratch stride
  Fact F;
  F.invd = sm;
  F.dl = sm + M;
  F.d = sm + 2 * M;
  F.du = sm + 3 * M;
  F.du2 = sm + 4 * M;
  double* x = sm + 5 * M;
  F.piv = (unsigned char*)(sm + 6 * M);
  // pivot guard of the inverse iteration: a shift equal to a leaf value (a
  // converged kept Ritz value with a negligible coupling) must give a large
  // but finite growth, so tiny pivots are replaced by eps * ||T||
  const double pivmin = eps * fmax(tnorm, 1e-300);
  const double pert = 10.0 * eps * tnorm;
  double lam_prev = -1e300;
  for (int i = i0; i < i1; ++i) {
    double lam = rz[i];
    if (i > i0 && lam - lam_prev < pert) lam = lam_prev + pert;
    lam_prev = lam;
    if (lane == 0) factor_tree(T, lam, pivmin, F);
    // deterministic start vector
    for (int t = lane; t < n; t += 32) {
      const uint64_t hsh = mix64((uint64_t)(i + 1) * 0x100000001b3ull + (uint64_t)t);
      x[t] = (double)(hsh >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    __syncwarp();
    for (int it = 0; it < 4; ++it) {
      // orthogonalise against the cluster's earlier vectors (twice), normalise
      for (int rep = 0; rep < 2; ++rep) {
        for (int c = i0; c < i; ++c) {
          const double* sc = ritz_vec(p, c);
          double dot = 0.0;
          for (int t = lane; t < n; t += 32) dot += sc[t] * x[t];
          dot = warp_sum(dot);
          for (int t = lane; t < n; t += 32) x[t] -= dot * sc[t];
          __syncwarp();
        }
      }
      double nr = 0.0;
      for (int t = lane; t < n; t += 32) nr += x[t] * x[t];
      nr = warp_sum(nr);
      const double inv = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
      for (int t = lane; t < n; t += 32) x[t] *= inv;
      __syncwarp();
      if (it == 3) break;
      if (lane == 0) solve_tree(T, F, x);
      __syncwarp();
    }
    double* out = ritz_vec(p, i);
    for (int t = lane; t < n; t += 32) out[t] = x[t];
    if (is_gk(p)) {
      // even-side (u~_k.., hub, u_{l+1}..) and odd-side (w~_k.., w_l..) coefficients, each
      // of norm 1 after the factor sqrt 2
      const int h = st->l - st->k, nt = st->m - st->l;
      const double s2 = 1.41421356237309504880;
      double* Se = p.S + (int64_t)i * p.ncv;
      double* So = p.S2 + (int64_t)i * p.ncv;
      for (int c = lane; c < h; c += 32) {
        Se[c] = x[c] + x[h + c];
        So[c] = x[c] - x[h + c];
      }
      for (int t = lane; t < nt; t += 32) {
        So[h + t] = s2 * x[2 * h + 1 + 2 * t];
        Se[h + t] = s2 * x[2 * h + 2 * t];
      }
      if (lane == 0) p.rest[i] = fabs(p.beta[st->m - 1] * s2 * x[n - 1]);
    } else if (lane == 0) {
      p.rest[i] = fabs(p.beta[st->m - 1] * x[n - 1]);
    }
    __syncwarp();
  }
}

// Lock the leading converged Ritz pairs, choose what to keep, and write the
// restarted arrow (theta, b).  One thread per problem.
__global__ void k_lock_decide(const Prob* __restrict__ probs, int nprob, int ph) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= nprob) return;
  const Prob& p = probs[ip];
  KState* st = p.st;
  if (st->done || st->status != ST_OK) return;
  const int k = st->k, m = st->m, n = m - k;
  const int nw = nwanted(st);
  if (ph && p.ritz[0] <= 0.0) { st->status = ST_NOTPD; return; }
  int nl = 0;
  while (nl < nw && k + nl < st->nev && p.rest[nl] <= st->lock_tol * fabs(p.ritz[nl])) ++nl;
  int nkeep;
  if (k + nl >= st->nev) {
    nkeep = nl;
  } else {
    nkeep = st->r_pkeep - k;
    if (nkeep < nl + 1) nkeep = nl + 1;
    if (nkeep > nw) nkeep = nw;
  }
  const double bl = p.beta[m - 1];
  for (int i = 0; i < nkeep; ++i) {
    p.theta[k + i] = p.ritz[i];
    const double* Sl = is_gk(p) ? p.S2 : p.S;   // the last basis vector's side
    p.barrow[k + i] = i < nl ? 0.0 : bl * Sl[(int64_t)i * p.ncv + (n - 1)];
  }
  st->beta_last = bl;
  st->r_k0 = k;
  st->r_nl = nl;
  st->r_nkeep = nkeep;
  st->r_go = 1;
}

void launch_ritz(const Prob* dprobs, int nprob, int ncv, bool gruning, cudaStream_t s) {
  if (gruning) {
    count_launch();
    k_gk_form<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob);
  }
  count_launch(2);
  k_ritz_values<<<dim3(ncv, nprob), 32, 0, s>>>(dprobs);
  const size_t M = gruning ? (size_t)(2 * ncv + 2) : (size_t)ncv;
  const size_t sm = M * 6 * sizeof(double) + M + 16;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_ritz_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_ritz_vectors<<<dim3(ncv, nprob), 32, sm, s>>>(dprobs);
}

void launch_lock_decide(const Prob* dprobs, int nprob, cudaStream_t s) {
  count_launch();
  k_lock_decide<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob, 1);
}

void launch_lock_decide_form(const Prob* dprobs, int nprob, int ph, cudaStream_t s) {
  count_launch();
  k_lock_decide<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob, ph);
}

}  // namespace bse
