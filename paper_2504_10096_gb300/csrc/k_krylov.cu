// Krylov-basis kernels of the thick-restart Lanczos iteration.
//
// Inner product: TDA uses the Euclidean one; the pseudo-Hermitian (folded)
// iteration uses <x, y>_K = Re(x^H M+ y) on C^N viewed as R^2N, in which the
// folded operator T = M- M+ (eigenvalues omega^2, Sec. 2.2.1) is self-adjoint.
// P = M+ V is stored next to V, so every K-inner product against the basis is
// Re(P^H w): one pass over the stored blocks per Krylov step is spent on
// M- p_j, the other on M+ w for the norm (the "two passes" of the step).
//
// Re-orthogonalisation is classical Gram-Schmidt done twice (CGS2).  On the
// pseudo-Hermitian path every omega^2 of T is double: with u an eigenvector,
// so is its "twin" i M+ u (M+(i x) = i M- x and M-(i x) = i M+ x give
// T(i M+ u) = i M+ T u), and a Krylov space of one start vector holds one
// direction per pair.  The
// twins of the whole basis, i P, are K-orthogonal to the Krylov space in
// exact arithmetic, but rounding noise along them is amplified like any
// wanted component and would surface as duplicate Ritz values.  Each CGS
// pass therefore also removes the K-projection of w onto span(i P): since
// M+(i P_c) = i T v_c, <i P_c, w>_K = Im((T v_c)^H w), and the K-Gram matrix
// of the twins, <i P_a, i P_b>_K = <v_a, T v_b>_K, is the projected matrix
// H of the Krylov relation T V = V H + (last column); so the projection's
// coefficients y solve H y = H s with s = Im(V^H w), i.e. y = s and
//     w -= V Re(P^H w) + i P Im(V^H w)
// (one extra set of Euclidean dots against V and one extra update from P,
// no small solve).
//
// Gruning variant (Lanczos recurrence of H in the M inner product, M of
// Eq. 2 positive definite, in which H = Omega M is self-adjoint).  From an
// even start vector (u; conj(u)) the recurrence alternates between even
// vectors (u; conj(u)) and odd ones (w; -conj(w)): H maps an even vector to
// the odd one with top M+ u and an odd one to the even one with top M- w.
// Only the tops are stored: V (even, M+-orthonormal, P = M+ V) and W (odd,
// M- -orthonormal, Z = M- W); the M inner products are 2 Re(u^H M+ u') and
// 2 Re(w^H M- w'), and H's projection is the tridiagonal with zero diagonal
// and couplings alpha_j (u_j -> w_j) and beta_j (w_j -> u_{j+1}):
//   odd half:  r = M+ u_j, orthogonalised against W and the twins i V,
//              alpha_j = |r|_-, w_j = r / alpha_j, z_j = M- r / alpha_j;
//   even half: s = z_j, orthogonalised against V and the twins i W,
//              beta_j = |s|_+, u_{j+1} = s / beta_j, p_{j+1} = M+ s / beta_j.
// The twins of the odd space are i V (M-(i v) = i M+ v, so i V is
// M- -orthonormal) and <i v_c, r>_- = Im(p_c^H r); those of the even space
// are i W with <i w_c, s>_+ = Im(z_c^H s).  In exact arithmetic both twin
// spaces are orthogonal to the Krylov vectors (Im(P^H P) = 0 and
// Im(V^H V) = 0 there), so each pass removes
//   r -= W Re(Z^H r) + i V Im(P^H r),    s -= V Re(P^H s) + i W Im(Z^H s).
#include "bse_internal.cuh"

namespace bse {

template <typename ST> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

__device__ __forceinline__ bool kactive(const KState* st) {
  return !st->done && st->status == ST_OK && !st->breakdown && st->j < st->m;
}
// problems that need a fresh basis vector: the very first one (j < 0) or a
// replacement after an invariant subspace was found (breakdown)
__device__ __forceinline__ bool kfresh(const KState* st) {
  return !st->done && st->status == ST_OK && (st->j < 0 || st->breakdown);
}
__device__ __forceinline__ bool kphase(const KState* st, int fresh) {
  return fresh ? kfresh(st) : kactive(st);
}

__device__ __forceinline__ double2 dshfl(double2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

// ---------------------------------------------------------------- CGS2 sets
// The vectors of one Gram-Schmidt pass: x -= Um Re(Dm^H x) + i Ut Im(Dt^H x) on the PH
// paths (real coefficients), x -= Um (Um^H x) on the TDA path (complex ones).  The
// set entries are c < nm (main) and nm <= c < nm + nt (twins).  The input x of the first
// pass of a Gruning half is a basis column (p_j, z_j); the result always goes to w.
struct CgsSet {
  const void* dm; const void* dt;   // dot sources
  const void* um; const void* ut;   // update bases (the twins enter as i * Ut)
  int nm, nt;
};

__device__ __forceinline__ CgsSet cgs_set(const Prob& p, const KState* st, int ph, int half) {
  const int j = st->j;
  CgsSet c;
  if (!ph) {
    c.dm = c.um = p.V; c.dt = c.ut = nullptr; c.nm = j + 1; c.nt = 0;
  } else if (half == 0) {
    c.dm = p.P; c.dt = p.V; c.um = p.V; c.ut = p.P; c.nm = c.nt = j + 1;
  } else if (half == 1) {
    c.dm = p.Z; c.dt = p.P; c.um = p.W; c.ut = p.V; c.nm = j; c.nt = j + 1;
  } else {
    c.dm = p.P; c.dt = p.Z; c.um = p.V; c.ut = p.W; c.nm = c.nt = j + 1;
  }
  return c;
}

// the input of the first pass of a Gruning half (a basis column), else w
template <typename ST>
__device__ __forceinline__ const ST* cgs_src(const Prob& p, const KState* st, int half, int pass, int newvec) {
  if (pass == 0 && !newvec) {
    if (half == 1) return (const ST*)p.P + (int64_t)st->j * p.Npad;
    if (half == 2) return (const ST*)p.Z + (int64_t)st->j * p.Npad;
  }
  return (const ST*)p.w;
}

// ---------------------------------------------------------------- CGS2 dots
// PH: cpart[rb][c] = sum_{rows in block rb} Re(conj(Dm[row, c]) x[row]) for c < nm and
// Im(conj(Dt[row, c']) x[row]) for c = nm + c' (the twin coefficients), nm + nt in all;
// TDA: the complex conj(V[row, c]) x[row], c <= j.  grid (ceil(maxcols/2), maxnrb, nprob),
// 8 warps: two columns per CTA, four warps per column, each warp a quarter of the block
// rows; the four partial sums meet in shared memory (fixed order).
template <typename ST>
__global__ void __launch_bounds__(256)
k_cgs_dot(const Prob* __restrict__ probs, int ph, int newvec, int half, int pass) {
  using R = typename RealOf<ST>::T;
  __shared__ double2 red[2][4];
  const Prob& p = probs[blockIdx.z];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  const int rb = blockIdx.y;
  if (rb >= p.nrb) return;
  const CgsSet cs = cgs_set(p, st, ph, half);
  const int nset = cs.nm + cs.nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hw = warp >> 2, quarter = warp & 3;
  const int c = blockIdx.x * 2 + hw;
  if (blockIdx.x * 2 >= nset) return;                     // whole CTA
  double2 a = mk(0.0, 0.0);
  if (c < nset) {
    const bool twin = c >= cs.nm;                         // warp-uniform
    const int col = twin ? c - cs.nm : c;
    const ST* Q = (const ST*)(twin ? cs.dt : cs.dm) + (int64_t)col * p.Npad;
    const ST* w = cgs_src<ST>(p, st, half, pass, newvec);
    const int64_t r0 = (int64_t)rb * ROWBLK + quarter * (ROWBLK / 4);
    const int64_t r1 = min((int64_t)p.Npad, r0 + ROWBLK / 4);
    // rounds of 8 rows per lane: all 16 loads of a round are issued before its arithmetic
    int64_t r = r0 + lane;
    if (ph) {   // real coefficients: Re(conj(q) x), or Im(conj(q) x) = Re(conj(q) (-i x)) for twins
      R a1 = 0, a2 = 0;   // two chains (x and y products) for more ILP
      for (; r + 7 * 32 < r1; r += 8 * 32) {
        ST q[8], x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          q[u] = __ldg(Q + r + 32 * u);
          x[u] = __ldg(w + r + 32 * u);
        }
        if (twin) {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const R t = x[u].x;
            x[u].x = x[u].y;
            x[u].y = -t;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a1 = fma(q[u].x, x[u].x, a1);
          a2 = fma(q[u].y, x[u].y, a2);
        }
      }
      for (; r < r1; r += 32) {
        const ST q = __ldg(Q + r);
        ST x = __ldg(w + r);
        if (twin) {
          const R t = x.x;
          x.x = x.y;
          x.y = -t;
        }
        a1 = fma(q.x, x.x, a1);
        a2 = fma(q.y, x.y, a2);
      }
      a = mk((double)a1 + (double)a2, 0.0);
    } else {
      ST acc = czero<ST>();
      for (; r + 7 * 32 < r1; r += 8 * 32) {
        ST q[8], x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          q[u] = __ldg(Q + r + 32 * u);
          x[u] = __ldg(w + r + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) cfmac(acc, q[u], x[u]);
      }
      for (; r < r1; r += 32) cfmac(acc, __ldg(Q + r), __ldg(w + r));
      a = mk((double)acc.x, (double)acc.y);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) a = cadd(a, dshfl(a, m));
  }
  if (lane == 0) red[hw][quarter] = a;
  __syncthreads();
  if (threadIdx.x < 2) {
    const int cc = blockIdx.x * 2 + threadIdx.x;
    if (cc < nset) {
      double2 t = red[threadIdx.x][0];
#pragma unroll
      for (int q = 1; q < 4; ++q) t = cadd(t, red[threadIdx.x][q]);
      ((double2*)p.cpart)[(int64_t)rb * p.ncol + cc] = t;
    }
  }
}


// w[row] = x[row] - sum_{c < nm} Um[row, c] coef[pass][c] (- i sum_{c'} Ut[row, c'] coef[pass][nm+c']
// on the PH paths: the twin projection).  grid (ceil(maxNpad/32), nprob), 8 warps: lane = row of a
// 32-row slab, warp w takes the set entries c = w mod 8 (six or eight loads in flight each),
// and the eight partial sums meet in shared memory.  Spreading the columns over warps keeps
// enough loads in flight when N is only a few hundred slabs; three CTAs per SM keep N = 10^4
// (316 slabs) in one wave (ncu: at two per SM the last 12 CTAs ran as a second wave).
template <typename ST>
__global__ void __launch_bounds__(256, 3)
k_cgs_update(const Prob* __restrict__ probs, int ph, int pass, int newvec, int half) {
  using R = typename RealOf<ST>::T;
  __shared__ ST cf[2 * MAXM + 2];
  __shared__ ST red[8][32];
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  const int64_t row = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  if ((int64_t)blockIdx.x * 32 >= p.Npad) return;     // whole block (Npad is a multiple of 128)
  const CgsSet cs = cgs_set(p, st, ph, half);
  const int nm = cs.nm;
  const int nset = nm + cs.nt;
  // coefficients: the row-block partial sums of the dots, added in row-block order (PH: real
  // part only); the first row slab also stores them for k_step_finish
  const double2* cp = (const double2*)p.cpart;
  double2* coef = (double2*)p.coef + (int64_t)(pass & 1) * p.ncol;
  for (int c = threadIdx.x; c < nset; c += blockDim.x) {
    double2 sc = mk(0.0, 0.0);
    for (int rb = 0; rb < p.nrb; ++rb) sc = cadd(sc, cp[(int64_t)rb * p.ncol + c]);
    if (ph) sc.y = 0.0;
    cf[c] = ccvt<ST>(sc);
    if (blockIdx.x == 0) coef[c] = sc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ST* vb = (const ST*)cs.um + row;
  const ST* pb = ph ? (const ST*)cs.ut + row : nullptr;
  constexpr int U = sizeof(ST) == 16 ? 6 : 8;   // loads in flight per thread (registers for 3 CTAs/SM)
  const int64_t ld = p.Npad;
  // entry cc of the set: Um[:, cc] for cc < nm, else the twin i Ut[:, cc - nm] (as (-t.y, t.x))
  auto colval = [&](int cc) -> ST {
    if (cc < nm) return __ldg(vb + (int64_t)cc * ld);
    const ST q = __ldg(pb + (int64_t)(cc - nm) * ld);
    ST t;
    t.x = -q.y;
    t.y = q.x;
    return t;
  };
  ST part = czero<ST>();
  int c = warp;
  // all U loads of a round are issued before any of their arithmetic
  if (ph) {                                 // real coefficients (K-inner products, twin projections)
    R ax[U], ay[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ax[u] = ay[u] = (R)0;
    for (; c + 8 * (U - 1) < nset; c += 8 * U) {
      ST v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = colval(c + 8 * u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const R f = cf[c + 8 * u].x;
        ax[u] = fma(v[u].x, f, ax[u]);
        ay[u] = fma(v[u].y, f, ay[u]);
      }
    }
    for (; c < nset; c += 8) {
      const ST v = colval(c);
      const R f = cf[c].x;
      ax[0] = fma(v.x, f, ax[0]);
      ay[0] = fma(v.y, f, ay[0]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      part.x += ax[u];
      part.y += ay[u];
    }
  } else {
    ST acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = czero<ST>();
    for (; c + 8 * (U - 1) < nset; c += 8 * U) {
      ST v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = __ldg(vb + (int64_t)(c + 8 * u) * ld);
#pragma unroll
      for (int u = 0; u < U; ++u) cfma(acc[u], v[u], cf[c + 8 * u]);
    }
    for (; c < nset; c += 8) cfma(acc[0], __ldg(vb + (int64_t)c * ld), cf[c]);
#pragma unroll
    for (int u = 0; u < U; ++u) part = cadd(part, acc[u]);
  }
  red[warp][lane] = part;
  __syncthreads();
  if (warp == 0) {
    ST tot = red[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) tot = cadd(tot, red[q][lane]);
    const ST* x = cgs_src<ST>(p, st, half, pass, newvec);
    ST* w = (ST*)p.w;
    w[row] = csub(x[row], tot);
  }
}

// ---------------------------------------------------------------- norms
// cpart[rb].x = sum over rows of Re(conj(w) pw) (PH) or |w|^2 (TDA).
template <typename ST>
__global__ void __launch_bounds__(256)
k_norm_partial(const Prob* __restrict__ probs, int ph, int start) {
  __shared__ double red[8];
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (!kphase(st, start)) return;
  const int rb = blockIdx.x;
  if (rb >= p.nrb) return;
  const ST* w = (const ST*)p.w;
  const ST* pw = (const ST*)(ph ? p.pw : p.w);
  const int64_t r0 = (int64_t)rb * ROWBLK;
  const int64_t r1 = min((int64_t)p.Npad, r0 + ROWBLK);
  double s = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += 256) {
    const ST a = w[r], b = pw[r];
    s += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    ((double2*)p.cpart)[rb] = mk(t, 0.0);
  }
}

__device__ __forceinline__ double sum_norm_parts(const Prob& p) {
  const double2* cp = (const double2*)p.cpart;
  double s = 0.0;
  for (int rb = 0; rb < p.nrb; ++rb) s += cp[rb].x;
  return s;
}

// Where a normalised vector goes: V[:, j+1] (and P) for the folded / TDA step and the even
// half of a Gruning step, W[:, j] (and Z) for the odd half.
template <typename ST>
__device__ __forceinline__ void norm_dest(const Prob& p, const KState* st, int half, ST*& X, ST*& Y) {
  if (half == 1) {
    X = (ST*)p.W + (int64_t)st->j * p.Npad;
    Y = (ST*)p.Z + (int64_t)st->j * p.Npad;
  } else {
    X = (ST*)p.V + (int64_t)(st->j + 1) * p.Npad;
    Y = p.ph ? (ST*)p.P + (int64_t)(st->j + 1) * p.Npad : nullptr;
  }
}

// X = w / beta, Y = pw / beta (norm_dest) when beta^2 is usable.
template <typename ST>
__global__ void __launch_bounds__(256)
k_normalize(const Prob* __restrict__ probs, int ph, int start, int half) {
  using R = typename RealOf<ST>::T;
  __shared__ double sb2;
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (!kphase(st, start)) return;
  if (threadIdx.x == 0) sb2 = sum_norm_parts(p);
  __syncthreads();
  const double b2 = sb2;
  if (!(b2 > 0.0) || !isfinite(b2)) return;   // k_step_finish records the outcome
  const R inv = (R)(1.0 / sqrt(b2));
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= p.Npad) return;
  ST *X, *Y;
  norm_dest<ST>(p, st, half, X, Y);
  X[row] = cscale(((const ST*)p.w)[row], inv);
  if (ph) Y[row] = cscale(((const ST*)p.pw)[row], inv);
}

// Record alpha_j, beta_j, advance j, given beta^2 = b2 of the new vector.  fresh = 0:
// regular step; fresh = 1: a first or replacement vector was just normalised.
__device__ void step_finish_one(const Prob& p, int ph, int fresh, double b2) {
  KState* st = p.st;
  const int j = st->j;
  if (!fresh) {
    const double2* coef = (const double2*)p.coef;
    const double a = coef[j].x + coef[p.ncol + j].x;
    if (!isfinite(a) || !isfinite(b2)) { st->status = ST_NOTFINITE; return; }
    p.alpha[j] = a;
    st->passes += ph ? 2 : 1;
    st->steps += 1;
    // scale of the projected matrix for the breakdown test
    double scale = fabs(a);
    for (int i = st->k; i < st->l; ++i) scale = fmax(scale, fabs(p.theta[i]));
    if (j > 0) scale = fmax(scale, fabs(p.beta[j - 1]));
    const double tiny = 1e-26 * scale * scale + 1e-300;
    if (ph && b2 < -1e6 * tiny) { st->status = ST_NOTPD; return; }
    if (b2 <= tiny) {                 // invariant subspace: the chain restarts
      p.beta[j] = 0.0;                // with a fresh vector (host-driven)
      st->breakdown = 1;
      return;
    }
    p.beta[j] = sqrt(b2);
    st->j = j + 1;
  } else {
    if (!isfinite(b2)) { st->status = ST_NOTFINITE; return; }
    if (!(b2 > 0.0)) { st->status = ph ? ST_NOTPD : ST_NOTFINITE; return; }
    st->breakdown = 0;
    st->passes += ph ? 1 : 0;
    st->j = j + 1;
  }
  if (st->steps >= st->maxit && !st->done) { st->done = 1; st->status = ST_NOCONV; }
}

// Gruning step: record alpha_j (odd half) or beta_j and advance j (even half), given the
// squared M-norm b2 of the new vector; fresh = 1: a first or replacement even vector.
// An odd vector cannot vanish when M+ is positive definite (M+ maps the j + 1 even
// vectors onto j + 1 independent odd ones), so a vanishing alpha means not definite.
__device__ void gk_finish_one(const Prob& p, int half, int fresh, double b2) {
  KState* st = p.st;
  const int j = st->j;
  if (!isfinite(b2)) { st->status = ST_NOTFINITE; return; }
  if (fresh) {
    if (!(b2 > 0.0)) { st->status = ST_NOTPD; return; }
    st->breakdown = 0;
    st->passes += 1;
    st->j = j + 1;
  } else {
    double scale = 0.0;
    for (int i = st->k; i < st->l; ++i) scale = fmax(scale, fabs(p.theta[i]));
    if (j > 0) scale = fmax(scale, p.beta[j - 1]);
    if (half == 2) scale = fmax(scale, p.alpha[j]);
    const double tiny = 1e-26 * scale * scale + 1e-300;
    if (b2 < -1e6 * tiny) { st->status = ST_NOTPD; return; }
    if (half == 1) {
      if (b2 <= tiny) { st->status = ST_NOTPD; return; }
      p.alpha[j] = sqrt(b2);
      return;                           // the even half follows in the same step
    }
    st->passes += 2;
    st->steps += 1;
    if (b2 <= tiny) {                   // invariant subspace: the chain restarts
      p.beta[j] = 0.0;                  // with a fresh vector (host-driven)
      st->breakdown = 1;
      return;
    }
    p.beta[j] = sqrt(b2);
    st->j = j + 1;
  }
  if (st->steps >= st->maxit && !st->done) { st->done = 1; st->status = ST_NOCONV; }
}

__device__ __forceinline__ void finish_one(const Prob& p, int ph, int fresh, int half, double b2) {
  if (half) gk_finish_one(p, half, fresh, b2);
  else step_finish_one(p, ph, fresh, b2);
}

// One thread per problem.
__global__ void k_step_finish(const Prob* __restrict__ probs, int nprob, int ph, int fresh, int half) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= nprob) return;
  const Prob& p = probs[ip];
  if (!kphase(p.st, fresh)) return;
  finish_one(p, ph, fresh, half, sum_norm_parts(p));
}

// Problems of at most one reduction row block (Npad <= ROWBLK): the norm, the scaling of
// the new basis vector and the state update in one CTA per problem (one launch instead of
// three per Krylov step; the same arithmetic as k_norm_partial, k_normalize, k_step_finish).
template <typename ST>
__global__ void __launch_bounds__(256)
k_norm_fused(const Prob* __restrict__ probs, int ph, int start, int half) {
  using R = typename RealOf<ST>::T;
  __shared__ double red[8];
  __shared__ double sb2;
  const Prob& p = probs[blockIdx.x];
  const KState* st = p.st;
  if (!kphase(st, start)) return;
  const ST* w = (const ST*)p.w;
  const ST* pw = (const ST*)(ph ? p.pw : p.w);
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < p.Npad; r += 256) {
    const ST a = w[r], b = pw[r];
    s += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    sb2 = t;
  }
  __syncthreads();
  const double b2 = sb2;
  if (b2 > 0.0 && isfinite(b2)) {
    const R inv = (R)(1.0 / sqrt(b2));
    ST *X, *Y;
    norm_dest<ST>(p, st, half, X, Y);
    for (int64_t r = threadIdx.x; r < p.Npad; r += 256) {
      X[r] = cscale(w[r], inv);
      if (ph) Y[r] = cscale(((const ST*)p.pw)[r], inv);
    }
  }
  __syncthreads();                     // every thread has read st->j
  if (threadIdx.x == 0) finish_one(p, ph, start, half, b2);
}

// ---------------------------------------------------------------- start vector
// Counter-based complex Gaussian-like entries: splitmix64 of (seed, row),
// Box-Muller on two 53-bit uniforms.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ double2 hash_normal(uint64_t seed, uint64_t i) {
  const uint64_t a = splitmix64(seed ^ splitmix64(2 * i));
  const uint64_t b = splitmix64(seed ^ splitmix64(2 * i + 1));
  const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);
  const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return mk(r * c, r * s);
}

// w = v0 (if given, single problem) or random; rows >= N are zero.
template <typename ST>
__global__ void k_start_fill(const Prob* __restrict__ probs, uint64_t seed, const ST* __restrict__ v0) {
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (!kfresh(st)) return;
  if (st->j >= 0) v0 = nullptr;     // replacement vectors are always random
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= p.Npad) return;
  ST v = czero<ST>();
  if (row < p.N) {
    if (v0) v = v0[row];
    else v = ccvt<ST>(hash_normal(seed + 0x51ed27ull * (uint64_t)(blockIdx.y + 1) + (uint64_t)st->restarts, row));
  }
  ((ST*)p.w)[row] = v;
}

// ---------------------------------------------------------------- restart
// V2[:, i] = sum_{c < n} V[:, k0 + c] S[c, i], i < nkeep (which = 0; P2 from P: 1; on the
// Gruning path W2 from W and Z2 from Z with the odd-side coefficients S2: 2, 3).
// grid (ceil(maxNpad/64), ceil(ncv/16), nprob), 256 threads: 64 rows x 16 cols,
// each thread 1 row x 4 columns.
template <typename ST>
__global__ void __launch_bounds__(256)
k_restart_gemm(const Prob* __restrict__ probs, int which) {
  using R = typename RealOf<ST>::T;
  __shared__ ST sv[32][64];
  __shared__ R ss[32][16];
  const Prob& p = probs[blockIdx.z];
  const KState* st = p.st;
  if (st->status != ST_OK || !st->r_go) return;   // decided in this restart only
  const int k0 = st->r_k0, nkeep = st->r_nkeep;
  const int n = st->m - k0;
  const int i0 = blockIdx.y * 16;
  if (i0 >= nkeep) return;
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  if (r0 >= p.Npad) return;
  const void* srcs[4] = {p.V, p.P, p.W, p.Z};
  void* dsts[4] = {p.V2, p.P2, p.W2, p.Z2};
  const ST* src = (const ST*)srcs[which] + (int64_t)k0 * p.Npad;
  ST* dst = (ST*)dsts[which];
  const double* Sc = which >= 2 ? p.S2 : p.S;
  const int tid = threadIdx.x, rr = tid & 63, cg = tid >> 6;
  ST acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = czero<ST>();
  for (int c0 = 0; c0 < n; c0 += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * 64; e += 256) {
      const int cc = e >> 6, r = e & 63;
      const int64_t row = r0 + r;
      sv[cc][r] = (c0 + cc < n && row < p.Npad) ? src[(int64_t)(c0 + cc) * p.Npad + row] : czero<ST>();
    }
    for (int e = tid; e < 32 * 16; e += 256) {
      const int cc = e >> 4, ii = e & 15;
      ss[cc][ii] = (c0 + cc < n && i0 + ii < nkeep) ? (R)Sc[(int64_t)(i0 + ii) * p.ncv + c0 + cc] : (R)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int cc = 0; cc < 32; ++cc) {
      const ST v = sv[cc][rr];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const R f = ss[cc][cg * 4 + q];
        acc[q].x = fma(v.x, f, acc[q].x);
        acc[q].y = fma(v.y, f, acc[q].y);
      }
    }
  }
  const int64_t row = r0 + rr;
  if (row < p.Npad) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + cg * 4 + q;
      if (i < nkeep) dst[(int64_t)i * p.Npad + row] = acc[q];
    }
  }
}

// V[:, k0+i] = V2[:, i]; V[:, k0+nkeep] = V[:, m]; same for P; W[:, k0+i] = W2[:, i] and
// Z from Z2 on the Gruning path (the odd basis has no extra column).
template <typename ST>
__global__ void k_restart_copy(const Prob* __restrict__ probs, int ph, int gk) {
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (st->status != ST_OK || !st->r_go) return;   // decided in this restart only
  const int k0 = st->r_k0, nkeep = st->r_nkeep, m = st->m;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= p.Npad) return;
  ST* V = (ST*)p.V;
  const ST* V2 = (const ST*)p.V2;
  const ST vm = V[(int64_t)m * p.Npad + row];
  for (int i = 0; i < nkeep; ++i) V[(int64_t)(k0 + i) * p.Npad + row] = V2[(int64_t)i * p.Npad + row];
  V[(int64_t)(k0 + nkeep) * p.Npad + row] = vm;
  if (ph) {
    ST* P = (ST*)p.P;
    const ST* P2 = (const ST*)p.P2;
    const ST pm = P[(int64_t)m * p.Npad + row];
    for (int i = 0; i < nkeep; ++i) P[(int64_t)(k0 + i) * p.Npad + row] = P2[(int64_t)i * p.Npad + row];
    P[(int64_t)(k0 + nkeep) * p.Npad + row] = pm;
  }
  if (gk) {
    ST* W = (ST*)p.W;
    ST* Z = (ST*)p.Z;
    const ST* W2 = (const ST*)p.W2;
    const ST* Z2 = (const ST*)p.Z2;
    for (int i = 0; i < nkeep; ++i) {
      W[(int64_t)(k0 + i) * p.Npad + row] = W2[(int64_t)i * p.Npad + row];
      Z[(int64_t)(k0 + i) * p.Npad + row] = Z2[(int64_t)i * p.Npad + row];
    }
  }
}

__global__ void k_restart_commit(const Prob* __restrict__ probs, int nprob, int ph) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= nprob) return;
  const Prob& p = probs[ip];
  KState* st = p.st;
  if (st->status != ST_OK || !st->r_go) return;   // decided in this restart only
  const int k0 = st->r_k0;
  st->k = k0 + st->r_nl;
  st->l = k0 + st->r_nkeep;
  st->j = st->l;
  st->restarts += 1;
  st->r_go = 0;
  if (st->k >= st->nev) st->done = 1;
  else if (st->steps >= st->maxit) { st->done = 1; st->status = ST_NOCONV; }
}

// ---------------------------------------------------------------- launchers
template <typename ST>
void launch_step_cgs(const Prob* dprobs, int nprob, int ph, int maxnrb, int64_t maxNpad, int ncol,
                     int pass, int half, cudaStream_t s) {
  // pass: 0/1 regular step passes; 2/3 the same for a fresh (replacement) vector
  count_launch(2);
  const int newvec = pass >= 2 ? 1 : 0;
  const int ps = pass & 1;
  k_cgs_dot<ST><<<dim3((ncol + 1) / 2, maxnrb, nprob), 256, 0, s>>>(dprobs, ph, newvec, half, ps);
  k_cgs_update<ST><<<dim3((unsigned)((maxNpad + 31) / 32), nprob), 256, 0, s>>>(dprobs, ph, ps, newvec, half);
}

template <typename ST>
void launch_step_normalize(const Prob* dprobs, int nprob, int ph, int maxnrb, int64_t maxNpad,
                           int start, int half, cudaStream_t s) {
  if (maxnrb == 1) {
    count_launch();
    k_norm_fused<ST><<<nprob, 256, 0, s>>>(dprobs, ph, start, half);
    return;
  }
  count_launch(3);
  // start: 0 regular step, 1 fresh (first or replacement) vector
  k_norm_partial<ST><<<dim3(maxnrb, nprob), 256, 0, s>>>(dprobs, ph, start);
  k_normalize<ST><<<dim3((unsigned)((maxNpad + 255) / 256), nprob), 256, 0, s>>>(dprobs, ph, start, half);
  k_step_finish<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob, ph, start, half);
}

template <typename ST>
void launch_start_vector(const Prob* dprobs, int nprob, int64_t maxNpad, uint64_t seed, const void* v0,
                         cudaStream_t s) {
  count_launch();
  // fills w for every problem that needs a fresh vector
  k_start_fill<ST><<<dim3((unsigned)((maxNpad + 255) / 256), nprob), 256, 0, s>>>(
      dprobs, seed, (const ST*)v0);
}

template <typename ST>
void launch_restart(const Prob* dprobs, int nprob, int ph, int64_t maxNpad, int ncv, bool gruning,
                    cudaStream_t s) {
  const int ngemm = ph ? (gruning ? 4 : 2) : 1;
  count_launch(ngemm + 2);
  const unsigned gx = (unsigned)((maxNpad + 63) / 64);
  for (int which = 0; which < ngemm; ++which)
    k_restart_gemm<ST><<<dim3(gx, (ncv + 15) / 16, nprob), 256, 0, s>>>(dprobs, which);
  const unsigned gr = (unsigned)((maxNpad + 255) / 256);
  k_restart_copy<ST><<<dim3(gr, nprob), 256, 0, s>>>(dprobs, ph, gruning ? 1 : 0);
  k_restart_commit<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob, ph);
}

#define INST(ST)                                                                                        \
  template void launch_step_cgs<ST>(const Prob*, int, int, int, int64_t, int, int, int, cudaStream_t); \
  template void launch_step_normalize<ST>(const Prob*, int, int, int, int64_t, int, int, cudaStream_t); \
  template void launch_start_vector<ST>(const Prob*, int, int64_t, uint64_t, const void*,              \
                                        cudaStream_t);                                                  \
  template void launch_restart<ST>(const Prob*, int, int, int64_t, int, bool, cudaStream_t);
INST(float2)
INST(double2)
#undef INST

}  // namespace bse
