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

// ---------------------------------------------------------------- CGS2 dots
// PH: cpart[rb][c] = sum_{rows in block rb} Re(conj(P[row, c]) w[row]) for
// c <= j (the K-inner products with the basis) and Im(conj(V[row, c']) w[row])
// for c = j + 1 + c' (the twin coefficients s of the header), 2 (j + 1) in
// all; TDA: the complex conj(V[row, c]) w[row], c <= j.  grid (ceil(maxcols/2),
// maxnrb, nprob), 8 warps: two columns per CTA, four warps per column, each
// warp a quarter of the block rows; the four partial sums meet in shared
// memory (fixed order).
template <typename ST>
__global__ void __launch_bounds__(256)
k_cgs_dot(const Prob* __restrict__ probs, int ph, int newvec) {
  using R = typename RealOf<ST>::T;
  __shared__ double2 red[2][4];
  const Prob& p = probs[blockIdx.z];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  const int rb = blockIdx.y;
  if (rb >= p.nrb) return;
  const int j = st->j;
  const int nset = ph ? 2 * (j + 1) : j + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = warp >> 2, quarter = warp & 3;
  const int c = blockIdx.x * 2 + half;
  if (blockIdx.x * 2 >= nset) return;                     // whole CTA
  double2 a = mk(0.0, 0.0);
  if (c < nset) {
    const bool twin = c > j;                              // warp-uniform
    const int col = twin ? c - (j + 1) : c;
    const ST* Q = (const ST*)(ph && !twin ? p.P : p.V) + (int64_t)col * p.Npad;
    const ST* w = (const ST*)p.w;
    const int64_t r0 = (int64_t)rb * ROWBLK + quarter * (ROWBLK / 4);
    const int64_t r1 = min((int64_t)p.Npad, r0 + ROWBLK / 4);
    // rounds of 8 rows per lane: all 16 loads of a round are issued before its arithmetic
    int64_t r = r0 + lane;
    if (ph) {   // real coefficients: Re(conj(q) w), or Im(conj(v) w) = Re(conj(v) (-i w)) for twins
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
  if (lane == 0) red[half][quarter] = a;
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


// w[row] -= sum_{c <= j} V[row, c] coef[pass][c] (+ i sum_{c'} P[row, c'] coef[pass][j+1+c'] on the
// PH path: the twin projection).  grid (ceil(maxNpad/32), nprob), 8 warps: lane = row of a
// 32-row slab, warp w takes the set entries c = w mod 8 (six or eight loads in flight each),
// and the eight partial sums meet in shared memory.  Spreading the columns over warps keeps
// enough loads in flight when N is only a few hundred slabs; three CTAs per SM keep N = 10^4
// (316 slabs) in one wave (ncu: at two per SM the last 12 CTAs ran as a second wave).
template <typename ST>
__global__ void __launch_bounds__(256, 3)
k_cgs_update(const Prob* __restrict__ probs, int ph, int pass, int newvec) {
  using R = typename RealOf<ST>::T;
  __shared__ ST cf[2 * MAXM + 2];
  __shared__ ST red[8][32];
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  const int64_t row = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  if ((int64_t)blockIdx.x * 32 >= p.Npad) return;     // whole block (Npad is a multiple of 128)
  const int j = st->j;
  const int nj = j + 1;                     // basis columns [0, j]
  const int nset = ph ? 2 * nj : nj;
  // coefficients: the row-block partial sums of the dots, added in row-block order (PH: real
  // part only); the first row slab also stores them for k_step_finish
  const double2* cp = (const double2*)p.cpart;
  double2* coef = (double2*)p.coef + (int64_t)pass * p.ncol;
  for (int c = threadIdx.x; c < nset; c += blockDim.x) {
    double2 sc = mk(0.0, 0.0);
    for (int rb = 0; rb < p.nrb; ++rb) sc = cadd(sc, cp[(int64_t)rb * p.ncol + c]);
    if (ph) sc.y = 0.0;
    cf[c] = ccvt<ST>(sc);
    if (blockIdx.x == 0) coef[c] = sc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ST* vb = (const ST*)p.V + row;
  const ST* pb = ph ? (const ST*)p.P + row : nullptr;
  constexpr int U = sizeof(ST) == 16 ? 6 : 8;   // loads in flight per thread (registers for 3 CTAs/SM)
  const int64_t ld = p.Npad;
  // entry cc of the set: V[:, cc] for cc < nj, else the twin i P[:, cc - nj] (as (-p.y, p.x))
  auto colval = [&](int cc) -> ST {
    if (cc < nj) return __ldg(vb + (int64_t)cc * ld);
    const ST q = __ldg(pb + (int64_t)(cc - nj) * ld);
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
    ST* w = (ST*)p.w;
    w[row] = csub(w[row], tot);
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

// V[:, j+1] = w / beta, P[:, j+1] = pw / beta when beta^2 is usable.
template <typename ST>
__global__ void __launch_bounds__(256)
k_normalize(const Prob* __restrict__ probs, int ph, int start) {
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
  const int col = st->j + 1;
  ST* V = (ST*)p.V + (int64_t)col * p.Npad;
  V[row] = cscale(((const ST*)p.w)[row], inv);
  if (ph) {
    ST* P = (ST*)p.P + (int64_t)col * p.Npad;
    P[row] = cscale(((const ST*)p.pw)[row], inv);
  }
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

// One thread per problem.
__global__ void k_step_finish(const Prob* __restrict__ probs, int nprob, int ph, int fresh) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= nprob) return;
  const Prob& p = probs[ip];
  if (!kphase(p.st, fresh)) return;
  step_finish_one(p, ph, fresh, sum_norm_parts(p));
}

// Problems of at most one reduction row block (Npad <= ROWBLK): the norm, the scaling of
// the new basis vector and the state update in one CTA per problem (one launch instead of
// three per Krylov step; the same arithmetic as k_norm_partial, k_normalize, k_step_finish).
template <typename ST>
__global__ void __launch_bounds__(256)
k_norm_fused(const Prob* __restrict__ probs, int ph, int start) {
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
    const int col = st->j + 1;
    ST* V = (ST*)p.V + (int64_t)col * p.Npad;
    ST* P = ph ? (ST*)p.P + (int64_t)col * p.Npad : nullptr;
    for (int64_t r = threadIdx.x; r < p.Npad; r += 256) {
      V[r] = cscale(w[r], inv);
      if (ph) P[r] = cscale(((const ST*)p.pw)[r], inv);
    }
  }
  __syncthreads();                     // every thread has read st->j
  if (threadIdx.x == 0) step_finish_one(p, ph, start, b2);
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
// V2[:, i] = sum_{c < n} V[:, k0 + c] S[c, i], i < nkeep (and P2 from P).
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
  const ST* src = (const ST*)(which ? p.P : p.V) + (int64_t)k0 * p.Npad;
  ST* dst = (ST*)(which ? p.P2 : p.V2);
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
      ss[cc][ii] = (c0 + cc < n && i0 + ii < nkeep) ? (R)p.S[(int64_t)(i0 + ii) * p.ncv + c0 + cc] : (R)0;
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

// V[:, k0+i] = V2[:, i]; V[:, k0+nkeep] = V[:, m]; same for P.
template <typename ST>
__global__ void k_restart_copy(const Prob* __restrict__ probs, int ph) {
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
                     int pass, cudaStream_t s) {
  // pass: 0/1 regular step passes; 2/3 the same for a fresh (replacement) vector
  count_launch(2);
  const int newvec = pass >= 2 ? 1 : 0;
  const int ps = pass & 1;
  k_cgs_dot<ST><<<dim3((ncol + 1) / 2, maxnrb, nprob), 256, 0, s>>>(dprobs, ph, newvec);
  k_cgs_update<ST><<<dim3((unsigned)((maxNpad + 31) / 32), nprob), 256, 0, s>>>(dprobs, ph, ps, newvec);
}

template <typename ST>
void launch_step_normalize(const Prob* dprobs, int nprob, int ph, int maxnrb, int64_t maxNpad,
                           int start, cudaStream_t s) {
  if (maxnrb == 1) {
    count_launch();
    k_norm_fused<ST><<<nprob, 256, 0, s>>>(dprobs, ph, start);
    return;
  }
  count_launch(3);
  // start: 0 regular step, 1 fresh (first or replacement) vector
  k_norm_partial<ST><<<dim3(maxnrb, nprob), 256, 0, s>>>(dprobs, ph, start);
  k_normalize<ST><<<dim3((unsigned)((maxNpad + 255) / 256), nprob), 256, 0, s>>>(dprobs, ph, start);
  k_step_finish<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob, ph, start);
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
void launch_restart(const Prob* dprobs, int nprob, int ph, int64_t maxNpad, int ncv, cudaStream_t s) {
  count_launch(ph ? 4 : 3);
  const unsigned gx = (unsigned)((maxNpad + 63) / 64);
  k_restart_gemm<ST><<<dim3(gx, (ncv + 15) / 16, nprob), 256, 0, s>>>(dprobs, 0);
  if (ph) k_restart_gemm<ST><<<dim3(gx, (ncv + 15) / 16, nprob), 256, 0, s>>>(dprobs, 1);
  const unsigned gr = (unsigned)((maxNpad + 255) / 256);
  k_restart_copy<ST><<<dim3(gr, nprob), 256, 0, s>>>(dprobs, ph);
  k_restart_commit<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob, ph);
}

#define INST(ST)                                                                                   \
  template void launch_step_cgs<ST>(const Prob*, int, int, int, int64_t, int, int, cudaStream_t); \
  template void launch_step_normalize<ST>(const Prob*, int, int, int, int64_t, int, cudaStream_t); \
  template void launch_start_vector<ST>(const Prob*, int, int64_t, uint64_t, const void*,         \
                                        cudaStream_t);                                             \
  template void launch_restart<ST>(const Prob*, int, int, int64_t, int, cudaStream_t);
INST(float2)
INST(double2)
#undef INST

}  // namespace bse
