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
#include "bse_phases.cuh"

namespace bse {

// ---------------------------------------------------------------- one kernel per phase
// The bodies (bse_phases.cuh) on the grids of the launchers below.
template <typename ST>
__global__ void __launch_bounds__(256)
k_cgs_dot(const Prob* __restrict__ probs, int ph, int newvec, int half, int pass) {
  __shared__ double2 red[2][4];
  cgs_dot_body<ST, false>(probs, ph, newvec, half, pass, blockIdx.x, blockIdx.y, blockIdx.z, red);
}

// three CTAs per SM keep N = 10^4 (316 slabs of 32 rows) in one wave (ncu: at two per SM the
// last 12 CTAs ran as a second wave)
template <typename ST>
__global__ void __launch_bounds__(256, 3)
k_cgs_update(const Prob* __restrict__ probs, int ph, int pass, int newvec, int half) {
  __shared__ ST cf[2 * MAXM + 2];
  __shared__ ST red[8][32];
  cgs_update_body<ST, false>(probs, ph, pass, newvec, half, blockIdx.x, blockIdx.y, cf, red);
}

// ---------------------------------------------------------------- double-FP32 Gram-Schmidt
// The folded step's CGS passes on the mixed path, on the double-FP32 shadows of V, P and w
// (48 bits of each FP64 value): a product a b of two (hi, lo) numbers is hi*hi exactly (its FMA
// residual) plus the two cross terms, sums are (hi, lo) pairs kept with Knuth's TwoSum, about
// 2^-44 relative per term.  GB300 runs FP64 at 1/64 of the FP32 rate, and the FP64 passes were
// bound by it, not by HBM; here the FP32 pipes carry them.  Same units, same partial-sum slots
// and the same fixed summation orders as k_cgs_dot / k_cgs_update.
__device__ __forceinline__ void df_madd(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float pr = ah * bh;
  const float e = __fmaf_rn(ah, bh, -pr);
  const float t = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  const float su = sh + pr;
  const float bb = su - sh;
  const float err = (sh - (su - bb)) + (pr - bb);
  sh = su;
  sl += err + t;
}
__device__ __forceinline__ void df_add(float& sh, float& sl, float bh, float bl) {
  const float su = sh + bh;
  const float bb = su - sh;
  const float err = (sh - (su - bb)) + (bh - bb);
  sh = su;
  sl += err + bl;
}

// units and output as k_cgs_dot (folded step, half 0: Re(P^H w) and Im(V^H w))
__global__ void __launch_bounds__(256)
k_cgs_dot_dfs(const Prob* __restrict__ probs, int newvec) {
  __shared__ double red[2][4];
  const Prob& p = probs[blockIdx.z];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  const int rb = blockIdx.y;
  if (rb >= p.nrb) return;
  const int j = st->j;
  const int nset = 2 * (j + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hw = warp >> 2, quarter = warp & 3;
  const int c = blockIdx.x * 2 + hw;
  if (blockIdx.x * 2 >= nset) return;                     // whole CTA
  double a = 0.0;
  if (c < nset) {
    const bool twin = c > j;                              // warp-uniform
    const int col = twin ? c - (j + 1) : c;
    const float4* Q = (twin ? p.Vs : p.Ps) + (int64_t)col * p.Npad;
    const float4* w = p.ws;
    const int64_t r0 = (int64_t)rb * ROWBLK + quarter * (ROWBLK / 4);
    const int64_t r1 = min((int64_t)p.Npad, r0 + ROWBLK / 4);
    float sh = 0.f, sl = 0.f;
    int64_t r = r0 + lane;
    for (; r + 3 * 32 < r1; r += 4 * 32) {
      float4 q[4], x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        q[u] = __ldg(Q + r + 32 * u);
        x[u] = __ldg(w + r + 32 * u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (twin) {              // Im(conj(q) x) = q_re x_im - q_im x_re
          df_madd(sh, sl, q[u].x, q[u].z, x[u].y, x[u].w);
          df_madd(sh, sl, -q[u].y, -q[u].w, x[u].x, x[u].z);
        } else {                 // Re(conj(q) x) = q_re x_re + q_im x_im
          df_madd(sh, sl, q[u].x, q[u].z, x[u].x, x[u].z);
          df_madd(sh, sl, q[u].y, q[u].w, x[u].y, x[u].w);
        }
      }
    }
    for (; r < r1; r += 32) {
      const float4 q = __ldg(Q + r), x = __ldg(w + r);
      if (twin) {
        df_madd(sh, sl, q.x, q.z, x.y, x.w);
        df_madd(sh, sl, -q.y, -q.w, x.x, x.z);
      } else {
        df_madd(sh, sl, q.x, q.z, x.x, x.z);
        df_madd(sh, sl, q.y, q.w, x.y, x.w);
      }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, sh, m), ol = __shfl_xor_sync(0xffffffffu, sl, m);
      df_add(sh, sl, oh, ol);
    }
    a = (double)sh + (double)sl;
  }
  if (lane == 0) red[hw][quarter] = a;
  __syncthreads();
  if (threadIdx.x < 2) {
    const int cc = blockIdx.x * 2 + threadIdx.x;
    if (cc < nset) {
      double t = red[threadIdx.x][0];
#pragma unroll
      for (int q = 1; q < 4; ++q) t += red[threadIdx.x][q];
      ((double2*)p.cpart)[(int64_t)rb * p.ncol + cc] = mk(t, 0.0);
    }
  }
}

// units as k_cgs_update: w = w - V c - i P d (c, d the pass's real coefficients), and ws
__global__ void __launch_bounds__(256, 3)
k_cgs_update_dfs(const Prob* __restrict__ probs, int pass, int newvec) {
  __shared__ float2 cf[2 * MAXM + 2];
  __shared__ float4 red[8][32];
  const Prob& p = probs[blockIdx.y];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  const int64_t row = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  if ((int64_t)blockIdx.x * 32 >= p.Npad) return;     // whole block (Npad is a multiple of 128)
  const int nj = st->j + 1;
  const int nset = 2 * nj;
  const double2* cp = (const double2*)p.cpart;
  double2* coef = (double2*)p.coef + (int64_t)(pass & 1) * p.ncol;
  for (int c = threadIdx.x; c < nset; c += blockDim.x) {
    double sc = 0.0;
    int rb = 0;
    for (; rb + 8 <= p.nrb; rb += 8) {      // eight loads in flight, then the sums in order
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = cp[(int64_t)(rb + u) * p.ncol + c].x;
#pragma unroll
      for (int u = 0; u < 8; ++u) sc += v[u];
    }
    for (; rb < p.nrb; ++rb) sc += cp[(int64_t)rb * p.ncol + c].x;
    const float h = (float)sc;
    cf[c] = make_float2(h, (float)(sc - (double)h));
    if (blockIdx.x == 0) coef[c] = mk(sc, 0.0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // entry cc: V[:, cc] (cc < nj) or the twin i P[:, cc - nj] = (-P_im, P_re)
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  for (int c = warp; c < nset; c += 8) {
    const bool tw = c >= nj;
    const float4 v = __ldg((tw ? p.Ps : p.Vs) + (int64_t)(tw ? c - nj : c) * p.Npad + row);
    const float2 f = cf[c];
    if (tw) {
      df_madd(rh, rl, -v.y, -v.w, f.x, f.y);
      df_madd(ih, il, v.x, v.z, f.x, f.y);
    } else {
      df_madd(rh, rl, v.x, v.z, f.x, f.y);
      df_madd(ih, il, v.y, v.w, f.x, f.y);
    }
  }
  red[warp][lane] = make_float4(rh, rl, ih, il);
  __syncthreads();
  if (warp == 0) {
    float4 t = red[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      const float4 o = red[q][lane];
      df_add(t.x, t.y, o.x, o.y);
      df_add(t.z, t.w, o.z, o.w);
    }
    double2* w = (double2*)p.w;
    const double2 x = w[row];
    const double2 y = mk(x.x - ((double)t.x + (double)t.y), x.y - ((double)t.z + (double)t.w));
    w[row] = y;
    p.ws[row] = dsplit(y);
  }
}

template <typename ST>
__global__ void __launch_bounds__(256)
k_norm_partial(const Prob* __restrict__ probs, int ph, int start) {
  __shared__ double red[8];
  norm_partial_body<ST>(probs, ph, start, blockIdx.x, blockIdx.y, red);
}

template <typename ST>
__global__ void __launch_bounds__(256)
k_normalize(const Prob* __restrict__ probs, int ph, int start, int half) {
  __shared__ double sb2;
  normalize_body<ST>(probs, ph, start, half, blockIdx.x, blockIdx.y, &sb2);
}

// One thread per problem.
__global__ void k_step_finish(const Prob* __restrict__ probs, int nprob, int ph, int fresh, int half) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= nprob) return;
  const Prob& p = probs[ip];
  if (!kphase(p.st, fresh)) return;
  finish_one(p, ph, fresh, half, sum_norm_parts(p));
}

template <typename ST>
__global__ void __launch_bounds__(256)
k_norm_fused(const Prob* __restrict__ probs, int ph, int start, int half) {
  __shared__ double red[8];
  __shared__ double sb2;
  norm_fused_body<ST>(probs, ph, start, half, blockIdx.x, red, &sb2);
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
  if constexpr (std::is_same<ST, double2>::value)
    if (p.ws) p.ws[row] = dsplit(v);
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

// The same product for an FP64 basis in double-FP32 arithmetic (the mixed path, whose basis and
// coefficients need far less than FP64's 2^-53): V and S are split into FP32 (hi, lo) pairs once
// when staged, each term v s is formed as hi*hi exactly (its FMA residual) plus the two cross
// terms, and the sums are kept as (hi, lo) pairs with Knuth's TwoSum, about 2^-44 relative per
// term; the FP32 pipes run this about five times faster than GB300's FP64 pipe runs the FP64 FMAs.
__device__ __forceinline__ void df_acc(float& ah, float& al, float vh, float vl, float sh, float sl) {
  const float pr = vh * sh;
  const float e = __fmaf_rn(vh, sh, -pr);
  const float t = __fmaf_rn(vh, sl, __fmaf_rn(vl, sh, e));
  const float su = ah + pr;
  const float bb = su - ah;
  const float err = (ah - (su - bb)) + (pr - bb);
  ah = su;
  al += err + t;
}

__global__ void __launch_bounds__(256)
k_restart_gemm_df(const Prob* __restrict__ probs, int which) {
  __shared__ float4 sv[32][64];      // {re_hi, im_hi, re_lo, im_lo}
  __shared__ float2 ss[32][16];      // {hi, lo}
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
  const double2* src = (const double2*)srcs[which] + (int64_t)k0 * p.Npad;
  double2* dst = (double2*)dsts[which];
  const double* Sc = which >= 2 ? p.S2 : p.S;
  const int tid = threadIdx.x, rr = tid & 63, cg = tid >> 6;
  float ah[4][2], al[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q) ah[q][0] = ah[q][1] = al[q][0] = al[q][1] = 0.f;
  for (int c0 = 0; c0 < n; c0 += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * 64; e += 256) {
      const int cc = e >> 6, r = e & 63;
      const int64_t row = r0 + r;
      const double2 v = (c0 + cc < n && row < p.Npad) ? src[(int64_t)(c0 + cc) * p.Npad + row] : czero<double2>();
      const float xh = __double2float_rn(v.x), yh = __double2float_rn(v.y);
      sv[cc][r] = make_float4(xh, yh, __double2float_rn(v.x - (double)xh), __double2float_rn(v.y - (double)yh));
    }
    for (int e = tid; e < 32 * 16; e += 256) {
      const int cc = e >> 4, ii = e & 15;
      const double f = (c0 + cc < n && i0 + ii < nkeep) ? Sc[(int64_t)(i0 + ii) * p.ncv + c0 + cc] : 0.0;
      const float fh = __double2float_rn(f);
      ss[cc][ii] = make_float2(fh, __double2float_rn(f - (double)fh));
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < 32; ++cc) {
      const float4 v = sv[cc][rr];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 f = ss[cc][cg * 4 + q];
        df_acc(ah[q][0], al[q][0], v.x, v.z, f.x, f.y);
        df_acc(ah[q][1], al[q][1], v.y, v.w, f.x, f.y);
      }
    }
  }
  const int64_t row = r0 + rr;
  if (row < p.Npad) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + cg * 4 + q;
      if (i < nkeep)
        dst[(int64_t)i * p.Npad + row] =
            make_double2((double)ah[q][0] + (double)al[q][0], (double)ah[q][1] + (double)al[q][1]);
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
  if constexpr (std::is_same<ST, double2>::value) {
    if (p.Vs) {                         // the double-FP32 shadows follow
      for (int i = 0; i < nkeep; ++i)
        p.Vs[(int64_t)(k0 + i) * p.Npad + row] = dsplit(((const double2*)p.V2)[(int64_t)i * p.Npad + row]);
      p.Vs[(int64_t)(k0 + nkeep) * p.Npad + row] = dsplit(vm);
      if (ph) {
        for (int i = 0; i < nkeep; ++i)
          p.Ps[(int64_t)(k0 + i) * p.Npad + row] = dsplit(((const double2*)p.P2)[(int64_t)i * p.Npad + row]);
        p.Ps[(int64_t)(k0 + nkeep) * p.Npad + row] = dsplit(((const double2*)p.P)[(int64_t)(k0 + nkeep) * p.Npad + row]);
      }
    }
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
  double ts = 0.0;
  for (int i = st->k; i < st->l; ++i) ts = fmax(ts, fabs(p.theta[i]));
  st->theta_scale = ts;
  st->j = st->l;
  st->restarts += 1;
  st->r_go = 0;
  if (st->k >= st->nev) st->done = 1;
  else if (st->steps >= st->maxit) { st->done = 1; st->status = ST_NOCONV; }
}

// ---------------------------------------------------------------- launchers
template <typename ST>
void launch_step_cgs(const Prob* dprobs, int nprob, int ph, int maxnrb, int64_t maxNpad, int ncol,
                     int pass, int half, bool dfs, cudaStream_t s) {
  // pass: 0/1 regular step passes; 2/3 the same for a fresh (replacement) vector
  count_launch(2);
  const int newvec = pass >= 2 ? 1 : 0;
  const int ps = pass & 1;
  if (dfs && ph && half == 0) {        // the double-FP32 shadows of the mixed path
    k_cgs_dot_dfs<<<dim3((ncol + 1) / 2, maxnrb, nprob), 256, 0, s>>>(dprobs, newvec);
    k_cgs_update_dfs<<<dim3((unsigned)((maxNpad + 31) / 32), nprob), 256, 0, s>>>(dprobs, ps, newvec);
    return;
  }
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
void launch_restart(const Prob* dprobs, int nprob, int ph, int64_t maxNpad, int ncv, bool gruning, bool df,
                    cudaStream_t s) {
  const int ngemm = ph ? (gruning ? 4 : 2) : 1;
  count_launch(ngemm + 2);
  const unsigned gx = (unsigned)((maxNpad + 63) / 64);
  for (int which = 0; which < ngemm; ++which) {
    if (df && std::is_same<ST, double2>::value)
      k_restart_gemm_df<<<dim3(gx, (ncv + 15) / 16, nprob), 256, 0, s>>>(dprobs, which);
    else
      k_restart_gemm<ST><<<dim3(gx, (ncv + 15) / 16, nprob), 256, 0, s>>>(dprobs, which);
  }
  const unsigned gr = (unsigned)((maxNpad + 255) / 256);
  k_restart_copy<ST><<<dim3(gr, nprob), 256, 0, s>>>(dprobs, ph, gruning ? 1 : 0);
  k_restart_commit<<<(nprob + 127) / 128, 128, 0, s>>>(dprobs, nprob, ph);
}

#define INST(ST)                                                                                        \
  template void launch_step_cgs<ST>(const Prob*, int, int, int, int64_t, int, int, int, bool, cudaStream_t); \
  template void launch_step_normalize<ST>(const Prob*, int, int, int, int64_t, int, int, cudaStream_t); \
  template void launch_start_vector<ST>(const Prob*, int, int64_t, uint64_t, const void*,              \
                                        cudaStream_t);                                                  \
  template void launch_restart<ST>(const Prob*, int, int, int64_t, int, bool, bool, cudaStream_t);
INST(float2)
INST(double2)
#undef INST

}  // namespace bse
