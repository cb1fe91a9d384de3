// Phase bodies of the Krylov step, shared by the one-kernel-per-phase launches (k_product.cu,
// k_krylov.cu: the kernels there are thin wrappers that map blockIdx onto a body's unit
// arguments and declare its shared memory) and the persistent step kernel (k_persist.cu: one
// cooperative launch runs whole Krylov steps, every phase a loop of its CTAs over the units,
// the phases separated by a grid barrier).  A body computes the same bits in either setting:
// it takes its work unit and shared memory as arguments and keeps the summation order of the
// unit fixed.  Loads of data that a persistent launch rewrites between its phases (the Krylov
// basis, the work vectors, the partial sums) go through ldv / ldp<COH>: L2 loads (ordered by
// the barrier's fences, and never served from a stale L1 line) when COH.
#pragma once

#include <type_traits>

#include "bse_internal.cuh"

namespace bse {

template <bool COH, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
// the same for loads that take the ordinary path outside a persistent launch
template <bool COH, typename T>
__device__ __forceinline__ T ldp(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

template <typename R> struct Acc;
template <> struct Acc<float> { using T = float2; };
template <> struct Acc<double> { using T = double2; };

template <typename T>
__device__ __forceinline__ T shfl_xor_c(T v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

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

// Resolve the input / output vectors of a product for problem p.
// Returns false if the problem takes no part in this launch.
template <typename ST, typename R>
__device__ __forceinline__ bool prod_operands(const Prob& p, int mode, const GenericIO& io,
                                              const ST*& x, ST*& y, R& sB) {
  const KState* st = p.st;
  if (mode == PM_GENERIC) {
    x = (const ST*)io.xa; y = (ST*)io.y; sB = (R)io.sB; return true;
  }
  if (st->done || st->status != ST_OK) return false;
  const int j = st->j;
  const bool fresh = j < 0 || st->breakdown;
  switch (mode) {
    case PM_STEP_MMINUS:
      if (fresh || j >= p.ncv) return false;
      x = (const ST*)p.P + (int64_t)j * p.Npad; y = (ST*)p.w; sB = (R)-1; return true;
    case PM_STEP_MPLUS:
      if (fresh || j >= p.ncv) return false;
      x = (const ST*)p.w; y = (ST*)p.pw; sB = (R)1; return true;
    case PM_STEP_A:
      if (fresh || j >= p.ncv) return false;
      x = (const ST*)p.V + (int64_t)j * p.Npad; y = (ST*)p.w; sB = (R)0; return true;
    case PM_START_MPLUS:
      if (!fresh) return false;
      x = (const ST*)p.w; y = (ST*)p.pw; sB = (R)1; return true;
    case PM_STEP_MMINUS_W:
      if (fresh || j >= p.ncv) return false;
      x = (const ST*)p.w; y = (ST*)p.pw; sB = (R)-1; return true;
  }
  return false;
}

// A CTA walks the global job list either as one contiguous run or with stride
// gridDim.x (ProdShape).  Registers allow one FP64 CTA per SM (FP64-pipe
// bound) and two FP32 ones, so that twice as many tile loads are in flight
// (the FP32 product is HBM-latency bound).
// The tile walk of CTA bid of nblk; shared memory: xc, xr (column block J and row block I of
// x, TS entries each) and red (8 x TS, the column reduction across warps).
template <typename ST, typename R, bool HASB, bool COH = false>
__device__ __forceinline__ void prod_tiles_body(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs,
                                                int njobs, int mode, const GenericIO& io, int strided, int bid,
                                                int nblk, typename Acc<R>::T* xc, typename Acc<R>::T* xr,
                                                typename Acc<R>::T (*red)[TS]) {
  using CT = typename Acc<R>::T;
  // complex128 PH tiles hold P = A + B and Q = A - B; complex64 PH tiles hold A and B
  constexpr bool PQ = HASB && std::is_same<ST, double2>::value;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
  const int per = strided ? 1 : (njobs + nblk - 1) / nblk;
  const int t0 = strided ? bid : bid * per;
  const int t1 = strided ? njobs : min(njobs, t0 + per);
  const int dt = strided ? nblk : 1;
  for (int t = t0; t < t1; t += dt) {
    const TileJob jb = jobs[t];
    const Prob& p = probs[jb.prob];
    const ST* x; ST* yout; R sB;
    if (!prod_operands<ST, R>(p, mode, io, x, yout, sB)) continue;   // uniform per CTA
    const bool diag = (jb.I == jb.J);
    __syncthreads();                       // smem of the previous tile is free
    if (tid < TS) xc[tid] = ccvt<CT>(ldp<COH>(x + (int64_t)jb.J * TS + tid));
    else xr[tid - TS] = ccvt<CT>(ldp<COH>(x + (int64_t)jb.I * TS + tid - TS));
    __syncthreads();
    // PH: M_s u = A u + s B conj(u) is real-linear; in (Re, Im) form its block
    // row is [[U_re, -V_im], [U_im, V_re]] with U = A + s B, V = A - s B (the
    // real matrix M_r of Eq. 5 for s = +1), and the transpose use of the same
    // tile is [[U_re, U_im], [-V_im, V_re]].  That is 8 real FMAs per stored
    // element pair instead of the 16 of A u + s B conj(u) as two complex
    // products.  Complex128 tiles store P = A + B and Q = A - B, so U, V are
    // P, Q (s = +1) or Q, P (s = -1); complex64 tiles keep A and B exact and
    // form U, V in registers.
    const bool pos = sB > (R)0;
    const ST* At = (const ST*)(PQ && !pos ? p.B : p.A) + (int64_t)jb.t * (TS * TS);
    const ST* Bt = HASB ? (const ST*)(PQ && !pos ? p.A : p.B) + (int64_t)jb.t * (TS * TS) : nullptr;
    CT racc[8], cacc[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) cacc[b] = czero<CT>();
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int r = ty + 16 * a;
      ST av[8], bv[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        av[b] = __ldg(At + r * TS + tx + 16 * b);
        if (HASB) bv[b] = __ldg(Bt + r * TS + tx + 16 * b);
      }
      CT ra = czero<CT>();
      const CT y = xr[r];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int c = tx + 16 * b;
        const CT xv = xc[c];
        if (HASB) {
          CT u, v;
          if constexpr (PQ) {
            u = ccvt<CT>(av[b]);
            v = ccvt<CT>(bv[b]);
          } else {
            const CT a0 = ccvt<CT>(av[b]), b0 = ccvt<CT>(bv[b]);
            u.x = fma(sB, b0.x, a0.x); u.y = fma(sB, b0.y, a0.y);
            v.x = fma(-sB, b0.x, a0.x); v.y = fma(-sB, b0.y, a0.y);
          }
          ra.x = fma(u.x, xv.x, ra.x); ra.x = fma(-v.y, xv.y, ra.x);    // (M_s x_J)_r
          ra.y = fma(u.y, xv.x, ra.y); ra.y = fma(v.x, xv.y, ra.y);
          if (!diag) {                                                  // (M_s^T x_I)_c
            cacc[b].x = fma(u.x, y.x, cacc[b].x); cacc[b].x = fma(u.y, y.y, cacc[b].x);
            cacc[b].y = fma(v.x, y.y, cacc[b].y); cacc[b].y = fma(-v.y, y.x, cacc[b].y);
          }
        } else {
          const CT A = ccvt<CT>(av[b]);
          cfma(ra, A, xv);                      // (A_IJ x_J)_r
          if (!diag) cfmac(cacc[b], A, y);      // (A_IJ^H x_I)_c
        }
      }
      racc[a] = ra;
    }
    // ---- row sums: reduce-scatter over the 16 tx lanes (xor 8, 4, 2, 1)
    {
      const bool u8 = tx & 8;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        CT send = u8 ? racc[q] : racc[q + 4];
        CT keep = u8 ? racc[q + 4] : racc[q];
        racc[q] = cadd(keep, shfl_xor_c(send, 8));
      }
      const bool u4 = tx & 4;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        CT send = u4 ? racc[q] : racc[q + 2];
        CT keep = u4 ? racc[q + 2] : racc[q];
        racc[q] = cadd(keep, shfl_xor_c(send, 4));
      }
      const bool u2 = tx & 2;
      {
        CT send = u2 ? racc[0] : racc[1];
        CT keep = u2 ? racc[1] : racc[0];
        racc[0] = cadd(keep, shfl_xor_c(send, 2));
      }
      racc[0] = cadd(racc[0], shfl_xor_c(racc[0], 1));
      if ((tx & 1) == 0) {
        const int a = (tx >> 1) & 7;
        const int r = ty + 16 * a;
        CT* part = (CT*)p.part;
        part[((int64_t)jb.I * p.nT + jb.J) * TS + r] = racc[0];
      }
    }
    if (!diag) {
      // ---- column sums: pair the two ty of a warp (xor 16), then across warps
      const bool up = lane & 16;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        CT send = up ? cacc[q] : cacc[q + 4];
        CT keep = up ? cacc[q + 4] : cacc[q];
        cacc[q] = cadd(keep, shfl_xor_c(send, 16));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) red[warp][tx + 16 * (q + (up ? 4 : 0))] = cacc[q];
      __syncthreads();
      if (tid < TS) {
        CT s = red[0][tid];
#pragma unroll
        for (int w = 1; w < 8; ++w) s = cadd(s, red[w][tid]);
        CT* part = (CT*)p.part;
        part[((int64_t)jb.J * p.nT + jb.I) * TS + tid] = s;
      }
    }
  }
}

// y[I*TS + r] = sum_J part[I][J][r]; grid (maxnT, nprob).
constexpr int REDUCE_GROUPS = 8;

// One unit: block row I of problem ip, with any multiple of TS threads (each thread takes
// the groups g = threadIdx.x / TS + k blockDim.x / TS); grp: (REDUCE_GROUPS - 1) x TS entries
// of shared memory.  The group sums and their order are those of the REDUCE_GROUPS * TS
// thread launch, so the result is the same bits for any thread count.
template <typename ST, typename R, bool COH = false>
__device__ __forceinline__ void prod_reduce_body(const Prob* __restrict__ probs, int mode, const GenericIO& io,
                                                 int I, int ip, typename Acc<R>::T (*grp)[TS]) {
  using CT = typename Acc<R>::T;
  const Prob& p = probs[ip];
  if (I >= p.nT) return;
  const ST* x; ST* y; R sB;
  if (!prod_operands<ST, R>(p, mode, io, x, y, sB)) return;
  // REDUCE_GROUPS groups of 128 threads sum the slots J = g, g + G, ... in
  // order; the group sums are then added in group order (fixed rounding order)
  const int r = threadIdx.x & (TS - 1);
  const CT* part = (const CT*)p.part + (int64_t)I * p.nT * TS;
  CT acc0 = czero<CT>();
  for (int g = threadIdx.x >> 7; g < REDUCE_GROUPS; g += blockDim.x >> 7) {
    CT acc = czero<CT>();
    int J = g;
    for (; J + 3 * REDUCE_GROUPS < p.nT; J += 4 * REDUCE_GROUPS) {   // four loads in flight, then the sums
      CT v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = ldp<COH>(part + (int64_t)(J + u * REDUCE_GROUPS) * TS + r);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = cadd(acc, v[u]);
    }
    for (; J < p.nT; J += REDUCE_GROUPS) acc = cadd(acc, ldp<COH>(part + (int64_t)J * TS + r));
    if (g > 0) grp[g - 1][r] = acc;
    else acc0 = acc;
  }
  __syncthreads();
  if (threadIdx.x < TS) {
#pragma unroll
    for (int q = 0; q < REDUCE_GROUPS - 1; ++q) acc0 = cadd(acc0, grp[q][r]);
    y[(int64_t)I * TS + r] = ccvt<ST>(acc0);
  }
  __syncthreads();                     // grp is rewritten by the next unit
}

// ---------------------------------------------------------------- CGS2 dots
// PH: cpart[rb][c] = sum_{rows in block rb} Re(conj(Dm[row, c]) x[row]) for c < nm and
// Im(conj(Dt[row, c']) x[row]) for c = nm + c' (the twin coefficients), nm + nt in all;
// TDA: the complex conj(V[row, c]) x[row], c <= j.  grid (ceil(maxcols/2), maxnrb, nprob),
// 8 warps: two columns per CTA, four warps per column, each warp a quarter of the block
// rows; the four partial sums meet in shared memory (fixed order).
// One unit: column pair bx, row block rb of problem ip (the kernel's blockIdx (x, y, z));
// red: 2 x 4 double2 of shared memory.
template <typename ST, bool COH>
__device__ __forceinline__ void cgs_dot_body(const Prob* __restrict__ probs, int ph, int newvec, int half, int pass,
                                             int bx, int rb, int ip, double2 (*red)[4]) {
  using R = typename RealOf<ST>::T;
  const Prob& p = probs[ip];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  if (rb >= p.nrb) return;
  const CgsSet cs = cgs_set(p, st, ph, half);
  const int nset = cs.nm + cs.nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hw = warp >> 2, quarter = warp & 3;
  const int c = bx * 2 + hw;
  if (bx * 2 >= nset) return;                     // whole CTA
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
          q[u] = ldv<COH>(Q + r + 32 * u);
          x[u] = ldv<COH>(w + r + 32 * u);
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
        const ST q = ldv<COH>(Q + r);
        ST x = ldv<COH>(w + r);
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
          q[u] = ldv<COH>(Q + r + 32 * u);
          x[u] = ldv<COH>(w + r + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) cfmac(acc, q[u], x[u]);
      }
      for (; r < r1; r += 32) cfmac(acc, ldv<COH>(Q + r), ldv<COH>(w + r));
      a = mk((double)acc.x, (double)acc.y);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) a = cadd(a, dshfl(a, m));
  }
  if (lane == 0) red[hw][quarter] = a;
  __syncthreads();
  if (threadIdx.x < 2) {
    const int cc = bx * 2 + threadIdx.x;
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
// One unit: 32-row slab bx of problem ip; cf: 2 MAXM + 2 entries and red: 8 x 32 entries
// of shared memory.
template <typename ST, bool COH>
__device__ __forceinline__ void cgs_update_body(const Prob* __restrict__ probs, int ph, int pass, int newvec,
                                                int half, int bx, int ip, ST* cf, ST (*red)[32]) {
  using R = typename RealOf<ST>::T;
  const Prob& p = probs[ip];
  const KState* st = p.st;
  if (!kphase(st, newvec)) return;
  const int64_t row = (int64_t)bx * 32 + (threadIdx.x & 31);
  if ((int64_t)bx * 32 >= p.Npad) return;     // whole block (Npad is a multiple of 128)
  const CgsSet cs = cgs_set(p, st, ph, half);
  const int nm = cs.nm;
  const int nset = nm + cs.nt;
  // coefficients: the row-block partial sums of the dots, added in row-block order (PH: real
  // part only); the first row slab also stores them for k_step_finish
  const double2* cp = (const double2*)p.cpart;
  double2* coef = (double2*)p.coef + (int64_t)(pass & 1) * p.ncol;
  for (int c = threadIdx.x; c < nset; c += blockDim.x) {
    double2 sc = mk(0.0, 0.0);
    int rb = 0;
    for (; rb + 8 <= p.nrb; rb += 8) {      // eight loads in flight, then the sums in order
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = ldp<COH>(cp + (int64_t)(rb + u) * p.ncol + c);
#pragma unroll
      for (int u = 0; u < 8; ++u) sc = cadd(sc, v[u]);
    }
    for (; rb < p.nrb; ++rb) sc = cadd(sc, ldp<COH>(cp + (int64_t)rb * p.ncol + c));
    if (ph) sc.y = 0.0;
    cf[c] = ccvt<ST>(sc);
    if (bx == 0) coef[c] = sc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ST* vb = (const ST*)cs.um + row;
  const ST* pb = ph ? (const ST*)cs.ut + row : nullptr;
  constexpr int U = sizeof(ST) == 16 ? 6 : 8;   // loads in flight per thread (registers for 3 CTAs/SM)
  const int64_t ld = p.Npad;
  // entry cc of the set: Um[:, cc] for cc < nm, else the twin i Ut[:, cc - nm] (as (-t.y, t.x))
  auto colval = [&](int cc) -> ST {
    if (cc < nm) return ldv<COH>(vb + (int64_t)cc * ld);
    const ST q = ldv<COH>(pb + (int64_t)(cc - nm) * ld);
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
      for (int u = 0; u < U; ++u) v[u] = ldv<COH>(vb + (int64_t)(c + 8 * u) * ld);
#pragma unroll
      for (int u = 0; u < U; ++u) cfma(acc[u], v[u], cf[c + 8 * u]);
    }
    for (; c < nset; c += 8) cfma(acc[0], ldv<COH>(vb + (int64_t)c * ld), cf[c]);
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
    w[row] = csub(ldp<COH>(x + row), tot);
  }
}

// ---------------------------------------------------------------- norms
// cpart[rb].x = sum over rows of Re(conj(w) pw) (PH) or |w|^2 (TDA).
// One unit: row block rb of problem ip; red: 8 doubles of shared memory.
template <typename ST, bool COH = false>
__device__ __forceinline__ void norm_partial_body(const Prob* __restrict__ probs, int ph, int start, int rb, int ip,
                                                  double* red) {
  const Prob& p = probs[ip];
  const KState* st = p.st;
  if (!kphase(st, start)) return;
  if (rb >= p.nrb) return;
  const ST* w = (const ST*)p.w;
  const ST* pw = (const ST*)(ph ? p.pw : p.w);
  const int64_t r0 = (int64_t)rb * ROWBLK;
  const int64_t r1 = min((int64_t)p.Npad, r0 + ROWBLK);
  double s = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += 256) {
    const ST a = ldp<COH>(w + r), b = ldp<COH>(pw + r);
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

template <bool COH = false>
__device__ __forceinline__ double sum_norm_parts(const Prob& p) {
  const double2* cp = (const double2*)p.cpart;
  double s = 0.0;
  for (int rb = 0; rb < p.nrb; ++rb) s += ldp<COH>(cp + rb).x;
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

// The double-FP32 shadows of a new V (and P) column, where the problem keeps them.
template <typename ST>
__device__ __forceinline__ void shadow_store(const Prob& p, const KState* st, int half, int64_t row, ST xv, ST yv) {
  if constexpr (std::is_same<ST, double2>::value) {
    if (p.Vs && half != 1) {
      const int64_t o = (int64_t)(st->j + 1) * p.Npad + row;
      p.Vs[o] = dsplit(xv);
      if (p.ph) p.Ps[o] = dsplit(yv);
    }
  }
}

// X = w / beta, Y = pw / beta (norm_dest) when beta^2 is usable.
// One unit: rows bx * blockDim.x ... of problem ip; sb2: one double of shared memory.
template <typename ST, bool COH = false>
__device__ __forceinline__ void normalize_body(const Prob* __restrict__ probs, int ph, int start, int half, int bx,
                                               int ip, double* sb2) {
  using R = typename RealOf<ST>::T;
  const Prob& p = probs[ip];
  const KState* st = p.st;
  if (!kphase(st, start)) return;
  if (threadIdx.x == 0) *sb2 = sum_norm_parts<COH>(p);
  __syncthreads();
  const double b2 = *sb2;
  __syncthreads();                              // sb2 is rewritten by the next unit
  if (!(b2 > 0.0) || !isfinite(b2)) return;   // k_step_finish records the outcome
  const R inv = (R)(1.0 / sqrt(b2));
  const int64_t row = (int64_t)bx * blockDim.x + threadIdx.x;
  if (row >= p.Npad) return;
  ST *X, *Y;
  norm_dest<ST>(p, st, half, X, Y);
  const ST xv = cscale(ldp<COH>((const ST*)p.w + row), inv);
  X[row] = xv;
  ST yv = czero<ST>();
  if (ph) Y[row] = yv = cscale(ldp<COH>((const ST*)p.pw + row), inv);
  shadow_store<ST>(p, st, half, row, xv, yv);
}

// Record alpha_j, beta_j, advance j, given beta^2 = b2 of the new vector.  fresh = 0:
// regular step; fresh = 1: a first or replacement vector was just normalised.
__device__ __forceinline__ void step_finish_one(const Prob& p, int ph, int fresh, double b2) {
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
    scale = fmax(scale, st->theta_scale);   // max |theta| of the kept Ritz values
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
__device__ __forceinline__ void gk_finish_one(const Prob& p, int half, int fresh, double b2) {
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
    scale = fmax(scale, st->theta_scale);   // max |theta| of the kept Ritz values
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


// Problems of at most one reduction row block (Npad <= ROWBLK): the norm, the scaling of
// the new basis vector and the state update in one CTA per problem (one launch instead of
// three per Krylov step; the same arithmetic as k_norm_partial, k_normalize, k_step_finish).
// One unit: problem ip; red: 8 doubles and sb2p: one double of shared memory.
template <typename ST, bool COH = false>
__device__ __forceinline__ void norm_fused_body(const Prob* __restrict__ probs, int ph, int start, int half, int ip,
                                                double* red, double* sb2p) {
  using R = typename RealOf<ST>::T;
  double& sb2 = *sb2p;
  const Prob& p = probs[ip];
  const KState* st = p.st;
  if (!kphase(st, start)) return;
  const ST* w = (const ST*)p.w;
  const ST* pw = (const ST*)(ph ? p.pw : p.w);
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < p.Npad; r += 256) {
    const ST a = ldp<COH>(w + r), b = ldp<COH>(pw + r);
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
      const ST xv = cscale(ldp<COH>(w + r), inv);
      X[r] = xv;
      ST yv = czero<ST>();
      if (ph) Y[r] = yv = cscale(ldp<COH>((const ST*)p.pw + r), inv);
      shadow_store<ST>(p, st, half, r, xv, yv);
    }
  }
  __syncthreads();                     // every thread has read st->j
  if (threadIdx.x == 0) finish_one(p, ph, start, half, b2);
}

}  // namespace bse
