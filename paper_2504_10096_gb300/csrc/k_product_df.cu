// Complex128 structured product in double-FP32 ("df64") arithmetic.
//
// GB300 executes 2 FP64 FMAs per SM per clock but 128 FP32 operations, so
// the FP64 product (8 FMAs per stored element pair in the real form of Eq. 5)
// is bound by the FP64 pipe at about 1/2.7 of the HBM rate.  The kernels here
// stream the same packed tiles -- split at creation into float pairs
// a = a_hi + a_lo (|a_lo| <= 2^-24 |a_hi|, exact to 2^-48 relative) for
// complex128 handles (k_prod_tiles_df), or the exact complex64 A and B
// (k_prod_tiles_df2, packed f32x2) -- and evaluate every real multiply-
// accumulate with error-free transformations on the FP32 pipes:
//   p = fl(a_hi x_hi),  e = fma(a_hi, x_hi, -p) + a_hi x_lo + a_lo x_hi
//   (s_hi, err) = TwoSum(s_hi, p),  s_lo += err + e
// (Dekker's product, Knuth's TwoSum; the dropped a_lo x_lo is 2^-48 of the
// term).  Partial sums leave the kernel as FP64 and are reduced in FP64 by
// the same k_prod_reduce.  Explicit __f*_rn intrinsics keep the compiler from
// contracting the transformations.
//
// The Krylov basis, Gram-Schmidt, projected problem and the final residuals
// of this path stay in FP64; only the streaming product changes arithmetic.
#include <algorithm>

#include "bse_internal.cuh"

namespace bse {
namespace {

// LO = false: the stored element is exact in FP32 (complex64 tiles), a_lo = 0
template <bool LO>
__device__ __forceinline__ void df_acc(float& h, float& l, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = __fmaf_rn(ah, xh, -p);
  e = __fmaf_rn(ah, xl, e);
  if (LO) e = __fmaf_rn(al, xh, e);
  const float t = __fadd_rn(h, p);
  const float bp = __fsub_rn(t, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  h = t;
  l = __fadd_rn(l, __fadd_rn(err, e));
}

struct DFC { float rh, rl, ih, il; };

__device__ __forceinline__ DFC dfc_zero() { return DFC{0.f, 0.f, 0.f, 0.f}; }

// y += a x ; a, x as float4 {re_hi, im_hi, re_lo, im_lo}
template <bool LO>
__device__ __forceinline__ void dfc_fma(DFC& y, float4 a, float4 x) {
  df_acc<LO>(y.rh, y.rl, a.x, a.z, x.x, x.z);
  df_acc<LO>(y.rh, y.rl, -a.y, -a.w, x.y, x.w);
  df_acc<LO>(y.ih, y.il, a.x, a.z, x.y, x.w);
  df_acc<LO>(y.ih, y.il, a.y, a.w, x.x, x.z);
}
// y += conj(a) x
template <bool LO>
__device__ __forceinline__ void dfc_fmac(DFC& y, float4 a, float4 x) {
  df_acc<LO>(y.rh, y.rl, a.x, a.z, x.x, x.z);
  df_acc<LO>(y.rh, y.rl, a.y, a.w, x.y, x.w);
  df_acc<LO>(y.ih, y.il, a.x, a.z, x.y, x.w);
  df_acc<LO>(y.ih, y.il, -a.y, -a.w, x.x, x.z);
}

__device__ __forceinline__ float4 widen(float4 v) { return v; }
__device__ __forceinline__ float4 widen(float2 v) { return make_float4(v.x, v.y, 0.f, 0.f); }

__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  const float t = __fadd_rn(h, bh);
  const float bp = __fsub_rn(t, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(bh, bp));
  const float lo = __fadd_rn(err, __fadd_rn(l, bl));
  h = __fadd_rn(t, lo);                  // renormalise (fast two-sum, |t| >= |lo|)
  l = __fsub_rn(lo, __fsub_rn(h, t));
}

__device__ __forceinline__ DFC dfc_add(DFC a, const DFC& b) {
  df_add(a.rh, a.rl, b.rh, b.rl);
  df_add(a.ih, a.il, b.ih, b.il);
  return a;
}

__device__ __forceinline__ DFC dfc_shfl(DFC v, int m) {
  v.rh = __shfl_xor_sync(0xffffffffu, v.rh, m);
  v.rl = __shfl_xor_sync(0xffffffffu, v.rl, m);
  v.ih = __shfl_xor_sync(0xffffffffu, v.ih, m);
  v.il = __shfl_xor_sync(0xffffffffu, v.il, m);
  return v;
}

__device__ __forceinline__ double2 dfc_to_d(const DFC& v) {
  return make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
}

__device__ __forceinline__ float4 split_d(double2 a) {
  const float rh = __double2float_rn(a.x), ih = __double2float_rn(a.y);
  return make_float4(rh, ih, __double2float_rn(a.x - (double)rh), __double2float_rn(a.y - (double)ih));
}

__device__ __forceinline__ bool df_operands(const Prob& p, int mode, const GenericIO& io, const double2*& x,
                                            double& sB) {
  const KState* st = p.st;
  if (mode == PM_GENERIC) { x = (const double2*)io.xa; sB = io.sB; return true; }
  if (st->done || st->status != ST_OK) return false;
  const int j = st->j;
  const bool fresh = j < 0 || st->breakdown;
  switch (mode) {
    case PM_STEP_MMINUS:
      if (fresh || j >= p.ncv) return false;
      x = (const double2*)p.P + (int64_t)j * p.Npad; sB = -1.0; return true;
    case PM_STEP_MPLUS:
      if (fresh || j >= p.ncv) return false;
      x = (const double2*)p.w; sB = 1.0; return true;
    case PM_STEP_A:
      if (fresh || j >= p.ncv) return false;
      x = (const double2*)p.V + (int64_t)j * p.Npad; sB = 0.0; return true;
    case PM_START_MPLUS:
      if (!fresh) return false;
      x = (const double2*)p.w; sB = 1.0; return true;
  }
  return false;
}

// Cross-lane reduction of a tile's partial sums into the two partial-sum
// slots (I, J) and (J, I): racc[a] = this thread's sum of row ty + 16a over
// its 8 columns, cacc[b] = its sum of column tx + 16b over its 8 rows.
// `red` is shared scratch of 8 x TS DFC (callers alias it with their row park).
__device__ __forceinline__ void df_tile_reduce(DFC (&racc)[8], DFC (&cacc)[8], DFC (*red)[TS], bool diag,
                                               const Prob& p, const TileJob& jb) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
  {
    const bool u8 = tx & 8;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      DFC s = u8 ? racc[q] : racc[q + 4], k = u8 ? racc[q + 4] : racc[q];
      racc[q] = dfc_add(k, dfc_shfl(s, 8));
    }
    const bool u4 = tx & 4;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      DFC s = u4 ? racc[q] : racc[q + 2], k = u4 ? racc[q + 2] : racc[q];
      racc[q] = dfc_add(k, dfc_shfl(s, 4));
    }
    const bool u2 = tx & 2;
    DFC s = u2 ? racc[0] : racc[1], k = u2 ? racc[1] : racc[0];
    racc[0] = dfc_add(k, dfc_shfl(s, 2));
    racc[0] = dfc_add(racc[0], dfc_shfl(racc[0], 1));
    if ((tx & 1) == 0) {
      double2* part = (double2*)p.part;
      part[((int64_t)jb.I * p.nT + jb.J) * TS + ty + 16 * ((tx >> 1) & 7)] = dfc_to_d(racc[0]);
    }
  }
  if (!diag) {
    const bool up = lane & 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      DFC s = up ? cacc[q] : cacc[q + 4], k = up ? cacc[q + 4] : cacc[q];
      cacc[q] = dfc_add(k, dfc_shfl(s, 16));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[warp][tx + 16 * (q + (up ? 4 : 0))] = cacc[q];
    __syncthreads();
    if (tid < TS) {
      DFC s = red[0][tid];
#pragma unroll
      for (int w = 1; w < 8; ++w) s = dfc_add(s, red[w][tid]);
      double2* part = (double2*)p.part;
      part[((int64_t)jb.J * p.nT + jb.I) * TS + tid] = dfc_to_d(s);
    }
  }
}

// SPLIT: float4 split complex128 tiles (p.Ahl); otherwise complex64 tiles (p.A)
template <bool HASB, bool SPLIT>
__global__ void __launch_bounds__(PROD_THREADS, 2)
k_prod_tiles_df(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs, int njobs, int mode,
                GenericIO io, int strided) {
  static_assert(!HASB || SPLIT, "complex64 PH tiles go through k_prod_tiles_df2");
  __shared__ float4 xc[TS], xr[TS];
  // per-thread row partial sums (own slots only); after a barrier the same
  // storage holds the cross-warp column reduction
  __shared__ DFC rpark[8][PROD_THREADS];
  DFC(*red)[TS] = reinterpret_cast<DFC(*)[TS]>(&rpark[0][0]);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int per = strided ? 1 : (njobs + gridDim.x - 1) / gridDim.x;
  const int t0 = strided ? blockIdx.x : blockIdx.x * per;
  const int t1 = strided ? njobs : min(njobs, t0 + per);
  const int dt = strided ? gridDim.x : 1;
  for (int t = t0; t < t1; t += dt) {
    const TileJob jb = jobs[t];
    const Prob& p = probs[jb.prob];
    const double2* x;
    double sB;
    if (!df_operands(p, mode, io, x, sB)) continue;   // uniform per CTA
    const bool diag = jb.I == jb.J;
    __syncthreads();
    {
      const int r = tid & (TS - 1);
      const double2 a = x[(int64_t)(tid < TS ? jb.J : jb.I) * TS + r];
      if (tid < TS) xc[r] = split_d(a);
      else xr[r] = split_d(a);
    }
    __syncthreads();
    using TT = typename std::conditional<SPLIT, float4, float2>::type;
    const bool swap = SPLIT && HASB && sB < 0.0;      // split tiles hold P, Q: U, V = Q, P for s = -1
    const TT* At = (const TT*)(SPLIT ? (swap ? p.Bhl : p.Ahl) : p.A) + (int64_t)jb.t * (TS * TS);
    const TT* Bt = HASB ? (const TT*)(SPLIT ? (swap ? p.Ahl : p.Bhl) : p.B) + (int64_t)jb.t * (TS * TS) : nullptr;
    DFC racc[8], cacc[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) cacc[b] = dfc_zero();
    // rows are not unrolled: the error-free transformations make one row of
    // 8 elements about 1.4k instructions, and a fully unrolled tile would not
    // fit the instruction cache.  Each row's partial sum is parked in shared
    // memory and read back for the cross-lane reduction.
    // complex64 tiles: the next row's elements are loaded before this row is
    // processed, so that their latency hides behind ~1.4k instructions of
    // arithmetic (the split float4 tiles have no registers left for that)
    constexpr bool PF = !SPLIT;
    TT av[8], bv[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      av[b] = __ldg(At + ty * TS + tx + 16 * b);
      if (HASB) bv[b] = __ldg(Bt + ty * TS + tx + 16 * b);
    }
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
      const int r = ty + 16 * a;
      TT an[8], bn[8];
      if (PF) {
        if (a < 7) {
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            an[b] = __ldg(At + (r + 16) * TS + tx + 16 * b);
            if (HASB) bn[b] = __ldg(Bt + (r + 16) * TS + tx + 16 * b);
          }
        }
      } else if (a > 0) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          av[b] = __ldg(At + r * TS + tx + 16 * b);
          if (HASB) bv[b] = __ldg(Bt + r * TS + tx + 16 * b);
        }
      }
      DFC ra = dfc_zero();
      const float4 y = xr[r];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int c = tx + 16 * b;
        const float4 x = xc[c];
        if (HASB) {
          // U = A + s B, V = A - s B: the real block row [[U_re, -V_im], [U_im, V_re]]
          // of M_s (Eq. 5 for s = +1) and its transpose, 8 multiply-accumulates
          // split P = A + B, Q = A - B, chosen by pointer (complex64 PH tiles use k_prod_tiles_df2)
          const float4 u = widen(av[b]), v = widen(bv[b]);
          df_acc<true>(ra.rh, ra.rl, u.x, u.z, x.x, x.z);
          df_acc<true>(ra.rh, ra.rl, -v.y, -v.w, x.y, x.w);
          df_acc<true>(ra.ih, ra.il, u.y, u.w, x.x, x.z);
          df_acc<true>(ra.ih, ra.il, v.x, v.z, x.y, x.w);
          if (!diag) {
            df_acc<true>(cacc[b].rh, cacc[b].rl, u.x, u.z, y.x, y.z);
            df_acc<true>(cacc[b].rh, cacc[b].rl, u.y, u.w, y.y, y.w);
            df_acc<true>(cacc[b].ih, cacc[b].il, v.x, v.z, y.y, y.w);
            df_acc<true>(cacc[b].ih, cacc[b].il, -v.y, -v.w, y.x, y.z);
          }
        } else {
          const float4 aw = widen(av[b]);
          dfc_fma<SPLIT>(ra, aw, x);
          if (!diag) dfc_fmac<SPLIT>(cacc[b], aw, y);
        }
      }
      rpark[a][tid] = ra;
      if (PF) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          av[b] = an[b];
          if (HASB) bv[b] = bn[b];
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) racc[a] = rpark[a][tid];
    __syncthreads();   // rpark is reused below as the column-reduction buffer
    df_tile_reduce(racc, cacc, red, diag, p, jb);
  }
}

// ---------------------------------------------------------------------------
// Packed variant for the PH product (A and B): the two lanes of the PTX
// f32x2 instructions (add/sub/mul/fma.rn.f32x2, each lane one IEEE
// round-to-nearest FP32 operation) carry two independent double-FP32
// accumulations, which halves the instructions of the error-free
// transformations.  With the pairs
//     UVr = (U_re, V_re), UVi = (U_im, V_im)    (U = A + sB, V = A - sB)
// the real form of Eq. 5 needs no lane shuffles per element:
//     row:    A1 += UVr (x_re, x_im),  A2 += UVi (x_re, -x_im)
//             (y_re, y_im) = (A1.0 + A2.1, A1.1 + A2.0)   once per row
//     column: C  += UVr (y_re, y_im) + UVi (y_im, -y_re)
// Every product takes a negated hi operand from shared memory, so the
// Dekker error is fma(a, x, -fl(a x)) without a negation instruction.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// (H, L) += (ah + al) (xh + xl), lane-wise; xn = -xh
__device__ __forceinline__ void acc2(f2& H, f2& L, f2 ah, f2 al, f2 xh, f2 xl, f2 xn) {
  const f2 q = mul2(ah, xn);              // -fl(ah xh)
  f2 e = fma2(ah, xh, q);                 // its rounding error, exactly
  e = fma2(ah, xl, e);
  e = fma2(al, xh, e);
  const f2 t = sub2(H, q);                // TwoSum(H, fl(ah xh))
  const f2 bp = sub2(t, H);
  const f2 err = sub2(sub2(H, sub2(t, bp)), add2(q, bp));
  H = t;
  L = add2(L, add2(err, e));
}

// exact (s, e) with s + e = a + b, lane-wise
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2& s, f2& e) {
  s = add2(a, b);
  const f2 bp = sub2(s, a);
  e = add2(sub2(a, sub2(s, bp)), sub2(b, bp));
}

struct XPack {       // one vector entry, as the packed operands the kernel needs
  f2 h1, l1, n1;     // (re, im) hi / lo / -hi
  f2 h2, l2, n2;     // second pairing: (re, -im) for x_J, (im, -re) for x_I
};

__device__ __forceinline__ XPack xpack(double2 v, bool row) {
  const float4 s = split_d(v);            // {re_hi, im_hi, re_lo, im_lo}
  XPack o;
  o.h1 = pk(s.x, s.y);
  o.l1 = pk(s.z, s.w);
  o.n1 = pk(-s.x, -s.y);
  if (!row) {
    o.h2 = pk(s.x, -s.y);
    o.l2 = pk(s.z, -s.w);
    o.n2 = pk(-s.x, s.y);
  } else {
    o.h2 = pk(s.y, -s.x);
    o.l2 = pk(s.w, -s.z);
    o.n2 = pk(-s.y, s.x);
  }
  return o;
}

__global__ void __launch_bounds__(PROD_THREADS, 2)
k_prod_tiles_df2(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs, int njobs, int mode,
                 GenericIO io, int strided) {
  __shared__ XPack xc[TS], xr[TS];
  __shared__ DFC rpark[8][PROD_THREADS];
  DFC(*red)[TS] = reinterpret_cast<DFC(*)[TS]>(&rpark[0][0]);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int per = strided ? 1 : (njobs + gridDim.x - 1) / gridDim.x;
  const int t0 = strided ? blockIdx.x : blockIdx.x * per;
  const int t1 = strided ? njobs : min(njobs, t0 + per);
  const int dt = strided ? gridDim.x : 1;
  const f2 zero = pk(0.f, 0.f);
  for (int t = t0; t < t1; t += dt) {
    const TileJob jb = jobs[t];
    const Prob& p = probs[jb.prob];
    const double2* x;
    double sB;
    if (!df_operands(p, mode, io, x, sB)) continue;   // uniform per CTA
    const bool diag = jb.I == jb.J;
    __syncthreads();
    {
      const int r = tid & (TS - 1);
      const double2 v = x[(int64_t)(tid < TS ? jb.J : jb.I) * TS + r];
      if (tid < TS) xc[r] = xpack(v, false);
      else xr[r] = xpack(v, true);
    }
    __syncthreads();
    using TT = float2;                              // exact complex64 A and B
    const TT* At = (const TT*)p.A + (int64_t)jb.t * (TS * TS);
    const TT* Bt = (const TT*)p.B + (int64_t)jb.t * (TS * TS);
    // (s b_re, -s b_re) pairs via a lane sign
    const float sg = sB > 0.0 ? 1.f : -1.f;
    const f2 spm = pk(sg, -sg);
    f2 cH[8], cL[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) cH[b] = cL[b] = zero;
    // rows stay rolled (instruction cache); the next row is prefetched
    constexpr bool PF = true;
    TT av[8], bv[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      av[b] = __ldg(At + ty * TS + tx + 16 * b);
      bv[b] = __ldg(Bt + ty * TS + tx + 16 * b);
    }
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
      const int r = ty + 16 * a;
      TT an[8], bn[8];
      if (PF) {
        if (a < 7) {
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            an[b] = __ldg(At + (r + 16) * TS + tx + 16 * b);
            bn[b] = __ldg(Bt + (r + 16) * TS + tx + 16 * b);
          }
        }
      } else if (a > 0) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          av[b] = __ldg(At + r * TS + tx + 16 * b);
          bv[b] = __ldg(Bt + r * TS + tx + 16 * b);
        }
      }
      const XPack y = xr[r];
      f2 H1 = zero, L1 = zero, H2 = zero, L2 = zero;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const XPack xv = xc[tx + 16 * b];
        f2 rh, rl, ih, il;                 // UVr and UVi, hi and lo, exact by TwoSum
        two_sum2(pk(av[b].x, av[b].x), mul2(pk(bv[b].x, bv[b].x), spm), rh, rl);
        two_sum2(pk(av[b].y, av[b].y), mul2(pk(bv[b].y, bv[b].y), spm), ih, il);
        acc2(H1, L1, rh, rl, xv.h1, xv.l1, xv.n1);
        acc2(H2, L2, ih, il, xv.h2, xv.l2, xv.n2);
        if (!diag) {
          acc2(cH[b], cL[b], rh, rl, y.h1, y.l1, y.n1);
          acc2(cH[b], cL[b], ih, il, y.h2, y.l2, y.n2);
        }
      }
      // (re, im) = (A1.0 + A2.1, A1.1 + A2.0)
      float h1a, h1b, l1a, l1b, h2a, h2b, l2a, l2b;
      upk(H1, h1a, h1b);
      upk(L1, l1a, l1b);
      upk(H2, h2a, h2b);
      upk(L2, l2a, l2b);
      DFC ra;
      ra.rh = h1a; ra.rl = l1a; ra.ih = h1b; ra.il = l1b;
      df_add(ra.rh, ra.rl, h2b, l2b);
      df_add(ra.ih, ra.il, h2a, l2a);
      rpark[a][tid] = ra;
      if (PF) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          av[b] = an[b];
          bv[b] = bn[b];
        }
      }
    }
    DFC racc[8], cacc[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      float hr, hi, lr, li;
      upk(cH[b], hr, hi);
      upk(cL[b], lr, li);
      cacc[b].rh = hr; cacc[b].rl = lr; cacc[b].ih = hi; cacc[b].il = li;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) racc[a] = rpark[a][tid];
    __syncthreads();   // rpark is reused below as the column-reduction buffer
    df_tile_reduce(racc, cacc, red, diag, p, jb);
  }
}

// ---------------------------------------------------------------------------
// Mixed-path product on "coarse" tiles (complex64 PH tiles whose entries are
// small against the largest tile of the problem): the same real form, but
// (1) U = A + sB and V = A - sB are rounded to FP32 -- a fixed perturbation of
//     the operator of at most 2^-24 |U| per entry, consistent between the
//     passes (it is the operator of the rounded blocks), and allowed only on
//     tiles whose entries are a small fraction tau of the largest ones;
// (2) every product of U with the double-FP32 vector x = xh + xl is
//     accumulated on a fixed-point grid: each chain starts at sigma = 1.5 2^e
//     with 2^(e-1) above the largest partial sum the chain can reach (from the
//     tile's bound on |U| and the staged chunk's max |xh|), so the chain value
//     H = sigma + S stays in [2^e, 2^(e+1)) and every
//         t = fma(U, xh, H)   (H + U xh rounded to the grid 2^(e-23))
//         d = t - H           (exact: both on the grid, |d| < 2^e)
//         r = fma(U, xh, -d)  (U xh - d, |r| <= 2^(e-24), rounded at 2^(e-48))
//     moves the part of the product below the grid into a plain FP32 tail L,
//     with U xl added there too (ExtractScalar-style splitting, Rump, Ogita
//     and Oishi, "Accurate floating-point summation", 2008, used here as an
//     accumulator).  Five packed f32x2 instructions per pair of
//     multiply-accumulates, against twelve for Dekker's product and Knuth's
//     TwoSum in k_prod_tiles_df2; the chain error is about 2^-35 of
//     max|U| max|xh| (the tail's own FP32 rounding), so tiles with big
//     entries stay on k_prod_tiles_df2.
// Row and column chain results leave as normalised double-FP32 pairs and go
// through the same cross-lane reduction and FP64 partial-sum slots as the
// other double-FP32 kernels.
__device__ __forceinline__ float grid_sigma(float m, int headroom) {
  // 1.5 2^e with e = exponent(m) + headroom; m >= 0 (0 for an all-zero operand)
  int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127 + headroom;
  e = max(-100, min(e, 120));
  return __uint_as_float(((unsigned)(e + 127) << 23) | 0x400000u);
}

struct XMix { f2 h1, l1, h2, l2; };   // hi / lo of the two operand pairings of one vector entry

__device__ __forceinline__ XMix xmix(double2 v, bool row) {
  const float4 s = split_d(v);           // {re_hi, im_hi, re_lo, im_lo}
  XMix o;
  o.h1 = pk(s.x, s.y);
  o.l1 = pk(s.z, s.w);
  if (!row) {                            // column block x_J: (re, -im)
    o.h2 = pk(s.x, -s.y);
    o.l2 = pk(s.z, -s.w);
  } else {                               // row block x_I: (im, -re)
    o.h2 = pk(s.y, -s.x);
    o.l2 = pk(s.w, -s.z);
  }
  return o;
}

// (H, L) += u (xh + xl) on the grid of H (see above), lane-wise
__device__ __forceinline__ void gacc(f2& H, f2& L, f2 u, f2 xh, f2 xl) {
  const f2 t = fma2(u, xh, H);
  const f2 nd = sub2(H, t);               // -(t - H), exact
  const f2 r = fma2(u, xh, nd);           // u xh - (t - H)
  L = add2(L, r);
  L = fma2(u, xl, L);
  H = t;
}

__device__ __forceinline__ void two_sum1(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__global__ void __launch_bounds__(PROD_THREADS, 2)
k_prod_tiles_mx(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs, int njobs, int mode,
                GenericIO io, int strided) {
  __shared__ XMix xc[TS], xr[TS];
  __shared__ DFC rpark[8][PROD_THREADS];
  __shared__ float smax[8];
  DFC(*red)[TS] = reinterpret_cast<DFC(*)[TS]>(&rpark[0][0]);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int per = strided ? 1 : (njobs + gridDim.x - 1) / gridDim.x;
  const int t0 = strided ? blockIdx.x : blockIdx.x * per;
  const int t1 = strided ? njobs : min(njobs, t0 + per);
  const int dt = strided ? gridDim.x : 1;
  const f2 zero = pk(0.f, 0.f);
  for (int t = t0; t < t1; t += dt) {
    const TileJob jb = jobs[t];
    const Prob& p = probs[jb.prob];
    const double2* x;
    double sB;
    if (!df_operands(p, mode, io, x, sB)) continue;   // uniform per CTA
    const bool diag = jb.I == jb.J;
    __syncthreads();
    float mx;
    {
      const int r = tid & (TS - 1);
      const double2 v = x[(int64_t)(tid < TS ? jb.J : jb.I) * TS + r];
      const XMix o = xmix(v, tid >= TS);
      if (tid < TS) xc[r] = o;
      else xr[r] = o;
      float a0, a1;
      upk(o.h1, a0, a1);
      mx = fmaxf(fabsf(a0), fabsf(a1));
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, m));
      if ((tid & 31) == 0) smax[tid >> 5] = mx;
    }
    __syncthreads();
    mx = smax[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = fmaxf(mx, smax[w]);
    // bound on every |U xh| of this tile; row chains sum 8 such products per lane,
    // column chains 16; one more bit absorbs the roundings of U, of the bound and
    // of the grid itself
    const float m = p.tmax[jb.t] * mx;
    const float sgr = grid_sigma(m, 6), sgc = grid_sigma(m, 7);
    const f2 sr2 = pk(sgr, sgr), sc2 = pk(sgc, sgc);
    const float2* At = (const float2*)p.A + (int64_t)jb.t * (TS * TS);
    const float2* Bt = (const float2*)p.B + (int64_t)jb.t * (TS * TS);
    const float sg = sB > 0.0 ? 1.f : -1.f;
    const f2 spm = pk(sg, -sg);
    f2 cH[8], cL[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      cH[b] = sc2;
      cL[b] = zero;
    }
    float2 av[8], bv[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      av[b] = __ldg(At + ty * TS + tx + 16 * b);
      bv[b] = __ldg(Bt + ty * TS + tx + 16 * b);
    }
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
      const int r = ty + 16 * a;
      float2 an[8], bn[8];
      if (a < 7) {                          // the next row's elements are in flight meanwhile
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          an[b] = __ldg(At + (r + 16) * TS + tx + 16 * b);
          bn[b] = __ldg(Bt + (r + 16) * TS + tx + 16 * b);
        }
      }
      const XMix y = xr[r];
      f2 H1 = sr2, L1 = zero, H2 = sr2, L2 = zero;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const XMix xv = xc[tx + 16 * b];
        // (U_re, V_re) and (U_im, V_im), rounded
        const f2 uvr = fma2(pk(bv[b].x, bv[b].x), spm, pk(av[b].x, av[b].x));
        const f2 uvi = fma2(pk(bv[b].y, bv[b].y), spm, pk(av[b].y, av[b].y));
        gacc(H1, L1, uvr, xv.h1, xv.l1);
        gacc(H2, L2, uvi, xv.h2, xv.l2);
        if (!diag) {
          gacc(cH[b], cL[b], uvr, y.h1, y.l1);
          gacc(cH[b], cL[b], uvi, y.h2, y.l2);
        }
      }
      // y_re = lane 0 of chain 1 + lane 1 of chain 2, y_im = lane 1 of 1 + lane 0 of 2;
      // the grid parts add exactly, then (grid, tail) is normalised
      const f2 S1 = sub2(H1, sr2), S2 = sub2(H2, sr2);
      float s1a, s1b, s2a, s2b, l1a, l1b, l2a, l2b;
      upk(S1, s1a, s1b);
      upk(S2, s2a, s2b);
      upk(L1, l1a, l1b);
      upk(L2, l2a, l2b);
      DFC ra;
      two_sum1(__fadd_rn(s1a, s2b), __fadd_rn(l1a, l2b), ra.rh, ra.rl);
      two_sum1(__fadd_rn(s1b, s2a), __fadd_rn(l1b, l2a), ra.ih, ra.il);
      rpark[a][tid] = ra;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        av[b] = an[b];
        bv[b] = bn[b];
      }
    }
    DFC racc[8], cacc[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      float hr, hi, lr, li;
      upk(sub2(cH[b], sc2), hr, hi);
      upk(cL[b], lr, li);
      two_sum1(hr, lr, cacc[b].rh, cacc[b].rl);
      two_sum1(hi, li, cacc[b].ih, cacc[b].il);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) racc[a] = rpark[a][tid];
    __syncthreads();   // rpark is reused below as the column-reduction buffer
    df_tile_reduce(racc, cacc, red, diag, p, jb);
  }
}

// per-tile bound max over the tile of max(|A_re| + |B_re|, |A_im| + |B_im|)
// (>= every |U| and |V| component for s = +-1); one CTA per tile
__global__ void __launch_bounds__(256)
k_tile_bound(const float2* __restrict__ A, const float2* __restrict__ B, int64_t ntiles, float* __restrict__ out) {
  __shared__ float sm[8];
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const float2* a = A + t * (TS * TS);
    const float2* b = B + t * (TS * TS);
    float m = 0.f;
    for (int e = threadIdx.x; e < TS * TS; e += 256) {
      const float2 x = a[e], y = b[e];
      m = fmaxf(m, fmaxf(fabsf(x.x) + fabsf(y.x), fabsf(x.y) + fabsf(y.y)));
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float r = sm[0];
      for (int w = 1; w < 8; ++w) r = fmaxf(r, sm[w]);
      // one ulp up: the sums above were rounded to nearest
      out[t] = r > 0.f ? __uint_as_float(__float_as_uint(r) + 1u) : 0.f;
    }
    __syncthreads();
  }
}

__global__ void k_split_tiles(const double2* __restrict__ in, int64_t n, float4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = split_d(in[i]);
}

}  // namespace

template <bool HASB, bool SPLIT>
int df_occupancy() {
  static int occ = 0;
  if (!occ) {
    int o = 0;
    if constexpr (HASB && !SPLIT)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_prod_tiles_df2, PROD_THREADS, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_prod_tiles_df<HASB, SPLIT>, PROD_THREADS, 0);
    occ = o > 0 ? o : 1;
  }
  return occ;
}

int product_df_occupancy(bool hasB, bool split) {
  if (split) return hasB ? df_occupancy<true, true>() : df_occupancy<false, true>();
  return hasB ? df_occupancy<true, false>() : df_occupancy<false, false>();
}

template <bool HASB, bool SPLIT>
void launch_df(const Prob* dprobs, const TileJob* jobs, int njobs, int mode, const GenericIO& io, ProdShape shape,
               cudaStream_t s) {
  const int grid = product_grid(df_occupancy<HASB, SPLIT>(), shape, njobs);
  // complex64 PH tiles: the packed kernel (measured 11 % faster per product at N = 2e4); split
  // complex128 tiles: the scalar kernel (its float4 rows leave the packed one no registers for
  // latency hiding: 0.274 vs 0.250 ms at N = 8000)
  if constexpr (HASB && !SPLIT)
    k_prod_tiles_df2<<<grid, PROD_THREADS, 0, s>>>(dprobs, jobs, njobs, mode, io, shape.strided);
  else
    k_prod_tiles_df<HASB, SPLIT><<<grid, PROD_THREADS, 0, s>>>(dprobs, jobs, njobs, mode, io, shape.strided);
}

void launch_product_df(const Prob* dprobs, const TileJob* jobs, int njobs, int nprob, int maxnT, int mode,
                       const GenericIO* io_host, bool hasB, bool split, ProdShape shape, cudaStream_t s) {
  count_launch(2);
  GenericIO io{};
  if (io_host) io = *io_host;
  if (split) {
    if (hasB) launch_df<true, true>(dprobs, jobs, njobs, mode, io, shape, s);
    else launch_df<false, true>(dprobs, jobs, njobs, mode, io, shape, s);
  } else {
    if (hasB) launch_df<true, false>(dprobs, jobs, njobs, mode, io, shape, s);
    else launch_df<false, false>(dprobs, jobs, njobs, mode, io, shape, s);
  }
  launch_prod_reduce_d(dprobs, nprob, maxnT, mode, io, s);
}

int product_mx_occupancy() {
  static int occ = 0;
  if (!occ) {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_prod_tiles_mx, PROD_THREADS, 0);
    occ = o > 0 ? o : 1;
  }
  return occ;
}

void launch_product_mixed(const Prob* dprobs, const TileJob* fine, int nfine, const TileJob* coarse, int ncoarse,
                          int nprob, int maxnT, int mode, const GenericIO* io_host, ProdShape shape, cudaStream_t s) {
  GenericIO io{};
  if (io_host) io = *io_host;
  if (nfine > 0) {
    count_launch();
    const ProdShape fs{0, 1};
    k_prod_tiles_df2<<<product_grid(df_occupancy<true, false>(), fs, nfine), PROD_THREADS, 0, s>>>(
        dprobs, fine, nfine, mode, io, 1);
  }
  if (ncoarse > 0) {
    count_launch();
    k_prod_tiles_mx<<<product_grid(product_mx_occupancy(), shape, ncoarse), PROD_THREADS, 0, s>>>(
        dprobs, coarse, ncoarse, mode, io, shape.strided);
  }
  count_launch();
  launch_prod_reduce_d(dprobs, nprob, maxnT, mode, io, s);
}

void launch_tile_bound(const float2* A, const float2* B, int64_t ntiles, float* out, cudaStream_t s) {
  count_launch();
  const int grid = (int)std::min<int64_t>(ntiles, 4096);
  k_tile_bound<<<grid, 256, 0, s>>>(A, B, ntiles, out);
}

void launch_split_tiles(const double2* packed, int64_t nelem, float4* split, cudaStream_t s) {
  count_launch();
  k_split_tiles<<<1024, 256, 0, s>>>(packed, nelem, split);
}

}  // namespace bse
