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

// partial-sum slots of the double-FP32 kernels hold the (hi, lo) pairs as
// float4 {re_hi, re_lo, im_hi, im_lo}; k_prod_reduce_dfc adds them in FP64
__device__ __forceinline__ float4 dfc_pack(const DFC& v) { return make_float4(v.rh, v.rl, v.ih, v.il); }

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
    case PM_STEP_MMINUS_W:
      if (fresh || j >= p.ncv) return false;
      x = (const double2*)p.w; sB = -1.0; return true;
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
      float4* part = (float4*)p.part;
      part[((int64_t)jb.I * p.nT + jb.J) * TS + ty + 16 * ((tx >> 1) & 7)] = dfc_pack(racc[0]);
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
      float4* part = (float4*)p.part;
      part[((int64_t)jb.J * p.nT + jb.I) * TS + tid] = dfc_pack(s);
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
//     tile's bound on |U| and the chunk's max |xh|), so the chain value
//     H = sigma + S stays in [2^e, 2^(e+1)) and every
//         t = fma(U, xh, H)   (H + U xh rounded to the grid 2^(e-23))
//         d = t - H           (exact: both on the grid, |d| < 2^e)
//         r = fma(U, xh, -d)  (U xh - d, |r| <= 2^(e-24), rounded at 2^(e-48))
//     moves the part of the product below the grid into a plain FP32 tail L,
//     with U xl added there too (ExtractScalar-style splitting, Rump, Ogita
//     and Oishi, "Accurate floating-point summation", 2008, used here as an
//     accumulator).  Five packed f32x2 instructions per pair of
//     multiply-accumulates, against twelve for Dekker's product and Knuth's
//     TwoSum in k_prod_tiles_df2.  The cross-lane sums of a tile use the same
//     idea one level up: every chain value is split at a grid 2^5 coarser than
//     the chains' (regrid), so the 16 or 32 grid parts of a row or column add
//     exactly with plain FP32 adds and only the tails round.  The error is
//     about 2^-30 of max|U| max|xh| in the worst case (the tails' FP32
//     rounding), so tiles with big entries stay on k_prod_tiles_df2.
//
// Data movement: one CTA of 512 threads per SM walks its tile jobs; the tile
// rows stream through a three-stage shared-memory pipeline of 32-row slabs of
// A and B (64 KiB a stage) filled by bulk asynchronous copies (cp.async.bulk,
// completion counted on an mbarrier), so up to 192 KiB per SM are in flight
// while the registers hold only accumulators.  The vector enters pre-split
// (k_mx_stage_x, once per product: hi/lo pairs in both pairings, and the max
// |xh| of every 128-entry chunk) and its two chunks ride along with a tile's
// first slab.  Every wait is bounded: on expiry the CTA stops, waits (bounded)
// for its copies in flight, and raises the caller's error flag.
__device__ __forceinline__ float grid_sigma(float m, int headroom) {
  // 1.5 2^e with e = exponent(m) + headroom; m >= 0 (0 for an all-zero operand)
  int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127 + headroom;
  e = max(-100, min(e, 120));
  return __uint_as_float(((unsigned)(e + 127) << 23) | 0x400000u);
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

// (grid part, tail) pairs of the coarse kernel's cross-lane sums: the grid parts of all lanes
// lie on one grid coarse enough that their sums are exact, so the pairs add with plain adds
__device__ __forceinline__ DFC gadd(DFC a, const DFC& b) {
  a.rh = __fadd_rn(a.rh, b.rh);
  a.rl = __fadd_rn(a.rl, b.rl);
  a.ih = __fadd_rn(a.ih, b.ih);
  a.il = __fadd_rn(a.il, b.il);
  return a;
}

// split an exact chain value S (|S| < 2^e, on the grid 2^(e-23)) at the grid of gs = 1.5 2^(e+5):
// g = the part on the grid 2^(e-18) (exact), and the rest (|.| <= 2^(e-19), exact) added to l
__device__ __forceinline__ void regrid(float S, float l, float gs, float& g, float& lo) {
  g = __fsub_rn(__fadd_rn(gs, S), gs);
  lo = __fadd_rn(l, __fsub_rn(S, g));
}

// x of every active problem, split once per product into chunks of 128 entries, one float4
// record {hi_re, hi_im, lo_re, lo_im} per entry (2 KiB a chunk, so one bulk copy stages it),
// with re and im exchanged in both pairs for the minus half (s = -1; see k_prod_tiles_mx),
// and xmax[I] = max |hi| over chunk I; grid (maxnT, nprob), TS threads
__global__ void __launch_bounds__(TS)
k_mx_stage_x(const Prob* __restrict__ probs, int mode, GenericIO io) {
  __shared__ float sm[TS / 32];
  const Prob& p = probs[blockIdx.y];
  const int I = blockIdx.x;
  if (I >= p.nT) return;
  const double2* x;
  double sB;
  if (!df_operands(p, mode, io, x, sB)) return;
  const int64_t r = (int64_t)I * TS + threadIdx.x;
  const float4 v = split_d(x[r]);          // {re_hi, im_hi, re_lo, im_lo}
  float4* xs = (float4*)p.xs + (int64_t)I * TS;
  xs[threadIdx.x] = sB > 0.0 ? v : make_float4(v.y, v.x, v.w, v.z);
  float m = fmaxf(fabsf(v.x), fabsf(v.y));
#pragma unroll
  for (int k = 16; k >= 1; k >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, k));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = sm[0];
#pragma unroll
    for (int w = 1; w < TS / 32; ++w) t = fmaxf(t, sm[w]);
    p.xmax[I] = t;
  }
}

// Two shapes of the coarse-tile kernel (the launch-shape tuner picks one per handle by timing):
// NT = 512 threads with 32-row slabs, one CTA per SM (216 KiB of shared memory), or NT = 256
// with 16-row slabs, two CTAs per SM (112 KiB each), whose block barriers overlap the other
// CTA's work.  16 column lanes x NT / 16 row lanes; the row lanes are the rows of a slab.
template <int NT>
struct Mx {
  static constexpr int THREADS = NT;
  static constexpr int CTAS = 512 / NT;                  // CTAs per SM
  static constexpr int WARPS = NT / 32;
  static constexpr int ROWS = NT / 16;                   // rows of a slab
  static constexpr int SLABS = TS / ROWS;                // slabs per tile (a multiple of 4)
  static constexpr int NST = 3;                          // pipeline stages
  static constexpr uint32_t HALF = ROWS * TS * 8;        // one matrix's slab
  static constexpr uint32_t STAGE = 2 * HALF;            // A and B
  static constexpr uint32_t XBYTES = 2 * TS * 8;         // one staged vector chunk (hi, lo): 2 KiB
  static constexpr uint32_t XOFF = NST * STAGE;          // two x buffers of (column, row) chunks
  static constexpr uint32_t REDOFF = XOFF + 2 * 2 * XBYTES;
  static constexpr int REDW = WARPS / 2;                 // column-reduction buffer: half the warps
  static constexpr uint32_t SMEM = REDOFF + REDW * TS * sizeof(DFC);
  // column chains sum 2 SLABS products per lane: |S| < 2^(k + 1 + log2(2 SLABS)), grid e below
  static constexpr int COLHEAD = SLABS == 4 ? 6 : 7;
};
constexpr long long MX_SPIN = 1ll << 26;              // polls of a bounded wait

__device__ __forceinline__ uint32_t mx_s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mx_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mx_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < MX_SPIN; ++i)
    if (mx_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mx_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// The tiles are streamed as the records UV = {U_re, V_re, U_im, V_im} of U = fl(A + B),
// V = fl(A - B) (Prob::UV), so that (U_re, V_re) and (U_im, V_im) are register pairs as
// loaded.  For the minus half (s = -1) U and V trade places; instead of swapping them, x is
// staged with re and im exchanged (k_mx_stage_x), which exchanges the two lanes of every
// chain, and the combinations below read the lanes the other way round.
// Thread (tx, ty) = (tid % 16, tid / 16) takes row ty of each slab and the columns
// c_b = tx + 16 b, b < 8: one 16-byte shared load brings one record (UV and x alike), and the
// 16 lanes of a row read 256 contiguous bytes.  Stage release: each warp arrives on empty[s]
// when it is done with stage s; the producer (thread 0) waits for all warps before refilling.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
k_prod_tiles_mx(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs, int njobs, int mode,
                GenericIO io, int strided, int* __restrict__ err) {
  using C = Mx<NT>;
  extern __shared__ __align__(128) unsigned char smx[];
  __shared__ uint64_t full[C::NST], empty[C::NST];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
  const int per = strided ? 1 : (njobs + gridDim.x - 1) / gridDim.x;
  const int t0 = strided ? blockIdx.x : blockIdx.x * per;
  const int t1 = strided ? njobs : min(njobs, t0 + per);
  const int dt = strided ? gridDim.x : 1;
  if (tid == 0) {
    for (int s = 0; s < C::NST; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mx_s32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mx_s32(&empty[s])), "r"(C::WARPS) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto active = [&](int t) {
    const double2* xx;
    double sb;
    return df_operands(probs[jobs[t].prob], mode, io, xx, sb);
  };
  // producer cursor (thread 0): the next (job, slab) to copy, and the active-tile ordinal
  int pt = t0, pa = 0, ptile = 0;
  long long issued = 0;
  bool pok = true;
  // issue every slab below `must` (waiting, bounded, for its stage to be released), then more
  // while stages happen to be free
  auto produce = [&](long long must) {
    while (pok) {
      if (pa == 0) {
        while (pt < t1 && !active(pt)) pt += dt;
        if (pt >= t1) return;
      }
      const int s = (int)(issued % C::NST);
      if (issued >= C::NST) {     // every warp is done with the previous use of stage s?
        const uint32_t bar = mx_s32(&empty[s]);
        const uint32_t par = (uint32_t)(((issued - C::NST) / C::NST) & 1);
        if (issued < must) {
          if (!mx_wait(bar, par)) { pok = false; return; }
        } else if (!mx_try(bar, par)) {
          return;
        }
      }
      const TileJob jb = jobs[pt];
      const Prob& p = probs[jb.prob];
      const uint32_t bar = mx_s32(&full[s]);
      const uint32_t st = mx_s32(smx) + (uint32_t)s * C::STAGE;
      const size_t off = ((size_t)jb.t * TS + (size_t)pa * C::ROWS) * TS;
      const uint32_t bytes = C::STAGE + (pa == 0 ? 2 * C::XBYTES : 0u);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
      mx_copy(st, (const float4*)p.UV + off, C::STAGE, bar);
      if (pa == 0) {   // the tile's two vector chunks, into the x buffer of its parity
        const uint32_t xb = mx_s32(smx) + C::XOFF + (uint32_t)(ptile & 1) * 2 * C::XBYTES;
        const float4* xs = (const float4*)p.xs;
        mx_copy(xb, xs + (int64_t)jb.J * TS, C::XBYTES, bar);
        mx_copy(xb + C::XBYTES, xs + (int64_t)jb.I * TS, C::XBYTES, bar);
      }
      ++issued;
      if (++pa == C::SLABS) {
        pa = 0;
        pt += dt;
        ++ptile;
      }
    }
  };
  if (tid == 0) produce(0);
  DFC(*red)[TS] = reinterpret_cast<DFC(*)[TS]>(smx + C::REDOFF);
  const f2 zero = pk(0.f, 0.f);
  long long consumed = 0;
  int ctile = 0;
  bool ok = true;
  for (int t = t0; t < t1 && ok; t += dt) {
    const TileJob jb = jobs[t];
    const Prob& p = probs[jb.prob];
    const double2* x;
    double sB;
    if (!df_operands(p, mode, io, x, sB)) continue;   // uniform per CTA
    const bool diag = jb.I == jb.J;
    const float4* xc4 = reinterpret_cast<const float4*>(smx + C::XOFF + (ctile & 1) * 2 * C::XBYTES) + tx;
    const float4* xr4 = xc4 - tx + TS;                                       // row chunk I
    // bound m on every |U xh| of this tile (m < 2^(k+1), k its exponent); row chains sum 8
    // such products per lane, so |S| < 2^(k+4) (1 + 3 u) and the grid 2^e with e = k + 6
    // keeps |S| below 2^(e-1) with a factor 2 to spare; column chains sum 16 (8 rows x 2):
    // e = k + 7
    const float m = p.tmax[jb.t] * fmaxf(p.xmax[jb.I], p.xmax[jb.J]);
    const float sg = grid_sigma(m, 6);
    const f2 sg2 = pk(sg, sg);
    const float sgc = grid_sigma(m, C::COLHEAD);
    const f2 sgc2 = pk(sgc, sgc);
    // grid of the cross-lane sums: at most 16 chain values are added (16 column lanes of a
    // row, 16 row lanes of a column), each below 2^(k+7), so every partial sum stays below
    // 2^(k+11) and 1.5 2^(k+11) leaves a factor 2 to spare
    const float gs = grid_sigma(m, 11);
    const bool neg = sB < 0.0;                       // minus half: chain lanes exchanged
    const float sgn = neg ? -1.f : 1.f;
    f2 cH[8], cL[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      cH[b] = sgc2;
      cL[b] = zero;
    }
    DFC racc[4];                      // this thread's rows of four consecutive slabs
    // groups of four slabs (the group loop is not unrolled: one copy of the slab code)
#pragma unroll 1
    for (int a0 = 0; a0 < C::SLABS; a0 += 4) {
#pragma unroll
    for (int a4 = 0; a4 < 4; ++a4) {
      const int a = a0 + a4;
      const int s = (int)(consumed % C::NST);
      if (tid == 0) produce(consumed + 1);     // this slab is issued before anyone waits for it
      // a wait that expires raises the error flag; the warp goes on (its reads stay inside
      // shared memory) and the CTA stops at the end of the tile
      if (__any_sync(0xffffffffu, !mx_wait(mx_s32(&full[s]), (uint32_t)((consumed / C::NST) & 1)))) {
        if (lane == 0) atomicExch(err, 1);
        ok = false;
      }
      const float4* Us = reinterpret_cast<const float4*>(smx + (size_t)s * C::STAGE) + ty * TS + tx;
      // row entry of x_I, staged as (y_re, y_im) (minus half: (y_im, y_re)); the column chains
      // take y1 = that pair and y2 = s (y.1, -y.0), hi and lo
      const float4 yv = xr4[ty + C::ROWS * a];
      const f2 y1h = pk(yv.x, yv.y), y1l = pk(yv.z, yv.w);
      const f2 y2h = pk(sgn * yv.y, -sgn * yv.x), y2l = pk(sgn * yv.w, -sgn * yv.z);
      // plus half: chain 1 (U_re x_re, V_re x_im), chain 2 (U_im x_re, V_im x_im)
      f2 H1 = sg2, L1 = zero, H2 = sg2, L2 = zero;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float4 uv = Us[16 * b], xv = xc4[16 * b];
        const f2 uvr = pk(uv.x, uv.y), uvi = pk(uv.z, uv.w);
        const f2 xh = pk(xv.x, xv.y), xl = pk(xv.z, xv.w);
        gacc(H1, L1, uvr, xh, xl);
        gacc(H2, L2, uvi, xh, xl);
        if (!diag) {
          gacc(cH[b], cL[b], uvr, y1h, y1l);
          gacc(cH[b], cL[b], uvi, y2h, y2l);
        }
      }
      // stage s is no longer read by this warp
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mx_s32(&empty[s])) : "memory");
      // y_re = U_re x_re - V_im x_im = lane 0 of chain 1 - lane 1 of chain 2,
      // y_im = V_re x_im + U_im x_re = lane 1 of chain 1 + lane 0 of chain 2;
      // the grid parts add exactly, then (grid, tail) is normalised
      float s1a, s1b, s2a, s2b, l1a, l1b, l2a, l2b;
      upk(sub2(H1, sg2), s1a, s1b);
      upk(sub2(H2, sg2), s2a, s2b);
      upk(L1, l1a, l1b);
      upk(L2, l2a, l2b);
      if (neg) {                     // the minus half accumulated with the chain lanes exchanged
        float t;
        t = s1a; s1a = s1b; s1b = t;
        t = s2a; s2a = s2b; s2b = t;
        t = l1a; l1a = l1b; l1b = t;
        t = l2a; l2a = l2b; l2b = t;
      }
      regrid(__fsub_rn(s1a, s2b), __fsub_rn(l1a, l2b), gs, racc[a4].rh, racc[a4].rl);
      regrid(__fadd_rn(s1b, s2a), __fadd_rn(l1b, l2a), gs, racc[a4].ih, racc[a4].il);
      ++consumed;
    }
      // ---- row sums of slabs a0 .. a0 + 3: reduce-scatter of the 4 rows over the 16 column
      // lanes, then the remaining pairs; lanes tx % 4 == 0 write row
      // ty + ROWS (a0 + (tx >> 3) * 2 + ((tx >> 2) & 1))
      const bool u8 = tx & 8;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const DFC snd = u8 ? racc[q] : racc[q + 2], kp = u8 ? racc[q + 2] : racc[q];
        racc[q] = gadd(kp, dfc_shfl(snd, 8));
      }
      const bool u4 = tx & 4;
      {
        const DFC snd = u4 ? racc[0] : racc[1], kp = u4 ? racc[1] : racc[0];
        racc[0] = gadd(kp, dfc_shfl(snd, 4));
      }
      racc[0] = gadd(racc[0], dfc_shfl(racc[0], 2));
      racc[0] = gadd(racc[0], dfc_shfl(racc[0], 1));
      if ((tx & 3) == 0) {
        const int as = a0 + (u8 ? 2 : 0) + (u4 ? 1 : 0);
        float4* part = (float4*)p.part;
        part[((int64_t)jb.I * p.nT + jb.J) * TS + ty + C::ROWS * as] = dfc_pack(racc[0]);
      }
    }
    if (__syncthreads_or(ok ? 0 : 1)) {
      ok = false;
      break;
    }
    ++ctile;
    if (!diag) {
      // ---- column sums over the 16 row lanes: the two of a warp (xor 16), then 8 warps in
      // two rounds through a REDW x TS buffer.  Column of entry b: tx + 16 b; the minus half
      // holds (im, re) in the chain lanes
      DFC cacc[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        float hr, hi, lr, li;
        upk(sub2(cH[b], sgc2), hr, hi);
        upk(cL[b], lr, li);
        if (neg) {
          float t;
          t = hr; hr = hi; hi = t;
          t = lr; lr = li; li = t;
        }
        regrid(hr, lr, gs, cacc[b].rh, cacc[b].rl);
        regrid(hi, li, gs, cacc[b].ih, cacc[b].il);
      }
      const bool up = lane & 16;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const DFC snd = up ? cacc[q] : cacc[q + 4], kp = up ? cacc[q + 4] : cacc[q];
        cacc[q] = gadd(kp, dfc_shfl(snd, 16));
      }
      // lane keeps entries b = q + 4 up, q < 4
      auto col = [&](int b) { return tx + 16 * b; };
      if (warp >= C::REDW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp - C::REDW][col(q + (up ? 4 : 0))] = cacc[q];
      }
      __syncthreads();
      if (warp < C::REDW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = col(q + (up ? 4 : 0));
          red[warp][c] = gadd(cacc[q], red[warp][c]);
        }
      }
      __syncthreads();
      if (tid < TS) {
        DFC sum = red[0][tid];
#pragma unroll
        for (int w = 1; w < C::REDW; ++w) sum = gadd(sum, red[w][tid]);
        float4* part = (float4*)p.part;
        part[((int64_t)jb.J * p.nT + jb.I) * TS + tid] = dfc_pack(sum);
      }
      // red is next written after the next tile's block barrier
    }
  }
  if (tid == 0) {
    // finish the producer's work only as far as needed to leave no copy in flight
    if (!ok) pok = false;
    for (long long g = consumed; g < issued; ++g)
      mx_wait(mx_s32(&full[g % C::NST]), (uint32_t)((g / C::NST) & 1));
  }
  __syncthreads();
}

// records {U_re, V_re, U_im, V_im} of U = fl(A + B), V = fl(A - B) for every packed element
// (the values the coarse-tile kernel multiplies, rounded once at ingest)
__global__ void k_uv_pack(const float2* __restrict__ A, const float2* __restrict__ B, int64_t n,
                          float4* __restrict__ uv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = A[i], b = B[i];
    uv[i] = make_float4(__fadd_rn(a.x, b.x), __fsub_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fsub_rn(a.y, b.y));
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

int product_mx_occupancy() { return 2; }   // shapes: 1 (512 threads) or 2 (256 threads) CTAs per SM

template <int NT>
void launch_mx(const Prob* dprobs, const TileJob* coarse, int ncoarse, int mode, const GenericIO& io,
               ProdShape shape, int* err, cudaStream_t s) {
  using C = Mx<NT>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_prod_tiles_mx<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    cudaFuncSetAttribute(k_prod_tiles_mx<NT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = true;
  }
  const ProdShape ms{shape.ctas_per_sm < 0 ? -1 : C::CTAS, shape.strided};
  k_prod_tiles_mx<NT><<<product_grid(C::CTAS, ms, ncoarse), NT, C::SMEM, s>>>(dprobs, coarse, ncoarse, mode, io,
                                                                            shape.strided, err);
}

void launch_product_mixed(const Prob* dprobs, const TileJob* fine, int nfine, const TileJob* coarse, int ncoarse,
                          int nprob, int maxnT, int mode, const GenericIO* io_host, ProdShape shape, int* err,
                          cudaStream_t s) {
  GenericIO io{};
  if (io_host) io = *io_host;
  if (nfine > 0) {
    count_launch();
    const ProdShape fs{0, 1};
    k_prod_tiles_df2<<<product_grid(df_occupancy<true, false>(), fs, nfine), PROD_THREADS, 0, s>>>(
        dprobs, fine, nfine, mode, io, 1);
  }
  if (ncoarse > 0) {
    count_launch(2);
    k_mx_stage_x<<<dim3(maxnT, nprob), TS, 0, s>>>(dprobs, mode, io);
    // shape.ctas_per_sm: 1 -> the 512-thread kernel, otherwise the 256-thread one (two CTAs per
    // SM; -1: one CTA per tile)
    if (shape.ctas_per_sm == 1) launch_mx<512>(dprobs, coarse, ncoarse, mode, io, shape, err, s);
    else launch_mx<256>(dprobs, coarse, ncoarse, mode, io, shape, err, s);
  }
  count_launch();
  launch_prod_reduce_d(dprobs, nprob, maxnT, mode, io, s);
}

void launch_tile_bound(const float2* A, const float2* B, int64_t ntiles, float* out, cudaStream_t s) {
  count_launch();
  const int grid = (int)std::min<int64_t>(ntiles, 4096);
  k_tile_bound<<<grid, 256, 0, s>>>(A, B, ntiles, out);
}

void launch_uv_pack(const float2* A, const float2* B, int64_t nelem, float4* uv, cudaStream_t s) {
  count_launch();
  k_uv_pack<<<1024, 256, 0, s>>>(A, B, nelem, uv);
}

void launch_split_tiles(const double2* packed, int64_t nelem, float4* split, cudaStream_t s) {
  count_launch();
  k_split_tiles<<<1024, 256, 0, s>>>(packed, nelem, split);
}

}  // namespace bse
