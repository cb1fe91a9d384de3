// Complex128 structured product in double-FP32 ("df64") arithmetic.
//
// GB300 executes 2 FP64 FMAs per SM per clock but 128 FP32 operations, so
// the FP64 product (16 FMAs per stored element pair of A and B) is bound by
// the FP64 pipe at about 1/5 of the HBM rate.  This kernel streams the same
// packed tiles, pre-split at creation into float pairs a = a_hi + a_lo
// (|a_lo| <= 2^-24 |a_hi|, exact to 2^-48 relative), and evaluates every
// complex multiply-accumulate with error-free transformations on the FP32
// pipes:
//   p = fl(a_hi x_hi),  e = fma(a_hi, x_hi, -p) + a_hi x_lo + a_lo x_hi
//   (s_hi, err) = TwoSum(s_hi, p),  s_lo += err + e
// (Dekker's product, Knuth's TwoSum; the dropped a_lo x_lo is 2^-48 of the
// term).  Partial sums leave the kernel as FP64 and are reduced in FP64 by
// the same k_prod_reduce.  Explicit __f*_rn intrinsics keep the compiler from
// contracting the transformations.
//
// The Krylov basis, Gram-Schmidt, projected problem and the final residuals
// of this path stay in FP64; only the streaming product changes arithmetic.
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

// Knuth's TwoSum: s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

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

// SPLIT: float4 split complex128 tiles (p.Ahl); otherwise complex64 tiles (p.A)
template <bool HASB, bool SPLIT>
__global__ void __launch_bounds__(PROD_THREADS, 2)
k_prod_tiles_df(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs, int njobs, int mode,
                GenericIO io, int strided) {
  __shared__ float4 xc[TS], xr[TS];
  // per-thread row partial sums (own slots only); after a barrier the same
  // storage holds the cross-warp column reduction
  __shared__ DFC rpark[8][PROD_THREADS];
  DFC(*red)[TS] = reinterpret_cast<DFC(*)[TS]>(&rpark[0][0]);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
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
          float4 u, v;
          if constexpr (SPLIT) {           // split P = A + B, Q = A - B, chosen by pointer
            u = widen(av[b]);
            v = widen(bv[b]);
          } else {                         // exact complex64 A, B: TwoSum gives U, V exactly
            const float4 a0 = widen(av[b]), b0 = widen(bv[b]);
            const float sb = sB > 0.0 ? b0.x : -b0.x, sbi = sB > 0.0 ? b0.y : -b0.y;
            two_sum(a0.x, sb, u.x, u.z);
            two_sum(a0.y, sbi, u.y, u.w);
            two_sum(a0.x, -sb, v.x, v.z);
            two_sum(a0.y, -sbi, v.y, v.w);
          }
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

void launch_split_tiles(const double2* packed, int64_t nelem, float4* split, cudaStream_t s) {
  count_launch();
  k_split_tiles<<<1024, 256, 0, s>>>(packed, nelem, split);
}

}  // namespace bse
