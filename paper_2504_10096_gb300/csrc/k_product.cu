// Structured products with the packed A and B (BSE Eq. 1 blocks).
//
// The hot kernel k_prod_tiles streams every stored upper-triangle tile of A
// (and of B) exactly once per product and uses it for both block rows:
//     y_I += A_IJ x_J + s B_IJ conj(x_J)
//     y_J += A_IJ^H x_I + s B_IJ^T conj(x_I)        (I < J)
// because A = A^H and B = B^T, applied in the real form of Eq. 5 (U = A + sB,
// V = A - sB; 8 FMAs per stored element pair, see k_prod_tiles).  This is the
// matrix-vector product that the paper identifies as the most expensive step
// of the iterative solver (Sec. 2.2.2, last paragraph).  Each tile writes its two partial block-row
// results into a scratch buffer part[I][J][:] (slot (I,J) receives the
// contribution of column block J to row block I), and k_prod_reduce sums the
// nT slots of every block row: no atomics, deterministic rounding order.
//
// k_prod_rowblock is the wide-block variant (k columns, GEMM-like): one CTA
// owns an output block row and reads tile (I,J) or the transpose of (J,I).
#include <type_traits>

#include "bse_phases.cuh"

namespace bse {

// (P, Q) = (A + B, A - B) -> (A, B)
template <typename CT>
__device__ __forceinline__ void unpack_pq(CT& a, CT& b) {
  const CT pv = a, qv = b;
  a.x = 0.5 * (pv.x + qv.x); a.y = 0.5 * (pv.y + qv.y);
  b.x = 0.5 * (pv.x - qv.x); b.y = 0.5 * (pv.y - qv.y);
}

// A CTA walks the global job list either as one contiguous run or with stride
// gridDim.x (ProdShape).  Registers allow one FP64 CTA per SM (FP64-pipe
// bound) and two FP32 ones, so that twice as many tile loads are in flight
// (the FP32 product is HBM-latency bound).  The arithmetic is prod_tiles_body.
template <typename ST, typename R, bool HASB>
__global__ void __launch_bounds__(PROD_THREADS, sizeof(R) == 4 ? 2 : 1)
k_prod_tiles(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs, int njobs,
             int mode, GenericIO io, int strided) {
  using CT = typename Acc<R>::T;
  __shared__ CT xc[TS];      // column block J of x
  __shared__ CT xr[TS];      // row block I of x
  __shared__ CT red[8][TS];  // column reduction across warps
  prod_tiles_body<ST, R, HASB>(probs, jobs, njobs, mode, io, strided, blockIdx.x, gridDim.x, xc, xr, red);
}

// y[I*TS + r] = sum_J part[I][J][r]; grid (maxnT, nprob) (prod_reduce_body).
template <typename ST, typename R>
__global__ void __launch_bounds__(REDUCE_GROUPS * TS)
k_prod_reduce(const Prob* __restrict__ probs, int mode, GenericIO io) {
  using CT = typename Acc<R>::T;
  __shared__ CT grp[REDUCE_GROUPS - 1][TS];
  prod_reduce_body<ST, R>(probs, mode, io, blockIdx.x, blockIdx.y, grp);
}

// Same reduction for the double-FP32 kernels, whose slots hold (hi, lo) float
// pairs {re_hi, re_lo, im_hi, im_lo}: each slot is widened to FP64 and the slots
// are summed in FP64 in the fixed order above.
__global__ void __launch_bounds__(REDUCE_GROUPS * TS)
k_prod_reduce_dfc(const Prob* __restrict__ probs, int mode, GenericIO io) {
  __shared__ double2 grp[REDUCE_GROUPS - 1][TS];
  const Prob& p = probs[blockIdx.y];
  const int I = blockIdx.x;
  if (I >= p.nT) return;
  const double2* x; double2* y; double sB;
  if (!prod_operands<double2, double>(p, mode, io, x, y, sB)) return;
  const int r = threadIdx.x & (TS - 1), g = threadIdx.x >> 7;
  const float4* part = (const float4*)p.part + (int64_t)I * p.nT * TS;
  double2 acc = make_double2(0.0, 0.0);
  auto wide = [](float4 v) { return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w); };
  int J = g;
  for (; J + 3 * REDUCE_GROUPS < p.nT; J += 4 * REDUCE_GROUPS) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = part[(int64_t)(J + u * REDUCE_GROUPS) * TS + r];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc = cadd(acc, wide(v[u]));
  }
  for (; J < p.nT; J += REDUCE_GROUPS) acc = cadd(acc, wide(part[(int64_t)J * TS + r]));
  if (g > 0) grp[g - 1][r] = acc;
  __syncthreads();
  if (g == 0) {
#pragma unroll
    for (int q = 0; q < REDUCE_GROUPS - 1; ++q) acc = cadd(acc, grp[q][r]);
    y[(int64_t)I * TS + r] = acc;
    if (p.ws && y == (double2*)p.w) p.ws[(int64_t)I * TS + r] = dsplit(acc);   // its double-FP32 shadow
  }
}

// ---------------------------------------------------------------- wide blocks
// Y[:, c0:c0+16] of block row I = sum_J Ablk(I,J) XA_J + sB Bblk(I,J) XB_J,
// Ablk(I,J) = tile(I,J) for J >= I, tile(J,I)^H otherwise; Bblk uses ^T.
// XA, XB, Y: compute-type complex, column-major, Npad rows.
constexpr int RB_Q = 16;   // q-chunk staged in shared memory
template <typename ST, typename R, bool HASB>
__global__ void __launch_bounds__(256)
k_prod_rowblock(const Prob* __restrict__ probs, int prob, const typename Acc<R>::T* __restrict__ xa,
                const typename Acc<R>::T* __restrict__ xb, int ldx, R sB,
                typename Acc<R>::T* __restrict__ y, int ldy, int K) {
  using CT = typename Acc<R>::T;
  constexpr bool PQ = HASB && std::is_same<ST, double2>::value;   // tiles hold A + B, A - B
  extern __shared__ unsigned char smem_raw[];
  CT* sA = (CT*)smem_raw;                 // [RB_Q][TS]
  CT* sB_ = sA + RB_Q * TS;               // [RB_Q][TS]
  CT* sXa = sB_ + RB_Q * TS;              // [RB_Q][16]
  CT* sXb = sXa + RB_Q * 16;              // [RB_Q][16]
  const Prob& p = probs[prob];
  const int I = blockIdx.x, c0 = blockIdx.y * 16;
  const int tid = threadIdx.x;
  const int c = tid >> 4, rr = tid & 15;
  const int nT = p.nT;
  CT acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a] = czero<CT>();
  for (int J = 0; J < nT; ++J) {
    const bool upper = J >= I;
    const int ti = upper ? I : J, tj = upper ? J : I;
    const int64_t tix = (int64_t)ti * nT - (int64_t)ti * (ti - 1) / 2 + (tj - ti);
    const ST* At = (const ST*)p.A + tix * (TS * TS);
    const ST* Bt = HASB ? (const ST*)p.B + tix * (TS * TS) : nullptr;
    for (int q0 = 0; q0 < TS; q0 += RB_Q) {
      __syncthreads();
      if (upper) {
        // Ablk[r][q] = tile[r][q]
        for (int e = tid; e < TS * RB_Q; e += 256) {
          const int qq = e & (RB_Q - 1), r = e >> 4;
          CT a = ccvt<CT>(At[r * TS + q0 + qq]), b;
          if (HASB) b = ccvt<CT>(Bt[r * TS + q0 + qq]);
          if constexpr (PQ) unpack_pq(a, b);
          sA[qq * TS + r] = a;
          if (HASB) sB_[qq * TS + r] = b;
        }
      } else {
        // Ablk[r][q] = conj(tile[q][r]); Bblk[r][q] = tile[q][r]
        for (int e = tid; e < TS * RB_Q; e += 256) {
          const int r = e & (TS - 1), qq = e >> 7;
          CT a = ccvt<CT>(At[(q0 + qq) * TS + r]), b;
          if (HASB) b = ccvt<CT>(Bt[(q0 + qq) * TS + r]);
          if constexpr (PQ) unpack_pq(a, b);
          sA[qq * TS + r] = conjc(a);
          if (HASB) sB_[qq * TS + r] = b;
        }
      }
      {
        const int qq = tid & (RB_Q - 1), cc = tid >> 4;
        const int64_t row = (int64_t)J * TS + q0 + qq;
        CT va = czero<CT>(), vb = czero<CT>();
        if (c0 + cc < K) {
          va = xa[(int64_t)(c0 + cc) * ldx + row];
          vb = xb ? xb[(int64_t)(c0 + cc) * ldx + row] : conjc(va);
        }
        sXa[qq * 16 + cc] = va;
        sXb[qq * 16 + cc] = cscale(vb, sB);
      }
      __syncthreads();
#pragma unroll 4
      for (int qq = 0; qq < RB_Q; ++qq) {
        const CT xv = sXa[qq * 16 + c];
        const CT xw = sXb[qq * 16 + c];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          cfma(acc[a], sA[qq * TS + rr + 16 * a], xv);
          if (HASB) cfma(acc[a], sB_[qq * TS + rr + 16 * a], xw);
        }
      }
    }
  }
  if (c0 + c < K) {
#pragma unroll
    for (int a = 0; a < 8; ++a) y[(int64_t)(c0 + c) * ldy + (int64_t)I * TS + rr + 16 * a] = acc[a];
  }
}

// ---------------------------------------------------------------- packing
// Pack the tiles (I, J >= I) of block row I from `rows` (TS rows of the full
// row-major matrix starting at row I*TS, leading dimension N).
template <typename TIn, typename TSt>
__global__ void __launch_bounds__(256)
k_pack_row(const TIn* __restrict__ rows, int64_t N, int nT, int I, int herm, TSt* __restrict__ dst) {
  const int J = I + blockIdx.x;
  const int64_t t = (int64_t)I * nT - (int64_t)I * (I - 1) / 2 + (J - I);
  TSt* out = dst + t * (TS * TS);
  for (int e = threadIdx.x; e < TS * TS; e += 256) {
    const int r = e >> 7, c = e & (TS - 1);
    const int64_t gi = (int64_t)I * TS + r, gj = (int64_t)J * TS + c;
    TSt v = czero<TSt>();
    if (gi < N && gj < N) {
      if (I != J || r < c) {
        v = ccvt<TSt>(rows[(int64_t)r * N + gj]);
      } else if (r == c) {
        v = ccvt<TSt>(rows[(int64_t)r * N + gj]);
        if (herm) v.y = 0;
      } else {  // lower half of a diagonal tile: mirror of (c, r)
        v = ccvt<TSt>(rows[(int64_t)c * N + (int64_t)I * TS + r]);
        if (herm) v.y = -v.y;
      }
    }
    out[e] = v;
  }
}

// element (r, c) of tile (I, J >= I) from a full row-major matrix: the upper
// triangle as stored, the lower half of a diagonal tile mirrored (conjugated for
// a Hermitian matrix, whose diagonal's imaginary part is dropped)
template <typename TIn, typename TSt>
__device__ __forceinline__ TSt pack_elem(const TIn* __restrict__ src, int64_t N, int I, int J, int r, int c,
                                         int herm) {
  const int64_t gi = (int64_t)I * TS + r, gj = (int64_t)J * TS + c;
  TSt v = czero<TSt>();
  if (gi < N && gj < N) {
    if (I != J || r < c) {
      v = ccvt<TSt>(src[gi * N + gj]);
    } else if (r == c) {
      v = ccvt<TSt>(src[gi * N + gj]);
      if (herm) v.y = 0;
    } else {
      v = ccvt<TSt>(src[((int64_t)I * TS + c) * N + (int64_t)I * TS + r]);
      if (herm) v.y = -v.y;
    }
  }
  return v;
}

// every tile (I, J >= I) of a device-resident matrix in one launch: grid (nT, nT)
template <typename TIn, typename TSt>
__global__ void __launch_bounds__(256)
k_pack_all(const TIn* __restrict__ src, int64_t N, int nT, int herm, TSt* __restrict__ dst) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (J < I) return;
  const int64_t t = (int64_t)I * nT - (int64_t)I * (I - 1) / 2 + (J - I);
  TSt* out = dst + t * (TS * TS);
  for (int e = threadIdx.x; e < TS * TS; e += 256) out[e] = pack_elem<TIn, TSt>(src, N, I, J, e >> 7, e & (TS - 1), herm);
}

// complex128 PH from device memory: the tiles of P = A + B and Q = A - B directly
__global__ void __launch_bounds__(256)
k_pack_pq(const double2* __restrict__ A, const double2* __restrict__ B, int64_t N, int nT, double2* __restrict__ P,
          double2* __restrict__ Q) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (J < I) return;
  const int64_t t = (int64_t)I * nT - (int64_t)I * (I - 1) / 2 + (J - I);
  for (int e = threadIdx.x; e < TS * TS; e += 256) {
    const double2 a = pack_elem<double2, double2>(A, N, I, J, e >> 7, e & (TS - 1), 1);
    const double2 b = pack_elem<double2, double2>(B, N, I, J, e >> 7, e & (TS - 1), 0);
    P[t * (TS * TS) + e] = make_double2(a.x + b.x, a.y + b.y);
    Q[t * (TS * TS) + e] = make_double2(a.x - b.x, a.y - b.y);
  }
}

template <typename TIn, typename TSt>
void launch_pack_all(const TIn* src, int64_t N, int nT, int herm, TSt* dst, cudaStream_t s) {
  count_launch();
  k_pack_all<TIn, TSt><<<dim3(nT, nT), 256, 0, s>>>(src, N, nT, herm, dst);
}

void launch_pack_pq(const double2* A, const double2* B, int64_t N, int nT, double2* P, double2* Q, cudaStream_t s) {
  count_launch();
  k_pack_pq<<<dim3(nT, nT), 256, 0, s>>>(A, B, N, nT, P, Q);
}

template void launch_pack_all<double2, double2>(const double2*, int64_t, int, int, double2*, cudaStream_t);
template void launch_pack_all<float2, float2>(const float2*, int64_t, int, int, float2*, cudaStream_t);

template <typename TIn, typename TSt>
void launch_pack_row(const TIn* rows, int64_t N, int nT, int I, int herm, TSt* dst, cudaStream_t s) {
  count_launch();
  k_pack_row<TIn, TSt><<<nT - I, 256, 0, s>>>(rows, N, nT, I, herm, dst);
}

template void launch_pack_row<double2, double2>(const double2*, int64_t, int, int, int, double2*, cudaStream_t);
template void launch_pack_row<float2, float2>(const float2*, int64_t, int, int, int, float2*, cudaStream_t);

// complex128 PH tiles: (A, B) -> (P, Q) = (A + B, A - B), element by element
__global__ void k_pq_combine(double2* __restrict__ a, double2* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = a[i], y = b[i];
    a[i] = make_double2(x.x + y.x, x.y + y.y);
    b[i] = make_double2(x.x - y.x, x.y - y.y);
  }
}

void launch_pq_combine(double2* a, double2* b, int64_t n, cudaStream_t s) {
  count_launch();
  k_pq_combine<<<1024, 256, 0, s>>>(a, b, n);
}

// ---------------------------------------------------------------- launchers
static int g_num_sms = 0;
static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

int product_grid(int occ, ProdShape shape, int njobs) {
  int64_t grid;
  if (shape.ctas_per_sm < 0) grid = njobs;                       // one CTA per tile
  else grid = (int64_t)(shape.ctas_per_sm == 0 || shape.ctas_per_sm > occ ? occ : shape.ctas_per_sm) * num_sms();
  if (grid > njobs) grid = njobs;
  if (grid < 1) grid = 1;
  return (int)grid;
}

template <typename ST, typename R>
int product_occupancy(bool hasB) {
  static int occ[2] = {0, 0};
  const int ib = hasB ? 1 : 0;
  if (!occ[ib]) {
    int o = 0;
    if (hasB)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_prod_tiles<ST, R, true>, PROD_THREADS, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_prod_tiles<ST, R, false>, PROD_THREADS, 0);
    occ[ib] = o > 0 ? o : 1;
  }
  return occ[ib];
}

template <typename ST, typename R>
void launch_product(const Prob* dprobs, const TileJob* jobs, int njobs, int nprob, int maxnT,
                    int mode, int K, const GenericIO* io_host, bool hasB, ProdShape shape, cudaStream_t s) {
  count_launch(2);
  GenericIO io{};
  if (io_host) io = *io_host;
  (void)K;
  // registers bound the FP64 variant to one CTA per SM and the FP32 one to two
  const int grid = product_grid(product_occupancy<ST, R>(hasB), shape, njobs);
  if (hasB)
    k_prod_tiles<ST, R, true><<<grid, PROD_THREADS, 0, s>>>(dprobs, jobs, njobs, mode, io, shape.strided);
  else
    k_prod_tiles<ST, R, false><<<grid, PROD_THREADS, 0, s>>>(dprobs, jobs, njobs, mode, io, shape.strided);
  k_prod_reduce<ST, R><<<dim3(maxnT, nprob), REDUCE_GROUPS * TS, 0, s>>>(dprobs, mode, io);
}

void launch_prod_reduce_d(const Prob* dprobs, int nprob, int maxnT, int mode, GenericIO io, cudaStream_t s) {
  k_prod_reduce_dfc<<<dim3(maxnT, nprob), REDUCE_GROUPS * TS, 0, s>>>(dprobs, mode, io);
}

template void launch_product<double2, double>(const Prob*, const TileJob*, int, int, int, int, int,
                                              const GenericIO*, bool, ProdShape, cudaStream_t);
template void launch_product<float2, float>(const Prob*, const TileJob*, int, int, int, int, int,
                                            const GenericIO*, bool, ProdShape, cudaStream_t);
template int product_occupancy<double2, double>(bool);
template int product_occupancy<float2, float>(bool);

template <typename ST, typename R>
void launch_rowblock(const Prob* dprobs, int prob, int nT, const void* xa, const void* xb, int ldx,
                     double sB, void* y, int ldy, int K, bool hasB, cudaStream_t s) {
  using CT = typename Acc<R>::T;
  count_launch();
  const size_t sm = (size_t)(2 * RB_Q * TS + 2 * RB_Q * 16) * sizeof(CT);
  dim3 grid(nT, (K + 15) / 16);
  if (hasB) {
    cudaFuncSetAttribute(k_prod_rowblock<ST, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_prod_rowblock<ST, R, true><<<grid, 256, sm, s>>>(dprobs, prob, (const CT*)xa, (const CT*)xb, ldx,
                                                       (R)sB, (CT*)y, ldy, K);
  } else {
    cudaFuncSetAttribute(k_prod_rowblock<ST, R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_prod_rowblock<ST, R, false><<<grid, 256, sm, s>>>(dprobs, prob, (const CT*)xa, (const CT*)xb, ldx,
                                                        (R)sB, (CT*)y, ldy, K);
  }
}

template void launch_rowblock<double2, double>(const Prob*, int, int, const void*, const void*, int,
                                               double, void*, int, int, bool, cudaStream_t);
template void launch_rowblock<float2, double>(const Prob*, int, int, const void*, const void*, int,
                                              double, void*, int, int, bool, cudaStream_t);
template void launch_rowblock<float2, float>(const Prob*, int, int, const void*, const void*, int,
                                             double, void*, int, int, bool, cudaStream_t);

}  // namespace bse
