// Allocation-free structured product (bse_apply_noalloc, see include/bse.h).
//
// Some callers cannot let a library call cudaMalloc: a serving process whose
// device memory is entirely reserved up front by its own pool allocator, or a
// latency-bound loop where a cudaMalloc (which may synchronise the device and
// has unbounded cost) is not acceptable.  For them this file offers one
// product, y = A x + s B conj(x), that reads the caller's full row-major A and
// B directly and keeps its only scratch -- the per-tile partial sums of the
// streaming product -- in a file-scope __device__ array of fixed size.
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code cannot use its name as a device address: the address is
// looked up once per device with cudaGetSymbolAddress (first call on that
// device, with the device current) and passed to the kernels.  All calls share
// the array, so calls that overlap on the GPU (different streams, or threads)
// race on it.  Every partial-sum slot a call reads is written earlier in the
// same call, so nothing has to be cleared between calls.  The looked-up
// address is cached per device for the life of the process, so this entry
// point does not support cudaDeviceReset (the cached address would be stale).
#include <mutex>

#include "../../include/bse.h"
#include "bse_internal.cuh"

namespace bse {
namespace {

constexpr int NA_MAXT = BSE_NOALLOC_MAX_N / TS;                         // tiles per dimension
constexpr size_t NA_SCRATCH = (size_t)NA_MAXT * NA_MAXT * TS * sizeof(double2);  // 2 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH];

constexpr int NA_MAXDEV = 64;
std::mutex g_na_mutex;
void* g_na_ptr[NA_MAXDEV] = {};

int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAXDEV) return BSE_ECUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BSE_ECUDA;
    }
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return BSE_OK;
}

template <typename R> struct NAC;
template <> struct NAC<float> { using T = float2; };
template <> struct NAC<double> { using T = double2; };

template <typename T>
__device__ __forceinline__ T na_shfl(T v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

// element (gi, gj) of the Hermitian (herm = 1) or symmetric (herm = 0) matrix
// M, reading only its upper triangle; zero outside [0, N)^2
template <typename CT>
__device__ __forceinline__ CT na_elem(const CT* M, int64_t N, int64_t gi, int64_t gj, int herm) {
  if (gi >= N || gj >= N) return czero<CT>();
  if (gi < gj) return M[gi * N + gj];
  CT v = M[gj * N + gi];
  if (herm) v.y = (gi == gj) ? (decltype(v.y))0 : -v.y;
  return v;
}

// one CTA per upper tile (I <= J); same per-tile arithmetic as the solver's
// streaming product: y_I += A_IJ x_J + s B_IJ conj(x_J), y_J += A_IJ^H x_I + s B_IJ^T conj(x_I)
template <typename R, bool HASB>
__global__ void __launch_bounds__(256)
k_na_tiles(int64_t N, int nT, const typename NAC<R>::T* __restrict__ A, const typename NAC<R>::T* __restrict__ B,
           R sB, const typename NAC<R>::T* __restrict__ x, typename NAC<R>::T* __restrict__ part) {
  using CT = typename NAC<R>::T;
  __shared__ CT xc[2][TS], xr[2][TS], red[8][TS];
  int t = blockIdx.x, I = 0;
  while (t >= nT - I) { t -= nT - I; ++I; }
  const int J = I + t;
  const bool diag = I == J;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
  {
    const int r = tid & (TS - 1);
    const int64_t g = (int64_t)(tid < TS ? J : I) * TS + r;
    const CT a = g < N ? x[g] : czero<CT>();
    CT b = conjc(a);
    b.x *= sB; b.y *= sB;
    if (tid < TS) { xc[0][r] = a; xc[1][r] = b; } else { xr[0][r] = a; xr[1][r] = b; }
  }
  __syncthreads();
  CT racc[8], cacc[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) cacc[b] = czero<CT>();
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int r = ty + 16 * a;
    const int64_t gi = (int64_t)I * TS + r;
    CT ra = czero<CT>();
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int c = tx + 16 * b;
      const int64_t gj = (int64_t)J * TS + c;
      const CT av = na_elem(A, N, gi, gj, 1);
      cfma(ra, av, xc[0][c]);
      if (!diag) cfmac(cacc[b], av, xr[0][r]);
      if (HASB) {
        const CT bv = na_elem(B, N, gi, gj, 0);
        cfma(ra, bv, xc[1][c]);
        if (!diag) cfma(cacc[b], bv, xr[1][r]);
      }
    }
    racc[a] = ra;
  }
  // row sums over the 16 tx lanes (reduce-scatter), written by even lanes
  {
    const bool u8 = tx & 8;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      CT s = u8 ? racc[q] : racc[q + 4], k = u8 ? racc[q + 4] : racc[q];
      racc[q] = cadd(k, na_shfl(s, 8));
    }
    const bool u4 = tx & 4;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      CT s = u4 ? racc[q] : racc[q + 2], k = u4 ? racc[q + 2] : racc[q];
      racc[q] = cadd(k, na_shfl(s, 4));
    }
    const bool u2 = tx & 2;
    CT s = u2 ? racc[0] : racc[1], k = u2 ? racc[1] : racc[0];
    racc[0] = cadd(k, na_shfl(s, 2));
    racc[0] = cadd(racc[0], na_shfl(racc[0], 1));
    if ((tx & 1) == 0) part[((int64_t)I * nT + J) * TS + ty + 16 * ((tx >> 1) & 7)] = racc[0];
  }
  if (!diag) {
    const bool up = lane & 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      CT s = up ? cacc[q] : cacc[q + 4], k = up ? cacc[q + 4] : cacc[q];
      cacc[q] = cadd(k, na_shfl(s, 16));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[warp][tx + 16 * (q + (up ? 4 : 0))] = cacc[q];
    __syncthreads();
    if (tid < TS) {
      CT s = red[0][tid];
#pragma unroll
      for (int w = 1; w < 8; ++w) s = cadd(s, red[w][tid]);
      part[((int64_t)J * nT + I) * TS + tid] = s;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(128)
k_na_reduce(int64_t N, int nT, const typename NAC<R>::T* __restrict__ part, typename NAC<R>::T* __restrict__ y) {
  using CT = typename NAC<R>::T;
  const int I = blockIdx.x, r = threadIdx.x;
  const int64_t g = (int64_t)I * TS + r;
  if (g >= N) return;
  CT acc = czero<CT>();
  for (int J = 0; J < nT; ++J) acc = cadd(acc, part[((int64_t)I * nT + J) * TS + r]);
  y[g] = acc;
}

template <typename R>
int na_run(int64_t N, const void* A, const void* B, int op, const void* x, void* y, cudaStream_t s,
           void* scratch) {
  using CT = typename NAC<R>::T;
  const int nT = (int)((N + TS - 1) / TS);
  const int ntiles = nT * (nT + 1) / 2;
  const R sB = op == BSE_OP_MPLUS ? (R)1 : (op == BSE_OP_MMINUS ? (R)-1 : (R)0);
  CT* part = (CT*)scratch;
  // an error pending from the caller's own earlier work is left for the caller to read
  if (cudaPeekAtLastError() != cudaSuccess) return BSE_ECUDA;
  if (op == BSE_OP_A)
    k_na_tiles<R, false><<<ntiles, 256, 0, s>>>(N, nT, (const CT*)A, nullptr, sB, (const CT*)x, part);
  else
    k_na_tiles<R, true><<<ntiles, 256, 0, s>>>(N, nT, (const CT*)A, (const CT*)B, sB, (const CT*)x, part);
  k_na_reduce<R><<<nT, TS, 0, s>>>(N, nT, part, (CT*)y);
  return cudaGetLastError() == cudaSuccess ? BSE_OK : BSE_ECUDA;   // no error was pending: it is ours
}

}  // namespace
}  // namespace bse

extern "C" int bse_apply_noalloc(int64_t N, const void* A, const void* B, int dtype, int op, const void* x,
                                 void* y, void* stream) {
  if (N < 1 || N > BSE_NOALLOC_MAX_N || !A || !x || !y) return BSE_EINVAL;
  if (op != BSE_OP_A && op != BSE_OP_MPLUS && op != BSE_OP_MMINUS) return BSE_EINVAL;
  if (op != BSE_OP_A && !B) return BSE_EINVAL;
  if (dtype != BSE_C64 && dtype != BSE_C128) return BSE_EINVAL;
  void* scratch = nullptr;
  const int rc = bse::scratch_address(&scratch);
  if (rc != BSE_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BSE_C128) return bse::na_run<double>(N, A, B, op, x, y, s, scratch);
  return bse::na_run<float>(N, A, B, op, x, y, s, scratch);
}
