// Persistent Krylov steps for one small problem.
//
// A Lanczos step of a problem of a few thousand rows is a chain of short phases -- the
// structured product (tiles, then the block-row reduction), two Gram-Schmidt passes (dots,
// then the update), the second product on the folded path, the norm and the new basis
// vector -- each far too small to fill the GPU, so with one kernel per phase the launch
// and drain gaps cost more than the work.  Here one cooperative launch runs all the steps of
// a restart cycle: every CTA loops over the units of a phase (the same bodies and unit
// decomposition as the per-phase kernels, bse_phases.cuh, so the result is the same bits),
// and the phases are separated by a grid barrier.  The state machine is the device-resident
// KState: the step loop stops when the subspace is full, a breakdown asks the host for a fresh
// vector, or the problem is done; the restart itself stays with the per-phase kernels.
//
// The grid barrier counts arrivals with an atomic and releases a generation number; every
// wait is bounded (about a second of polling), after which the CTA raises the barrier's error
// flag and the whole launch returns, so a wait can never hang the device.  The launch is
// cooperative, so all CTAs are resident together.
#include <algorithm>

#include "bse_phases.cuh"

namespace bse {
namespace {

constexpr int PS_THREADS = 256;
constexpr long long PS_SPIN = 1ll << 22;   // polls of one barrier wait

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// All CTAs of the launch meet here; false (in every thread of the CTA) when some wait expired.
__device__ __forceinline__ bool grid_sync(GridBar* gb, unsigned int nblk, unsigned int& gen, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = gen;
    __threadfence();                                   // this CTA's writes before the arrival
    if (atomicAdd(&gb->count, 1u) == nblk - 1) {
      atomicExch(&gb->count, 0u);                      // nobody arrives again before the release
      __threadfence();
      atomicAdd(&gb->gen, 1u);                         // release generation g
    } else {
      long long i = 0;
      while (ld_acquire_u32(&gb->gen) == g) {
        if (++i > PS_SPIN) {
          atomicExch(&gb->err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    gen = g + 1;
    if (ok && *(volatile int*)&gb->err) ok = 0;
    *s_ok = ok;
  }
  __syncthreads();
  __threadfence();                                     // every thread orders its later loads
  return *s_ok != 0;
}

template <typename ST, typename R, bool HASB>
__global__ void __launch_bounds__(PS_THREADS, 1)
k_steps_persist(const Prob* __restrict__ probs, const TileJob* __restrict__ jobs, int njobs, int steps,
                GridBar* gb) {
  using CT = typename Acc<R>::T;
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ int s_ok;
  const int bid = blockIdx.x;
  const unsigned int nblk = gridDim.x;
  unsigned int gen = 0;
  const Prob& p = probs[0];
  const KState* st = p.st;
  const int ph = HASB ? 1 : 0;
  const GenericIO io{};
  // one shared-memory region, carved per phase
  CT* xc = reinterpret_cast<CT*>(psm);
  CT* xr = xc + TS;
  CT(*pred)[TS] = reinterpret_cast<CT(*)[TS]>(xr + TS);
  CT(*grp)[TS] = reinterpret_cast<CT(*)[TS]>(psm);
  double2(*dred)[4] = reinterpret_cast<double2(*)[4]>(psm);
  ST* cf = reinterpret_cast<ST*>(psm);
  ST(*ured)[32] = reinterpret_cast<ST(*)[32]>(cf + 2 * MAXM + 2);
  double* nred = reinterpret_cast<double*>(psm);
  double* sb2 = nred + 8;
  const int nT = p.nT, nrb = p.nrb;
  const int nslab = (int)(p.Npad / 32);
  const int nrow = (int)((p.Npad + PS_THREADS - 1) / PS_THREADS);
  const int ncp = (p.ncol + 1) / 2;
  const int m1 = HASB ? PM_STEP_MMINUS : PM_STEP_A;
  for (int s = 0; s < steps; ++s) {
    if (!kactive(st)) break;                          // the same state in every CTA
    prod_tiles_body<ST, R, HASB, true>(probs, jobs, njobs, m1, io, 1, bid, nblk, xc, xr, pred);
    if (!grid_sync(gb, nblk, gen, &s_ok)) return;
    for (int I = bid; I < nT; I += nblk) prod_reduce_body<ST, R, true>(probs, m1, io, I, 0, grp);
    if (!grid_sync(gb, nblk, gen, &s_ok)) return;
    for (int pass = 0; pass < 2; ++pass) {
      for (int u = bid; u < ncp * nrb; u += nblk) {
        cgs_dot_body<ST, true>(probs, ph, 0, 0, pass, u % ncp, u / ncp, 0, dred);
        __syncthreads();
      }
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
      for (int u = bid; u < nslab; u += nblk) {
        cgs_update_body<ST, true>(probs, ph, pass, 0, 0, u, 0, cf, ured);
        __syncthreads();
      }
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
    }
    if (HASB) {
      prod_tiles_body<ST, R, HASB, true>(probs, jobs, njobs, PM_STEP_MPLUS, io, 1, bid, nblk, xc, xr, pred);
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
      for (int I = bid; I < nT; I += nblk) prod_reduce_body<ST, R, true>(probs, PM_STEP_MPLUS, io, I, 0, grp);
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
    }
    if (nrb == 1) {
      if (bid == 0) norm_fused_body<ST, true>(probs, ph, 0, 0, 0, nred, sb2);
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
    } else {
      for (int rb = bid; rb < nrb; rb += nblk) {
        norm_partial_body<ST, true>(probs, ph, 0, rb, 0, nred);
        __syncthreads();
      }
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
      for (int u = bid; u < nrow; u += nblk) normalize_body<ST, true>(probs, ph, 0, 0, u, 0, sb2);
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
      if (bid == 0 && threadIdx.x == 0 && kphase(st, 0)) finish_one(p, ph, 0, 0, sum_norm_parts<true>(p));
      if (!grid_sync(gb, nblk, gen, &s_ok)) return;
    }
  }
}

template <typename ST, typename R, bool HASB>
size_t persist_smem() {
  using CT = typename Acc<R>::T;
  const size_t prod = (size_t)10 * TS * sizeof(CT);
  const size_t red = (size_t)(REDUCE_GROUPS - 1) * TS * sizeof(CT);
  const size_t upd = (size_t)(2 * MAXM + 2) * sizeof(ST) + (size_t)8 * 32 * sizeof(ST);
  return std::max(std::max(prod, red), std::max(upd, (size_t)(9 * sizeof(double) + 8 * sizeof(double2))));
}

template <typename ST, typename R, bool HASB>
int persist_grid() {
  static int grid = -1;
  if (grid < 0) {
    const size_t sm = persist_smem<ST, R, HASB>();
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_steps_persist<ST, R, HASB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int occ = 0, dev = 0, nsm = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_steps_persist<ST, R, HASB>, PS_THREADS, sm);
    grid = (coop && occ >= 1) ? nsm : 0;    // one CTA per SM: every CTA resident
    cudaGetLastError();
  }
  return grid;
}

template <typename ST, typename R, bool HASB>
int launch_persist_t(const Prob* dprobs, const TileJob* jobs, int njobs, int steps, GridBar* gb, cudaStream_t s) {
  const int grid = persist_grid<ST, R, HASB>();
  if (grid <= 0) return 1;
  if (cudaMemsetAsync(gb, 0, sizeof(GridBar), s) != cudaSuccess) return -1;
  const size_t sm = persist_smem<ST, R, HASB>();
  void* args[] = {(void*)&dprobs, (void*)&jobs, (void*)&njobs, (void*)&steps, (void*)&gb};
  count_launch();
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_steps_persist<ST, R, HASB>, dim3(grid),
                                                    dim3(PS_THREADS), args, sm, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return 0;
}

}  // namespace

template <typename ST, typename R>
int launch_steps_persist(const Prob* dprobs, const TileJob* jobs, int njobs, bool ph, int steps, GridBar* gb,
                         cudaStream_t s) {
  return ph ? launch_persist_t<ST, R, true>(dprobs, jobs, njobs, steps, gb, s)
            : launch_persist_t<ST, R, false>(dprobs, jobs, njobs, steps, gb, s);
}

template int launch_steps_persist<double2, double>(const Prob*, const TileJob*, int, bool, int, GridBar*,
                                                   cudaStream_t);
template int launch_steps_persist<float2, float>(const Prob*, const TileJob*, int, bool, int, GridBar*,
                                                 cudaStream_t);

}  // namespace bse
