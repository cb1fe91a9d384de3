// Hellmann-Feynman adjoint on the 5th-generation tensor cores (complex64 outputs).
//
// With L = [X g, conj(Y) g], R_A = [X, conj(Y)], R_B = [Y, conj(X)] (N x 2k),
//     dA = L R_A^H,  dB = L R_B^H      (TDA: L = X g, R_A = X)
// and, in real arithmetic,  Re(L R^H) = L_re R_re^T + L_im R_im^T,
//                           Im(L R^H) = L_im R_re^T - L_re R_im^T.
//
// k_adj_panels writes the operands once, split into TF32 hi + lo parts (3xTF32:
// hi*hi + hi*lo + lo*hi, about FP32 accuracy), already in the shared-memory
// image the tensor cores read: the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices), in 8 KiB blocks of 128 rows x 16 K.
//
// k_adjoint_tc: one persistent CTA per SM, warp-specialised.  The work unit is
// a half-tile (128 output rows x 64 columns of a 128 x 128 tile I <= J), whose
// FP32 accumulators (dA re/im, dB re/im) take 256 TMEM columns, so two sets
// fit in the SM's 512: while warps 0-3 drain one set (tcgen05.ld) and write
// the half-tile and its mirror (dA Hermitian, dB symmetric), warp 4 already
// runs the next half-tile's tcgen05.mma (M = 128, N = 64, K = 8) into the
// other.  Warp 4 also feeds a three-stage shared-memory pipeline with bulk
// asynchronous copies (cp.async.bulk, completion on mbarriers); tcgen05.commit
// releases a stage when its MMAs finish and publishes a finished accumulator
// set.  Every wait is bounded; on expiry the CTA records an error, stops, waits
// (bounded) for what it has in flight and releases its TMEM, and the host
// returns a timeout.
#include <cstdint>

#include "bse_internal.cuh"

namespace bse {
namespace {

constexpr int TCM = 128;                  // tile rows (M) and columns (N)
constexpr int KC = 16;                    // K elements per pipeline chunk
constexpr int TC_THREADS = 160;           // warps 0-3 epilogue, warp 4 copies + MMAs
constexpr int NSTAGE = 3;                 // shared-memory pipeline stages
constexpr int BLK = TCM * KC * 4;         // bytes of one operand block (8 KiB)
constexpr int EPI_BYTES = 4 * 32 * 33 * 8;   // per-warp transpose buffers of the epilogue
constexpr long long TC_SPIN = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major, no swizzle: core matrix (row/8, k/4) at ((row/8)*4 + k/4)*128 bytes;
// K-direction neighbours 128 B apart (LBO), 8-row groups 512 B apart (SBO)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for this architecture
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// offset (in floats) of element (row r, K index q) in a panel plane of nk chunks
__host__ __device__ __forceinline__ int64_t plane_off(int64_t r, int q, int nk) {
  const int64_t blk = (r >> 7) * nk + (q >> 4);
  const int ri = (int)(r & 127), ki = q & 15;
  return blk * (TCM * KC) + (((ri >> 3) * 4 + (ki >> 2)) * 32 + (ri & 7) * 4 + (ki & 3));
}

__host__ __device__ constexpr uint32_t instr_desc(bool neg_a) {
  return (1u << 4)                          // D: F32
         | (2u << 7)                        // A: TF32
         | (2u << 10)                       // B: TF32
         | ((neg_a ? 1u : 0u) << 13)        // negate A
         | ((uint32_t)(64 >> 3) << 17)      // N / 8 (half-tile: 64 output columns)
         | ((uint32_t)(TCM >> 4) << 24);    // M / 16   (A and B K-major)
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < TC_SPIN; ++i)
    if (mbar_test(mbar, parity)) return true;
  return false;
}

__device__ __forceinline__ float tf32_hi(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Operand planes (rows padded to a multiple of 128, K to a multiple of 16, zeros beyond),
// each in 8 KiB blocks [row block][K chunk] of the layout plane_off describes:
//   2j = hi part, 2j + 1 = lo part of  j = 0 L_re, 1 L_im, 2 RA_re, 3 RA_im, 4 RB_re, 5 RB_im
__global__ void k_adj_panels(const double2* __restrict__ Z, int64_t ldz, int64_t Npad, int64_t N, int k,
                             const double* __restrict__ g, int ph, int nk, int64_t rows, float* __restrict__ P) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int kk = ph ? 2 * k : k;
  const int kp = nk * KC;
  const int64_t plane = rows * kp;
  const int nj = ph ? 6 : 4;
  for (int q = 0; q < kp; ++q) {
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r < N && q < kk) {
      const int c = q < k ? q : q - k;
      const double2 x = Z[(int64_t)c * ldz + r];
      const double2 y = ph ? Z[(int64_t)c * ldz + Npad + r] : make_double2(0.0, 0.0);
      const double gc = g[c];
      if (q < k) {               // L = X g, R_A = X, R_B = Y
        v[0] = (float)(gc * x.x); v[1] = (float)(gc * x.y);
        v[2] = (float)x.x; v[3] = (float)x.y;
        v[4] = (float)y.x; v[5] = (float)y.y;
      } else {                   // L = conj(Y) g, R_A = conj(Y), R_B = conj(X)
        v[0] = (float)(gc * y.x); v[1] = (float)(-gc * y.y);
        v[2] = (float)y.x; v[3] = (float)(-y.y);
        v[4] = (float)x.x; v[5] = (float)(-x.y);
      }
    }
    const int64_t o = plane_off(r, q, nk);
    for (int j = 0; j < nj; ++j) {
      const float hi = tf32_hi(v[j]);
      P[(int64_t)(2 * j) * plane + o] = hi;
      P[(int64_t)(2 * j + 1) * plane + o] = v[j] - hi;
    }
  }
}

// Half-tile unit h = 2 * (tile iteration) + q: output rows of block I, columns
// J * 128 + 64 q ... + 63 (M = 128, N = 64), so that two accumulator sets fit
// in the 512 TMEM columns and the epilogue of one half-tile overlaps the MMAs
// of the next.  Warps 0-3 drain TMEM and write; warp 4 (one lane) issues the
// bulk copies and the MMAs.  Barriers: full[s] / empty[s] for the three
// shared-memory stages (copies landed / MMAs done reading), tfull[b] /
// tempty[b] for the two accumulator buffers (MMAs done / epilogue done).
template <bool PH>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_adjoint_tc(const float* __restrict__ P, int64_t rows, int nk, int64_t N, const int2* __restrict__ tiles,
             int ntiles, float2* __restrict__ dA, float2* __restrict__ dB, int* __restrict__ err) {
  constexpr int NR = PH ? 8 : 4;                     // R planes (R_A, and R_B for PH)
  constexpr uint32_t LBYTES = 4 * BLK;               // L: 4 planes x 128 rows
  constexpr uint32_t RBLK = BLK / 2;                 // one R plane, 64 rows
  constexpr uint32_t STAGE = LBYTES + NR * RBLK;
  constexpr uint32_t ACC = PH ? 256 : 128;           // TMEM columns of one accumulator set
  constexpr uint32_t TMEM_COLS = 2 * ACC;
  extern __shared__ __align__(1024) unsigned char sm[];   // NSTAGE stages, then the epilogue buffers
  __shared__ uint64_t full[NSTAGE], empty[NSTAGE], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t plane = rows * (int64_t)nk * KC;   // floats per plane
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty[b])), "r"(128) : "memory");
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_slot;
  const uint32_t s0 = smem_u32(sm);
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nhalf = 2 * my_tiles;
  volatile int* vabort = &abort_flag;

  if (warp == 4) {
    // ------------------------------------------------ copies and MMAs (one lane)
    if (lane == 0) {
      const uint32_t idp = instr_desc(false), idn = instr_desc(true);
      const long long nb = (long long)nhalf * nk;     // batches: (half-tile, K-chunk)
      auto issue_tma = [&](long long g) {
        const int h = (int)(g / nk), c = (int)(g % nk);
        const int2 tl = tiles[blockIdx.x + (int64_t)(h >> 1) * gridDim.x];
        const int q = h & 1;
        const int s = (int)(g % NSTAGE);
        const uint32_t bar = smem_u32(&full[s]);
        const uint32_t st = s0 + (uint32_t)s * STAGE;
        mbar_expect_tx(bar, STAGE);
#pragma unroll 1
        for (int p = 0; p < 4; ++p)           // L: block row I, all 128 rows
          bulk_g2s(st + (uint32_t)p * BLK, P + (int64_t)p * plane + ((int64_t)tl.x * nk + c) * (TCM * KC), BLK,
                   bar);
#pragma unroll 1
        for (int p = 0; p < NR; ++p)          // R: block row J, rows 64 q ... 64 q + 63
          bulk_g2s(st + LBYTES + (uint32_t)p * RBLK,
                   reinterpret_cast<const char*>(P + (int64_t)(4 + p) * plane + ((int64_t)tl.y * nk + c) * (TCM * KC)) +
                       q * RBLK,
                   RBLK, bar);
      };
      long long issued = 0, committed = 0;
      for (; issued < nb && issued < NSTAGE; ++issued) issue_tma(issued);
      bool ok = true;
      for (long long g = 0; g < nb && ok; ++g) {
        const int h = (int)(g / nk), c = (int)(g % nk);
        const int s = (int)(g % NSTAGE), b = h & 1;
        if (*vabort) { ok = false; break; }
        if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((g / NSTAGE) & 1))) { ok = false; break; }
        if (c == 0 && !mbar_wait(smem_u32(&tempty[b]), (uint32_t)(((h >> 1) & 1) ^ 1))) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = s0 + (uint32_t)s * STAGE;
#pragma unroll 1
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t koff = (uint32_t)ks * 256u;
          auto dl = [&](int p) { return smem_desc(st + (uint32_t)p * BLK + koff); };
          auto dr = [&](int p) { return smem_desc(st + LBYTES + (uint32_t)p * RBLK + koff); };
          const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
#pragma unroll 1
          for (int m = 0; m < (PH ? 2 : 1); ++m) {
            const int rr = 4 * m, ri = 4 * m + 2;            // R_re / R_im hi planes of this matrix
            const uint32_t d_re = tbase + (uint32_t)b * ACC + (uint32_t)(128 * m), d_im = d_re + 64u;
            // Re += L_re R_re^T + L_im R_im^T   (3xTF32 each)
            mma_tf32(d_re, dl(0), dr(rr), idp, first);
            mma_tf32(d_re, dl(0), dr(rr + 1), idp, 1u);
            mma_tf32(d_re, dl(1), dr(rr), idp, 1u);
            mma_tf32(d_re, dl(2), dr(ri), idp, 1u);
            mma_tf32(d_re, dl(2), dr(ri + 1), idp, 1u);
            mma_tf32(d_re, dl(3), dr(ri), idp, 1u);
            // Im += L_im R_re^T - L_re R_im^T
            mma_tf32(d_im, dl(2), dr(rr), idp, first);
            mma_tf32(d_im, dl(2), dr(rr + 1), idp, 1u);
            mma_tf32(d_im, dl(3), dr(rr), idp, 1u);
            mma_tf32(d_im, dl(0), dr(ri), idn, 1u);
            mma_tf32(d_im, dl(0), dr(ri + 1), idn, 1u);
            mma_tf32(d_im, dl(1), dr(ri), idn, 1u);
          }
        }
        mma_commit(smem_u32(&empty[s]));              // stage s may be refilled once these finish
        if (c == nk - 1) mma_commit(smem_u32(&tfull[b]));   // the half-tile's accumulators are final
        committed = g + 1;
        // refill the stage of batch g - 1 (its MMAs finish while batch g's run)
        if (g >= 1 && issued < nb) {
          const long long gp = g - 1;
          if (!mbar_wait(smem_u32(&empty[gp % NSTAGE]), (uint32_t)((gp / NSTAGE) & 1))) { ok = false; break; }
          issue_tma(issued);
          ++issued;
        }
      }
      if (!ok) {
        *vabort = 1;
        atomicExch(err, 1);
      }
      // nothing may be in flight when the shared memory and TMEM go away
      if (issued > 0) {
        const long long gi = issued - 1;
        mbar_wait(smem_u32(&full[gi % NSTAGE]), (uint32_t)((gi / NSTAGE) & 1));
      }
      if (committed > 0) {
        const long long gc = committed - 1;
        mbar_wait(smem_u32(&empty[gc % NSTAGE]), (uint32_t)((gc / NSTAGE) & 1));
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 0-3)
    float2* buf = reinterpret_cast<float2*>(sm + NSTAGE * STAGE) + warp * (32 * 33);
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    for (int h = 0; h < nhalf; ++h) {
      const int b = h & 1;
      if (*vabort) break;
      // warp-uniform outcome: tcgen05.ld below needs the whole warp
      const bool ready = __all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[b]), (uint32_t)((h >> 1) & 1)) ? 1 : 0);
      if (!ready) {
        *vabort = 1;
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int2 tl = tiles[blockIdx.x + (int64_t)(h >> 1) * gridDim.x];
      const int I = tl.x, J = tl.y, q = h & 1;
      const int64_t gi = (int64_t)I * TCM + warp * 32 + lane;
      // the mirror block is written from registers (lanes run along its rows); the tile goes
      // through a per-warp transpose so that lanes run along its rows too.  A diagonal tile keeps
      // its upper triangle and mirrors it (dA exactly Hermitian with a real diagonal, dB symmetric)
#pragma unroll 1
      for (int m = 0; m < (PH ? 2 : 1); ++m) {
        float2* out = m == 0 ? dA : dB;
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 32) {
          float re[32], im[32];
          tmem_ld32(tbase + lane_off + (uint32_t)b * ACC + (uint32_t)(128 * m + c0), re);
          tmem_ld32(tbase + lane_off + (uint32_t)b * ACC + (uint32_t)(128 * m + 64 + c0), im);
          const int64_t jb = (int64_t)J * TCM + 64 * q + c0;
          if (gi < N) {
#pragma unroll
            for (int qq = 0; qq < 32; ++qq) {
              const int64_t gj = jb + qq;
              if (gj < N && (I != J || gj > gi)) out[gj * N + gi] = make_float2(re[qq], m == 0 ? -im[qq] : im[qq]);
            }
          }
#pragma unroll
          for (int qq = 0; qq < 32; ++qq) buf[lane * 33 + qq] = make_float2(re[qq], im[qq]);
          __syncwarp();
          const int64_t gj = jb + lane;
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t row = (int64_t)I * TCM + warp * 32 + rr;
            if (row < N && gj < N && (I != J || gj >= row)) {
              float2 v = buf[rr * 33 + lane];
              if (m == 0 && gj == row) v.y = 0.f;
              out[row * N + gj] = v;
            }
          }
          __syncwarp();
        }
      }
      // this accumulator set may be overwritten by the half-tile after next
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS));
}

// Self-test of the bounded mbarrier wait every pipeline above relies on: with
// arrive = 0 nothing ever completes the barrier, the wait gives up after
// `spins` polls and the kernel reports it; with arrive = 1 the single expected
// arrival comes first and the wait succeeds.  No fault, no unbounded loop.
__global__ void k_wait_selftest(int arrive, long long spins, int* __restrict__ expired) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
  bool ok = false;
  for (long long i = 0; i < spins && !ok; ++i) ok = mbar_test(b, 0u);
  *expired = ok ? 0 : 1;
}

int g_tc_sms = 0;

}  // namespace

int selftest_bounded_wait(int arrive, int* expired_host) {
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return -1;
  count_launch();
  k_wait_selftest<<<1, 32>>>(arrive, 1ll << 20, d);
  int h = -1;
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d);
  if (!ok) return -1;
  *expired_host = h;
  return 0;
}

size_t adjoint_tc_panel_bytes(int64_t N, int k, int ph) {
  const int64_t rows = ((N + TCM - 1) / TCM) * TCM;
  const int kk = ph ? 2 * k : k;
  const int nk = (kk + KC - 1) / KC;
  return (size_t)(ph ? 12 : 8) * rows * nk * KC * sizeof(float);
}

// returns 0 on success, 1 if a bounded wait expired on the device, -1 on a launch error
int launch_adjoint_tc(const double2* Z, int64_t ldz, int64_t Npad, int64_t N, int k, const double* g, int ph,
                      const int2* tiles128, int64_t ntiles, float* panels, int* derr, float2* dA, float2* dB,
                      cudaStream_t s) {
  const int64_t rows = ((N + TCM - 1) / TCM) * TCM;
  const int kk = ph ? 2 * k : k;
  const int nk = (kk + KC - 1) / KC;
  count_launch(2);
  k_adj_panels<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(Z, ldz, Npad, N, k, g, ph, nk, rows, panels);
  if (!g_tc_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_tc_sms <= 0) g_tc_sms = 1;
  }
  // stage: L (4 planes x 8 KiB) + R (8 or 4 planes x 4 KiB)
  const size_t smem = (size_t)NSTAGE * (4 * BLK + (ph ? 8 : 4) * (BLK / 2)) + EPI_BYTES;
  cudaMemsetAsync(derr, 0, sizeof(int), s);
  const int grid = (int)(ntiles < g_tc_sms ? ntiles : g_tc_sms);
  if (ph) {
    cudaFuncSetAttribute(k_adjoint_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_adjoint_tc<true><<<grid, TC_THREADS, smem, s>>>(panels, rows, nk, N, tiles128, (int)ntiles, dA, dB, derr);
  } else {
    cudaFuncSetAttribute(k_adjoint_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_adjoint_tc<false><<<grid, TC_THREADS, smem, s>>>(panels, rows, nk, N, tiles128, (int)ntiles, dA, dB, derr);
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return herr;
}

}  // namespace bse
