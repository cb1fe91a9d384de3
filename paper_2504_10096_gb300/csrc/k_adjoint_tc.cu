// Hellmann-Feynman adjoint on the 5th-generation tensor cores (complex64 outputs).
//
// With L = [X g, conj(Y) g], R_A = [X, conj(Y)], R_B = [Y, conj(X)] (N x 2k),
//     dA = L R_A^H,  dB = L R_B^H      (TDA: L = X g, R_A = X)
// and, in real arithmetic,  Re(L R^H) = L_re R_re^T + L_im R_im^T,
//                           Im(L R^H) = L_im R_re^T - L_re R_im^T.
// One CTA (4 warps) owns a 128 x 128 output tile (I <= J) and keeps its four
// FP32 accumulators (dA re/im, dB re/im) in the 512 TMEM columns of its SM.
// Operands are staged in shared memory in the canonical K-major layout
// without swizzle (8-row x 16-byte core matrices), split into TF32 hi + lo
// parts (3xTF32: hi*hi + hi*lo + lo*hi, about FP32 accuracy), and one thread
// issues tcgen05.mma (M = 128, N = 128, K = 8) and commits to an mbarrier.
// The epilogue reads TMEM with tcgen05.ld and writes the tile and, for I < J,
// its mirror (dA Hermitian, dB symmetric).  Every wait is bounded; on expiry
// the CTA records an error, waits again (bounded) and releases its TMEM.
#include <cstdint>

#include "bse_internal.cuh"

namespace bse {
namespace {

constexpr int TCM = 128;         // tile rows (M) and columns (N)
constexpr int TCKC = 32;         // K elements (tf32) staged per round
constexpr int TC_THREADS = 128;
constexpr int OPND = TCM * TCKC * 4;   // bytes of one staged operand (16 KiB)
constexpr int NOPND = 12;              // L re/im hi/lo (4) + R_A (4) + R_B (4)
constexpr long long TC_SPIN = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major, no swizzle: core matrix (row/8, k/4) at ((row/8)*8 + k/4)*128 bytes;
// K-direction neighbours 128 B apart (LBO), 8-row groups 1024 B apart (SBO)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for this architecture
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

__host__ __device__ constexpr uint32_t instr_desc(bool neg_a) {
  return (1u << 4)                          // D: F32
         | (2u << 7)                        // A: TF32
         | (2u << 10)                       // B: TF32
         | ((neg_a ? 1u : 0u) << 13)        // negate A
         | ((uint32_t)(TCM >> 3) << 17)     // N / 8
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

// Panels (row-major, ld = kp, rows padded to a multiple of 128, zeros beyond):
//   P[0] = L_re, P[1] = L_im, P[2] = RA_re, P[3] = RA_im, P[4] = RB_re, P[5] = RB_im
__global__ void k_adj_panels(const double2* __restrict__ Z, int64_t ldz, int64_t Npad, int64_t N, int k,
                             const double* __restrict__ g, int ph, int kp, int64_t rows, float* __restrict__ P) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int kk = ph ? 2 * k : k;
  const int64_t plane = rows * kp;
  for (int q = 0; q < kp; ++q) {
    float lre = 0.f, lim = 0.f, are = 0.f, aim = 0.f, bre = 0.f, bim = 0.f;
    if (r < N && q < kk) {
      const int c = q < k ? q : q - k;
      const double2 x = Z[(int64_t)c * ldz + r];
      const double2 y = ph ? Z[(int64_t)c * ldz + Npad + r] : make_double2(0.0, 0.0);
      const double gc = g[c];
      if (q < k) {               // L = X g, R_A = X, R_B = Y
        lre = (float)(gc * x.x); lim = (float)(gc * x.y);
        are = (float)x.x; aim = (float)x.y;
        bre = (float)y.x; bim = (float)y.y;
      } else {                   // L = conj(Y) g, R_A = conj(Y), R_B = conj(X)
        lre = (float)(gc * y.x); lim = (float)(-gc * y.y);
        are = (float)y.x; aim = (float)(-y.y);
        bre = (float)x.x; bim = (float)(-x.y);
      }
    }
    const int64_t o = r * kp + q;
    P[o] = lre; P[plane + o] = lim; P[2 * plane + o] = are; P[3 * plane + o] = aim;
    P[4 * plane + o] = bre; P[5 * plane + o] = bim;
  }
}

template <bool PH>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_adjoint_tc(const float* __restrict__ P, int64_t rows, int kp, int64_t N, const int2* __restrict__ tiles,
             int ntiles, float2* __restrict__ dA, float2* __restrict__ dB, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nop = PH ? NOPND : 8;
  const int64_t plane = rows * kp;
  const uint32_t mb = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_slot;
  uint32_t phase = 0;
  bool ok = true;
  const uint32_t id_pos = instr_desc(false), id_neg = instr_desc(true);
  for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int I = tiles[t].x, J = tiles[t].y;
    for (int kc = 0; kc < kp && ok; kc += TCKC) {
      __syncthreads();   // the previous round's MMAs have completed (waited below)
      // stage: thread tid owns row tid of each operand (A operands: rows of block I, B: block J)
#pragma unroll 1
      for (int o = 0; o < nop / 2; ++o) {       // operand o reads panel o
        const int64_t row = (int64_t)(o < 2 ? I : J) * TCM + tid;
        const float* pr = P + (int64_t)o * plane + row * kp + kc;
        unsigned char* hi = sm + (size_t)(2 * o) * OPND;
        unsigned char* lo = sm + (size_t)(2 * o + 1) * OPND;
#pragma unroll
        for (int k4 = 0; k4 < TCKC / 4; ++k4) {
          const float4 v = *reinterpret_cast<const float4*>(pr + 4 * k4);
          float4 h, l;
          h.x = tf32_hi(v.x); h.y = tf32_hi(v.y); h.z = tf32_hi(v.z); h.w = tf32_hi(v.w);
          l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
          const int off = ((tid >> 3) * 8 + k4) * 128 + (tid & 7) * 16;
          *reinterpret_cast<float4*>(hi + off) = h;
          *reinterpret_cast<float4*>(lo + off) = l;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const uint32_t s0 = smem_u32(sm);
        // operand o: hi at 2o, lo at 2o+1; o = 0 L_re, 1 L_im, 2 RA_re, 3 RA_im, 4 RB_re, 5 RB_im
#pragma unroll 1
        for (int ks = 0; ks < TCKC / 8; ++ks) {
          const uint32_t koff = (uint32_t)ks * 256u;
          auto d = [&](int o, int part) { return smem_desc(s0 + (uint32_t)(2 * o + part) * OPND + koff); };
          const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
#pragma unroll 1
          for (int m = 0; m < (PH ? 2 : 1); ++m) {
            const int rr = 2 + 2 * m, ri = 3 + 2 * m;       // R_re, R_im operand of this matrix
            const uint32_t d_re = tbase + (uint32_t)(256 * m), d_im = d_re + 128u;
            // Re += L_re R_re^T + L_im R_im^T   (3xTF32 each)
            mma_tf32(d_re, d(0, 0), d(rr, 0), id_pos, first);
            mma_tf32(d_re, d(0, 0), d(rr, 1), id_pos, 1u);
            mma_tf32(d_re, d(0, 1), d(rr, 0), id_pos, 1u);
            mma_tf32(d_re, d(1, 0), d(ri, 0), id_pos, 1u);
            mma_tf32(d_re, d(1, 0), d(ri, 1), id_pos, 1u);
            mma_tf32(d_re, d(1, 1), d(ri, 0), id_pos, 1u);
            // Im += L_im R_re^T - L_re R_im^T
            mma_tf32(d_im, d(1, 0), d(rr, 0), id_pos, first);
            mma_tf32(d_im, d(1, 0), d(rr, 1), id_pos, 1u);
            mma_tf32(d_im, d(1, 1), d(rr, 0), id_pos, 1u);
            mma_tf32(d_im, d(0, 0), d(ri, 0), id_neg, 1u);
            mma_tf32(d_im, d(0, 0), d(ri, 1), id_neg, 1u);
            mma_tf32(d_im, d(0, 1), d(ri, 0), id_neg, 1u);
          }
        }
        mma_commit(mb);
      }
      const int mine = mbar_wait(mb, phase) ? 1 : 0;
      phase ^= 1u;
      ok = __syncthreads_and(mine) != 0;   // block-uniform outcome of the bounded wait
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok) break;
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (tile rows), 32 columns at a
    // time.  The mirror block is written straight from registers (lanes run
    // along its rows); the tile itself goes through a per-warp transpose in the
    // operand shared memory, idle until the next tile's staging, so that lanes
    // run along its rows too.
    const int64_t gi = (int64_t)I * TCM + warp * 32 + lane;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    float2* buf = reinterpret_cast<float2*>(sm) + warp * (32 * 33);
#pragma unroll 1
    for (int m = 0; m < (PH ? 2 : 1); ++m) {
      float2* out = m == 0 ? dA : dB;
#pragma unroll 1
      for (int c0 = 0; c0 < TCM; c0 += 32) {
        float re[32], im[32];
        tmem_ld32(tbase + lane_off + (uint32_t)(256 * m + c0), re);
        tmem_ld32(tbase + lane_off + (uint32_t)(256 * m + 128 + c0), im);
        // a diagonal tile keeps its upper triangle and mirrors it, so dA is
        // exactly Hermitian (real diagonal: g |x|^2 + g |y|^2) and dB exactly symmetric
        if (gi < N) {   // mirror: dA Hermitian (conjugate), dB symmetric
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int64_t gj = (int64_t)J * TCM + c0 + q;
            if (gj < N && (I != J || gj > gi)) out[gj * N + gi] = make_float2(re[q], m == 0 ? -im[q] : im[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) buf[lane * 33 + q] = make_float2(re[q], im[q]);
        __syncwarp();
        const int64_t gj = (int64_t)J * TCM + c0 + lane;
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  if (!ok) mbar_wait(mb, phase ^ 1u);   // let an outstanding commit land before releasing TMEM
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

int g_tc_sms = 0;

}  // namespace

size_t adjoint_tc_panel_bytes(int64_t N, int k, int ph) {
  const int64_t rows = ((N + TCM - 1) / TCM) * TCM;
  const int kk = ph ? 2 * k : k;
  const int kp = ((kk + TCKC - 1) / TCKC) * TCKC;
  return (size_t)6 * rows * kp * sizeof(float);
}

// returns 0 on success, 1 if a bounded wait expired on the device, -1 on a launch error
int launch_adjoint_tc(const double2* Z, int64_t ldz, int64_t Npad, int64_t N, int k, const double* g, int ph,
                      const int2* tiles128, int64_t ntiles, float* panels, int* derr, float2* dA, float2* dB,
                      cudaStream_t s) {
  const int64_t rows = ((N + TCM - 1) / TCM) * TCM;
  const int kk = ph ? 2 * k : k;
  const int kp = ((kk + TCKC - 1) / TCKC) * TCKC;
  count_launch(2);
  k_adj_panels<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(Z, ldz, Npad, N, k, g, ph, kp, rows, panels);
  if (!g_tc_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_tc_sms <= 0) g_tc_sms = 1;
  }
  const size_t smem = (size_t)(ph ? NOPND : 8) * OPND;
  cudaMemsetAsync(derr, 0, sizeof(int), s);
  const int grid = (int)(ntiles < g_tc_sms ? ntiles : g_tc_sms);
  if (ph) {
    cudaFuncSetAttribute(k_adjoint_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_adjoint_tc<true><<<grid, TC_THREADS, smem, s>>>(panels, rows, kp, N, tiles128, (int)ntiles, dA, dB, derr);
  } else {
    cudaFuncSetAttribute(k_adjoint_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_adjoint_tc<false><<<grid, TC_THREADS, smem, s>>>(panels, rows, kp, N, tiles128, (int)ntiles, dA, dB, derr);
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return herr;
}

}  // namespace bse
