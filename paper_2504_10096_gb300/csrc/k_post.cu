// Post-processing of the converged Krylov vectors.
//
// PH ("last step" of the folded method, Sec. 2.2.1): for a converged
// K-normalised u with M- M+ u = omega^2 u,
//     X = omega u + M+ u,   Y = conj(omega u - M+ u)
// satisfy H (X; Y) = omega (X; Y); the columns are then scaled so that
// z^H Omega z = |X|^2 - |Y|^2 = 1.  The -omega partner (conj Y; conj X) and the
// left eigenvectors (X; -Y) follow from Eq. 7 without further work.  On the
// Gruning path the converged pair (u, w) of even and odd tops gives
// X = u + w, Y = conj(u - w) directly (w = M+ u / omega).
//
// Final FP64 check: Hz from the stored blocks (Y1 = A X + B Y,
// Y2 = -conj(A conj(Y) + B conj(X))), the Omega-Rayleigh quotient
// rho = Re(z^H Omega H z) / (z^H Omega z) (Omega H = M of Eq. 3) and the
// relative residual ||Hz - rho z|| / (|rho| ||z||).
//
// Adjoint: d omega = z^H Omega dH z (left eigenvector Omega z, Eq. 7), giving
//     dA = X g X^H + conj(Y g Y^H),  dB = X g Y^H + (X g Y^H)^T.
#include "bse_internal.cuh"

namespace bse {

template <typename ST> struct RealOf2;
template <> struct RealOf2<float2> { using T = float; };
template <> struct RealOf2<double2> { using T = double; };

// Z[:, i] (FP64, ldz = 2 Npad for PH, Npad for TDA) from the locked basis.
template <typename ST>
__global__ void k_recover(const Prob* __restrict__ probs, int iprob, int ph, double2* __restrict__ Z,
                          int64_t ldz) {
  const Prob& p = probs[iprob];
  const int i = blockIdx.y;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= p.Npad) return;
  const double2 u = ccvt<double2>(((const ST*)p.V)[(int64_t)i * p.Npad + row]);
  double2* z = Z + (int64_t)i * ldz;
  if (!ph) { z[row] = u; return; }
  if (p.variant == VAR_GRUNING) {   // z = even + odd vector: (u + w; conj(u - w))
    const double2 w = ccvt<double2>(((const ST*)p.W)[(int64_t)i * p.Npad + row]);
    z[row] = cadd(u, w);
    z[p.Npad + row] = conjc(csub(u, w));
    return;
  }
  const double2 pu = ccvt<double2>(((const ST*)p.P)[(int64_t)i * p.Npad + row]);
  const double om = sqrt(p.theta[i]);
  const double2 X = mk(om * u.x + pu.x, om * u.y + pu.y);
  const double2 Yc = mk(om * u.x - pu.x, om * u.y - pu.y);
  z[row] = X;
  z[p.Npad + row] = conjc(Yc);
}

// part[i][rb] = sum over the block of |X|^2 - |Y|^2 (PH) or |X|^2 (TDA)
__global__ void k_colnorm_partial(const double2* __restrict__ Z, int64_t ldz, int64_t Npad, int ph,
                                  double* __restrict__ part, int nrb) {
  __shared__ double red[8];
  const int i = blockIdx.y, rb = blockIdx.x;
  const double2* z = Z + (int64_t)i * ldz;
  const int64_t r0 = (int64_t)rb * ROWBLK, r1 = min(Npad, r0 + ROWBLK);
  double s = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += 256) {
    const double2 x = z[r];
    s += x.x * x.x + x.y * x.y;
    if (ph) { const double2 y = z[Npad + r]; s -= y.x * y.x + y.y * y.y; }
  }
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[(int64_t)i * nrb + rb] = t;
  }
}

__global__ void k_colscale(double2* __restrict__ Z, int64_t ldz, int64_t Npad, int ph,
                           const double* __restrict__ part, int nrb) {
  __shared__ double sc;
  const int i = blockIdx.y;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int rb = 0; rb < nrb; ++rb) t += part[(int64_t)i * nrb + rb];
    sc = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
  }
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= Npad) return;
  double2* z = Z + (int64_t)i * ldz;
  z[row] = cscale(z[row], sc);
  if (ph) z[Npad + row] = cscale(z[Npad + row], sc);
}

// XA = [X | conj(Y)], XB = [Y | conj(X)]  (Npad x 2k, ld Npad)
__global__ void k_prepare_hz(const double2* __restrict__ Z, int64_t ldz, int64_t Npad, int k,
                             double2* __restrict__ XA, double2* __restrict__ XB) {
  const int i = blockIdx.y;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= Npad) return;
  const double2 x = Z[(int64_t)i * ldz + row];
  const double2 y = Z[(int64_t)i * ldz + Npad + row];
  XA[(int64_t)i * Npad + row] = x;
  XA[(int64_t)(k + i) * Npad + row] = conjc(y);
  XB[(int64_t)i * Npad + row] = y;
  XB[(int64_t)(k + i) * Npad + row] = conjc(x);
}

// Residual partials.  stage 0: part[i][rb] = (num, den, zz, 0);
// stage 1: part[i][rb].w = |Hz - rho z|^2.  U as produced by the row-block
// product: PH U (Npad x 2k): Hz1 = U[:, i], Hz2 = -conj(U[:, k+i]); TDA Hz = U[:, i].
__global__ void k_resid_partial(const double2* __restrict__ Z, int64_t ldz, const double2* __restrict__ U,
                                int64_t Npad, int k, int ph, const double* __restrict__ rho,
                                D4* __restrict__ part, int nrb, int stage) {
  __shared__ D4 red[8];
  const int i = blockIdx.y, rb = blockIdx.x;
  const double2* z = Z + (int64_t)i * ldz;
  const double2* u1 = U + (int64_t)i * Npad;
  const double2* u2 = ph ? U + (int64_t)(k + i) * Npad : nullptr;
  const int64_t r0 = (int64_t)rb * ROWBLK, r1 = min(Npad, r0 + ROWBLK);
  const double rh = stage ? rho[i] : 0.0;
  D4 s = D4{0.0, 0.0, 0.0, 0.0};
  for (int64_t r = r0 + threadIdx.x; r < r1; r += 256) {
    const double2 x = z[r];
    const double2 h1 = u1[r];
    if (stage == 0) {
      s.x += x.x * h1.x + x.y * h1.y;           // Re(conj x * Hz1)
      s.y += x.x * x.x + x.y * x.y;
      s.z += x.x * x.x + x.y * x.y;
    } else {
      const double dx = h1.x - rh * x.x, dy = h1.y - rh * x.y;
      s.w += dx * dx + dy * dy;
    }
    if (ph) {
      const double2 y = z[Npad + r];
      const double2 t = u2[r];
      const double2 h2 = mk(-t.x, t.y);       // -conj(U2)
      if (stage == 0) {
        s.x -= y.x * h2.x + y.y * h2.y;         // Omega weighting
        s.y -= y.x * y.x + y.y * y.y;
        s.z += y.x * y.x + y.y * y.y;
      } else {
        const double dx = h2.x - rh * y.x, dy = h2.y - rh * y.y;
        s.w += dx * dx + dy * dy;
      }
    }
  }
  for (int m = 16; m >= 1; m >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, m);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, m);
    s.z += __shfl_xor_sync(0xffffffffu, s.z, m);
    s.w += __shfl_xor_sync(0xffffffffu, s.w, m);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    D4 t = red[0];
    for (int w = 1; w < 8; ++w) { t.x += red[w].x; t.y += red[w].y; t.z += red[w].z; t.w += red[w].w; }
    D4* pp = part + (int64_t)i * nrb + rb;
    if (stage == 0) *pp = t;
    else pp->w = t.w;
  }
}

// stage 0: rho[i] = num / den, zz kept in znorm[i]; stage 1: res[i]
__global__ void k_resid_final(const D4* __restrict__ part, int nrb, int k, int stage,
                              double* __restrict__ rho, double* __restrict__ znorm2,
                              double* __restrict__ res) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  D4 t = D4{0.0, 0.0, 0.0, 0.0};
  for (int rb = 0; rb < nrb; ++rb) {
    const D4 q = part[(int64_t)i * nrb + rb];
    t.x += q.x; t.y += q.y; t.z += q.z; t.w += q.w;
  }
  if (stage == 0) {
    rho[i] = t.x / t.y;
    znorm2[i] = t.z;
  } else {
    res[i] = sqrt(t.w) / (fabs(rho[i]) * sqrt(znorm2[i]));
  }
}

// out[:, c] (ld ldo, rows < N, and for PH rows N..2N-1 from the Y half) = Z[:, perm[c]]
template <typename ST>
__global__ void k_store_vectors(const double2* __restrict__ Z, int64_t ldz, int64_t Npad, int64_t N, int ph,
                                const int* __restrict__ perm, ST* __restrict__ out, int64_t ldo) {
  const int c = blockIdx.y;
  const int i = perm ? perm[c] : c;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= N) return;
  const double2* z = Z + (int64_t)i * ldz;
  out[(int64_t)c * ldo + row] = ccvt<ST>(z[row]);
  if (ph) out[(int64_t)c * ldo + N + row] = ccvt<ST>(z[Npad + row]);
}

// ---------------------------------------------------------------- adjoint
// One CTA per 64 x 64 output tile (I <= J) of dA (and dB); 256 threads, 4 x 4
// outputs each; the mirror tile (J, I) is written from the same registers.
constexpr int ADJ_KC = 8;
template <typename ST, typename R>
__global__ void __launch_bounds__(256)
k_adjoint(const double2* __restrict__ Z, int64_t ldz, int64_t Npad, int64_t N, int k,
          const double* __restrict__ g, int ph, const int2* __restrict__ tiles, ST* __restrict__ dA,
          ST* __restrict__ dB) {
  using CT = typename C2<R>::T;
  __shared__ CT xi[ADJ_KC][64], yi[ADJ_KC][64], xj[ADJ_KC][64], yj[ADJ_KC][64];
  const int2 tl = tiles[blockIdx.x];
  const int I = tl.x, J = tl.y;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  CT accA[4][4], accB[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { accA[a][b] = czero<CT>(); accB[a][b] = czero<CT>(); }
  for (int k0 = 0; k0 < k; k0 += ADJ_KC) {
    __syncthreads();
    for (int e = tid; e < ADJ_KC * 64; e += 256) {
      const int q = e >> 6, r = e & 63;
      const int kk = k0 + q;
      const int64_t ri = (int64_t)I * 64 + r, rj = (int64_t)J * 64 + r;
      CT a = czero<CT>(), b = czero<CT>(), c = czero<CT>(), d = czero<CT>();
      if (kk < k) {
        const double gk = g[kk];
        const double2* z = Z + (int64_t)kk * ldz;
        if (ri < N) { a = ccvt<CT>(cscale(z[ri], gk)); if (ph) b = ccvt<CT>(cscale(z[Npad + ri], gk)); }
        if (rj < N) { c = ccvt<CT>(z[rj]); if (ph) d = ccvt<CT>(z[Npad + rj]); }
      }
      xi[q][r] = a; yi[q][r] = b; xj[q][r] = c; yj[q][r] = d;
    }
    __syncthreads();
#pragma unroll 2
    for (int q = 0; q < ADJ_KC; ++q) {
      CT vxi[4], vyi[4], vxj[4], vyj[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { vxi[a] = xi[q][ty * 4 + a]; vyi[a] = yi[q][ty * 4 + a]; }
#pragma unroll
      for (int b = 0; b < 4; ++b) { vxj[b] = xj[q][tx * 4 + b]; vyj[b] = yj[q][tx * 4 + b]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          // dA += g x_i conj(x_j) + conj(g y_i) y_j
          cfmac(accA[a][b], vxj[b], vxi[a]);
          if (ph) {
            cfmac(accA[a][b], vyi[a], vyj[b]);
            // dB += g x_i conj(y_j) + x_j conj(g y_i)
            cfmac(accB[a][b], vyj[b], vxi[a]);
            cfmac(accB[a][b], vyi[a], vxj[b]);
          }
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = (int64_t)I * 64 + ty * 4 + a;
    if (i >= N) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = (int64_t)J * 64 + tx * 4 + b;
      if (j >= N) continue;
      dA[i * N + j] = ccvt<ST>(accA[a][b]);
      if (ph) dB[i * N + j] = ccvt<ST>(accB[a][b]);
    }
  }
  if (I != J) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = (int64_t)J * 64 + tx * 4 + b;
      if (j >= N) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t i = (int64_t)I * 64 + ty * 4 + a;
        if (i >= N) continue;
        dA[j * N + i] = ccvt<ST>(conjc(accA[a][b]));
        if (ph) dB[j * N + i] = ccvt<ST>(accB[a][b]);
      }
    }
  }
}

// ---------------------------------------------------------------- launchers
template <typename ST>
void launch_recover(const Prob* dprobs, int iprob, int ph, int64_t Npad, int64_t N, int nev, double2* Z,
                    int ldz, cudaStream_t s) {
  (void)N;
  count_launch();
  k_recover<ST><<<dim3((unsigned)((Npad + 255) / 256), nev), 256, 0, s>>>(dprobs, iprob, ph, Z, ldz);
}

void launch_colnormalize(double2* Z, int64_t ldz, int64_t Npad, int k, int ph, double* part, int nrb,
                         cudaStream_t s) {
  count_launch(2);
  k_colnorm_partial<<<dim3(nrb, k), 256, 0, s>>>(Z, ldz, Npad, ph, part, nrb);
  k_colscale<<<dim3((unsigned)((Npad + 255) / 256), k), 256, 0, s>>>(Z, ldz, Npad, ph, part, nrb);
}

void launch_prepare_hz2(const double2* Z, int64_t ldz, int64_t Npad, int k, double2* XA, double2* XB,
                        cudaStream_t s) {
  count_launch();
  k_prepare_hz<<<dim3((unsigned)((Npad + 255) / 256), k), 256, 0, s>>>(Z, ldz, Npad, k, XA, XB);
}

void launch_residuals2(const double2* Z, int64_t ldz, const double2* U, int64_t Npad, int k, int ph,
                       D4* part, int nrb, double* rho, double* znorm2, double* res, cudaStream_t s) {
  count_launch(4);
  k_resid_partial<<<dim3(nrb, k), 256, 0, s>>>(Z, ldz, U, Npad, k, ph, rho, part, nrb, 0);
  k_resid_final<<<(k + 127) / 128, 128, 0, s>>>(part, nrb, k, 0, rho, znorm2, res);
  k_resid_partial<<<dim3(nrb, k), 256, 0, s>>>(Z, ldz, U, Npad, k, ph, rho, part, nrb, 1);
  k_resid_final<<<(k + 127) / 128, 128, 0, s>>>(part, nrb, k, 1, rho, znorm2, res);
}

template <typename ST>
void launch_store_vectors2(const double2* Z, int64_t ldz, int64_t Npad, int64_t N, int ph, int k,
                           const int* perm, ST* out, int64_t ldo, cudaStream_t s) {
  count_launch();
  k_store_vectors<ST><<<dim3((unsigned)((N + 255) / 256), k), 256, 0, s>>>(Z, ldz, Npad, N, ph, perm, out, ldo);
}

template <typename ST, typename R>
void launch_adjoint2(const double2* Z, int64_t ldz, int64_t Npad, int64_t N, int k, const double* g, int ph,
                     const int2* tiles, int64_t ntiles, ST* dA, ST* dB, cudaStream_t s) {
  count_launch();
  k_adjoint<ST, R><<<(unsigned)ntiles, 256, 0, s>>>(Z, ldz, Npad, N, k, g, ph, tiles, dA, dB);
}

template void launch_recover<float2>(const Prob*, int, int, int64_t, int64_t, int, double2*, int, cudaStream_t);
template void launch_recover<double2>(const Prob*, int, int, int64_t, int64_t, int, double2*, int, cudaStream_t);
template void launch_store_vectors2<float2>(const double2*, int64_t, int64_t, int64_t, int, int, const int*,
                                            float2*, int64_t, cudaStream_t);
template void launch_store_vectors2<double2>(const double2*, int64_t, int64_t, int64_t, int, int, const int*,
                                             double2*, int64_t, cudaStream_t);
template void launch_adjoint2<float2, float>(const double2*, int64_t, int64_t, int64_t, int, const double*, int,
                                             const int2*, int64_t, float2*, float2*, cudaStream_t);
template void launch_adjoint2<double2, double>(const double2*, int64_t, int64_t, int64_t, int, const double*,
                                               int, const int2*, int64_t, double2*, double2*, cudaStream_t);

}  // namespace bse
