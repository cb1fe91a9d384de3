// Lanczos-Haydock absorption spectrum (Sec. 2.2: the iterative route that
// gives the optical spectrum from Lanczos coefficients without eigenvectors).
//
// TDA:  three-term Lanczos on A from q_0 = d / |d|; F(z) = |d|^2 CF(z).
// PH:   three-term Lanczos on the folded operator K' K (K, K' = M-, M+ or
//       M+, M-), self-adjoint in <x, y>_K = Re(x^H K y), from d;
//       F(z) = 2 <d, d>_K CF(z^2) = D^H Omega (z - H)^{-1} D, D = (d; s conj d)
//       (s = -1: K = M-, s = +1: K = M+).  Each step keeps p = K q beside q,
//       so one step is two structured products (w = K' p, then K r), the
//       same two passes per step as the eigensolver.
// CF(zeta) = 1/(zeta - a_0 - b_0^2/(zeta - a_1 - ...)).  No
// re-orthogonalisation: the recurrence is the method; with enough steps its
// continued fraction converges to the resolvent despite the loss of
// orthogonality.
//
// All scalars stay on the device (HdState, alpha, beta): every kernel reads
// the step index there, so one captured step replays as a CUDA graph.
#include "bse_internal.cuh"

namespace bse {
namespace {

constexpr int HD_THREADS = 256;

template <typename ST>
__global__ void __launch_bounds__(HD_THREADS) k_hd_dot(const ST* __restrict__ x, const ST* __restrict__ y,
                                                       int64_t n, double* __restrict__ partial) {
  __shared__ double red[HD_THREADS / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ST a = x[i], b = y[i];
    s += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < HD_THREADS / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// which = 0: <d, d>_K (start); 1: alpha_j; 2: beta_j and the step advance
__global__ void k_hd_scalar(HdState* __restrict__ st, const double* __restrict__ partial, int np,
                            double* __restrict__ alpha, double* __restrict__ beta, int which) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < np; ++i) s += partial[i];
  if (which == 0) {
    st->n2 = s;
    st->j = 0;
    st->nsteps = 0;
    st->done = (s > 0.0 && isfinite(s)) ? 0 : 1;
    return;
  }
  if (st->done || st->j >= st->m) return;
  const int j = st->j;
  if (which == 1) {
    alpha[j] = s;
    return;
  }
  // an (almost) invariant Krylov space ends the fraction exactly here
  const double scale = fabs(alpha[j]) + (j > 0 ? beta[j - 1] : 0.0);
  st->nsteps = j + 1;
  if (!(s > 1e-28 * scale * scale) || !isfinite(s)) {
    beta[j] = 0.0;
    st->done = 1;
    return;
  }
  beta[j] = sqrt(s);
  st->j = j + 1;
}

// r = w - alpha_j q - beta_{j-1} q_prev
template <typename ST>
__global__ void k_hd_axpy(const HdState* __restrict__ st, const double* __restrict__ alpha,
                          const double* __restrict__ beta, const ST* __restrict__ w, const ST* __restrict__ q,
                          const ST* __restrict__ qprev, ST* __restrict__ r, int64_t n) {
  if (st->done || st->j >= st->m) return;
  const int j = st->j;
  using R = decltype(w[0].x);
  const R a = (R)alpha[j], b = (R)(j > 0 ? beta[j - 1] : 0.0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ST v = w[i];
    const ST x = q[i], y = qprev[i];
    v.x = v.x - a * x.x - b * y.x;
    v.y = v.y - a * x.y - b * y.y;
    r[i] = v;
  }
}

// start (init = 1): q = r / sqrt(n2), p = pr / sqrt(n2), q_prev = 0;
// step: q_prev = q, q = r / beta_{j-1}, p = pr / beta_{j-1} (j already advanced)
template <typename ST>
__global__ void k_hd_scale(const HdState* __restrict__ st, const double* __restrict__ beta, const ST* __restrict__ r,
                           const ST* __restrict__ pr, ST* __restrict__ q, ST* __restrict__ qprev, ST* __restrict__ p,
                           int64_t n, int init) {
  if (st->done) return;
  double s;
  if (init) {
    s = 1.0 / sqrt(st->n2);
  } else {
    if (st->j <= 0) return;
    s = 1.0 / beta[st->j - 1];
  }
  using R = decltype(r[0].x);
  const R f = (R)s;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ST x = r[i];
    qprev[i] = init ? czero<ST>() : q[i];
    q[i] = cscale(x, f);
    if (p) p[i] = cscale(pr[i], f);
  }
}

// d (complex128, N) -> x (ST, Npad, zero padded)
template <typename ST>
__global__ void k_hd_load(const double2* __restrict__ d, int64_t N, int64_t Npad, ST* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Npad; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = i < N ? ccvt<ST>(d[i]) : czero<ST>();
}

// F(omega_i + i eta) from the continued fraction; out[2i], out[2i+1] = Re, Im
__global__ void k_hd_cf(const HdState* __restrict__ st, const double* __restrict__ alpha,
                        const double* __restrict__ beta, int nw, const double* __restrict__ omega, double eta,
                        int ph, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int n = st->nsteps;
  const double zr = omega[i], zi = eta;
  const double xr = ph ? zr * zr - zi * zi : zr, xi = ph ? 2.0 * zr * zi : zi;   // zeta = z^2 (PH) or z
  double tr = 0.0, ti = 0.0;
  for (int j = n - 1; j >= 0; --j) {
    double dr = xr - alpha[j], di = xi;
    if (j < n - 1) {
      const double b2 = beta[j] * beta[j];
      dr -= b2 * tr;
      di -= b2 * ti;
    }
    const double den = dr * dr + di * di;     // t = 1 / (dr + i di)
    tr = dr / den;
    ti = -di / den;
  }
  const double f = (ph ? 2.0 : 1.0) * (n > 0 ? st->n2 : 0.0);
  out[2 * i] = f * tr;
  out[2 * i + 1] = f * ti;
}

int g_hd_sms = 0;
int hd_grid() {
  if (!g_hd_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_hd_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_hd_sms <= 0) g_hd_sms = 1;
  }
  return 2 * g_hd_sms;
}

}  // namespace

int haydock_partials() { return hd_grid(); }

template <typename ST>
void launch_hd_dot(const ST* x, const ST* y, int64_t n, double* partial, cudaStream_t s) {
  count_launch();
  k_hd_dot<ST><<<hd_grid(), HD_THREADS, 0, s>>>(x, y, n, partial);
}

void launch_hd_scalar(HdState* st, const double* partial, double* alpha, double* beta, int which, cudaStream_t s) {
  count_launch();
  k_hd_scalar<<<1, 32, 0, s>>>(st, partial, hd_grid(), alpha, beta, which);
}

template <typename ST>
void launch_hd_axpy(const HdState* st, const double* alpha, const double* beta, const ST* w, const ST* q,
                    const ST* qprev, ST* r, int64_t n, cudaStream_t s) {
  count_launch();
  k_hd_axpy<ST><<<hd_grid(), HD_THREADS, 0, s>>>(st, alpha, beta, w, q, qprev, r, n);
}

template <typename ST>
void launch_hd_scale(const HdState* st, const double* beta, const ST* r, const ST* pr, ST* q, ST* qprev, ST* p,
                     int64_t n, int init, cudaStream_t s) {
  count_launch();
  k_hd_scale<ST><<<hd_grid(), HD_THREADS, 0, s>>>(st, beta, r, pr, q, qprev, p, n, init);
}

template <typename ST>
void launch_hd_load(const double2* d, int64_t N, int64_t Npad, ST* x, cudaStream_t s) {
  count_launch();
  k_hd_load<ST><<<hd_grid(), HD_THREADS, 0, s>>>(d, N, Npad, x);
}

void launch_hd_cf(const HdState* st, const double* alpha, const double* beta, int nw, const double* omega,
                  double eta, int ph, double* out, cudaStream_t s) {
  count_launch();
  k_hd_cf<<<(nw + 127) / 128, 128, 0, s>>>(st, alpha, beta, nw, omega, eta, ph, out);
}

#define HD_INST(ST)                                                                                           \
  template void launch_hd_dot<ST>(const ST*, const ST*, int64_t, double*, cudaStream_t);                     \
  template void launch_hd_axpy<ST>(const HdState*, const double*, const double*, const ST*, const ST*,        \
                                   const ST*, ST*, int64_t, cudaStream_t);                                    \
  template void launch_hd_scale<ST>(const HdState*, const double*, const ST*, const ST*, ST*, ST*, ST*,       \
                                    int64_t, int, cudaStream_t);                                              \
  template void launch_hd_load<ST>(const double2*, int64_t, int64_t, ST*, cudaStream_t);
HD_INST(float2)
HD_INST(double2)
#undef HD_INST

}  // namespace bse
