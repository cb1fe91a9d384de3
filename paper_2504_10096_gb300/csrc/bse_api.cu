// C ABI and host-side driver of the iterative BSE eigensolver (see bse.h).
//
// The host only sequences launches and reads a few bytes of per-problem
// state once per restart cycle; every arithmetic step of the method (products,
// Gram-Schmidt, projected eigenproblem, restart, recovery, residuals, adjoint)
// runs in the kernels of this library.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bse.h"
#include "bse_internal.cuh"

using namespace bse;

namespace {

struct ProbHost {
  int64_t N = 0;
  int nT = 0;
  int64_t Npad = 0;
  int64_t ntiles = 0;
  void* A = nullptr;
  void* B = nullptr;
  void* Ahl = nullptr;   // split tiles (BSE_C128_DF)
  void* Bhl = nullptr;
  // solve buffers
  int ncv = 0;
  void *V = nullptr, *P = nullptr, *V2 = nullptr, *P2 = nullptr, *w = nullptr, *pw = nullptr;
  void* part = nullptr;
  double *cpart = nullptr, *coef = nullptr, *small = nullptr, *S = nullptr;
  // results
  double2* Z = nullptr;
  int zcols = 0;
  int nconv = 0;
  int* perm = nullptr;   // device, output column -> Z column
  std::vector<double> eval, res;
};

}  // namespace

struct bse_handle {
  int count = 0, form = 0, dtype = 0, ph = 0;
  bool df = false;       // Lanczos products in double-FP32 arithmetic
  bool split = false;    // ... on split complex128 tiles (else on complex64 tiles)
  bool tiles64 = false;  // packed tiles are complex64
  size_t vs = 0;         // bytes per complex element of the Krylov vectors
  size_t es = 0;  // bytes per stored complex element
  cudaStream_t stream = nullptr;
  std::vector<ProbHost> p;
  std::vector<Prob> hprobs;
  Prob* dprobs = nullptr;
  KState* dstate = nullptr;
  std::vector<KState> hstate;
  TileJob* djobs = nullptr;
  int njobs = 0;
  int maxnT = 0;
  int64_t maxNpad = 0;
  int maxnrb = 1;
  int ncv = 0;
  int nev = 0;
  bool solved = false;
  bse_stats stats{};
  // post-processing scratch (single problem at a time)
  void* post = nullptr;
  size_t post_bytes = 0;
  // adjoint tile list
  int2* adj_tiles = nullptr;
  int64_t adj_ntiles = 0;
  double* gdev = nullptr;
  // product timing ring
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  double ms_product = 0.0;
};

namespace {

#define CK(x)                                         \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return BSE_ECUDA;          \
  } while (0)

int dalloc(void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return e == cudaErrorMemoryAllocation ? BSE_ENOMEM : BSE_ECUDA;
  }
  return BSE_OK;
}

void dfree(void*& ptr) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
}
template <typename T>
void dfreet(T*& ptr) {
  if (ptr) cudaFree((void*)ptr);
  ptr = nullptr;
}

bool is_c64(int dtype) { return dtype == BSE_C64 || dtype == BSE_C64_MIXED; }

void free_solve_buffers(ProbHost& q) {
  dfree(q.V); dfree(q.P); dfree(q.V2); dfree(q.P2); dfree(q.w); dfree(q.pw); dfree(q.part);
  dfreet(q.cpart); dfreet(q.coef); dfreet(q.small); dfreet(q.S);
  q.ncv = 0;
}

void free_results(ProbHost& q) {
  dfreet(q.Z);
  dfreet(q.perm);
  q.zcols = 0;
  q.nconv = 0;
}

int nrb_of(int64_t Npad) { return (int)((Npad + ROWBLK - 1) / ROWBLK); }

// ------------------------------------------------------------------ packing
template <typename T>
int pack_matrix(bse_handle* h, const T* src, int64_t N, int nT, int herm, int where, T* dst) {
  if (where == BSE_DEVICE) {
    for (int I = 0; I < nT; ++I)
      launch_pack_row<T, T>(src + (int64_t)I * TS * N, N, nT, I, herm, dst, h->stream);
    CK(cudaGetLastError());
    return BSE_OK;
  }
  // host source: stage one block row (TS x N) at a time
  void* stage = nullptr;
  int rc = dalloc(&stage, (size_t)TS * N * sizeof(T));
  if (rc) return rc;
  for (int I = 0; I < nT; ++I) {
    const int64_t rows = std::min<int64_t>(TS, N - (int64_t)I * TS);
    cudaError_t e = cudaMemcpyAsync(stage, src + (int64_t)I * TS * N, (size_t)rows * N * sizeof(T),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) { cudaFree(stage); return BSE_ECUDA; }
    launch_pack_row<T, T>((const T*)stage, N, nT, I, herm, dst, h->stream);
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  cudaFree(stage);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return BSE_ECUDA;
  return BSE_OK;
}

int map_status(int st) {
  switch (st) {
    case ST_OK: return BSE_OK;
    case ST_NOTPD: return BSE_ENOTPD;
    case ST_NOCONV: return BSE_ENOCONV;
    case ST_TIMEOUT: return BSE_ETIMEOUT;
    case ST_NOTFINITE: return BSE_ENOTFINITE;
  }
  return BSE_ECUDA;
}

// ------------------------------------------------------------------ solve pieces
template <typename ST>
struct Driver {
  using R = typename std::conditional<std::is_same<ST, float2>::value, float, double>::type;
  bse_handle* h;
  explicit Driver(bse_handle* hh) : h(hh) {}

  void product(int mode) {
    const bool timed = h->ev_used + 2 <= (int)h->ev.size();
    if (timed) cudaEventRecord(h->ev[h->ev_used], h->stream);
    if (h->df)
      launch_product_df(h->dprobs, h->djobs, h->njobs, h->count, h->maxnT, mode, nullptr, h->ph != 0, h->split,
                        h->stream);
    else
      launch_product<ST, R>(h->dprobs, h->djobs, h->njobs, h->count, h->maxnT, mode, 1, nullptr, h->ph != 0,
                            h->stream);
    if (timed) {
      cudaEventRecord(h->ev[h->ev_used + 1], h->stream);
      h->ev_used += 2;
    }
  }

  void harvest_events() {
    for (int i = 0; i + 1 < h->ev_used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) == cudaSuccess) h->ms_product += ms;
    }
    h->ev_used = 0;
  }

  void cgs(int pass) {
    const int ncol = h->ncv + 1 + h->ncv;
    launch_step_cgs<ST>(h->dprobs, h->count, h->ph, h->maxnrb, h->maxNpad, ncol, pass, h->stream);
  }

  void step() {
    product(h->ph ? PM_STEP_MMINUS : PM_STEP_A);
    cgs(0);
    cgs(1);
    if (h->ph) product(PM_STEP_MPLUS);
    launch_step_normalize<ST>(h->dprobs, h->count, h->ph, h->maxnrb, h->maxNpad, 0, h->stream);
  }

  void fresh_chain(uint64_t seed, const void* v0) {
    launch_start_vector<ST>(h->dprobs, h->count, h->maxNpad, seed, v0, h->stream);
    cgs(2);
    cgs(3);
    if (h->ph) product(PM_START_MPLUS);
    launch_step_normalize<ST>(h->dprobs, h->count, h->ph, h->maxnrb, h->maxNpad, 1, h->stream);
  }

  int read_state() {
    CK(cudaMemcpyAsync(h->hstate.data(), h->dstate, sizeof(KState) * h->count, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    harvest_events();
    return BSE_OK;
  }

  int iterate(uint64_t seed, const void* v0) {
    fresh_chain(seed, v0);
    int guard = 0;
    long long rounds = 0;
    long long maxit = 0;
    for (int i = 0; i < h->count; ++i) maxit = std::max(maxit, h->hstate[i].maxit);
    for (;;) {
      // every round either adds Krylov steps or restarts; a round without
      // progress cannot repeat more often than this bound
      if (++rounds > 4 * maxit + 4096) return BSE_ETIMEOUT;
      int rc = read_state();
      if (rc) return rc;
      bool any_active = false, any_bd = false;
      int steps = 0;
      for (int i = 0; i < h->count; ++i) {
        const KState& s = h->hstate[i];
        if (s.done || s.status != ST_OK) continue;
        any_active = true;
        if (s.breakdown || s.j < 0) any_bd = true;
        else steps = std::max(steps, s.m - s.j);
      }
      if (!any_active) break;
      if (any_bd) {
        if (++guard > 4 * h->ncv + 64) return BSE_ETIMEOUT;
        fresh_chain(seed + 0x9e3779b9ull * (uint64_t)guard, nullptr);
        continue;
      }
      if (steps > 0) {
        for (int s = 0; s < steps; ++s) step();
        continue;
      }
      launch_ritz(h->dprobs, h->count, h->ncv, h->stream);
      launch_lock_decide_form(h->dprobs, h->count, h->ph, h->stream);
      launch_restart<ST>(h->dprobs, h->count, h->ph, h->maxNpad, h->ncv, h->stream);
    }
    return BSE_OK;
  }

  // recover eigenvectors, FP64 residuals and Rayleigh quotients of problem i
  int finalize(int i, int nev) {
    ProbHost& q = h->p[i];
    const KState& s = h->hstate[i];
    free_results(q);
    const int k = std::min(s.k, nev);
    q.nconv = k;
    q.eval.assign(k, 0.0);
    q.res.assign(k, 0.0);
    if (k == 0) return BSE_OK;
    const int64_t Npad = q.Npad;
    const int64_t ldz = h->ph ? 2 * Npad : Npad;
    int rc = dalloc((void**)&q.Z, sizeof(double2) * (size_t)ldz * k);
    if (rc) return rc;
    rc = dalloc((void**)&q.perm, sizeof(int) * k);
    if (rc) return rc;
    q.zcols = k;
    const int nrb = nrb_of(Npad);
    const int kc = h->ph ? 2 * k : k;
    // scratch: XA, XB, U (Npad x kc FP64 complex), part4 (k x nrb double4), rho, z2, res
    const size_t need = sizeof(double2) * (size_t)Npad * kc * 3 + sizeof(D4) * (size_t)k * nrb +
                        sizeof(double) * 3 * (size_t)k + 1024;
    if (need > h->post_bytes) {
      dfree(h->post);
      h->post_bytes = 0;
      rc = dalloc(&h->post, need);
      if (rc) return rc;
      h->post_bytes = need;
    }
    double2* XA = (double2*)h->post;
    double2* XB = XA + (size_t)Npad * kc;
    double2* U = XB + (size_t)Npad * kc;
    D4* part4 = (D4*)(U + (size_t)Npad * kc);
    double* rho = (double*)(part4 + (size_t)k * nrb);
    double* z2 = rho + k;
    double* res = z2 + k;
    launch_recover<ST>(h->dprobs, i, h->ph, Npad, q.N, k, q.Z, (int)ldz, h->stream);
    launch_colnormalize(q.Z, ldz, Npad, k, h->ph, (double*)part4, nrb, h->stream);
    // FP64 products with the stored tiles (complex64 or complex128)
    const void* xa = h->ph ? (const void*)XA : (const void*)q.Z;
    const void* xb = h->ph ? (const void*)XB : nullptr;
    const double sgn = h->ph ? 1.0 : 0.0;
    if (h->ph) launch_prepare_hz2(q.Z, ldz, Npad, k, XA, XB, h->stream);
    if (h->tiles64)
      launch_rowblock<float2, double>(h->dprobs, i, q.nT, xa, xb, (int)Npad, sgn, U, (int)Npad, kc, h->ph != 0,
                                      h->stream);
    else
      launch_rowblock<double2, double>(h->dprobs, i, q.nT, xa, xb, (int)Npad, sgn, U, (int)Npad, kc, h->ph != 0,
                                       h->stream);
    launch_residuals2(q.Z, ldz, U, Npad, k, h->ph, part4, nrb, rho, z2, res, h->stream);
    CK(cudaGetLastError());
    std::vector<double> hr(k), hres(k);
    CK(cudaMemcpyAsync(hr.data(), rho, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(hres.data(), res, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::vector<int> perm(k);
    for (int c = 0; c < k; ++c) perm[c] = c;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return hr[a] < hr[b]; });
    for (int c = 0; c < k; ++c) {
      q.eval[c] = hr[perm[c]];
      q.res[c] = hres[perm[c]];
    }
    CK(cudaMemcpyAsync(q.perm, perm.data(), sizeof(int) * k, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return BSE_OK;
  }

  int store(int i, void* out) {
    ProbHost& q = h->p[i];
    if (!out || q.nconv == 0) return BSE_OK;
    const int64_t ldz = h->ph ? 2 * q.Npad : q.Npad;
    const int64_t ldo = h->ph ? 2 * q.N : q.N;
    if (is_c64(h->dtype))   // caller-facing vectors in the handle's dtype
      launch_store_vectors2<float2>(q.Z, ldz, q.Npad, q.N, h->ph, q.nconv, q.perm, (float2*)out, ldo, h->stream);
    else
      launch_store_vectors2<double2>(q.Z, ldz, q.Npad, q.N, h->ph, q.nconv, q.perm, (double2*)out, ldo,
                                     h->stream);
    CK(cudaGetLastError());
    return BSE_OK;
  }
};

int alloc_solve(bse_handle* h, int ncv) {
  const size_t es = h->vs;  // Krylov vectors
  const size_t cs = es;     // product partials in the vectors' precision
  for (int i = 0; i < h->count; ++i) {
    ProbHost& q = h->p[i];
    if (q.ncv == ncv) continue;
    free_solve_buffers(q);
    const int ncol = 2 * ncv + 1;
    const int nrb = nrb_of(q.Npad);
    int rc;
    if ((rc = dalloc(&q.V, es * (size_t)q.Npad * ncol))) return rc;
    if (h->ph && (rc = dalloc(&q.P, es * (size_t)q.Npad * ncol))) return rc;
    if ((rc = dalloc(&q.V2, es * (size_t)q.Npad * ncv))) return rc;
    if (h->ph && (rc = dalloc(&q.P2, es * (size_t)q.Npad * ncv))) return rc;
    if ((rc = dalloc(&q.w, es * (size_t)q.Npad))) return rc;
    if ((rc = dalloc(&q.pw, es * (size_t)q.Npad))) return rc;
    if ((rc = dalloc(&q.part, cs * (size_t)q.nT * q.nT * TS))) return rc;
    if ((rc = dalloc((void**)&q.cpart, sizeof(double2) * (size_t)nrb * ncol))) return rc;
    if ((rc = dalloc((void**)&q.coef, sizeof(double2) * 2 * (size_t)ncol))) return rc;
    if ((rc = dalloc((void**)&q.small, sizeof(double) * 6 * (size_t)(ncv + 1)))) return rc;
    if ((rc = dalloc((void**)&q.S, sizeof(double) * (size_t)ncv * ncv))) return rc;
    CK(cudaMemsetAsync(q.V, 0, es * (size_t)q.Npad * ncol, h->stream));
    if (h->ph) CK(cudaMemsetAsync(q.P, 0, es * (size_t)q.Npad * ncol, h->stream));
    CK(cudaMemsetAsync(q.small, 0, sizeof(double) * 6 * (size_t)(ncv + 1), h->stream));
    CK(cudaMemsetAsync(q.S, 0, sizeof(double) * (size_t)ncv * ncv, h->stream));
    q.ncv = ncv;
  }
  return BSE_OK;
}

int upload_probs(bse_handle* h) {
  h->hprobs.resize(h->count);
  for (int i = 0; i < h->count; ++i) {
    ProbHost& q = h->p[i];
    Prob& d = h->hprobs[i];
    d.N = q.N;
    d.nT = q.nT;
    d.Npad = q.Npad;
    d.ph = h->ph;
    d.ncv = q.ncv;
    d.ncol = 2 * q.ncv + 1;
    d.A = q.A;
    d.B = q.B;
    d.V = q.V; d.P = q.P; d.V2 = q.V2; d.P2 = q.P2; d.w = q.w; d.pw = q.pw; d.part = q.part;
    d.cpart = q.cpart;
    d.coef = q.coef;
    const int64_t m1 = q.ncv + 1;
    d.theta = q.small;
    d.barrow = q.small + m1;
    d.alpha = q.small + 2 * m1;
    d.beta = q.small + 3 * m1;
    d.ritz = q.small + 4 * m1;
    d.rest = q.small + 5 * m1;
    d.S = q.S;
    d.nrb = nrb_of(q.Npad);
    d.st = h->dstate + i;
    d.Ahl = q.Ahl;
    d.Bhl = q.Bhl;
  }
  CK(cudaMemcpyAsync(h->dprobs, h->hprobs.data(), sizeof(Prob) * h->count, cudaMemcpyHostToDevice,
                     h->stream));
  return BSE_OK;
}

template <typename ST>
int solve_impl(bse_handle* h, int nev, double tol, const bse_solve_opts* opts, double* eval_out,
               void* const* evec_out, int* nconv_out) {
  int64_t minN = h->p[0].N;
  for (auto& q : h->p) minN = std::min(minN, q.N);
  if (nev < 1 || nev > minN || !(tol > 0.0) || !eval_out) return BSE_EINVAL;
  int ncv = opts && opts->ncv > 0 ? opts->ncv : std::max(2 * nev, nev + 32);
  if (ncv > minN) ncv = (int)minN;
  if (ncv > MAXM) ncv = MAXM;
  if (ncv < nev) return BSE_EINVAL;
  const long long maxit = opts && opts->maxit > 0 ? opts->maxit : 20000;
  const uint64_t seed = opts && opts->seed ? opts->seed : 12345ull;
  const double lock_tol = opts && opts->lock_tol > 0.0 ? opts->lock_tol : tol * 0.25;
  const void* v0 = (opts && h->count == 1) ? opts->v0 : nullptr;
  int rc = alloc_solve(h, ncv);
  if (rc) return rc;
  h->ncv = ncv;
  h->nev = nev;
  h->solved = false;
  for (int i = 0; i < h->count; ++i) {
    KState& s = h->hstate[i];
    std::memset(&s, 0, sizeof(KState));
    s.k = 0; s.l = 0; s.j = -1; s.m = ncv; s.ntw = 0; s.nev = nev;
    s.r_pkeep = std::min(ncv - 1, nev + (ncv - nev) / 2);
    if (s.r_pkeep < nev) s.r_pkeep = nev;
    s.maxit = maxit;
    s.tol = tol;
    s.lock_tol = lock_tol;
  }
  CK(cudaMemcpyAsync(h->dstate, h->hstate.data(), sizeof(KState) * h->count, cudaMemcpyHostToDevice,
                     h->stream));
  if ((rc = upload_probs(h))) return rc;
  if (h->ev.empty()) {
    h->ev.resize(4 * MAXM + 8);
    for (auto& e : h->ev) cudaEventCreate(&e);
  }
  h->ev_used = 0;
  h->ms_product = 0.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, h->stream);
  const long long launches0 = launch_counter();
  Driver<ST> drv(h);
  rc = drv.iterate(seed, v0);
  if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
  int worst = BSE_OK;
  double maxres = 0.0;
  int64_t steps = 0, passes = 0, restarts = 0;
  int nconv_total = 0;
  for (int i = 0; i < h->count; ++i) {
    rc = drv.finalize(i, nev);
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    const KState& s = h->hstate[i];
    ProbHost& q = h->p[i];
    for (int c = 0; c < nev; ++c) eval_out[(size_t)i * nev + c] = c < q.nconv ? q.eval[c] : NAN;
    if (nconv_out) nconv_out[i] = q.nconv;
    for (double r : q.res) maxres = std::max(maxres, r);
    if (evec_out && evec_out[i]) {
      rc = drv.store(i, evec_out[i]);
      if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    }
    steps += s.steps;
    passes += s.passes;
    restarts += s.restarts;
    nconv_total += q.nconv;
    int st = map_status(s.status);
    if (st == BSE_OK && q.nconv < nev) st = BSE_ENOCONV;
    if (st != BSE_OK && worst == BSE_OK) worst = st;
    if (st == BSE_ENOTPD || st == BSE_ENOTFINITE) worst = st;
  }
  cudaEventRecord(e1, h->stream);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  h->stats.steps = steps;
  h->stats.passes = passes;
  h->stats.restarts = restarts;
  h->stats.nconv = nconv_total;
  h->stats.max_residual = maxres;
  h->stats.ms_total = ms;
  h->stats.ms_product = h->ms_product;
  h->stats.launches = launch_counter() - launches0;
  h->solved = true;
  return worst;
}

// ------------------------------------------------------------------ apply helpers
template <typename ST>
__global__ void k_pad_in(const ST* __restrict__ X, int64_t N, int64_t ldx, int64_t Npad, int k, int ph_half,
                         ST* __restrict__ out) {
  // out[:, c] (Npad rows) = X[half*N : half*N + N, c] with zero padding
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Npad) return;
  out[(int64_t)c * Npad + r] = r < N ? X[(int64_t)c * ldx + (int64_t)ph_half * N + r] : czero<ST>();
}

template <typename ST, typename CT>
__global__ void k_hz_in(const ST* __restrict__ X, int64_t N, int64_t Npad, int k, CT* __restrict__ XA,
                        CT* __restrict__ XB) {
  // X: 2N x k stacked (X1; X2).  XA = [X1 | conj X2], XB = [X2 | conj X1]
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Npad) return;
  CT x1 = czero<CT>(), x2 = czero<CT>();
  if (r < N) {
    x1 = ccvt<CT>(X[(int64_t)c * 2 * N + r]);
    x2 = ccvt<CT>(X[(int64_t)c * 2 * N + N + r]);
  }
  XA[(int64_t)c * Npad + r] = x1;
  XA[(int64_t)(k + c) * Npad + r] = conjc(x2);
  XB[(int64_t)c * Npad + r] = x2;
  XB[(int64_t)(k + c) * Npad + r] = conjc(x1);
}

template <typename ST, typename CT>
__global__ void k_hz_out(const CT* __restrict__ U, int64_t N, int64_t Npad, int k, int op, ST* __restrict__ Y) {
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  if (op == BSE_OP_H) {
    Y[(int64_t)c * 2 * N + r] = ccvt<ST>(U[(int64_t)c * Npad + r]);
    const CT u2 = U[(int64_t)(k + c) * Npad + r];
    CT y2;
    y2.x = -u2.x;
    y2.y = u2.y;
    Y[(int64_t)c * 2 * N + N + r] = ccvt<ST>(y2);
  } else {
    Y[(int64_t)c * N + r] = ccvt<ST>(U[(int64_t)c * Npad + r]);
  }
}

template <typename ST, typename CT>
__global__ void k_cvt_pad(const ST* __restrict__ X, int64_t N, int64_t Npad, int k, CT* __restrict__ out) {
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Npad) return;
  out[(int64_t)c * Npad + r] = r < N ? ccvt<CT>(X[(int64_t)c * N + r]) : czero<CT>();
}

template <typename ST>
int apply_impl(bse_handle* h, int op, int k, const void* X, void* Y) {
  using R = typename std::conditional<std::is_same<ST, float2>::value, float, double>::type;
  using CT = ST;
  ProbHost& q = h->p[0];
  const int64_t N = q.N, Npad = q.Npad;
  const bool hasB = h->ph != 0;
  if ((op != BSE_OP_A) && !hasB) return BSE_EINVAL;
  int rc;
  if (op != BSE_OP_H && k == 1) {
    // the streaming tile kernel (the solver's hot path), padded copies in/out
    if (!q.w || q.ncv == 0) {
      if ((rc = alloc_solve(h, std::min<int64_t>(q.N, 8) > 1 ? (int)std::min<int64_t>(q.N, 8) : 1))) return rc;
      if ((rc = upload_probs(h))) return rc;
    }
    count_launch();
    k_pad_in<ST><<<dim3((unsigned)((Npad + 255) / 256), 1), 256, 0, h->stream>>>(
        (const ST*)X, N, N, Npad, 1, 0, (ST*)q.w);
    GenericIO io{};
    io.xa = q.w;
    io.y = q.pw;
    io.sB = op == BSE_OP_A ? 0.0 : (op == BSE_OP_MPLUS ? 1.0 : -1.0);
    if (h->df && h->split)   // complex128 handle: the solver's double-FP32 product
      launch_product_df(h->dprobs, h->djobs, h->njobs, 1, h->maxnT, PM_GENERIC, &io, hasB && op != BSE_OP_A,
                        true, h->stream);
    else
      launch_product<ST, R>(h->dprobs, h->djobs, h->njobs, 1, h->maxnT, PM_GENERIC, 1, &io,
                            hasB && op != BSE_OP_A, h->stream);
    CK(cudaMemcpyAsync(Y, q.pw, h->es * (size_t)N, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return BSE_OK;
  }
  const int kc = op == BSE_OP_H ? 2 * k : k;
  const size_t need = sizeof(CT) * (size_t)Npad * kc * 3 + 1024;
  if (need > h->post_bytes) {
    dfree(h->post);
    h->post_bytes = 0;
    if ((rc = dalloc(&h->post, need))) return rc;
    h->post_bytes = need;
  }
  CT* XA = (CT*)h->post;
  CT* XB = XA + (size_t)Npad * kc;
  CT* U = XB + (size_t)Npad * kc;
  if (!q.w || q.ncv == 0) {
    if ((rc = alloc_solve(h, std::min<int64_t>(q.N, 8) > 1 ? (int)std::min<int64_t>(q.N, 8) : 1))) return rc;
  }
  if ((rc = upload_probs(h))) return rc;
  const dim3 g((unsigned)((Npad + 255) / 256), k);
  double sB = 0.0;
  const void* xb = nullptr;
  if (op == BSE_OP_H) {
    count_launch();
    k_hz_in<ST, CT><<<g, 256, 0, h->stream>>>((const ST*)X, N, Npad, k, XA, XB);
    sB = 1.0;
    xb = XB;
  } else {
    count_launch();
    k_cvt_pad<ST, CT><<<g, 256, 0, h->stream>>>((const ST*)X, N, Npad, k, XA);
    sB = op == BSE_OP_A ? 0.0 : (op == BSE_OP_MPLUS ? 1.0 : -1.0);
    xb = nullptr;  // conj(XA)
  }
  launch_rowblock<ST, R>(h->dprobs, 0, q.nT, XA, xb, (int)Npad, sB, U, (int)Npad, kc,
                         hasB && op != BSE_OP_A, h->stream);
  count_launch();
  k_hz_out<ST, CT><<<dim3((unsigned)((N + 255) / 256), k), 256, 0, h->stream>>>(U, N, Npad, k, op, (ST*)Y);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return BSE_OK;
}

template <typename ST>
int backward_impl(bse_handle* h, const double* g, int where, void* dA, void* dB) {
  using R = typename std::conditional<std::is_same<ST, float2>::value, float, double>::type;
  ProbHost& q = h->p[0];
  const int k = q.nconv;
  if (k == 0) return BSE_ESTATE;
  std::vector<double> gh(h->nev), gz(k, 0.0);
  if (where == BSE_DEVICE) {
    CK(cudaMemcpyAsync(gh.data(), g, sizeof(double) * h->nev, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } else {
    std::memcpy(gh.data(), g, sizeof(double) * h->nev);
  }
  std::vector<int> perm(k);
  CK(cudaMemcpy(perm.data(), q.perm, sizeof(int) * k, cudaMemcpyDeviceToHost));
  for (int c = 0; c < k; ++c) gz[perm[c]] = gh[c];
  int rc;
  if (!h->gdev && (rc = dalloc((void**)&h->gdev, sizeof(double) * MAXM))) return rc;
  CK(cudaMemcpyAsync(h->gdev, gz.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
  if (!h->adj_tiles) {
    const int nb = (int)((q.N + 63) / 64);
    std::vector<int2> t;
    t.reserve((size_t)nb * (nb + 1) / 2);
    for (int I = 0; I < nb; ++I)
      for (int J = I; J < nb; ++J) t.push_back(make_int2(I, J));
    h->adj_ntiles = (int64_t)t.size();
    if ((rc = dalloc((void**)&h->adj_tiles, sizeof(int2) * t.size()))) return rc;
    CK(cudaMemcpyAsync(h->adj_tiles, t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice, h->stream));
  }
  const int64_t ldz = h->ph ? 2 * q.Npad : q.Npad;
  launch_adjoint2<ST, R>(q.Z, ldz, q.Npad, q.N, k, h->gdev, h->ph, h->adj_tiles, h->adj_ntiles, (ST*)dA,
                         (ST*)dB, h->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return BSE_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* bse_strerror(int status) {
  switch (status) {
    case BSE_OK: return "success";
    case BSE_EINVAL: return "invalid argument";
    case BSE_ENOMEM: return "out of memory";
    case BSE_ENOTPD: return "M is not positive definite (the spectrum of H need not be real)";
    case BSE_ENOCONV: return "fewer than nev eigenpairs converged within maxit Krylov steps";
    case BSE_ETIMEOUT: return "device-side iteration limit expired";
    case BSE_ECUDA: return "CUDA runtime error";
    case BSE_ESTATE: return "call out of order (no completed solve)";
    case BSE_ENOTFINITE: return "NaN or Inf in the Lanczos coefficients";
  }
  return "unknown status";
}

int bse_create_batched(int count, const int64_t* N, const void* const* A, const void* const* B, int form,
                       int dtype, int where, void* stream, bse_handle** out) {
  if (!out) return BSE_EINVAL;
  *out = nullptr;
  if (count < 1 || !N || !A) return BSE_EINVAL;
  if (form != BSE_TDA && form != BSE_PH) return BSE_EINVAL;
  if (dtype != BSE_C64 && dtype != BSE_C128 && dtype != BSE_C64_MIXED && dtype != BSE_C128_DF)
    return BSE_EINVAL;
  if (where != BSE_HOST && where != BSE_DEVICE) return BSE_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (N[i] < 1 || N[i] > 2147483647LL || !A[i]) return BSE_EINVAL;
    if (form == BSE_PH && (!B || !B[i])) return BSE_EINVAL;
  }
  bse_handle* h = new (std::nothrow) bse_handle();
  if (!h) return BSE_ENOMEM;
  h->count = count;
  h->form = form;
  h->dtype = dtype;
  h->ph = form == BSE_PH;
  h->df = dtype == BSE_C128_DF || dtype == BSE_C64_MIXED;
  h->split = dtype == BSE_C128_DF;
  h->tiles64 = is_c64(dtype);
  h->es = is_c64(dtype) ? sizeof(float2) : sizeof(double2);   // stored (tile / caller) elements
  h->vs = dtype == BSE_C64 ? sizeof(float2) : sizeof(double2);  // Krylov vectors
  h->stream = (cudaStream_t)stream;
  h->p.resize(count);
  h->hstate.resize(count);
  std::vector<TileJob> jobs;
  int rc = BSE_OK;
  for (int i = 0; i < count && rc == BSE_OK; ++i) {
    ProbHost& q = h->p[i];
    q.N = N[i];
    q.nT = (int)((q.N + TS - 1) / TS);
    q.Npad = (int64_t)q.nT * TS;
    q.ntiles = (int64_t)q.nT * (q.nT + 1) / 2;
    h->maxnT = std::max(h->maxnT, q.nT);
    h->maxNpad = std::max(h->maxNpad, q.Npad);
    h->maxnrb = std::max(h->maxnrb, nrb_of(q.Npad));
    const size_t bytes = h->es * (size_t)q.ntiles * TS * TS;
    if ((rc = dalloc(&q.A, bytes))) break;
    if (h->ph && (rc = dalloc(&q.B, bytes))) break;
    if (is_c64(dtype)) {
      rc = pack_matrix<float2>(h, (const float2*)A[i], q.N, q.nT, 1, where, (float2*)q.A);
      if (!rc && h->ph) rc = pack_matrix<float2>(h, (const float2*)B[i], q.N, q.nT, 0, where, (float2*)q.B);
    } else {
      rc = pack_matrix<double2>(h, (const double2*)A[i], q.N, q.nT, 1, where, (double2*)q.A);
      if (!rc && h->ph) rc = pack_matrix<double2>(h, (const double2*)B[i], q.N, q.nT, 0, where, (double2*)q.B);
      if (!rc && h->df) {
        const int64_t nel = q.ntiles * TS * TS;
        if (!(rc = dalloc(&q.Ahl, sizeof(float4) * (size_t)nel)))
          launch_split_tiles((const double2*)q.A, nel, (float4*)q.Ahl, h->stream);
        if (!rc && h->ph && !(rc = dalloc(&q.Bhl, sizeof(float4) * (size_t)nel)))
          launch_split_tiles((const double2*)q.B, nel, (float4*)q.Bhl, h->stream);
      }
    }
    for (int I = 0; I < q.nT; ++I)
      for (int J = I; J < q.nT; ++J) {
        TileJob t;
        t.prob = i;
        t.I = I;
        t.J = J;
        t.t = (int)((int64_t)I * q.nT - (int64_t)I * (I - 1) / 2 + (J - I));
        jobs.push_back(t);
      }
  }
  if (rc == BSE_OK && jobs.size() > 2147483647ull) rc = BSE_EINVAL;
  if (rc == BSE_OK) {
    h->njobs = (int)jobs.size();
    rc = dalloc((void**)&h->djobs, sizeof(TileJob) * jobs.size());
  }
  if (rc == BSE_OK && cudaMemcpyAsync(h->djobs, jobs.data(), sizeof(TileJob) * jobs.size(),
                                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    rc = BSE_ECUDA;
  if (rc == BSE_OK) rc = dalloc((void**)&h->dprobs, sizeof(Prob) * count);
  if (rc == BSE_OK) rc = dalloc((void**)&h->dstate, sizeof(KState) * count);
  if (rc == BSE_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = BSE_ECUDA;
  if (rc != BSE_OK) {
    bse_destroy(h);
    return rc;
  }
  *out = h;
  return BSE_OK;
}

int bse_create(int64_t N, const void* A, const void* B, int form, int dtype, int where, void* stream,
               bse_handle** out) {
  const void* a[1] = {A};
  const void* b[1] = {B};
  return bse_create_batched(1, &N, a, form == BSE_PH ? b : nullptr, form, dtype, where, stream, out);
}

int bse_solve_ex(bse_handle* h, int nev, double tol, int which, const bse_solve_opts* opts, double* eval_out,
                 void* evec_out, int* nconv_out) {
  if (!h || which != BSE_LOWEST) return BSE_EINVAL;
  if (h->count != 1) return BSE_EINVAL;
  void* const ev[1] = {evec_out};
  if (h->vs == sizeof(float2)) return solve_impl<float2>(h, nev, tol, opts, eval_out, ev, nconv_out);
  return solve_impl<double2>(h, nev, tol, opts, eval_out, ev, nconv_out);
}

int bse_solve(bse_handle* h, int nev, double tol, int which, double* eval_out, void* evec_out, int* nconv_out) {
  return bse_solve_ex(h, nev, tol, which, nullptr, eval_out, evec_out, nconv_out);
}

int bse_solve_batched(bse_handle* h, int nev, double tol, int which, const bse_solve_opts* opts,
                      double* eval_out, void* const* evec_out, int* nconv_out) {
  if (!h || which != BSE_LOWEST) return BSE_EINVAL;
  if (h->vs == sizeof(float2)) return solve_impl<float2>(h, nev, tol, opts, eval_out, evec_out, nconv_out);
  return solve_impl<double2>(h, nev, tol, opts, eval_out, evec_out, nconv_out);
}

int bse_backward(bse_handle* h, const double* dL_dlambda, int where, void* dA, void* dB) {
  if (!h || !dL_dlambda || !dA) return BSE_EINVAL;
  if (where != BSE_HOST && where != BSE_DEVICE) return BSE_EINVAL;
  if (h->count != 1) return BSE_EINVAL;
  if (h->ph && !dB) return BSE_EINVAL;
  if (!h->ph && dB) return BSE_EINVAL;
  if (!h->solved) return BSE_ESTATE;
  if (is_c64(h->dtype)) return backward_impl<float2>(h, dL_dlambda, where, dA, dB);
  return backward_impl<double2>(h, dL_dlambda, where, dA, dB);
}

int bse_apply(bse_handle* h, int op, int k, const void* X, void* Y) {
  if (!h || !X || !Y || k < 1 || h->count != 1) return BSE_EINVAL;
  if (op < BSE_OP_A || op > BSE_OP_H) return BSE_EINVAL;
  if (is_c64(h->dtype)) return apply_impl<float2>(h, op, k, X, Y);
  return apply_impl<double2>(h, op, k, X, Y);
}

int bse_get_stats(const bse_handle* h, bse_stats* out) {
  if (!h || !out) return BSE_EINVAL;
  *out = h->stats;
  return BSE_OK;
}

int bse_destroy(bse_handle* h) {
  if (!h) return BSE_EINVAL;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& q : h->p) {
    free_solve_buffers(q);
    free_results(q);
    dfree(q.A);
    dfree(q.B);
    dfree(q.Ahl);
    dfree(q.Bhl);
  }
  dfreet(h->dprobs);
  dfreet(h->dstate);
  dfreet(h->djobs);
  dfree(h->post);
  dfreet(h->adj_tiles);
  dfreet(h->gdev);
  for (auto& e : h->ev) cudaEventDestroy(e);
  delete h;
  return BSE_OK;
}

}  // extern "C"
