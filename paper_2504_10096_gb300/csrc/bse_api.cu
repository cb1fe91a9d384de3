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
#include <map>
#include <mutex>
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
  float* tmax = nullptr;   // mixed PH path: per-tile bound on |U|, |V| (device)
  void* UV = nullptr;      // mixed PH path: {U_re, V_re, U_im, V_im} records of the packed tiles
  std::vector<float> htmax;
  float tref = 0.f;        // the largest of them
  // solve buffers
  int ncv = 0;
  void *V = nullptr, *P = nullptr, *V2 = nullptr, *P2 = nullptr, *w = nullptr, *pw = nullptr;
  void* part = nullptr;
  void* xs = nullptr;        // mixed PH path: pre-split product vector and chunk maxima
  float* xmax = nullptr;
  double *cpart = nullptr, *coef = nullptr, *small = nullptr, *S = nullptr;
  // Gruning variant: odd basis W, Z = M- W, their restart scratch, the projected tree and the
  // odd-side Ritz coefficients (allocated by the first solve that asks for the variant)
  void *W = nullptr, *Z2 = nullptr, *Zo = nullptr, *W2 = nullptr;
  double *jw = nullptr, *S2 = nullptr;
  // mixed PH path: double-FP32 shadows of V, P and w for the Gram-Schmidt passes
  float4 *Vs = nullptr, *Ps = nullptr, *ws = nullptr;
  // results
  double2* Z = nullptr;
  int zcols = 0;
  int nconv = 0;
  int* perm = nullptr;   // device, output column -> Z column
  std::vector<double> eval, res;
};

// A CUDA graph of 2^b consecutive Krylov steps.  The step kernels read the
// per-problem state on the device and do nothing once a problem's subspace
// is full, so one captured sequence serves every cycle of a solve.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;            // kernels per replay
  std::vector<cudaEvent_t> ev;       // product start/stop pairs recorded by the graph
  bool pending = false;              // replayed since the events were last read
};

constexpr int kMaxGraphLog = 10;     // 2^10 = MAXM steps

// Launch-shape tuner of the structured product.  While a handle is untuned,
// its successive products (the solver's own, no extra work) cycle through
// the candidate shapes; each product is timed by the CUDA events that also
// feed bse_stats.  Once every candidate has kTuneSamples timings after its
// first one, the shape with the lowest mean is kept for the handle and, keyed
// by kernel variant, tile-job count and problem count, for later handles.
constexpr int kTuneSamples = 3;

struct TuneKey {
  int variant, njobs, count;
  bool operator<(const TuneKey& o) const {
    if (variant != o.variant) return variant < o.variant;
    if (njobs != o.njobs) return njobs < o.njobs;
    return count < o.count;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, ProdShape> g_tuned;

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
  std::vector<TileJob> hjobs;
  // mixed PH path: the tile jobs split by precision for the current solve
  bool mixed = false;        // BSE_C64_MIXED with B
  TileJob* djobs_fine = nullptr;
  TileJob* djobs_coarse = nullptr;
  int njobs_fine = 0, njobs_coarse = 0;
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
  int2* adj_tiles128 = nullptr;   // tensor-core adjoint
  int64_t adj_ntiles128 = 0;
  void* adj_panels = nullptr;
  size_t adj_panel_bytes = 0;
  int* adj_err = nullptr;
  int* prod_err = nullptr;   // raised by a product kernel whose bounded wait expired
  double* gdev = nullptr;
  // product timing ring
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  double ms_product = 0.0;
  // product launch shape and its tuner state
  ProdShape shape{0, 0};
  bool tuned = false;
  TuneKey tkey{};
  std::vector<ProdShape> cands;
  std::vector<double> tsum;
  std::vector<int> tcnt, tseen;
  int tnext = 0;
  std::vector<int> ev_tag;   // candidate timed by each pair of the ring (-1: none)
  // step graphs (valid for one subspace size) and the stream they are captured on
  StepGraph sg[kMaxGraphLog + 1];
  StepGraph rg;              // the restart sequence (Ritz pairs, lock decision, restart)
  int sg_ncv = 0;
  bool graphs = true;
  cudaStream_t cap = nullptr;
  // structure-preserving variant of the current solve (PH handles) and the scratch of the
  // projected-BSE variant's dense solves
  int variant = 0;
  int sg_variant = 0;        // variant of the captured graphs
  // persistent steps (one cooperative launch per restart cycle) for one small problem, and
  // the grid barrier they meet at
  bool persist = true;
  GridBar* gbar = nullptr;
  double* pj_work = nullptr;
  size_t pj_doubles = 0;
  int* pj_flag = nullptr;
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
  dfree(q.V); dfree(q.P); dfree(q.V2); dfree(q.P2); dfree(q.w); dfree(q.pw); dfree(q.part); dfree(q.xs);
  dfreet(q.xmax);
  dfreet(q.cpart); dfreet(q.coef); dfreet(q.small); dfreet(q.S);
  dfree(q.W); dfree(q.Zo); dfree(q.W2); dfree(q.Z2); dfreet(q.jw); dfreet(q.S2);
  dfreet(q.Vs); dfreet(q.Ps); dfreet(q.ws);
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
    launch_pack_all<T, T>(src, N, nT, herm, dst, h->stream);
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
  cudaStream_t s;                          // the handle's stream, or the capture stream
  std::vector<cudaEvent_t>* cap_ev = nullptr;   // events of the graph being captured
  size_t cap_n = 0;
  explicit Driver(bse_handle* hh) : h(hh), s(hh->stream) {}

  void product(int mode) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ProdShape shape = h->shape;
    int tag = -1;
    if (!h->tuned && !cap_ev && !h->cands.empty()) {
      tag = h->tnext++ % (int)h->cands.size();
      shape = h->cands[tag];
    }
    if (cap_ev) {
      if (cap_n + 2 <= cap_ev->size()) {
        e0 = (*cap_ev)[cap_n];
        e1 = (*cap_ev)[cap_n + 1];
        cap_n += 2;
        cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
      }
    } else if (h->ev_used + 2 <= (int)h->ev.size()) {
      e0 = h->ev[h->ev_used];
      e1 = h->ev[h->ev_used + 1];
      h->ev_tag[h->ev_used / 2] = tag;
      h->ev_used += 2;
      cudaEventRecord(e0, s);
    }
    if (h->mixed)
      launch_product_mixed(h->dprobs, h->djobs_fine, h->njobs_fine, h->djobs_coarse, h->njobs_coarse, h->count,
                           h->maxnT, mode, nullptr, shape, h->prod_err, s);
    else if (h->df)
      launch_product_df(h->dprobs, h->djobs, h->njobs, h->count, h->maxnT, mode, nullptr, h->ph != 0, h->split,
                        shape, s);
    else
      launch_product<ST, R>(h->dprobs, h->djobs, h->njobs, h->count, h->maxnT, mode, 1, nullptr, h->ph != 0,
                            shape, s);
    if (e1) {
      if (cap_ev) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
      else cudaEventRecord(e1, s);
    }
  }

  static double elapsed(const std::vector<cudaEvent_t>& ev, size_t n) {
    double sum = 0.0;
    for (size_t i = 0; i + 1 < n; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) sum += ms;
    }
    return sum;
  }

  void harvest_events() {
    for (int i = 0; i + 1 < h->ev_used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) != cudaSuccess) continue;
      h->ms_product += ms;
      const int tag = h->ev_tag[i / 2];
      if (tag >= 0 && !h->tuned && h->tseen[tag]++ > 0) {   // the first timing of a shape is a warm-up
        h->tsum[tag] += ms;
        h->tcnt[tag] += 1;
      }
    }
    h->ev_used = 0;
    if (!h->tuned && !h->cands.empty() &&
        *std::min_element(h->tcnt.begin(), h->tcnt.end()) >= kTuneSamples) {
      int best = 0;
      for (int c = 1; c < (int)h->cands.size(); ++c)
        if (h->tsum[c] / h->tcnt[c] < h->tsum[best] / h->tcnt[best]) best = c;
      h->shape = h->cands[best];
      h->tuned = true;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[h->tkey] = h->shape;
    }
    for (StepGraph& g : h->sg) {
      if (!g.pending) continue;
      h->ms_product += elapsed(g.ev, g.ev.size());
      g.pending = false;
    }
  }

  bool gruning() const { return h->ph && h->variant == VAR_GRUNING; }

  void cgs(int pass, int half = 0) {
    const int ncol = h->ncv + 1 + h->ncv;
    launch_step_cgs<ST>(h->dprobs, h->count, h->ph, h->maxnrb, h->maxNpad, ncol, pass, half, h->mixed && h->ph,
                        s);
  }

  void normalize(int start, int half, cudaStream_t st) {
    launch_step_normalize<ST>(h->dprobs, h->count, h->ph, h->maxnrb, h->maxNpad, start, half, st);
  }

  void step() {
    if (gruning()) {
      // odd half: r = p_j against W and i V, pw = M- r, alpha_j, w_j = r / alpha_j, z_j
      cgs(0, 1);
      cgs(1, 1);
      product(PM_STEP_MMINUS_W);
      normalize(0, 1, s);
      // even half: s = z_j against V and i W, pw = M+ s, beta_j, u_{j+1}, p_{j+1}
      cgs(0, 2);
      cgs(1, 2);
      product(PM_STEP_MPLUS);
      normalize(0, 2, s);
      return;
    }
    product(h->ph ? PM_STEP_MMINUS : PM_STEP_A);
    cgs(0);
    cgs(1);
    if (h->ph) product(PM_STEP_MPLUS);
    normalize(0, 0, s);
  }

  // record 2^b steps into h->sg[b]; false (and graphs off for the handle)
  // when capture or instantiation is refused
  bool capture(int b) {
    StepGraph& g = h->sg[b];
    const int n = 1 << b;
    const size_t nev = (size_t)(h->ph ? 4 : 2) * n;
    while (g.ev.size() < nev) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); h->graphs = false; return false; }
      g.ev.push_back(e);
    }
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      h->cap = nullptr;
      h->graphs = false;
      return false;
    }
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      h->graphs = false;
      return false;
    }
    const long long c0 = launch_counter();
    s = h->cap;
    cap_ev = &g.ev;
    cap_n = 0;
    for (int i = 0; i < n; ++i) step();
    s = h->stream;
    cap_ev = nullptr;
    g.launches = launch_counter() - c0;
    launch_counter() = c0;                  // counted again at every replay
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g.exec = nullptr;
      h->graphs = false;
      return false;
    }
    return true;
  }

  // `steps` Krylov steps: graphs of 2^b steps for the binary digits of
  // `steps` (each replayed at most once per cycle, so every event pair of a
  // replay is read before it is recorded again), or plain launches
  int run_steps(int steps) {
    if (!h->tuned) {                       // shapes still being compared: one launch at a time
      for (; steps > 0; --steps) step();
      return BSE_OK;
    }
    if (persistent_ok()) {
      const int rc = run_steps_persistent(steps);
      if (rc == 0) return BSE_OK;
      if (rc != 1) return rc;
      h->persist = false;                  // not available on this device: graphs from now on
    }
    if (h->graphs && h->sg_ncv != h->ncv) {
      drop_graphs();
      h->sg_ncv = h->ncv;
    }
    for (int b = kMaxGraphLog; b >= 0 && steps > 0; --b) {
      const int n = 1 << b;
      if (steps < n) continue;
      StepGraph& g = h->sg[b];
      if (h->graphs && (g.exec || capture(b)) && cudaGraphLaunch(g.exec, h->stream) == cudaSuccess) {
        launch_counter() += g.launches;
        g.pending = true;
      } else {
        cudaGetLastError();
        for (int i = 0; i < n; ++i) step();
      }
      steps -= n;
    }
    for (; steps > 0; --steps) step();     // only when steps >= 2^(kMaxGraphLog+1)
    return BSE_OK;
  }

  void restart_seq(cudaStream_t st) {
    launch_ritz(h->dprobs, h->count, h->ncv, gruning(), st);
    launch_lock_decide_form(h->dprobs, h->count, h->ph, st);
    launch_restart<ST>(h->dprobs, h->count, h->ph, h->maxNpad, h->ncv, gruning(), h->mixed, st);
  }

  // projected-BSE variant: each active problem's projected matrix goes through the dense
  // structure-preserving solver (sizes from the Krylov state just read), then the same lock
  // decision and restart as the folded iteration; launched on the stream, not captured
  int run_restart_projected() {
    for (int i = 0; i < h->count; ++i) {
      const KState& st = h->hstate[i];
      if (st.done || st.status != ST_OK) continue;
      const int n = st.m - st.k;
      const int nw = std::min(st.r_pkeep - st.k, n);
      const int rc = projected_ritz(h->dprobs, i, n, nw, h->pj_work, h->pj_flag, h->stream);
      if (rc < 0) return BSE_ECUDA;
    }
    launch_lock_decide_form(h->dprobs, h->count, h->ph, h->stream);
    launch_restart<ST>(h->dprobs, h->count, h->ph, h->maxNpad, h->ncv, false, h->mixed, h->stream);
    CK(cudaGetLastError());
    return BSE_OK;
  }

  // the restart sequence reads every decision from KState, so it replays as
  // one graph too (captured with the step graphs, for one subspace size)
  void run_restart() {
    if (h->graphs && h->sg_ncv != h->ncv) {
      drop_graphs();
      h->sg_ncv = h->ncv;
    }
    StepGraph& g = h->rg;
    if (h->graphs && !g.exec && (h->cap || cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) == cudaSuccess) &&
        cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      const long long c0 = launch_counter();
      restart_seq(h->cap);
      g.launches = launch_counter() - c0;
      launch_counter() = c0;
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) g.exec = nullptr;
    }
    cudaGetLastError();
    if (h->graphs && g.exec && cudaGraphLaunch(g.exec, h->stream) == cudaSuccess) {
      launch_counter() += g.launches;
      return;
    }
    cudaGetLastError();
    restart_seq(h->stream);
  }

  // one small problem on the folded (Shao) or TDA recurrence with the plain FP64 / FP32
  // products: its steps run as one persistent launch per cycle
  static constexpr int64_t kPersistMaxNpad = 6144;
  bool persistent_ok() const {
    return h->persist && h->count == 1 && !h->mixed && !h->df && (!h->ph || h->variant == VAR_SHAO) &&
           h->p[0].Npad <= kPersistMaxNpad;
  }

  // 0: launched; 1: not available (the caller falls back); BSE_ECUDA/ENOMEM on errors
  int run_steps_persistent(int steps) {
    if (!h->gbar) {
      const int rc = dalloc((void**)&h->gbar, sizeof(GridBar));
      if (rc) return rc;
    }
    const int r = launch_steps_persist<ST, R>(h->dprobs, h->djobs, h->njobs, h->ph != 0, steps, h->gbar, h->stream);
    if (r < 0) return BSE_ECUDA;
    return r;
  }

  void drop_graphs() {
    for (StepGraph& g : h->sg) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
      g.pending = false;
    }
    if (h->rg.exec) cudaGraphExecDestroy(h->rg.exec);
    h->rg.exec = nullptr;
  }

  void fresh_chain(uint64_t seed, const void* v0) {
    // a fresh vector is even on the Gruning path: against V and the twins i W
    const int half = gruning() ? 2 : 0;
    launch_start_vector<ST>(h->dprobs, h->count, h->maxNpad, seed, v0, h->stream);
    cgs(2, half);
    cgs(3, half);
    if (h->ph) product(PM_START_MPLUS);
    normalize(1, half, h->stream);
  }

  int read_state() {
    CK(cudaMemcpyAsync(h->hstate.data(), h->dstate, sizeof(KState) * h->count, cudaMemcpyDeviceToHost,
                       h->stream));
    int perr = 0;
    GridBar gb{};
    if (h->prod_err) CK(cudaMemcpyAsync(&perr, h->prod_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (h->gbar) CK(cudaMemcpyAsync(&gb, h->gbar, sizeof(GridBar), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    harvest_events();
    return (perr || gb.err) ? BSE_ETIMEOUT : BSE_OK;
  }

  int iterate(uint64_t seed, const void* v0) {
    fresh_chain(seed, v0);
    int guard = 0;
    long long cycles = 0;
    long long maxit = 0;
    for (int i = 0; i < h->count; ++i) maxit = std::max(maxit, h->hstate[i].maxit);
    for (;;) {
      // every pass of this loop either adds Krylov steps or restarts; a pass
      // without progress cannot repeat more often than this bound
      if (++cycles > 4 * maxit + 4096) return BSE_ETIMEOUT;
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
        if ((rc = run_steps(steps))) return rc;
        continue;
      }
      if (h->ph && h->variant == VAR_PROJECTED) {
        if ((rc = run_restart_projected())) return rc;
        continue;
      }
      run_restart();
    }
    return BSE_OK;
  }

  // result buffers of problem i for k pairs
  int alloc_results(int i, int k) {
    ProbHost& q = h->p[i];
    free_results(q);
    q.nconv = k;
    q.eval.assign(k, 0.0);
    q.res.assign(k, 0.0);
    if (k == 0) return BSE_OK;
    const int64_t ldz = h->ph ? 2 * q.Npad : q.Npad;
    int rc = dalloc((void**)&q.Z, sizeof(double2) * (size_t)ldz * k);
    if (rc) return rc;
    rc = dalloc((void**)&q.perm, sizeof(int) * k);
    if (rc) return rc;
    q.zcols = k;
    return BSE_OK;
  }

  // recover eigenvectors, FP64 residuals and Rayleigh quotients of problem i;
  // a pair counts as converged only if its FP64 relative residual is <= tol
  int finalize(int i, int nev, double tol) {
    const KState& s = h->hstate[i];
    const int k = std::min(s.k, nev);
    int rc = alloc_results(i, k);
    if (rc || k == 0) return rc;
    return finish(i, k, tol, true);
  }

  // Omega- (or 2-) normalise the k columns of Z (recovered from the Krylov basis first when
  // `recover`), FP64 products H z, Rayleigh quotients, residuals, output order
  int finish(int i, int k, double tol, bool recover) {
    ProbHost& q = h->p[i];
    const int64_t Npad = q.Npad;
    const int64_t ldz = h->ph ? 2 * Npad : Npad;
    int rc;
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
    if (recover) launch_recover<ST>(h->dprobs, i, h->ph, Npad, q.N, k, q.Z, (int)ldz, h->stream);
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
    int good = 0;
    for (int c = 0; c < k; ++c) {
      q.eval[c] = hr[perm[c]];
      q.res[c] = hres[perm[c]];
      if (q.res[c] <= tol) ++good;      // NaN residuals never count
    }
    q.nconv = good;
    CK(cudaMemcpyAsync(q.perm, perm.data(), sizeof(int) * k, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return BSE_OK;
  }

  int store(int i, void* out) {
    ProbHost& q = h->p[i];
    if (!out || q.zcols == 0) return BSE_OK;
    const int64_t ldz = h->ph ? 2 * q.Npad : q.Npad;
    const int64_t ldo = h->ph ? 2 * q.N : q.N;
    if (is_c64(h->dtype))   // caller-facing vectors in the handle's dtype
      launch_store_vectors2<float2>(q.Z, ldz, q.Npad, q.N, h->ph, q.zcols, q.perm, (float2*)out, ldo, h->stream);
    else
      launch_store_vectors2<double2>(q.Z, ldz, q.Npad, q.N, h->ph, q.zcols, q.perm, (double2*)out, ldo,
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
    const int ncol = 2 * ncv + 1;          // stride of the CGS partial sums and coefficients
    const int nbas = ncv + 1;              // basis columns of V and P
    const int nrb = nrb_of(q.Npad);
    int rc;
    if ((rc = dalloc(&q.V, es * (size_t)q.Npad * nbas))) return rc;
    if (h->ph && (rc = dalloc(&q.P, es * (size_t)q.Npad * nbas))) return rc;
    if ((rc = dalloc(&q.V2, es * (size_t)q.Npad * ncv))) return rc;
    if (h->ph && (rc = dalloc(&q.P2, es * (size_t)q.Npad * ncv))) return rc;
    if ((rc = dalloc(&q.w, es * (size_t)q.Npad))) return rc;
    if ((rc = dalloc(&q.pw, es * (size_t)q.Npad))) return rc;
    if ((rc = dalloc(&q.part, cs * (size_t)q.nT * q.nT * TS))) return rc;
    if (h->mixed) {
      if ((rc = dalloc(&q.xs, sizeof(float4) * (size_t)q.Npad))) return rc;
      if ((rc = dalloc((void**)&q.Vs, sizeof(float4) * (size_t)q.Npad * nbas))) return rc;
      if ((rc = dalloc((void**)&q.Ps, sizeof(float4) * (size_t)q.Npad * nbas))) return rc;
      if ((rc = dalloc((void**)&q.ws, sizeof(float4) * (size_t)q.Npad))) return rc;
      CK(cudaMemsetAsync(q.Vs, 0, sizeof(float4) * (size_t)q.Npad * nbas, h->stream));
      CK(cudaMemsetAsync(q.Ps, 0, sizeof(float4) * (size_t)q.Npad * nbas, h->stream));
      if ((rc = dalloc((void**)&q.xmax, sizeof(float) * (size_t)q.nT))) return rc;
    }
    if ((rc = dalloc((void**)&q.cpart, sizeof(double2) * (size_t)nrb * ncol))) return rc;
    if ((rc = dalloc((void**)&q.coef, sizeof(double2) * 2 * (size_t)ncol))) return rc;
    if ((rc = dalloc((void**)&q.small, sizeof(double) * 6 * (size_t)(ncv + 1)))) return rc;
    if ((rc = dalloc((void**)&q.S, sizeof(double) * (size_t)ncv * ncv))) return rc;
    CK(cudaMemsetAsync(q.V, 0, es * (size_t)q.Npad * nbas, h->stream));
    if (h->ph) CK(cudaMemsetAsync(q.P, 0, es * (size_t)q.Npad * nbas, h->stream));
    CK(cudaMemsetAsync(q.small, 0, sizeof(double) * 6 * (size_t)(ncv + 1), h->stream));
    CK(cudaMemsetAsync(q.S, 0, sizeof(double) * (size_t)ncv * ncv, h->stream));
    q.ncv = ncv;
  }
  if (h->ph && h->variant == VAR_GRUNING) {
    for (int i = 0; i < h->count; ++i) {
      ProbHost& q = h->p[i];
      if (q.W) continue;
      const size_t vb = es * (size_t)q.Npad * ncv;
      const size_t jwld = 2 * (size_t)ncv + 2;
      int rc;
      if ((rc = dalloc(&q.W, vb)) || (rc = dalloc(&q.Zo, vb)) || (rc = dalloc(&q.W2, vb)) ||
          (rc = dalloc(&q.Z2, vb)) || (rc = dalloc((void**)&q.jw, sizeof(double) * jwld * (4 + (size_t)ncv))) ||
          (rc = dalloc((void**)&q.S2, sizeof(double) * (size_t)ncv * ncv)))
        return rc;
      CK(cudaMemsetAsync(q.W, 0, vb, h->stream));
      CK(cudaMemsetAsync(q.Zo, 0, vb, h->stream));
      CK(cudaMemsetAsync(q.S2, 0, sizeof(double) * (size_t)ncv * ncv, h->stream));
    }
  }
  if (h->ph && h->variant == VAR_PROJECTED) {
    const size_t need = (dense_scratch_doubles(ncv, ncv) + 31) / 32 * 32 + projected_scratch_doubles(ncv, ncv);
    if (need > h->pj_doubles) {
      dfreet(h->pj_work);
      h->pj_doubles = 0;
      int rc = dalloc((void**)&h->pj_work, sizeof(double) * need);
      if (rc) return rc;
      h->pj_doubles = need;
    }
    if (!h->pj_flag) {
      int rc = dalloc((void**)&h->pj_flag, sizeof(int));
      if (rc) return rc;
    }
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
    d.tmax = q.tmax;
    d.UV = q.UV;
    d.xs = q.xs;
    d.xmax = q.xmax;
    d.variant = h->ph ? h->variant : VAR_SHAO;
    d.W = q.W; d.Z = q.Zo; d.W2 = q.W2; d.Z2 = q.Z2;
    d.jw = q.jw;
    d.jwld = 2 * q.ncv + 2;
    d.S2 = q.S2;
    d.Vs = q.Vs; d.Ps = q.Ps; d.ws = q.ws;
  }
  CK(cudaMemcpyAsync(h->dprobs, h->hprobs.data(), sizeof(Prob) * h->count, cudaMemcpyHostToDevice,
                     h->stream));
  return BSE_OK;
}

// Mixed PH path: split the tile jobs by precision for a solve at `tol`.  A
// tile is "coarse" -- U, V rounded to FP32 and products accumulated on a
// fixed-point grid (k_prod_tiles_mx) -- when its bound on |U|, |V| is at most
// tau times the largest bound of its problem; the others ("fine") get exact
// double-FP32 products (k_prod_tiles_df2).  The rounding of U, V on coarse
// tiles is a fixed perturbation of at most 2^-24 tau max|U| per entry; with
// random signs its 2-norm grows like 2 sqrt(N) times that, and the default
// tau = min(2^-7, tol 2^24 / (16 sqrt(N))) keeps it near tol / 8 of the
// largest entry.  tau < 0 puts every tile on the exact path.
double default_tile_tau(double tol, int64_t N) {
  return std::min(std::ldexp(1.0, -7), tol * std::ldexp(1.0, 24) / (16.0 * std::sqrt((double)N)));
}

int split_mixed_jobs(bse_handle* h, double tol, double tau_opt) {
  std::vector<TileJob> fine, coarse;
  fine.reserve(h->hjobs.size());
  coarse.reserve(h->hjobs.size());
  for (const TileJob& j : h->hjobs) {
    const ProbHost& q = h->p[j.prob];
    const double tau = tau_opt != 0.0 ? tau_opt : default_tile_tau(tol, q.N);
    const bool exact = tau < 0.0 || !(q.htmax[j.t] <= tau * q.tref);
    (exact ? fine : coarse).push_back(j);
  }
  if (!h->djobs_fine) {
    int rc = dalloc((void**)&h->djobs_fine, sizeof(TileJob) * h->hjobs.size());
    if (!rc) rc = dalloc((void**)&h->djobs_coarse, sizeof(TileJob) * h->hjobs.size());
    if (rc) return rc;
  }
  h->njobs_fine = (int)fine.size();
  h->njobs_coarse = (int)coarse.size();
  if (!fine.empty())
    CK(cudaMemcpyAsync(h->djobs_fine, fine.data(), sizeof(TileJob) * fine.size(), cudaMemcpyHostToDevice, h->stream));
  if (!coarse.empty())
    CK(cudaMemcpyAsync(h->djobs_coarse, coarse.data(), sizeof(TileJob) * coarse.size(), cudaMemcpyHostToDevice,
                       h->stream));
  CK(cudaStreamSynchronize(h->stream));    // the host vectors go out of scope
  return BSE_OK;
}

template <typename ST>
int solve_impl(bse_handle* h, int nev, double tol, const bse_solve_opts* opts, double* eval_out,
               void* const* evec_out, int* nconv_out) {
  int64_t minN = h->p[0].N, maxN = h->p[0].N;
  for (auto& q : h->p) {
    minN = std::min(minN, q.N);
    maxN = std::max(maxN, q.N);
  }
  if (nev < 1 || nev > minN || !(tol > 0.0) || !eval_out) return BSE_EINVAL;
  int ncv = opts && opts->ncv > 0 ? opts->ncv : std::max(2 * nev, nev + 32);
  // a restart keeps at least nev vectors, so a cycle adds a new Lanczos
  // vector only when m > nev; m = nev is allowed only when it is the whole
  // space (m = N) of every problem, where one cycle is exact.  The subspace
  // never exceeds the smallest N: the Krylov space of one start vector has
  // dimension <= N (on the pseudo-Hermitian path every omega^2 of the folded
  // operator is double, one chain sees one copy, and the projection onto the
  // twins' space keeps the other copy out).
  if (ncv < nev + 1) ncv = nev + 1;
  const int64_t cap = std::min<int64_t>(minN, MAXM);
  if (ncv > cap) ncv = (int)cap;
  const bool whole = ncv == minN && minN == maxN;
  if (ncv < nev || (ncv < nev + 1 && !whole)) return BSE_EINVAL;
  const long long maxit = opts && opts->maxit > 0 ? opts->maxit : 20000;
  const uint64_t seed = opts && opts->seed ? opts->seed : 12345ull;
  const double lock_tol = opts && opts->lock_tol > 0.0 ? opts->lock_tol : tol * 0.25;
  const void* v0 = (opts && h->count == 1) ? opts->v0 : nullptr;
  const bool graphs = !(opts && opts->stream_launches == 1);
  h->persist = !(opts && opts->stream_launches);     // 2: graph replay even where steps could persist
  const int variant = opts ? opts->variant : BSE_VARIANT_SHAO;
  if (variant < BSE_VARIANT_SHAO || variant > BSE_VARIANT_PROJECTED) return BSE_EINVAL;
  h->variant = h->ph ? variant : BSE_VARIANT_SHAO;
  if (h->variant != h->sg_variant) {          // the captured graphs hold one variant's kernels
    Driver<ST>(h).drop_graphs();
    h->sg_variant = h->variant;
  }
  int rc = alloc_solve(h, ncv);
  if (rc) return rc;
  const double tau_opt = opts ? opts->tile_tau : 0.0;
  if (h->mixed && (rc = split_mixed_jobs(h, tol, tau_opt))) return rc;
  h->ncv = ncv;
  h->nev = nev;
  h->solved = false;
  for (int i = 0; i < h->count; ++i) {
    KState& s = h->hstate[i];
    std::memset(&s, 0, sizeof(KState));
    s.k = 0; s.l = 0; s.j = -1; s.m = ncv; s.nev = nev;
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
    h->ev_tag.assign(h->ev.size() / 2, -1);
  }
  h->ev_used = 0;
  h->ms_product = 0.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, h->stream);
  const long long launches0 = launch_counter();
  Driver<ST> drv(h);
  h->graphs = graphs;
  rc = drv.iterate(seed, v0);
  if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
  int worst = BSE_OK;
  double maxres = 0.0;
  int64_t steps = 0, passes = 0, restarts = 0;
  int nconv_total = 0;
  for (int i = 0; i < h->count; ++i) {
    rc = drv.finalize(i, nev, tol);
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    const KState& s = h->hstate[i];
    ProbHost& q = h->p[i];
    for (int c = 0; c < nev; ++c) eval_out[(size_t)i * nev + c] = c < (int)q.eval.size() ? q.eval[c] : NAN;
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
  h->stats.shape_ctas_per_sm = h->shape.ctas_per_sm;
  h->stats.shape_strided = h->shape.strided;
  h->stats.tuned = h->tuned ? 1 : 0;
  h->stats.tiles_fine = h->mixed ? h->njobs_fine : h->njobs;
  h->stats.tiles_coarse = h->mixed ? h->njobs_coarse : 0;
  h->stats.retried_exact = 0;
  h->solved = true;
  // the rounded blocks of the coarse tiles are a fixed perturbation of the
  // operator; if a pair then misses tol on the FP64 residual check (and not
  // because of maxit), solve again with every tile on the exact path
  if (h->mixed && h->njobs_coarse > 0 && worst == BSE_ENOCONV) {
    bool maxit_hit = false;
    for (const KState& s : h->hstate) maxit_hit |= s.steps >= s.maxit;
    if (!maxit_hit) {
      bse_solve_opts o{};
      if (opts) o = *opts;
      o.tile_tau = -1.0;
      const int rc2 = solve_impl<ST>(h, nev, tol, &o, eval_out, evec_out, nconv_out);
      h->stats.retried_exact = 1;
      return rc2;
    }
  }
  return worst;
}

// candidate launch shapes of the handle's product kernel (see TuneKey)
void setup_tuner(bse_handle* h) {
  const int occ = h->mixed ? product_mx_occupancy()
                 : h->df  ? product_df_occupancy(h->ph != 0, h->split)
                          : (h->vs == sizeof(float2) ? product_occupancy<float2, float>(h->ph != 0)
                                                     : product_occupancy<double2, double>(h->ph != 0));
  const bool batch = h->count > 1;
  h->cands.clear();
  for (int c = 1; c <= occ; ++c) {
    if (!batch) h->cands.push_back(ProdShape{c, 0});
    h->cands.push_back(ProdShape{c, 1});
  }
  h->cands.push_back(ProdShape{-1, 0});
  const size_t n = h->cands.size();
  h->tsum.assign(n, 0.0);
  h->tcnt.assign(n, 0);
  h->tseen.assign(n, 0);
  h->tnext = 0;
  h->shape = ProdShape{0, batch ? 1 : 0};
  h->tkey = TuneKey{h->dtype * 2 + h->ph, h->njobs, h->count};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(h->tkey);
  h->tuned = it != g_tuned.end();
  if (h->tuned) h->shape = it->second;
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
  // A alone on complex128 PH tiles (P, Q) goes through the row-block kernel, which unpacks A
  const bool pq_a = hasB && op == BSE_OP_A && !h->tiles64;
  if (op != BSE_OP_H && k == 1 && !pq_a) {
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
                        true, h->shape, h->stream);
    else
      launch_product<ST, R>(h->dprobs, h->djobs, h->njobs, 1, h->maxnT, PM_GENERIC, 1, &io,
                            hasB && op != BSE_OP_A, h->shape, h->stream);
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
  // P, Q tiles always go through the unpacking variant (sB = 0 drops the B half)
  launch_rowblock<ST, R>(h->dprobs, 0, q.nT, XA, xb, (int)Npad, sB, U, (int)Npad, kc,
                         hasB && (op != BSE_OP_A || !h->tiles64), h->stream);
  count_launch();
  k_hz_out<ST, CT><<<dim3((unsigned)((N + 255) / 256), k), 256, 0, h->stream>>>(U, N, Npad, k, op, (ST*)Y);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return BSE_OK;
}

template <typename ST>
int backward_impl(bse_handle* h, const double* g, int where, void* dA, void* dB, int impl) {
  using R = typename std::conditional<std::is_same<ST, float2>::value, float, double>::type;
  ProbHost& q = h->p[0];
  const int k = q.zcols;      // every returned pair (converged or not)
  if (k == 0) return BSE_ESTATE;
  std::vector<double> gh(h->nev), gz(k, 0.0);
  if (where == BSE_DEVICE) {
    CK(cudaMemcpyAsync(gh.data(), g, sizeof(double) * h->nev, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } else {
    std::memcpy(gh.data(), g, sizeof(double) * h->nev);
  }
  std::vector<int> perm(k);
  CK(cudaMemcpyAsync(perm.data(), q.perm, sizeof(int) * k, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
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
  const bool tensor = std::is_same<ST, float2>::value && impl != BSE_IMPL_CUDA_CORES;
  if (!tensor) {
    launch_adjoint2<ST, R>(q.Z, ldz, q.Npad, q.N, k, h->gdev, h->ph, h->adj_tiles, h->adj_ntiles, (ST*)dA,
                           (ST*)dB, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return BSE_OK;
  }
  // complex64 outputs: rank-2k update on the tensor cores (3xTF32)
  if (!h->adj_tiles128) {
    const int nb = (int)((q.N + 127) / 128);
    std::vector<int2> t;
    t.reserve((size_t)nb * (nb + 1) / 2);
    for (int I = 0; I < nb; ++I)
      for (int J = I; J < nb; ++J) t.push_back(make_int2(I, J));
    h->adj_ntiles128 = (int64_t)t.size();
    if ((rc = dalloc((void**)&h->adj_tiles128, sizeof(int2) * t.size()))) return rc;
    CK(cudaMemcpyAsync(h->adj_tiles128, t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice, h->stream));
  }
  const size_t pb = adjoint_tc_panel_bytes(q.N, k, h->ph);
  if (pb > h->adj_panel_bytes) {
    dfree(h->adj_panels);
    h->adj_panel_bytes = 0;
    if ((rc = dalloc(&h->adj_panels, pb))) return rc;
    h->adj_panel_bytes = pb;
  }
  if (!h->adj_err && (rc = dalloc((void**)&h->adj_err, sizeof(int)))) return rc;
  const int r = launch_adjoint_tc(q.Z, ldz, q.Npad, q.N, k, h->gdev, h->ph, h->adj_tiles128, h->adj_ntiles128,
                                  (float*)h->adj_panels, h->adj_err, (float2*)dA, (float2*)dB, h->stream);
  if (r < 0) return BSE_ECUDA;
  if (r > 0) return BSE_ETIMEOUT;
  return BSE_OK;
}

// ------------------------------------------------------------------ Haydock spectrum
template <typename ST>
int haydock_impl(bse_handle* h, const void* d, int where, int m, int sign, int nw, const double* omega, double eta,
                 double* spectrum_out, double* response_out, double* coef_out, int* steps_out) {
  using R = typename std::conditional<std::is_same<ST, float2>::value, float, double>::type;
  ProbHost& q0 = h->p[0];
  int rc;
  if (!q0.w || q0.ncv == 0) {      // the product's partial-sum scratch lives with the solve buffers
    if ((rc = alloc_solve(h, std::min<int64_t>(q0.N, 8) > 1 ? (int)std::min<int64_t>(q0.N, 8) : 1))) return rc;
    if ((rc = upload_probs(h))) return rc;
  }
  const int64_t N = q0.N, Npad = q0.Npad;
  const bool ph = h->ph != 0;
  const int np = haydock_partials();
  // one allocation: 6 vectors, partial sums, alpha, beta, state, frequencies, output, staged d
  const size_t vb = sizeof(ST) * (size_t)Npad;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t o_vec = take(6 * vb), o_part = take(sizeof(double) * np), o_al = take(sizeof(double) * m),
               o_be = take(sizeof(double) * m), o_st = take(sizeof(HdState)), o_om = take(sizeof(double) * nw),
               o_out = take(sizeof(double) * 2 * nw), o_d = take(where == BSE_HOST ? sizeof(double2) * N : 0);
  char* buf = nullptr;
  if ((rc = dalloc((void**)&buf, off))) return rc;
  struct Free { char* b; ~Free() { cudaFree(b); } } guard{buf};
  ST* r = (ST*)(buf + o_vec);
  ST* pr = r + Npad;
  ST* w = pr + Npad;
  ST* q = w + Npad;
  ST* qprev = q + Npad;
  ST* p = qprev + Npad;
  double* part = (double*)(buf + o_part);
  double* alpha = (double*)(buf + o_al);
  double* beta = (double*)(buf + o_be);
  HdState* st = (HdState*)(buf + o_st);
  double* om = (double*)(buf + o_om);
  double* out = (double*)(buf + o_out);
  const double2* dd = (const double2*)d;
  cudaStream_t s0 = h->stream;
  if (where == BSE_HOST) {
    CK(cudaMemcpyAsync(buf + o_d, d, sizeof(double2) * N, cudaMemcpyHostToDevice, s0));
    dd = (const double2*)(buf + o_d);
  }
  HdState hs{0, m, 0, 0, 0.0};
  CK(cudaMemcpyAsync(st, &hs, sizeof(HdState), cudaMemcpyHostToDevice, s0));
  CK(cudaMemcpyAsync(om, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, s0));
  const double sK = ph ? (double)sign : 0.0, sK2 = -sK;   // K = M- (s = -1) or M+ (s = +1); K' the other
  auto product = [&](const ST* x, ST* y, double sB, cudaStream_t s) {
    GenericIO io{};
    io.xa = x;
    io.y = y;
    io.sB = sB;
    if (h->df)
      launch_product_df(h->dprobs, h->djobs, h->njobs, 1, h->maxnT, PM_GENERIC, &io, ph, h->split, h->shape, s);
    else
      launch_product<ST, R>(h->dprobs, h->djobs, h->njobs, 1, h->maxnT, PM_GENERIC, 1, &io, ph, h->shape, s);
  };
  auto step = [&](cudaStream_t s) {
    if (ph) product(p, w, sK2, s);
    else product(q, w, 0.0, s);
    launch_hd_dot<ST>(ph ? p : q, w, Npad, part, s);
    launch_hd_scalar(st, part, alpha, beta, 1, s);
    launch_hd_axpy<ST>(st, alpha, beta, w, q, qprev, r, Npad, s);
    if (ph) {
      product(r, pr, sK, s);
      launch_hd_dot<ST>(r, pr, Npad, part, s);
    } else {
      launch_hd_dot<ST>(r, r, Npad, part, s);
    }
    launch_hd_scalar(st, part, alpha, beta, 2, s);
    launch_hd_scale<ST>(st, beta, r, ph ? pr : nullptr, q, qprev, ph ? p : nullptr, Npad, 0, s);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s0);
  const long long launches0 = launch_counter();
  // start: q_0 = d / sqrt(<d, d>_K), p_0 = K q_0
  launch_hd_load<ST>(dd, N, Npad, r, s0);
  if (ph) {
    product(r, pr, sK, s0);
    launch_hd_dot<ST>(r, pr, Npad, part, s0);
  } else {
    launch_hd_dot<ST>(r, r, Npad, part, s0);
  }
  launch_hd_scalar(st, part, alpha, beta, 0, s0);
  launch_hd_scale<ST>(st, beta, r, ph ? pr : nullptr, q, qprev, ph ? p : nullptr, Npad, 1, s0);
  // the steps: one captured step replayed m times (stream launches if capture is refused)
  cudaGraphExec_t exec = nullptr;
  long long per_step = 0;
  if (h->cap || cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) == cudaSuccess) {
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      const long long c0 = launch_counter();
      step(h->cap);
      per_step = launch_counter() - c0;
      launch_counter() = c0;
      cudaGraph_t graph = nullptr;
      if (cudaStreamEndCapture(h->cap, &graph) == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
        cudaGraphDestroy(graph);
      }
    }
  }
  cudaGetLastError();
  for (int j = 0; j < m; ++j) {
    if (exec && cudaGraphLaunch(exec, s0) == cudaSuccess) {
      launch_counter() += per_step;
    } else {
      cudaGetLastError();
      step(s0);
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  launch_hd_cf(st, alpha, beta, nw, om, eta, ph ? 1 : 0, out, s0);
  cudaEventRecord(e1, s0);
  std::vector<double> hout(2 * (size_t)nw);
  CK(cudaMemcpyAsync(hout.data(), out, sizeof(double) * 2 * nw, cudaMemcpyDeviceToHost, s0));
  CK(cudaMemcpyAsync(&hs, st, sizeof(HdState), cudaMemcpyDeviceToHost, s0));
  std::vector<double> hal, hbe;
  if (coef_out) {
    hal.resize(m);
    hbe.resize(m);
    CK(cudaMemcpyAsync(hal.data(), alpha, sizeof(double) * m, cudaMemcpyDeviceToHost, s0));
    CK(cudaMemcpyAsync(hbe.data(), beta, sizeof(double) * m, cudaMemcpyDeviceToHost, s0));
  }
  CK(cudaStreamSynchronize(s0));
  CK(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < nw; ++i) {
    spectrum_out[i] = -hout[2 * (size_t)i + 1] / M_PI;
    if (response_out) {
      response_out[2 * (size_t)i] = hout[2 * (size_t)i];
      response_out[2 * (size_t)i + 1] = hout[2 * (size_t)i + 1];
    }
  }
  if (coef_out) {
    for (int j = 0; j < m; ++j) {
      coef_out[j] = j < hs.nsteps ? hal[j] : 0.0;
      coef_out[m + j] = j + 1 < hs.nsteps ? hbe[j] : 0.0;
    }
    coef_out[2 * (size_t)m] = hs.n2;
  }
  if (steps_out) *steps_out = hs.nsteps;
  h->stats = bse_stats{};
  h->stats.steps = hs.nsteps;
  h->stats.passes = ph ? 2 * (int64_t)m + 1 : (int64_t)m;
  h->stats.ms_total = ms;
  h->stats.launches = launch_counter() - launches0;
  h->stats.shape_ctas_per_sm = h->shape.ctas_per_sm;
  h->stats.shape_strided = h->shape.strided;
  h->stats.tuned = h->tuned ? 1 : 0;
  if (!(hs.n2 > 0.0)) return BSE_ENOTPD;
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
  h->mixed = dtype == BSE_C64_MIXED && form == BSE_PH;
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
      // complex128 PH tiles are kept as P = A + B, Q = A - B (8 FMAs per element pair)
      if (h->ph && where == BSE_DEVICE) {
        launch_pack_pq((const double2*)A[i], (const double2*)B[i], q.N, q.nT, (double2*)q.A, (double2*)q.B,
                       h->stream);
        if (cudaGetLastError() != cudaSuccess) rc = BSE_ECUDA;
      } else {
        rc = pack_matrix<double2>(h, (const double2*)A[i], q.N, q.nT, 1, where, (double2*)q.A);
        if (!rc && h->ph) rc = pack_matrix<double2>(h, (const double2*)B[i], q.N, q.nT, 0, where, (double2*)q.B);
        if (!rc && h->ph) launch_pq_combine((double2*)q.A, (double2*)q.B, q.ntiles * TS * TS, h->stream);
      }
      if (!rc && h->df) {
        const int64_t nel = q.ntiles * TS * TS;
        if (!(rc = dalloc(&q.Ahl, sizeof(float4) * (size_t)nel)))
          launch_split_tiles((const double2*)q.A, nel, (float4*)q.Ahl, h->stream);
        if (!rc && h->ph && !(rc = dalloc(&q.Bhl, sizeof(float4) * (size_t)nel)))
          launch_split_tiles((const double2*)q.B, nel, (float4*)q.Bhl, h->stream);
      }
    }
    if (!rc && dtype == BSE_C64_MIXED && h->ph) {
      const int64_t nel = q.ntiles * TS * TS;
      if (!(rc = dalloc(&q.UV, sizeof(float4) * (size_t)nel)))
        launch_uv_pack((const float2*)q.A, (const float2*)q.B, nel, (float4*)q.UV, h->stream);
      if (!rc && !(rc = dalloc((void**)&q.tmax, sizeof(float) * (size_t)q.ntiles))) {
        launch_tile_bound((const float2*)q.A, (const float2*)q.B, q.ntiles, q.tmax, h->stream);
        q.htmax.resize(q.ntiles);
        if (cudaMemcpyAsync(q.htmax.data(), q.tmax, sizeof(float) * q.ntiles, cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
          rc = BSE_ECUDA;
        for (float v : q.htmax) q.tref = std::max(q.tref, v);
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
  if (rc == BSE_OK && h->mixed) {
    h->hjobs = jobs;
    rc = dalloc((void**)&h->prod_err, sizeof(int));
    if (rc == BSE_OK && cudaMemsetAsync(h->prod_err, 0, sizeof(int), h->stream) != cudaSuccess) rc = BSE_ECUDA;
  }
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
  if (rc == BSE_OK) setup_tuner(h);
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

int bse_backward_ex(bse_handle* h, const double* dL_dlambda, int where, void* dA, void* dB, int impl) {
  if (!h || !dL_dlambda || !dA) return BSE_EINVAL;
  if (impl < BSE_IMPL_AUTO || impl > BSE_IMPL_TENSOR_CORES) return BSE_EINVAL;
  if (impl == BSE_IMPL_TENSOR_CORES && !is_c64(h->dtype)) return BSE_EINVAL;
  if (where != BSE_HOST && where != BSE_DEVICE) return BSE_EINVAL;
  if (h->count != 1) return BSE_EINVAL;
  if (h->ph && !dB) return BSE_EINVAL;
  if (!h->ph && dB) return BSE_EINVAL;
  if (!h->solved) return BSE_ESTATE;
  if (is_c64(h->dtype)) return backward_impl<float2>(h, dL_dlambda, where, dA, dB, impl);
  return backward_impl<double2>(h, dL_dlambda, where, dA, dB, impl);
}

int bse_backward(bse_handle* h, const double* dL_dlambda, int where, void* dA, void* dB) {
  return bse_backward_ex(h, dL_dlambda, where, dA, dB, BSE_IMPL_AUTO);
}

int bse_apply(bse_handle* h, int op, int k, const void* X, void* Y) {
  if (!h || !X || !Y || k < 1 || h->count != 1) return BSE_EINVAL;
  if (op < BSE_OP_A || op > BSE_OP_H) return BSE_EINVAL;
  if (is_c64(h->dtype)) return apply_impl<float2>(h, op, k, X, Y);
  return apply_impl<double2>(h, op, k, X, Y);
}

int bse_solve_dense(bse_handle* h, int nev, double tol, double* eval_out, void* evec_out, int* nconv_out) {
  if (!h || h->count != 1 || !h->ph || !eval_out || !(tol > 0.0)) return BSE_EINVAL;
  ProbHost& q = h->p[0];
  if (nev < 1 || nev > q.N) return BSE_EINVAL;
  int rc;
  if (!q.w || q.ncv == 0) {      // partial-sum and vector buffers of the FP64 residual products
    if ((rc = alloc_solve(h, std::min<int64_t>(q.N, 8) > 1 ? (int)std::min<int64_t>(q.N, 8) : 1))) return rc;
  }
  if ((rc = upload_probs(h))) return rc;
  const size_t nd = dense_scratch_doubles(q.N, nev);
  void* work = nullptr;
  if ((rc = dalloc(&work, sizeof(double) * nd))) return rc;
  struct Free { void* b; ~Free() { cudaFree(b); } } guard{work};
  if (!h->adj_err && (rc = dalloc((void**)&h->adj_err, sizeof(int)))) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, h->stream);
  const long long launches0 = launch_counter();
  h->solved = false;
  h->nev = nev;
  int status = BSE_OK;
  if (h->vs == sizeof(float2)) {
    Driver<float2> drv(h);
    if ((rc = drv.alloc_results(0, nev))) return rc;
    const int r = dense_shao(h->dprobs, q.N, q.Npad, h->tiles64, !h->tiles64, nev, (double*)work, h->adj_err, q.Z,
                             nullptr, h->stream);
    if (r < 0) return BSE_ECUDA;
    if (r > 0) status = BSE_ENOTPD;
    if ((rc = drv.finish(0, nev, tol, false))) return rc;
    if (evec_out && (rc = drv.store(0, evec_out))) return rc;
  } else {
    Driver<double2> drv(h);
    if ((rc = drv.alloc_results(0, nev))) return rc;
    const int r = dense_shao(h->dprobs, q.N, q.Npad, h->tiles64, !h->tiles64, nev, (double*)work, h->adj_err, q.Z,
                             nullptr, h->stream);
    if (r < 0) return BSE_ECUDA;
    if (r > 0) status = BSE_ENOTPD;
    if ((rc = drv.finish(0, nev, tol, false))) return rc;
    if (evec_out && (rc = drv.store(0, evec_out))) return rc;
  }
  cudaEventRecord(e1, h->stream);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int c = 0; c < nev; ++c) eval_out[c] = c < (int)q.eval.size() ? q.eval[c] : NAN;
  if (nconv_out) *nconv_out = q.nconv;
  double maxres = 0.0;
  for (double r : q.res) maxres = std::max(maxres, r);
  h->stats = bse_stats{};
  h->stats.nconv = q.nconv;
  h->stats.max_residual = maxres;
  h->stats.ms_total = ms;
  h->stats.launches = launch_counter() - launches0;
  h->solved = true;
  if (status == BSE_OK && q.nconv < nev) status = BSE_ENOCONV;
  return status;
}

int bse_apply_mixed(bse_handle* h, int op, double tile_tau, const void* X, void* Y) {
  if (!h || !X || !Y || h->count != 1 || !h->mixed) return BSE_EINVAL;
  if (op != BSE_OP_MPLUS && op != BSE_OP_MMINUS) return BSE_EINVAL;
  if (!std::isfinite(tile_tau)) return BSE_EINVAL;
  ProbHost& q = h->p[0];
  int rc;
  if (!q.w || q.ncv == 0) {
    if ((rc = alloc_solve(h, std::min<int64_t>(q.N, 8) > 1 ? (int)std::min<int64_t>(q.N, 8) : 1))) return rc;
  }
  if ((rc = upload_probs(h))) return rc;
  if ((rc = split_mixed_jobs(h, 1e-6, tile_tau))) return rc;
  count_launch();
  k_pad_in<double2><<<dim3((unsigned)((q.Npad + 255) / 256), 1), 256, 0, h->stream>>>(
      (const double2*)X, q.N, q.N, q.Npad, 1, 0, (double2*)q.w);
  GenericIO io{};
  io.xa = q.w;
  io.y = q.pw;
  io.sB = op == BSE_OP_MPLUS ? 1.0 : -1.0;
  launch_product_mixed(h->dprobs, h->djobs_fine, h->njobs_fine, h->djobs_coarse, h->njobs_coarse, 1, h->maxnT,
                       PM_GENERIC, &io, h->shape, h->prod_err, h->stream);
  CK(cudaMemcpyAsync(Y, q.pw, sizeof(double2) * (size_t)q.N, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaGetLastError());
  int perr = 0;
  CK(cudaMemcpyAsync(&perr, h->prod_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (perr) return BSE_ETIMEOUT;
  h->stats.tiles_fine = h->njobs_fine;
  h->stats.tiles_coarse = h->njobs_coarse;
  return BSE_OK;
}

int bse_haydock(bse_handle* h, const void* d, int where, int m, int sign, int nw, const double* omega, double eta,
                double* spectrum_out, double* response_out, double* coef_out, int* steps_out) {
  if (!h || !d || !omega || !spectrum_out || h->count != 1) return BSE_EINVAL;
  if (where != BSE_HOST && where != BSE_DEVICE) return BSE_EINVAL;
  if (m < 1 || m > 1000000 || nw < 1 || !(eta > 0.0) || !std::isfinite(eta)) return BSE_EINVAL;
  if (h->ph && sign != 1 && sign != -1) return BSE_EINVAL;
  if (h->vs == sizeof(float2))
    return haydock_impl<float2>(h, d, where, m, sign, nw, omega, eta, spectrum_out, response_out, coef_out,
                                steps_out);
  return haydock_impl<double2>(h, d, where, m, sign, nw, omega, eta, spectrum_out, response_out, coef_out,
                               steps_out);
}

int bse_selftest_bounded_wait(int arrive, int* expired) {
  if (!expired || (arrive != 0 && arrive != 1)) return BSE_EINVAL;
  return selftest_bounded_wait(arrive, expired) == 0 ? BSE_OK : BSE_ECUDA;
}

int bse_get_residuals(const bse_handle* h, int problem, double* res_out, int n) {
  if (!h || !res_out || n < 0 || problem < 0 || problem >= h->count) return BSE_EINVAL;
  if (!h->solved) return BSE_ESTATE;
  const ProbHost& q = h->p[problem];
  for (int c = 0; c < n; ++c) res_out[c] = c < (int)q.res.size() ? q.res[c] : NAN;
  return BSE_OK;
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
    dfreet(q.tmax);
    dfree(q.UV);
  }
  dfreet(h->djobs_fine);
  dfreet(h->djobs_coarse);
  dfreet(h->prod_err);
  dfreet(h->dprobs);
  dfreet(h->dstate);
  dfreet(h->djobs);
  dfree(h->post);
  dfreet(h->pj_work);
  dfreet(h->pj_flag);
  dfreet(h->gbar);
  dfreet(h->adj_tiles);
  dfreet(h->adj_tiles128);
  dfree(h->adj_panels);
  dfreet(h->adj_err);
  dfreet(h->gdev);
  for (auto& e : h->ev) cudaEventDestroy(e);
  for (StepGraph& g : h->sg) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& e : g.ev) cudaEventDestroy(e);
  }
  if (h->rg.exec) cudaGraphExecDestroy(h->rg.exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
  return BSE_OK;
}

}  // extern "C"
