// C ABI of the least-action propagator: context, configuration checks, time-basis constants,
// and the per-step driver (factorisation, V-cycles, convergence test, step advance).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "la_internal.cuh"
#include "../../include/leastaction.h"

using namespace la;

#define LA_MAX_LEVELS 8

struct la_ctx {
  la_config cfg;
  cudaStream_t stream = 0;
  std::string err;
  int K = 0, L = 0, dim = 0, np0 = 0;
  long long nunk0 = 0;
  double hd = 1.0;          // h^d
  double nscale = 1.0;      // N = nscale * r~^dagger Wt r~
  FineOp fine{};
  LevelGeom geo[LA_MAX_LEVELS];
  TimeMats htm{};           // host copy of the static part
  TimeMats* d_tm = nullptr;
  double* d_V0 = nullptr;
  // finest level, FP64
  double2 *d_psi = nullptr, *d_f = nullptr, *d_c = nullptr, *d_r = nullptr, *d_z = nullptr, *d_s = nullptr;
  // finest level, FP32 (mixed precision correction problem)
  float2 *d_f32 = nullptr, *d_e32 = nullptr, *d_r32 = nullptr, *d_z32 = nullptr, *d_s32 = nullptr;
  // levels >= 1 (precision of the V-cycle), and factors of every level
  void* d_e[LA_MAX_LEVELS] = {};
  void* d_g[LA_MAX_LEVELS] = {};
  void* d_sl[LA_MAX_LEVELS] = {};
  void* d_fac[LA_MAX_LEVELS] = {};
  double* d_sigma[LA_MAX_LEVELS] = {};
  // complex64 path: the Galerkin stencils rounded to float once, as its kernels use them
  float* d_sigma32[LA_MAX_LEVELS] = {};
  double* d_partials = nullptr;
  double* d_N = nullptr;
  int* d_status = nullptr;
  int* d_perm = nullptr;            // square local form: row permutation of every finest factor
  int nparts = 0;
  bool have_ham = false;
  bool have_step = false;
  // adjoint relaxation mode: finest-level right-hand side is y (added), not f
  bool adj = false;
  const void* adj_y = nullptr;
  // forward recording for la_backward
  bool have_rec = false;
  double rec_t0 = 0.0;
  int rec_nsteps = 0;
  double2* d_ckpt = nullptr;        // checkpoints psi_{s C}
  int ckpt_cap = 0;
  double2 *d_seg_psi = nullptr, *d_seg_c = nullptr, *d_lam = nullptr, *d_y = nullptr, *d_rho = nullptr;
  double2* d_gpart = nullptr;
  double* d_grad = nullptr;
  int seg_cap = 0;
  double last_N = 0.0, last_rel = 0.0;
  // converged coefficients of the last steps of the current propagation (trial extrapolation)
  double2* d_hist[3] = {};
  int nhist = 0, hist_head = 0;     // valid vectors; slot of the next push
  double hist_t_next = 0.0;         // start time of the step the history continues into
  // factors of the steps of the segment being back-propagated (cfg.cache_factors)
  void* d_fcache = nullptr;
  size_t fcache_step = 0;           // bytes of one step's factors (all levels)
  int fcache_cap = 0;               // steps the cache holds
  // converged adjoint solutions z of the last backward steps (trial of the adjoint relaxation)
  double2* d_ahist[3] = {};
  int nahist = 0, ahist_head = 0;
  std::vector<void*> allocs;
  // profiling
  bool prof = false;
  long long launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  // a timed launch: kind 0 = finest sweep, 1 = FP64 residual stencil, 2 = complex64 residual stencil
  struct ProfPair {
    cudaEvent_t e0, e1;
    int kind;
    double bytes;
  };
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_factor;
  std::vector<ProfPair> ev_kern;
  size_t ev_next = 0;
  double ms_factor = 0.0, ms_sweep = 0.0, ms_resid = 0.0, bytes_resid = 0.0, ms_resid32 = 0.0, bytes_resid32 = 0.0;
  double ms_restrict = 0.0, bytes_restrict = 0.0, ms_prolong = 0.0, bytes_prolong = 0.0;
  int n_factor = 0, n_sweep = 0, n_resid = 0, n_resid32 = 0, n_restrict = 0, n_prolong = 0;
  double flops_factor = 0.0, flops_sweep = 0.0;
  // one captured cycle (V-cycle + action norm + read-back), replayed on an internal stream
  struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<ProfPair> pairs;  // profiling event nodes
    long long launches = 0;
  };
  CycleGraph cg[2];               // [0] plain, [1] with profiling events
  CycleGraph* pending_graph = nullptr;
  bool use_graph = true;
  bool capturing = false;
  long long cycles_run = 0;
  std::vector<ProfPair> cap_pairs;
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* h_N = nullptr;          // pinned
  // device-side relaxation loop (la_step_batch): one graph per context whose conditional WHILE node runs
  // cycles until the device-computed action meets the stopping rule; no host synchronisation per cycle
  cudaGraphExec_t loop_exec = nullptr;
  LoopState* d_lstate = nullptr;
  LoopRecord* d_lrec = nullptr;     // one record per step of the current batch call
  int lrec_cap = 0;
  bool device_norm = false;         // action evaluations stay on the device (no read-back)
  // TMA tensor maps of the complex64 fields the finest-level stencils read (mixed precision, 2D/3D)
  CUtensorMap map_e32, map_z32;
  bool have_map_e32 = false, have_map_z32 = false;
};

static cudaEvent_t prof_event(la_ctx* c) {
  if (c->ev_next == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_next++];
}
// Adds one completed timed launch to the totals of its kind.
static void prof_add(la_ctx* c, const la_ctx::ProfPair& p) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, p.e0, p.e1) != cudaSuccess) return;
  if (p.kind == 0) { c->ms_sweep += ms; ++c->n_sweep; }
  else if (p.kind == 1) { c->ms_resid += ms; ++c->n_resid; c->bytes_resid += p.bytes; }
  else if (p.kind == 2) { c->ms_resid32 += ms; ++c->n_resid32; c->bytes_resid32 += p.bytes; }
  else if (p.kind == 3) { c->ms_restrict += ms; ++c->n_restrict; c->bytes_restrict += p.bytes; }
  else { c->ms_prolong += ms; ++c->n_prolong; c->bytes_prolong += p.bytes; }
}
// Drain recorded event pairs into the totals (synchronises).
static void prof_drain(la_ctx* c) {
  if (c->ev_factor.empty() && c->ev_kern.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& p : c->ev_factor) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) { c->ms_factor += ms; ++c->n_factor; }
  }
  for (auto& p : c->ev_kern) prof_add(c, p);
  c->ev_factor.clear();
  c->ev_kern.clear();
  c->ev_next = 0;
}
// Start event of a timed launch on the context's stream (an external event node while a cycle is
// being captured; the graph keeps those events).  False when profiling is off or events fail.
static bool prof_begin(la_ctx* c, cudaEvent_t* e0, cudaEvent_t* e1) {
  *e0 = *e1 = nullptr;
  if (!c->prof) return false;
  if (c->capturing) {
    if (cudaEventCreate(e0) != cudaSuccess) return false;
    if (cudaEventCreate(e1) != cudaSuccess) { cudaEventDestroy(*e0); *e0 = nullptr; return false; }
    cudaEventRecordWithFlags(*e0, c->stream, cudaEventRecordExternal);
  } else {
    *e0 = prof_event(c);
    *e1 = *e0 ? prof_event(c) : nullptr;
    if (!*e1) return false;
    cudaEventRecord(*e0, c->stream);
  }
  return true;
}
static void prof_end(la_ctx* c, cudaEvent_t e0, cudaEvent_t e1, int kind, double bytes) {
  if (c->capturing) cudaEventRecordWithFlags(e1, c->stream, cudaEventRecordExternal);
  else cudaEventRecord(e1, c->stream);
  (c->capturing ? c->cap_pairs : c->ev_kern).push_back({e0, e1, kind, bytes});
}

static la_status fail(la_ctx* c, la_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}
#define LA_CUDA(ctx, call)                                                                       \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(ctx, LA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define LA_CHECK_LAUNCH(ctx) LA_CUDA(ctx, cudaGetLastError())
#define LA_TRY(expr)                   \
  do {                                 \
    la_status s_ = (expr);             \
    if (s_ != LA_OK) return s_;        \
  } while (0)

static la_status dalloc(la_ctx* c, void** p, size_t bytes) {
  if (getenv("LA_FAIL_ALLOC")) return fail(c, LA_ENOMEM, "allocation of %zu bytes refused (LA_FAIL_ALLOC)", bytes);
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, LA_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return LA_OK;
}

// The context's static time-basis constants (la_internal.cuh: fill_time_constants).
static bool build_time_constants(la_ctx* c) {
  return fill_time_constants(c->K, c->cfg.dt, c->cfg.weight, c->htm);
}

static int round_npad(int n) {
  const int sizes[8] = {16, 32, 48, 64, 96, 128, 192, 256};
  for (int s : sizes)
    if (n <= s) return s;
  return -1;
}

static size_t csize(const la_ctx* c) { return c->cfg.precision ? sizeof(float2) : sizeof(double2); }

// ------------------------------------------------------------------ ABI
extern "C" const char* la_version(void) { return "leastaction-gb300 0.1 (sm_103a)"; }

// message of the last failed la_init on this thread (the context does not exist then)
static thread_local std::string g_init_error = "no error";

extern "C" const char* la_last_error(const la_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

namespace la {
// time-basis constants of a configuration without a context (used by la_action_noalloc)
bool time_constants_for(const la_config& cfg, TimeMats& out) {
  la_ctx tmp;
  tmp.cfg = cfg;
  tmp.K = cfg.nt;
  if (!build_time_constants(&tmp)) return false;
  out = tmp.htm;
  return true;
}
void set_thread_error(const char* msg) { g_init_error = msg ? msg : "unknown error"; }
void gauss_legendre_rule(int q, double* x, double* w) { gauss_legendre(q, x, w); }
}  // namespace la

extern "C" la_status la_init(const la_config* cfg, void* stream, la_ctx** out) {
  if (!cfg || !out) return LA_EINVAL;
  *out = nullptr;
  la_ctx* c = new (std::nothrow) la_ctx();
  if (!c) return LA_ENOMEM;
  c->cfg = *cfg;
  c->stream = (cudaStream_t)stream;
  const la_config& k = *cfg;
  la_status st = LA_OK;
  auto bad = [&](const char* why) {
    st = fail(c, LA_EINVAL, "invalid configuration: %s", why);
  };
  if (k.dim < 1 || k.dim > 3) bad("dim must be 1, 2 or 3");
  else if (k.nt < 1 || k.nt > LA_KMAX) bad("nt must be in [1, 8]");
  else if (!(k.dt > 0)) bad("dt must be positive");
  else if (k.levels < 1 || k.levels > LA_MAX_LEVELS) bad("levels must be in [1, 8]");
  else if (k.max_cycles < 1) bad("max_cycles must be >= 1");
  else if (k.nu1 < 0 || k.nu2 < 0 || k.nu1 + k.nu2 < 1) bad("nu1, nu2 >= 0 with nu1 + nu2 >= 1");
  else if (k.levels > 1 && k.coarse_sweeps < 1) bad("coarse_sweeps must be >= 1 with multigrid");
  else if (k.weight < 0 || k.weight > 2) bad("weight must be 0, 1 or 2");
  else if (k.precision < 0 || k.precision > 1) bad("precision must be 0 or 1");
  else if (k.laser_axis < 0 || k.laser_axis >= k.dim) bad("laser_axis must be a used axis");
  else if (k.ckpt_every < 0) bad("ckpt_every must be >= 0");
  else if (k.trial < 0 || k.trial > 3) bad("trial must be 0..3");
  else if (k.coarse_cycle && (k.coarse_nu1 < 0 || k.coarse_nu2 < 0)) bad("coarse_nu1, coarse_nu2 must be >= 0");
  else if (k.local_form < 0 || k.local_form > 1) bad("local_form must be 0 or 1");
  else if (k.local_form == 1 && k.precision != 0) bad("the square local form runs in FP64 (precision 0)");
  else if (k.local_form == 1 && k.levels != 1) bad("the square local form is single-level (levels 1)");
  else if (k.factor_group < 0 || k.factor_group > 1) bad("factor_group must be 0 or 1");
  if (st == LA_OK) {
    for (int a = 0; a < 3 && st == LA_OK; ++a) {
      if (a < k.dim) {
        if (k.n[a] < 1) bad("n must be >= 1 on used axes");
        else if (!(k.h[a] > 0)) bad("h must be positive on used axes");
        else if (k.sub[a] < (k.local_form == 1 ? 1 : 2))
          bad("sub must be >= 2 on used axes (>= 1 in the square form): same-colour subvolumes must not interact");
        else if (k.coarse_sub[a] == 1 || k.coarse_sub[a] < 0) bad("coarse_sub must be 0 or >= 2 on used axes");
        else if (k.n[a] % (1 << (k.levels - 1))) bad("n must be divisible by 2^(levels-1) on used axes");
      } else if (k.n[a] != 1) bad("unused axes must have n = 1");
    }
  }
  if (st != LA_OK) {
    g_init_error = c->err;
    delete c;
    return st;
  }
  c->K = k.nt;
  c->L = k.levels;
  c->dim = k.dim;
  int subpts = 1, csubpts = 1;
  for (int a = 0; a < k.dim; ++a) {
    subpts *= k.sub[a];
    csubpts *= k.coarse_sub[a] > 0 ? k.coarse_sub[a] : k.sub[a];
  }
  // finest level: up to 64 points and 256 unknowns (more than 128 unknowns: factorised in global
  // memory); Galerkin levels: up to 32 points and 128 unknowns (factorised in shared memory)
  if (subpts > LA_NPTS_WIDE || round_npad(subpts * k.nt) < 0) {
    g_init_error = "invalid configuration: a finest-level subvolume may hold at most 64 points and 256 unknowns";
    delete c;
    return LA_EINVAL;
  }
  if (k.levels > 1 && (csubpts > LA_NPTS_MAX || round_npad(csubpts * k.nt) < 0 ||
                       round_npad(csubpts * k.nt) > LA_NPAD_MAX)) {
    g_init_error = "invalid configuration: a Galerkin-level subvolume may hold at most 32 points and 128 unknowns "
                   "(set coarse_sub)";
    delete c;
    return LA_EINVAL;
  }
  if (k.local_form == 1 && round_npad(subpts * k.nt) > 96) {
    g_init_error = "invalid configuration: the square local form allows at most 96 unknowns per subvolume";
    delete c;
    return LA_EINVAL;
  }
  // fine operator
  FineOp& g = c->fine;
  g.dim = k.dim;
  g.dsum = 0.0;
  c->hd = 1.0;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = a < k.dim ? k.n[a] : 1;
    g.h[a] = a < k.dim ? k.h[a] : 1.0;
    g.ih2[a] = a < k.dim ? 1.0 / (k.h[a] * k.h[a]) : 0.0;
    g.x0[a] = -0.5 * (g.n[a] - 1) * g.h[a];
    if (a < k.dim) {
      g.dsum += g.ih2[a];
      c->hd *= k.h[a];
    }
  }
  g.lax = k.laser_axis;
  c->np0 = g.n[0] * g.n[1] * g.n[2];
  c->nunk0 = (long long)c->np0 * c->K;
  c->nscale = k.weight == 0 ? c->hd : (k.weight == 1 ? c->hd * c->hd * c->hd : c->hd * c->hd);
  // levels
  for (int l = 0; l < c->L; ++l) {
    LevelGeom& G = c->geo[l];
    G.dim = k.dim;
    G.np = 1;
    for (int a = 0; a < 3; ++a) {
      G.n[a] = a < k.dim ? (g.n[a] >> l) : 1;
      G.sub[a] = a < k.dim ? ((l > 0 && k.coarse_sub[a] > 0) ? k.coarse_sub[a] : k.sub[a]) : 1;
      G.nb[a] = (G.n[a] + G.sub[a] - 1) / G.sub[a];
      G.np *= G.n[a];
    }
    G.nsub = G.nb[0] * G.nb[1] * G.nb[2];
    G.npad = round_npad((l > 0 ? csubpts : subpts) * k.nt);
    G.nblk = G.npad / LA_BLK;
    G.fsize = k.local_form == 1 ? (long long)G.npad * G.npad : (long long)G.nblk * (G.nblk + 1) / 2 * LA_BLK * LA_BLK;
    G.fd_K = make_fastdiv(k.nt);
    for (int a = 0; a < 2; ++a) {
      const bool used = a < k.dim;
      G.fd_c[a] = make_fastdiv(used ? G.sub[a] + 4 : 1);
      G.fd_f[a] = make_fastdiv(used ? G.sub[a] + 2 : 1);
      G.fd_u[a] = make_fastdiv(G.sub[a]);
    }
    G.fd_pair = make_fastdiv(LA_NPAIR * box5_count(k.dim));
    G.one_per_cta = k.factor_group == 1 ? 1 : 0;
    G.band = (l == 0 && k.local_form == 0 && G.npad > LA_NPAD_MAX) ? fine_band_blocks(k.dim, G.sub, k.nt, G.nblk)
                                                                  : G.nblk - 1;
  }
  if (!build_time_constants(c)) {
    g_init_error = "invalid configuration: singular time-basis Gram matrix";
    delete c;
    return LA_EINVAL;
  }
  // allocations
  const size_t v64 = sizeof(double2) * (size_t)c->nunk0;
  const size_t v32 = sizeof(float2) * (size_t)c->nunk0;
  void* p;
#define ALLOC(field, bytes)                                         \
  do {                                                              \
    st = dalloc(c, &p, (bytes));                                    \
    if (st != LA_OK) { g_init_error = c->err; la_finalize(c); return st; } \
    field = (decltype(field))p;                                     \
  } while (0)
  ALLOC(c->d_tm, sizeof(TimeMats));
  ALLOC(c->d_V0, sizeof(double) * c->np0);
  ALLOC(c->d_psi, sizeof(double2) * c->np0);
  ALLOC(c->d_f, v64);
  ALLOC(c->d_c, v64);
  ALLOC(c->d_r, v64);
  ALLOC(c->d_z, v64);
  ALLOC(c->d_s, v64);
  if (k.precision == 1) {
    ALLOC(c->d_f32, v32);
    ALLOC(c->d_e32, v32);
    ALLOC(c->d_r32, v32);
    ALLOC(c->d_z32, v32);
    ALLOC(c->d_s32, v32);
  }
  for (int l = 0; l < c->L; ++l) {
    const LevelGeom& G = c->geo[l];
    ALLOC(c->d_fac[l], csize(c) * (size_t)G.nsub * G.fsize);
    if (l >= 1) {
      const size_t vb = csize(c) * (size_t)G.np * c->K;
      ALLOC(c->d_e[l], vb);
      ALLOC(c->d_g[l], vb);
      ALLOC(c->d_sl[l], vb);
      ALLOC(c->d_sigma[l], sizeof(double) * (size_t)G.np * LA_NPAIR * box5_count(k.dim));
      if (k.precision == 1) ALLOC(c->d_sigma32[l], sizeof(float) * (size_t)G.np * LA_NPAIR * box5_count(k.dim));
    }
  }
  c->nparts = norm_blocks(c->np0);
  ALLOC(c->d_partials, sizeof(double) * c->nparts);
  ALLOC(c->d_N, sizeof(double) * 2);
  ALLOC(c->d_status, sizeof(int));
  if (k.local_form == 1) ALLOC(c->d_perm, sizeof(int) * (size_t)c->geo[0].nsub * c->geo[0].npad);
  for (int j = 0; j < k.trial; ++j) ALLOC(c->d_hist[j], sizeof(double2) * (size_t)c->nunk0);
#undef ALLOC
  c->fine.V0 = c->d_V0;
  c->use_graph = getenv("LA_NO_GRAPH") == nullptr;
  if (k.precision == 1) {
    c->have_map_e32 = encode_stencil_map(c->fine, c->K, c->d_e32, &c->map_e32);
    c->have_map_z32 = encode_stencil_map(c->fine, c->K, c->d_z32, &c->map_z32);
  }
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&c->h_N, sizeof(double) * 2) != cudaSuccess) {
    g_init_error = "stream, event or pinned-buffer creation failed";
    la_finalize(c);
    return LA_ECUDA;
  }
  cudaError_t e = cudaMemcpyAsync(c->d_tm, &c->htm, sizeof(TimeMats), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_V0, 0, sizeof(double) * c->np0, c->stream);
  if (e != cudaSuccess) {
    la_finalize(c);
    return LA_ECUDA;
  }
  *out = c;
  return LA_OK;
}

// Real flops (8 per complex multiply-add) of the block-banded factorisation of an n-unknown subvolume
// whose 16 x 16 blocks (I, J) with I - J > band are zero: block (I, J) of the band is updated with the
// block columns Kb = max(0, I - band) .. J - 1 (only the lower half of a diagonal block counts), divided by
// the diagonal block's triangular inverse, and every diagonal block is factorised and inverted (16^3 / 3).
// Without a band this is the dense Cholesky's 4/3 n^3 up to terms of order 16 n^2.
static double banded_factor_flops(double n, int band) {
  const int nb = (int)((n + LA_BLK - 1) / LA_BLK);
  const double b3 = (double)LA_BLK * LA_BLK * LA_BLK;
  double macs = 0.0;
  for (int J = 0; J < nb; ++J) {
    for (int I = J; I < nb && I - J <= band; ++I) {
      const int nk = J - std::max(0, I - band);
      if (nk > 0) macs += (I == J ? b3 * (LA_BLK + 1) / (2.0 * LA_BLK) : b3) * nk;
      if (I > J) macs += (double)LA_BLK * LA_BLK * (LA_BLK + 1) / 2.0;
    }
    macs += b3 / 3.0;
  }
  return 8.0 * macs;
}

// algorithmic flops of the finest-level factorisation and of one full sweep
static void finest_flops(la_ctx* c) {
  const LevelGeom& G = c->geo[0];
  const bool banded = G.band < G.nblk - 1;
  double ff = 0.0, fs = 0.0;
  for (int bz = 0; bz < G.nb[2]; ++bz)
    for (int by = 0; by < G.nb[1]; ++by)
      for (int bx = 0; bx < G.nb[0]; ++bx) {
        int e[3], bb[3] = {bx, by, bz};
        for (int a = 0; a < 3; ++a) e[a] = std::min(G.sub[a], G.n[a] - bb[a] * G.sub[a]);
        const double n = (double)e[0] * e[1] * e[2] * c->K;
        if (banded) {
          // the factor's nonzero blocks only: the banded factorisation, and two triangular solves over
          // the blocks of the band (8 flops per complex entry and solve)
          ff += banded_factor_flops(n, G.band);
          const int nb = (int)((n + LA_BLK - 1) / LA_BLK);
          double nz = 0.0;
          for (int I = 0; I < nb; ++I) nz += std::min(I, G.band) + 1;
          fs += 2.0 * 8.0 * LA_BLK * LA_BLK * nz * (n * n) / ((double)nb * nb * LA_BLK * LA_BLK);
        } else {
          // Cholesky (4/3 n^3) and two triangular solves (8 n^2); the square form's LU takes 8/3 n^3
          ff += (c->cfg.local_form == 1 ? 8.0 : 4.0) / 3.0 * n * n * n;
          fs += 8.0 * n * n;
        }
      }
  c->flops_factor = ff;
  c->flops_sweep = fs;
}

// Compulsory bytes of one k_mresid launch on the finest level: c in, r or z out, f in when present
// (csize bytes per complex), V0 in (8 bytes per point); stencil neighbours are re-reads.
static double resid_bytes(const la_ctx* c, size_t csize, bool with_f) {
  return (double)c->np0 * ((double)csize * c->K * (with_f ? 3 : 2) + sizeof(double));
}

extern "C" la_status la_profile_enable(la_ctx* c, int enable) {
  if (!c) return LA_EINVAL;
  prof_drain(c);
  c->prof = enable != 0;
  if (c->prof) {
    c->launches = 0;
    c->ms_factor = c->ms_sweep = c->ms_resid = c->bytes_resid = c->ms_resid32 = c->bytes_resid32 = 0.0;
    c->ms_restrict = c->bytes_restrict = c->ms_prolong = c->bytes_prolong = 0.0;
    c->n_factor = c->n_sweep = c->n_resid = c->n_resid32 = c->n_restrict = c->n_prolong = 0;
    finest_flops(c);
  }
  return LA_OK;
}

extern "C" la_status la_profile_read(la_ctx* c, la_profile* out) {
  if (!c || !out) return LA_EINVAL;
  prof_drain(c);
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  out->launches = c->launches;
  out->n_factor = c->n_factor;
  out->ms_factor = c->ms_factor;
  out->flops_factor = c->flops_factor;
  out->n_sweep = c->n_sweep;
  out->ms_sweep = c->ms_sweep;
  out->flops_sweep = c->flops_sweep;
  out->n_resid = c->n_resid;
  out->ms_resid = c->ms_resid;
  out->bytes_resid = c->bytes_resid;
  out->n_resid32 = c->n_resid32;
  out->ms_resid32 = c->ms_resid32;
  out->bytes_resid32 = c->bytes_resid32;
  out->n_restrict = c->n_restrict;
  out->ms_restrict = c->ms_restrict;
  out->bytes_restrict = c->bytes_restrict;
  out->n_prolong = c->n_prolong;
  out->ms_prolong = c->ms_prolong;
  out->bytes_prolong = c->bytes_prolong;
  return LA_OK;
}

extern "C" la_status la_finalize(la_ctx* c) {
  if (!c) return LA_EINVAL;
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->cap) cudaStreamSynchronize(c->cap);
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  for (auto& g : c->cg) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& p : g.pairs) { cudaEventDestroy(p.e0); cudaEventDestroy(p.e1); }
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->h_N) cudaFreeHost(c->h_N);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
  return LA_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy n bytes from a host-or-device pointer into device memory dst
static la_status load_any(la_ctx* c, void* dst, const void* src, size_t n) {
  LA_CUDA(c, cudaMemcpyAsync(dst, src, n, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
  return LA_OK;
}
static la_status store_any(la_ctx* c, void* dst, const void* src, size_t n) {
  LA_CUDA(c, cudaMemcpyAsync(dst, src, n, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
  return LA_OK;
}

extern "C" la_status la_set_hamiltonian(la_ctx* c, const double* V0, const la_pulse* pulse) {
  if (!c) return LA_EINVAL;
  if (!V0) return fail(c, LA_EINVAL, "V0 is null");
  int nc = pulse ? pulse->ncomp : 0;
  if (nc < 0 || nc > LA_NCOMP_MAX) return fail(c, LA_EINVAL, "pulse ncomp must be in [0, %d]", LA_NCOMP_MAX);
  if (nc > 0 && (!pulse->amp || !pulse->omega || !pulse->t_center || !pulse->sigma))
    return fail(c, LA_EINVAL, "pulse arrays must not be null");
  c->htm.ncomp = nc;
  for (int k = 0; k < nc; ++k) {
    c->htm.amp[k] = pulse->amp[k];
    c->htm.omega[k] = pulse->omega[k];
    c->htm.tc[k] = pulse->t_center[k];
    c->htm.sigma[k] = pulse->sigma[k];
  }
  LA_TRY(load_any(c, c->d_V0, V0, sizeof(double) * c->np0));
  LA_CUDA(c, cudaMemcpyAsync(c->d_tm, &c->htm, sizeof(TimeMats), cudaMemcpyHostToDevice, c->stream));
  // Galerkin spatial factors of every coarse level (static)
  for (int l = 1; l < c->L; ++l) {
    if (l == 1) launch_galerkin_from_fine(c->fine, c->geo[1], c->d_sigma[1], c->stream);
    else launch_galerkin_coarse(c->geo[l - 1], c->d_sigma[l - 1], c->geo[l], c->d_sigma[l], c->stream);
    LA_CHECK_LAUNCH(c);
  }
  // the complex64 kernels read the stencils as float: round them once here, which halves the bytes
  // every Galerkin-level sweep, residual and factorisation streams and changes no result
  if (c->cfg.precision == 1) {
    for (int l = 1; l < c->L; ++l) {
      launch_f64_to_f32((long long)c->geo[l].np * LA_NPAIR * box5_count(c->dim), c->d_sigma[l], c->d_sigma32[l],
                        c->stream);
      LA_CHECK_LAUNCH(c);
    }
  }
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_ham = true;
  c->nhist = 0;
  return LA_OK;
}

// ------------------------------------------------------------------ V-cycle
template <typename R> struct Fine;
template <> struct Fine<double> {
  static double2* f(la_ctx* c) { return c->d_f; }
  static double2* e(la_ctx* c) { return c->d_c; }
  static double2* r(la_ctx* c) { return c->d_r; }
  static double2* z(la_ctx* c) { return c->d_z; }
  static double2* s(la_ctx* c) { return c->d_s; }
};
template <> struct Fine<float> {
  static float2* f(la_ctx* c) { return c->d_f32; }
  static float2* e(la_ctx* c) { return c->d_e32; }
  static float2* r(la_ctx* c) { return c->d_r32; }
  static float2* z(la_ctx* c) { return c->d_z32; }
  static float2* s(la_ctx* c) { return c->d_s32; }
};

// The Galerkin stencils of level l in the precision R of the path that reads them.
template <typename R> static const R* sigma_of(const la_ctx* c, int l);
template <> const double* sigma_of<double>(const la_ctx* c, int l) { return c->d_sigma[l]; }
template <> const float* sigma_of<float>(const la_ctx* c, int l) { return c->d_sigma32[l]; }

template <typename R>
static la_status factor_all(la_ctx* c) {
  typedef typename C2<R>::T CT;
  // Galerkin levels are factored on the internal stream, concurrently with the finest level
  // (their few CTAs would otherwise leave most SMs idle); joined before returning.
  const bool side = !c->capturing && c->L > 1 && c->cap;
  if (side) {
    LA_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    LA_CUDA(c, cudaStreamWaitEvent(c->cap, c->ev_fork, 0));
    for (int l = 1; l < c->L; ++l) {
      cudaError_t e = launch_factor<R>(c->geo[l], nullptr, sigma_of<R>(c, l), c->d_tm, (CT*)c->d_fac[l], c->d_status,
                                       c->cap);
      if (e != cudaSuccess) return fail(c, LA_ECUDA, "factor level %d: %s", l, cudaGetErrorString(e));
      ++c->launches;
    }
  }
  for (int l = 0; l < (side ? 1 : c->L); ++l) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof && l == 0 && (e0 = prof_event(c)) && (e1 = prof_event(c))) cudaEventRecord(e0, c->stream);
    cudaError_t e = c->cfg.local_form == 1
                        ? launch_factor_square(c->geo[0], c->fine, c->d_tm, (double2*)c->d_fac[0], c->d_perm,
                                               c->d_status, c->stream)
                        : launch_factor<R>(c->geo[l], l == 0 ? &c->fine : nullptr, sigma_of<R>(c, l), c->d_tm,
                                           (CT*)c->d_fac[l], c->d_status, c->stream);
    if (e != cudaSuccess) return fail(c, LA_ECUDA, "factor level %d: %s", l, cudaGetErrorString(e));
    ++c->launches;
    if (e1) {
      cudaEventRecord(e1, c->stream);
      c->ev_factor.push_back({e0, e1});
    }
  }
  if (side) {
    LA_CUDA(c, cudaEventRecord(c->ev_join, c->cap));
    LA_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  }
  return LA_OK;
}

template <typename R>
static la_status sweep_level(la_ctx* c, int l, int nsweeps) {
  typedef typename C2<R>::T CT;
  const bool square = c->cfg.local_form == 1;
  const int ncol = square ? 2 : 1 << c->dim;
  for (int s = 0; s < nsweeps; ++s) {
    // one event pair around a whole finest-level sweep (all colours)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = l == 0 && prof_begin(c, &e0, &e1);
    for (int col = 0; col < ncol; ++col) {
      cudaError_t e;
      if (square || colour_count(c->geo[l], col) > 0) ++c->launches;
      if (square)
        e = launch_sweep_square(c->geo[0], c->fine, c->d_tm, c->K, c->d_f, c->d_c, (const double2*)c->d_fac[0],
                                c->d_perm, col, c->stream);
      else if (l == 0)
        e = launch_sweep_fine<R>(c->geo[0], c->fine, c->d_tm, c->K, c->adj ? nullptr : Fine<R>::f(c),
                                 c->adj ? (const CT*)c->adj_y : nullptr, Fine<R>::e(c), (const CT*)c->d_fac[0], col,
                                 c->d_status, c->stream);
      else
        e = launch_sweep_coarse<R>(c->geo[l], sigma_of<R>(c, l), c->d_tm, c->K, (const CT*)c->d_g[l], (CT*)c->d_e[l],
                                   (const CT*)c->d_fac[l], col, c->d_status, c->stream);
      if (e != cudaSuccess) return fail(c, LA_ECUDA, "sweep level %d colour %d: %s", l, col, cudaGetErrorString(e));
    }
    // inside a capture the records are graph nodes (external), not capture-internal joins
    if (timed) prof_end(c, e0, e1, 0, 0.0);
  }
  return LA_OK;
}

// Error for a nonzero device status word (flag 1: a subvolume matrix was not positive definite;
// flag 4: a staged copy did not arrive within its wait limit).
static la_status status_error(la_ctx* c, int status) {
  if (status & 1)
    return fail(c, LA_ECUDA, "a subvolume matrix was singular or not positive definite (status %d)", status);
  return fail(c, LA_ETIMEOUT, "a staged copy did not complete within its wait limit (status %d)", status);
}

// The TMA tensor map of a finest-level complex64 field, when one was encoded for it.
static const CUtensorMap* stencil_map(const la_ctx* c, const void* field) {
  if (c->have_map_e32 && field == c->d_e32) return &c->map_e32;
  if (c->have_map_z32 && field == c->d_z32) return &c->map_z32;
  return nullptr;
}

template <typename R>
static la_status vcycle(la_ctx* c, int l) {
  typedef typename C2<R>::T CT;
  const la_config& k = c->cfg;
  if (c->L == 1) return sweep_level<R>(c, 0, k.nu1 + k.nu2);
  if (l == c->L - 1) return sweep_level<R>(c, l, k.coarse_sweeps);
  const int nu1 = (l > 0 && k.coarse_cycle) ? k.coarse_nu1 : k.nu1;
  const int nu2 = (l > 0 && k.coarse_cycle) ? k.coarse_nu2 : k.nu2;
  LA_TRY(sweep_level<R>(c, l, nu1));
  CT* sfine;
  if (l == 0) {
    // normal residual s = M~^dagger Wt (f - M~ e) on the finest level
    // (adjoint mode: s = y - G~ e)
    cudaEvent_t e0, e1;
    const bool timed = prof_begin(c, &e0, &e1);
    launch_mresid<R>(c->fine, c->d_tm, c->K, c->adj ? nullptr : Fine<R>::f(c), Fine<R>::e(c), nullptr, Fine<R>::z(c),
                     nullptr, c->nparts, c->stream, stencil_map(c, Fine<R>::e(c)), c->d_status);
    if (timed) prof_end(c, e0, e1, sizeof(R) == 8 ? 1 : 2, resid_bytes(c, sizeof(CT), !c->adj));
    launch_mnormal<R>(c->fine, c->d_tm, c->K, Fine<R>::z(c), Fine<R>::s(c), c->stream,
                      c->adj ? (const CT*)c->adj_y : nullptr, stencil_map(c, Fine<R>::z(c)), c->d_status);
    c->launches += 2;
    sfine = Fine<R>::s(c);
  } else {
    cudaError_t ge = launch_gresid_tiles<R>(c->geo[l], sigma_of<R>(c, l), c->d_tm, c->K, (const CT*)c->d_g[l],
                                            (const CT*)c->d_e[l], (CT*)c->d_sl[l], c->stream);
    if (ge != cudaSuccess) return fail(c, LA_ECUDA, "coarse residual level %d: %s", l, cudaGetErrorString(ge));
    ++c->launches;
    sfine = (CT*)c->d_sl[l];
  }
  {
    // finest-level transfer timed for the roofline: s (fine) in, g (level 1) out
    cudaEvent_t e0, e1;
    const bool timed = l == 0 && prof_begin(c, &e0, &e1);
    launch_restrict<R>(c->geo[l], c->geo[l + 1], c->K, sfine, (CT*)c->d_g[l + 1], c->stream);
    if (timed)
      prof_end(c, e0, e1, 3, (double)sizeof(CT) * c->K * ((double)c->geo[0].np + (double)c->geo[1].np));
  }
  ++c->launches;
  LA_CHECK_LAUNCH(c);
  LA_CUDA(c, cudaMemsetAsync(c->d_e[l + 1], 0, sizeof(CT) * (size_t)c->geo[l + 1].np * c->K, c->stream));
  LA_TRY(vcycle<R>(c, l + 1));
  CT* efine = l == 0 ? Fine<R>::e(c) : (CT*)c->d_e[l];
  {
    // e (level 1) in, the fine correction read and written
    cudaEvent_t e0, e1;
    const bool timed = l == 0 && prof_begin(c, &e0, &e1);
    launch_prolong_add<R>(c->geo[l], c->geo[l + 1], c->K, (const CT*)c->d_e[l + 1], efine, c->stream);
    if (timed)
      prof_end(c, e0, e1, 4, (double)sizeof(CT) * c->K * (2.0 * c->geo[0].np + (double)c->geo[1].np));
  }
  ++c->launches;
  LA_CHECK_LAUNCH(c);
  return sweep_level<R>(c, l, nu2);
}

// N of the current FP64 iterate into h_N[slot] (stores r~ = f~ - M~ c in d_r); enqueue only.  zero_c:
// the iterate is known to be c = 0, so r~ = f~ and no stencil is applied.
static la_status action_enqueue(la_ctx* c, int slot = 0, bool zero_c = false) {
  cudaEvent_t e0, e1;
  const bool timed = !zero_c && prof_begin(c, &e0, &e1);   // the stencil launches carry the roofline
  launch_mresid<double>(c->fine, c->d_tm, c->K, c->d_f, zero_c ? nullptr : c->d_c, c->d_r, nullptr, c->d_partials,
                        c->nparts, c->stream);
  if (timed) prof_end(c, e0, e1, 1, resid_bytes(c, sizeof(double2), true));
  launch_norm_final(c->d_partials, c->nparts, c->nscale, c->d_N + slot, c->stream);
  c->launches += 2;
  LA_CHECK_LAUNCH(c);
  if (!c->device_norm)
    LA_CUDA(c, cudaMemcpyAsync(c->h_N + slot, c->d_N + slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return LA_OK;
}
// N of the current FP64 iterate; synchronises.
static la_status action_now(la_ctx* c, double* N) {
  LA_TRY(action_enqueue(c));
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  *N = *c->h_N;
  return LA_OK;
}

// One cycle: V-cycle (FP64) or complex64 correction V-cycle with FP64 refinement, then N.
static la_status cycle_body(la_ctx* c) {
  if (c->cfg.precision == 0) {
    LA_TRY(vcycle<double>(c, 0));
  } else {
    // refinement: correction problem M~ e = r~ (r~ from the last action evaluation) in complex64
    launch_c128_to_c64(c->nunk0, c->d_r, c->d_f32, c->stream);
    LA_CUDA(c, cudaMemsetAsync(c->d_e32, 0, sizeof(float2) * (size_t)c->nunk0, c->stream));
    LA_TRY(vcycle<float>(c, 0));
    launch_axpy_c64_to_c128(c->nunk0, c->d_e32, c->d_c, c->stream);
    c->launches += 2;
    LA_CHECK_LAUNCH(c);
  }
  return action_enqueue(c);
}

// Run one cycle and return N.  After the first cycle of a context the cycle is captured once into
// a CUDA graph and replayed on an internal stream joined to the caller's stream by events.
static la_status cycle_issue(la_ctx* c) {
  c->pending_graph = nullptr;
  if (!c->use_graph || c->cycles_run == 0) return cycle_body(c);
  la_ctx::CycleGraph& g = c->cg[c->prof ? 1 : 0];
  if (!g.exec) {
    cudaStream_t user = c->stream;
    const long long l0 = c->launches;
    c->stream = c->cap;
    c->capturing = true;
    c->cap_pairs.clear();
    LA_CUDA(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    la_status st = cycle_body(c);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(c->cap, &graph);
    c->stream = user;
    c->capturing = false;
    if (st != LA_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return fail(c, LA_ECUDA, "cycle capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(c, LA_ECUDA, "cycle graph instantiate: %s", cudaGetErrorString(ce));
    g.pairs.swap(c->cap_pairs);
    g.launches = c->launches - l0;
    c->launches = l0;
  }
  LA_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
  LA_CUDA(c, cudaStreamWaitEvent(c->cap, c->ev_fork, 0));
  LA_CUDA(c, cudaGraphLaunch(g.exec, c->cap));
  LA_CUDA(c, cudaEventRecord(c->ev_join, c->cap));
  LA_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  c->pending_graph = &g;
  return LA_OK;
}

static la_status cycle_complete(la_ctx* c, double* N) {
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  *N = *c->h_N;
  if (c->pending_graph) {
    la_ctx::CycleGraph& g = *c->pending_graph;
    c->launches += g.launches;
    if (c->prof) {
      for (auto& p : g.pairs) prof_add(c, p);
    }
    c->pending_graph = nullptr;
  }
  ++c->cycles_run;
  return LA_OK;
}

// Run one cycle and return N.  After the first cycle of a context the cycle is captured once into
// a CUDA graph and replayed on an internal stream joined to the caller's stream by events.
static la_status run_cycle(la_ctx* c, double* N) {
  LA_TRY(cycle_issue(c));
  return cycle_complete(c, N);
}

// time matrices and right-hand side for initial state d_psi at t0
static la_status setup_step(la_ctx* c, double t0) {
  launch_time_matrices(c->d_tm, t0, c->stream);
  launch_rhs(c->fine, c->d_tm, c->d_psi, c->d_f, c->stream);
  c->launches += 2;
  LA_CHECK_LAUNCH(c);
  return LA_OK;
}

// ------------------------------------------------------------------ trial iterate
// The relaxation corrects a trial function (Sec. IV, Eq. leastaction_correction).  The trial of a
// step is the polynomial in the step index through the last q converged coefficient vectors
// (q = 1, 2, 3: constant, linear, quadratic), evaluated at the new step.
static const double kTrialW[3][3] = {{1.0, 0.0, 0.0}, {2.0, -1.0, 0.0}, {3.0, -3.0, 1.0}};

static la_status hist_push(la_ctx* c) {
  const int T = c->cfg.trial;
  if (T <= 0) return LA_OK;
  LA_CUDA(c, cudaMemcpyAsync(c->d_hist[c->hist_head], c->d_c, sizeof(double2) * (size_t)c->nunk0,
                             cudaMemcpyDeviceToDevice, c->stream));
  c->hist_head = (c->hist_head + 1) % T;
  c->nhist = std::min(c->nhist + 1, T);
  return LA_OK;
}

// Enqueue the starting iterate of a step: N(0) into h_N[1]; with a history (and use_trial) the
// extrapolated trial into d_c and its action into h_N[0].  d_r ends as the residual of d_c.
static la_status seed_enqueue(la_ctx* c, bool use_trial, bool* tried) {
  LA_CUDA(c, cudaMemsetAsync(c->d_c, 0, sizeof(double2) * (size_t)c->nunk0, c->stream));
  LA_TRY(action_enqueue(c, 1, true));
  *tried = false;
  if (use_trial && c->cfg.trial > 0 && c->nhist > 0) {
    const int T = c->cfg.trial, q = c->nhist;
    const double2* h[3] = {nullptr, nullptr, nullptr};
    for (int j = 0; j < q; ++j) h[j] = c->d_hist[((c->hist_head - 1 - j) % T + T) % T];
    launch_trial(c->nunk0, kTrialW[q - 1], h[0], h[1], h[2], c->d_c, c->stream);
    ++c->launches;
    LA_CHECK_LAUNCH(c);
    LA_TRY(action_enqueue(c, 0));
    *tried = true;
  }
  return LA_OK;
}

// After the stream has synchronised: N0 = N(0); N = N of the starting iterate.  A trial whose
// action is not below N(0) is replaced by c = 0.
static la_status seed_finish(la_ctx* c, bool tried, double* N0, double* N) {
  *N0 = c->h_N[1];
  *N = *N0;
  if (!tried) return LA_OK;
  *N = c->h_N[0];
  if (!(*N < *N0)) {
    LA_CUDA(c, cudaMemsetAsync(c->d_c, 0, sizeof(double2) * (size_t)c->nunk0, c->stream));
    LA_TRY(action_now(c, N));
  }
  return LA_OK;
}

// Relax the step's coefficients from c = 0, or from the trial when use_trial.  ncycles > 0:
// exactly that many cycles.
static la_status solve_current(la_ctx* c, int ncycles, la_step_stats* st, bool use_trial = false) {
  const la_config& k = c->cfg;
  if (k.precision == 0) LA_TRY(factor_all<double>(c));
  else LA_TRY(factor_all<float>(c));
  bool tried = false;
  LA_TRY(seed_enqueue(c, use_trial, &tried));
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  double N0 = 0.0, N = 0.0;
  LA_TRY(seed_finish(c, tried, &N0, &N));
  int cyc = 0;
  const int maxc = ncycles > 0 ? ncycles : k.max_cycles;
  const bool check = ncycles <= 0 && k.tol > 0;
  while (cyc < maxc) {
    if (check && N <= k.tol * N0) break;
    if (!std::isfinite(N)) break;   // canary: a non-finite action ends the relaxation
    LA_TRY(run_cycle(c, &N));
    ++cyc;
  }
  int status = 0;
  LA_CUDA(c, cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status) {
    cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    return status_error(c, status);
  }
  c->last_N = N;
  c->last_rel = N0 > 0 ? N / N0 : 0.0;
  c->have_step = true;
  const int fine_per_cycle = c->L == 1 ? k.nu1 + k.nu2 : k.nu1 + k.nu2;
  if (st) {
    st->cycles = cyc;
    st->fine_sweeps = cyc * fine_per_cycle;
    st->action = N;
    st->rel_action = c->last_rel;
  }
  if (!std::isfinite(N)) return fail(c, LA_ENOTCONV, "the action is not finite after %d cycles", cyc);
  if (check && !(N <= k.tol * N0)) return fail(c, LA_ENOTCONV, "not converged after %d cycles (rel %.3e)", cyc, c->last_rel);
  return LA_OK;
}

extern "C" la_status la_step(la_ctx* c, void* psi, int nsteps, double t0, la_step_stats* per_step) {
  if (!c || !psi || nsteps < 0) return c ? fail(c, LA_EINVAL, "null psi or negative nsteps") : LA_EINVAL;
  if (!c->have_ham) return fail(c, LA_ESTATE, "la_set_hamiltonian must be called first");
  const bool dev = is_device_ptr(psi);
  const size_t bytes = sizeof(double2) * (size_t)c->np0;
  LA_CUDA(c, cudaMemcpyAsync(c->d_psi, psi, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  la_status worst = LA_OK;
  const int C = c->cfg.ckpt_every;
  // the trial history continues only a propagation that ended at t0
  if (!(std::fabs(t0 - c->hist_t_next) <= 1e-9 * std::fabs(c->cfg.dt))) c->nhist = 0;
  if (C > 0 && nsteps > 0) {
    const int need = (nsteps + C - 1) / C;
    if (need > c->ckpt_cap) {
      void* p = nullptr;
      LA_TRY(dalloc(c, &p, sizeof(double2) * (size_t)c->np0 * need));
      c->d_ckpt = (double2*)p;
      c->ckpt_cap = need;
    }
    c->rec_t0 = t0;
    c->rec_nsteps = nsteps;
    c->have_rec = true;
  }
  for (int s = 0; s < nsteps; ++s) {
    if (C > 0 && s % C == 0) {
      LA_CUDA(c, cudaMemcpyAsync(c->d_ckpt + (size_t)(s / C) * c->np0, c->d_psi, bytes, cudaMemcpyDeviceToDevice,
                                 c->stream));
      c->nhist = 0;   // a segment's iterates depend only on its checkpoint (exact recomputation)
    }
    LA_TRY(setup_step(c, t0 + s * c->cfg.dt));
    la_status st = solve_current(c, 0, per_step ? per_step + s : nullptr, true);
    if (st == LA_ENOTCONV) worst = LA_ENOTCONV;
    else if (st != LA_OK) return st;
    launch_advance(c->np0, c->d_tm, c->d_c, c->d_psi, c->stream);
    ++c->launches;
    LA_CHECK_LAUNCH(c);
    LA_TRY(hist_push(c));
    c->hist_t_next = t0 + (s + 1) * c->cfg.dt;
  }
  prof_drain(c);
  LA_CUDA(c, cudaMemcpyAsync(psi, c->d_psi, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  return worst;
}

// Relax G~ z = y~ (y~ in d_y) from z = 0 into d_c with the step's factors; on return d_z holds
// Wt (0 - M~ z) = -mu of the final z.  Stops when |y~ - G~ z|^2 <= tol |y~|^2 or at max_cycles.
// Relaxes from z = 0 or, with cfg.trial > 0 and an adjoint history, from the extrapolation of the
// last converged adjoint solutions (in the backward step order) when that trial's residual is
// below the one of z = 0; the stopping test stays relative to |y~|^2.
static la_status adjoint_solve(la_ctx* c, int* cycles) {
  const la_config& k = c->cfg;
  const long long n = c->nunk0;
  const int nb = (int)std::min<long long>((n + 255) / 256, 4096);
  LA_CUDA(c, cudaMemsetAsync(c->d_c, 0, sizeof(double2) * (size_t)n, c->stream));
  auto rho_norm = [&](double* out) -> la_status {
    launch_mresid<double>(c->fine, c->d_tm, c->K, nullptr, c->d_c, nullptr, c->d_z, nullptr, c->nparts, c->stream);
    launch_mnormal<double>(c->fine, c->d_tm, c->K, c->d_z, c->d_rho, c->stream, c->d_y);
    launch_norm2_partials(n, c->d_rho, c->d_partials, std::min(nb, c->nparts), c->stream);
    launch_norm_final(c->d_partials, std::min(nb, c->nparts), 1.0, c->d_N, c->stream);
    c->launches += 4;
    LA_CHECK_LAUNCH(c);
    LA_CUDA(c, cudaMemcpyAsync(c->h_N, c->d_N, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LA_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = *c->h_N;
    return LA_OK;
  };
  double N0 = 0.0, N = 0.0;
  LA_TRY(rho_norm(&N0));
  N = N0;
  const int T = k.trial;
  if (T > 0 && c->nahist > 0) {
    const int q = c->nahist;
    const double2* h[3] = {nullptr, nullptr, nullptr};
    for (int j = 0; j < q; ++j) h[j] = c->d_ahist[((c->ahist_head - 1 - j) % T + T) % T];
    launch_trial(n, kTrialW[q - 1], h[0], h[1], h[2], c->d_c, c->stream);
    ++c->launches;
    LA_CHECK_LAUNCH(c);
    double Nt = 0.0;
    LA_TRY(rho_norm(&Nt));
    if (Nt < N0) {
      N = Nt;
    } else {
      LA_CUDA(c, cudaMemsetAsync(c->d_c, 0, sizeof(double2) * (size_t)n, c->stream));
      LA_TRY(rho_norm(&N));
    }
  }
  int cyc = 0;
  while (cyc < k.max_cycles && N > k.tol * N0) {
    c->adj = true;
    la_status st;
    if (k.precision == 0) {
      c->adj_y = c->d_y;
      st = vcycle<double>(c, 0);
    } else {
      launch_c128_to_c64(n, c->d_rho, c->d_f32, c->stream);
      cudaMemsetAsync(c->d_e32, 0, sizeof(float2) * (size_t)n, c->stream);
      c->adj_y = c->d_f32;
      st = vcycle<float>(c, 0);
      launch_axpy_c64_to_c128(n, c->d_e32, c->d_c, c->stream);
      c->launches += 2;
    }
    c->adj = false;
    c->adj_y = nullptr;
    LA_TRY(st);
    ++cyc;
    LA_TRY(rho_norm(&N));
  }
  if (!std::isfinite(N)) return fail(c, LA_ENOTCONV, "the adjoint residual norm is not finite after %d cycles", cyc);
  if (cycles) *cycles = cyc;
  if (T > 0) {   // history of converged adjoint solutions
    LA_CUDA(c, cudaMemcpyAsync(c->d_ahist[c->ahist_head], c->d_c, sizeof(double2) * (size_t)n, cudaMemcpyDeviceToDevice,
                               c->stream));
    c->ahist_head = (c->ahist_head + 1) % T;
    c->nahist = std::min(c->nahist + 1, T);
  }
  return LA_OK;
}

extern "C" la_status la_backward(la_ctx* c, const void* dJ_dpsiT, double* grad_amp, void* dJ_dpsi0) {
  if (!c || !dJ_dpsiT) return c ? fail(c, LA_EINVAL, "null dJ/dpsi_T") : LA_EINVAL;
  if (c->cfg.local_form == 1)
    return fail(c, LA_EINVAL, "la_backward relaxes the adjoint with the least-squares factors (local_form 0)");
  if (!c->have_rec || c->rec_nsteps < 1)
    return fail(c, LA_ESTATE, "la_backward needs a preceding la_step with ckpt_every > 0");
  const int C = c->cfg.ckpt_every, nsteps = c->rec_nsteps, K = c->K;
  const size_t vb = sizeof(double2) * (size_t)c->np0, cb = sizeof(double2) * (size_t)c->nunk0;
  if (C > c->seg_cap) {
    void* p = nullptr;
    LA_TRY(dalloc(c, &p, vb * C)); c->d_seg_psi = (double2*)p;
    LA_TRY(dalloc(c, &p, cb * C)); c->d_seg_c = (double2*)p;
    if (!c->d_lam) {
      LA_TRY(dalloc(c, &p, vb)); c->d_lam = (double2*)p;
      LA_TRY(dalloc(c, &p, cb)); c->d_y = (double2*)p;
      LA_TRY(dalloc(c, &p, cb)); c->d_rho = (double2*)p;
      LA_TRY(dalloc(c, &p, sizeof(double2) * (size_t)((c->np0 + 255) / 256) * K * (K + 1))); c->d_gpart = (double2*)p;
      LA_TRY(dalloc(c, &p, sizeof(double) * LA_NCOMP_MAX)); c->d_grad = (double*)p;
    }
    c->seg_cap = C;
  }
  for (int j = 0; j < c->cfg.trial; ++j)
    if (!c->d_ahist[j]) {
      void* p = nullptr;
      LA_TRY(dalloc(c, &p, cb));
      c->d_ahist[j] = (double2*)p;
    }
  c->nahist = 0;
  // factor cache for one segment (cfg.cache_factors); allocation failure only disables it
  size_t lvl_bytes[LA_MAX_LEVELS] = {};
  bool cache = false;
  if (c->cfg.cache_factors) {
    size_t step = 0;
    for (int l = 0; l < c->L; ++l) {
      lvl_bytes[l] = csize(c) * (size_t)c->geo[l].nsub * c->geo[l].fsize;
      step += lvl_bytes[l];
    }
    if (c->fcache_cap < C || c->fcache_step != step) {
      if (c->d_fcache) {
        cudaFree(c->d_fcache);
        c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), c->d_fcache), c->allocs.end());
        c->d_fcache = nullptr;
        c->fcache_cap = 0;
      }
      void* p = nullptr;
      if (cudaMalloc(&p, step * (size_t)C) == cudaSuccess) {
        c->allocs.push_back(p);
        c->d_fcache = p;
        c->fcache_cap = C;
        c->fcache_step = step;
      } else {
        cudaGetLastError();
      }
    }
    cache = c->d_fcache != nullptr;
  }
  auto cache_slot = [&](int j, int l) -> unsigned char* {
    size_t off = c->fcache_step * (size_t)j;
    for (int m = 0; m < l; ++m) off += lvl_bytes[m];
    return static_cast<unsigned char*>(c->d_fcache) + off;
  };
  LA_TRY(load_any(c, c->d_lam, dJ_dpsiT, vb));
  LA_CUDA(c, cudaMemsetAsync(c->d_grad, 0, sizeof(double) * LA_NCOMP_MAX, c->stream));
  const int nseg = (nsteps + C - 1) / C;
  for (int sgm = nseg - 1; sgm >= 0; --sgm) {
    const int k0 = sgm * C, k1 = std::min(k0 + C, nsteps);
    // recompute the segment's states and converged coefficients from its checkpoint
    LA_CUDA(c, cudaMemcpyAsync(c->d_psi, c->d_ckpt + (size_t)sgm * c->np0, vb, cudaMemcpyDeviceToDevice, c->stream));
    c->nhist = 0;
    for (int kk = k0; kk < k1; ++kk) {
      LA_CUDA(c, cudaMemcpyAsync(c->d_seg_psi + (size_t)(kk - k0) * c->np0, c->d_psi, vb, cudaMemcpyDeviceToDevice,
                                 c->stream));
      LA_TRY(setup_step(c, c->rec_t0 + kk * c->cfg.dt));
      la_status st = solve_current(c, 0, nullptr, true);
      if (st != LA_OK && st != LA_ENOTCONV) return st;
      LA_CUDA(c, cudaMemcpyAsync(c->d_seg_c + (size_t)(kk - k0) * c->nunk0, c->d_c, cb, cudaMemcpyDeviceToDevice,
                                 c->stream));
      if (cache)
        for (int l = 0; l < c->L; ++l)
          LA_CUDA(c, cudaMemcpyAsync(cache_slot(kk - k0, l), c->d_fac[l], lvl_bytes[l], cudaMemcpyDeviceToDevice,
                                     c->stream));
      launch_advance(c->np0, c->d_tm, c->d_c, c->d_psi, c->stream);
      ++c->launches;
      LA_TRY(hist_push(c));
    }
    // backward through the segment
    for (int kk = k1 - 1; kk >= k0; --kk) {
      const double tk = c->rec_t0 + kk * c->cfg.dt;
      LA_CUDA(c, cudaMemcpyAsync(c->d_psi, c->d_seg_psi + (size_t)(kk - k0) * c->np0, vb, cudaMemcpyDeviceToDevice,
                                 c->stream));
      LA_TRY(setup_step(c, tk));
      void* own[LA_MAX_LEVELS] = {};
      if (cache) {
        // the adjoint V-cycles are launched directly (no captured graph), so they can read the
        // cached factors in place
        for (int l = 0; l < c->L; ++l) { own[l] = c->d_fac[l]; c->d_fac[l] = cache_slot(kk - k0, l); }
      } else if (c->cfg.precision == 0) {
        LA_TRY(factor_all<double>(c));
      } else {
        LA_TRY(factor_all<float>(c));
      }
      launch_bt_lambda(c->np0, c->d_tm, 1.0 / c->hd, c->d_lam, c->d_y, c->stream);
      ++c->launches;
      const la_status ast = adjoint_solve(c, nullptr);
      if (cache)
        for (int l = 0; l < c->L; ++l) c->d_fac[l] = own[l];
      LA_TRY(ast);
      launch_grad_contract(c->fine, c->d_tm, K, tk, c->hd, c->d_z, c->d_psi, c->d_seg_c + (size_t)(kk - k0) * c->nunk0,
                           c->d_gpart, c->d_grad, c->stream);
      launch_lambda_update(c->fine, c->d_tm, c->hd, c->d_z, c->d_lam, c->stream);
      c->launches += 3;
      LA_CHECK_LAUNCH(c);
    }
  }
  c->nhist = 0;   // the history now belongs to the recomputation
  if (dJ_dpsi0) LA_TRY(store_any(c, dJ_dpsi0, c->d_lam, vb));
  if (grad_amp && c->htm.ncomp > 0)
    LA_CUDA(c, cudaMemcpyAsync(grad_amp, c->d_grad, sizeof(double) * c->htm.ncomp, cudaMemcpyDeviceToHost, c->stream));
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  int status = 0;
  LA_CUDA(c, cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status) return status_error(c, status);
  return LA_OK;
}

// ------------------------------------------------------------------ device-side relaxation loop
// One graph per context: a kernel sets the loop condition from the starting iterate's action, then a
// conditional WHILE node repeats { cycle (V-cycle and action norm, on the device only), condition }.
// Launched once per step on the context's stream, it relaxes to the stopping rule without any host
// synchronisation; the step's cycles, N and N(0) are recorded on the device.
static la_status build_loop_graph(la_ctx* c) {
  if (c->loop_exec) return LA_OK;
  if (!c->d_lstate) {
    void* p = nullptr;
    LA_TRY(dalloc(c, &p, sizeof(LoopState)));
    c->d_lstate = (LoopState*)p;
  }
  const la_config& k = c->cfg;
  const int check = k.tol > 0 ? 1 : 0;
  cudaGraph_t g = nullptr;
  LA_CUDA(c, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  cudaStream_t user = c->stream;
  const long long l0 = c->launches;
  cudaGraphNode_t head = nullptr, wnode = nullptr;
  cudaGraph_t out = nullptr;
  la_status st = LA_OK;
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(c->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    launch_loop_cond(c->d_lstate, c->d_N, k.tol, k.max_cycles, check, 1, h, c->cap);
    e = cudaStreamEndCapture(c->cap, &out);
  }
  size_t nn = 1;
  if (e == cudaSuccess) e = cudaGraphGetNodes(g, &head, &nn);
  cudaGraphNodeParams cp = {};
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, g, &head, nullptr, 1, &cp);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      // a conditional body holds kernels, memsets and copies only: no profiling events
      const bool prof = c->prof;
      c->prof = false;
      c->stream = c->cap;
      c->capturing = true;
      c->device_norm = true;
      st = cycle_body(c);
      if (st == LA_OK) launch_loop_cond(c->d_lstate, c->d_N, k.tol, k.max_cycles, check, 0, h, c->cap);
      cudaError_t ee = cudaStreamEndCapture(c->cap, &out);
      c->stream = user;
      c->capturing = false;
      c->device_norm = false;
      c->prof = prof;
      if (e == cudaSuccess) e = ee;
    }
  }
  c->launches = l0;
  if (st == LA_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->loop_exec, g, 0);
  cudaGraphDestroy(g);
  if (st != LA_OK) return st;
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->loop_exec = nullptr;
    return fail(c, LA_ECUDA, "relaxation loop graph: %s", cudaGetErrorString(e));
  }
  return LA_OK;
}

extern "C" la_status la_step_batch(la_ctx* const* ctxs, int nctx, void* const* psis, int nsteps, const double* t0s,
                                   la_step_stats* stats) {
  if (!ctxs || !psis || !t0s || nctx < 1 || nsteps < 0) return LA_EINVAL;
  for (int i = 0; i < nctx; ++i) {
    if (!ctxs[i] || !psis[i]) return LA_EINVAL;
    if (!ctxs[i]->have_ham) return fail(ctxs[i], LA_ESTATE, "la_set_hamiltonian must be called first");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], LA_EINVAL, "a context appears twice in the batch");
  }
  std::vector<cudaStream_t> user(nctx);
  std::vector<char> dev(nctx);
  la_status st = LA_OK;
  // every context works on its own internal stream for the whole call (forked from its stream)
  for (int i = 0; i < nctx && st == LA_OK; ++i) {
    la_ctx* c = ctxs[i];
    st = build_loop_graph(c);
    if (st == LA_OK && nsteps > c->lrec_cap) {
      void* p = nullptr;
      st = dalloc(c, &p, sizeof(LoopRecord) * (size_t)nsteps);
      if (st == LA_OK) {
        c->d_lrec = (LoopRecord*)p;
        c->lrec_cap = nsteps;
      }
    }
  }
  if (st != LA_OK) return st;
  for (int i = 0; i < nctx; ++i) {
    la_ctx* c = ctxs[i];
    user[i] = c->stream;
    LA_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    LA_CUDA(c, cudaStreamWaitEvent(c->cap, c->ev_fork, 0));
    c->stream = c->cap;
    dev[i] = is_device_ptr(psis[i]);
    if (!(std::fabs(t0s[i] - c->hist_t_next) <= 1e-9 * std::fabs(c->cfg.dt))) c->nhist = 0;
    LA_CUDA(c, cudaMemcpyAsync(c->d_psi, psis[i], sizeof(double2) * (size_t)c->np0,
                               dev[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  }
  // Every step of every context is enqueued without waiting: time matrices, factorisation, the starting
  // iterate (trial or zero, decided on the device), the relaxation loop graph, the step record and the
  // advance.  The contexts' streams run concurrently; the host synchronises once, at the end.
  for (int s = 0; s < nsteps && st == LA_OK; ++s) {
    for (int i = 0; i < nctx && st == LA_OK; ++i) {
      la_ctx* c = ctxs[i];
      st = setup_step(c, t0s[i] + s * c->cfg.dt);
      if (st == LA_OK) st = c->cfg.precision == 0 ? factor_all<double>(c) : factor_all<float>(c);
      bool tried = false;
      if (st == LA_OK) {
        c->device_norm = true;
        st = seed_enqueue(c, true, &tried);
        c->device_norm = false;
      }
      if (st == LA_OK) {
        launch_seed_select(c->nunk0, c->d_N, tried ? 1 : 0, c->d_lstate, c->d_c, c->d_r, c->d_f, c->stream);
        const cudaError_t e = cudaGraphLaunch(c->loop_exec, c->stream);
        if (e != cudaSuccess) st = fail(c, LA_ECUDA, "relaxation loop launch: %s", cudaGetErrorString(e));
      }
      if (st == LA_OK) {
        launch_loop_record(c->d_lstate, c->d_lrec + s, c->stream);
        launch_advance(c->np0, c->d_tm, c->d_c, c->d_psi, c->stream);
        c->launches += 3;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(c, LA_ECUDA, "batch step: %s", cudaGetErrorString(e));
      }
      if (st == LA_OK) st = hist_push(c);
      c->hist_t_next = t0s[i] + (s + 1) * c->cfg.dt;
    }
  }
  // results back, streams restored and joined
  std::vector<std::vector<LoopRecord>> rec(nctx);
  for (int i = 0; i < nctx; ++i) {
    la_ctx* c = ctxs[i];
    rec[i].resize((size_t)std::max(nsteps, 1));
    if (st == LA_OK && nsteps > 0)
      cudaMemcpyAsync(rec[i].data(), c->d_lrec, sizeof(LoopRecord) * (size_t)nsteps, cudaMemcpyDeviceToHost, c->stream);
    if (st == LA_OK)
      cudaMemcpyAsync(psis[i], c->d_psi, sizeof(double2) * (size_t)c->np0,
                      dev[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
    cudaEventRecord(c->ev_join, c->cap);
    c->stream = user[i];
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  }
  for (int i = 0; i < nctx; ++i) {
    if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess && st == LA_OK)
      st = fail(ctxs[i], LA_ECUDA, "synchronisation failed");
  }
  if (st != LA_OK) return st;
  la_status worst = LA_OK;
  for (int i = 0; i < nctx; ++i) {
    la_ctx* c = ctxs[i];
    int status = 0;
    if (cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || status) {
      cudaMemset(c->d_status, 0, sizeof(int));
      return status_error(c, status);
    }
    for (int s = 0; s < nsteps; ++s) {
      const LoopRecord& r = rec[i][s];
      c->last_N = r.N;
      c->last_rel = r.N0 > 0 ? r.N / r.N0 : 0.0;
      c->have_step = true;
      if (stats) {
        la_step_stats& o = stats[(size_t)i * nsteps + s];
        o.cycles = r.cycles;
        o.fine_sweeps = r.cycles * (c->cfg.nu1 + c->cfg.nu2);
        o.action = r.N;
        o.rel_action = c->last_rel;
      }
      // canary as in la_step: a non-finite action fails the member whatever its tolerance
      if (!std::isfinite(r.N)) {
        fail(c, LA_ENOTCONV, "the action is not finite after %d cycles (step %d)", r.cycles, s);
        worst = LA_ENOTCONV;
      } else if (c->cfg.tol > 0 && !(r.N <= c->cfg.tol * r.N0)) {
        fail(c, LA_ENOTCONV, "not converged after %d cycles (step %d, rel %.3e)", r.cycles, s, c->last_rel);
        worst = LA_ENOTCONV;
      }
    }
  }
  return worst;
}

extern "C" la_status la_action(la_ctx* c, double* N, double* rel) {
  if (!c) return LA_EINVAL;
  if (!c->have_step) return fail(c, LA_ESTATE, "no step has been computed");
  if (N) *N = c->last_N;
  if (rel) *rel = c->last_rel;
  return LA_OK;
}

extern "C" la_status la_solve_step(la_ctx* c, const void* psi0, double t0, int ncycles, void* c_out,
                                   la_step_stats* stats) {
  if (!c || !psi0 || !c_out || ncycles < 0) return c ? fail(c, LA_EINVAL, "invalid argument") : LA_EINVAL;
  if (!c->have_ham) return fail(c, LA_ESTATE, "la_set_hamiltonian must be called first");
  LA_TRY(load_any(c, c->d_psi, psi0, sizeof(double2) * (size_t)c->np0));
  LA_TRY(setup_step(c, t0));
  la_status st = solve_current(c, ncycles, stats);
  if (st != LA_OK && st != LA_ENOTCONV) return st;
  LA_TRY(store_any(c, c_out, c->d_c, sizeof(double2) * (size_t)c->nunk0));
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  return st;
}

extern "C" la_status la_residual(la_ctx* c, const void* psi0, double t0, const void* cin, void* r_out,
                                 double* action) {
  if (!c || !psi0 || !cin) return c ? fail(c, LA_EINVAL, "invalid argument") : LA_EINVAL;
  if (!c->have_ham) return fail(c, LA_ESTATE, "la_set_hamiltonian must be called first");
  LA_TRY(load_any(c, c->d_psi, psi0, sizeof(double2) * (size_t)c->np0));
  LA_TRY(load_any(c, c->d_c, cin, sizeof(double2) * (size_t)c->nunk0));
  LA_TRY(setup_step(c, t0));
  double N = 0.0;
  LA_TRY(action_now(c, &N));
  if (action) *action = N;
  if (r_out) {
    // the kernels work with r~ = r / h^d (overlap factor O = h^d dropped); return the paper's r
    launch_scale_c128(c->nunk0, c->hd, c->d_r, c->d_z, c->stream);
    LA_CHECK_LAUNCH(c);
    LA_TRY(store_any(c, r_out, c->d_z, sizeof(double2) * (size_t)c->nunk0));
  }
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  return LA_OK;
}

extern "C" la_status la_relax_colour(la_ctx* c, const void* psi0, double t0, int colour, void* cio) {
  if (!c || !psi0 || !cio) return c ? fail(c, LA_EINVAL, "invalid argument") : LA_EINVAL;
  if (colour < 0 || colour >= (c->cfg.local_form == 1 ? 2 : (1 << c->dim)))
    return fail(c, LA_EINVAL, "colour out of range");
  if (!c->have_ham) return fail(c, LA_ESTATE, "la_set_hamiltonian must be called first");
  LA_TRY(load_any(c, c->d_psi, psi0, sizeof(double2) * (size_t)c->np0));
  LA_TRY(load_any(c, c->d_c, cio, sizeof(double2) * (size_t)c->nunk0));
  LA_TRY(setup_step(c, t0));
  cudaError_t e;
  if (c->cfg.local_form == 1) {
    LA_TRY(factor_all<double>(c));
    e = launch_sweep_square(c->geo[0], c->fine, c->d_tm, c->K, c->d_f, c->d_c, (const double2*)c->d_fac[0],
                            c->d_perm, colour, c->stream);
  } else if (c->cfg.precision == 0) {
    LA_TRY(factor_all<double>(c));
    e = launch_sweep_fine<double>(c->geo[0], c->fine, c->d_tm, c->K, c->d_f, nullptr, c->d_c,
                                  (const double2*)c->d_fac[0], colour, c->d_status, c->stream);
  } else {
    LA_TRY(factor_all<float>(c));
    launch_c128_to_c64(c->nunk0, c->d_f, c->d_f32, c->stream);
    launch_c128_to_c64(c->nunk0, c->d_c, c->d_e32, c->stream);
    e = launch_sweep_fine<float>(c->geo[0], c->fine, c->d_tm, c->K, c->d_f32, nullptr, c->d_e32,
                                 (const float2*)c->d_fac[0], colour, c->d_status, c->stream);
    LA_CUDA(c, cudaMemsetAsync(c->d_c, 0, sizeof(double2) * (size_t)c->nunk0, c->stream));
    launch_axpy_c64_to_c128(c->nunk0, c->d_e32, c->d_c, c->stream);
  }
  if (e != cudaSuccess) return fail(c, LA_ECUDA, "sweep: %s", cudaGetErrorString(e));
  LA_CHECK_LAUNCH(c);
  LA_TRY(store_any(c, cio, c->d_c, sizeof(double2) * (size_t)c->nunk0));
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  int status = 0;
  LA_CUDA(c, cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status) return status_error(c, status);
  return LA_OK;
}

extern "C" la_status la_time_matrices(la_ctx* c, double t0, double* out) {
  if (!c || !out) return LA_EINVAL;
  launch_time_matrices(c->d_tm, t0, c->stream);
  LA_CHECK_LAUNCH(c);
  TimeMats t;
  LA_CUDA(c, cudaMemcpyAsync(&t, c->d_tm, sizeof(TimeMats), cudaMemcpyDeviceToHost, c->stream));
  LA_CUDA(c, cudaStreamSynchronize(c->stream));
  const int K = c->K, KK = K * K;
  memcpy(out, t.Ub, sizeof(double) * KK);
  memcpy(out + KK, t.Qb, sizeof(double) * KK);
  memcpy(out + 2 * KK, t.Eb, sizeof(double) * KK);
  memcpy(out + 3 * KK, t.Ub0, sizeof(double) * K);
  memcpy(out + 3 * KK + K, t.Eb0, sizeof(double) * K);
  memcpy(out + 3 * KK + 2 * K, t.Wt, sizeof(double) * KK);
  return LA_OK;
}
