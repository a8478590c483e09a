// Residual norm N for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc: code that runs inside a host framework which owns all
// device memory through its own pool, or a process that has exhausted or pinned its device
// budget.  la_action_noalloc gives them the action residual norm N of trial coefficients without
// any allocation.  Its scratch (the per-step time matrices, the per-block partial sums and the
// result) lives in one file-scope __device__ array of fixed size.
//
// Limits and sharing rules:
//   * at most LA_NOALLOC_MAX_POINTS grid points; larger grids are rejected with LA_EINVAL;
//   * V0, psi0 and c must be device (or managed) memory; host pointers are rejected with LA_EINVAL;
//   * every GPU that loads this library holds the array (about 140 KB) until the process exits;
//   * all calls share the array: each call overwrites it completely before reading it, so no state
//     leaks between calls, but calls that overlap on the GPU (different streams or host threads)
//     race on it and must be serialised by the caller;
//   * set-up: the first call in a CUDA context (normally the primary context of a device) looks up
//     the array's device address (cudaGetSymbolAddress) with that device current and keeps it for
//     that context.  The address is keyed by the context's unique id, so a context created later on
//     the same device (after cudaDeviceReset, or a caller-created context) gets its own lookup
//     instead of a stale address;
//   * under lazy module loading (the CUDA default) the first call in a context may load this
//     library's module, which takes device memory for its code and this array; a process that must
//     not allocate at all sets CUDA_MODULE_LOADING=EAGER or makes one call early.
#include <mutex>
#include <string>

#include "la_internal.cuh"
#include "../../include/leastaction.h"

namespace la {
bool time_constants_for(const la_config& cfg, TimeMats& out);
void set_thread_error(const char* msg);
}

using namespace la;

namespace {

constexpr int kMaxPoints = LA_NOALLOC_MAX_POINTS;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = (kMaxPoints + kThreads - 1) / kThreads;
constexpr size_t kTmBytes = (sizeof(TimeMats) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kTmBytes + sizeof(double) * (kMaxBlocks + 32);

// Host code sees only a stand-in for this symbol; its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
// (context id, scratch address) of the contexts seen so far; a small ring, newest overwriting oldest
constexpr int kCacheSlots = 64;
struct CacheSlot {
  unsigned long long id;
  void* addr;
};
CacheSlot g_cache[kCacheSlots] = {};
int g_cache_next = 0;

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

// Unique id of the CUDA context current on this thread (0 when none is current or the driver
// entry points are unavailable).
unsigned long long current_context_id() {
  static PfnCtxGetCurrent get_cur = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PfnCtxGetCurrent>(f1);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PfnCtxGetId>(f2);
    cudaGetLastError();
    looked_up = true;
  }
  if (!get_cur || !get_id) return 0;
  CUcontext cu = nullptr;
  if (get_cur(&cu) != CUDA_SUCCESS || !cu) return 0;
  unsigned long long id = 0;
  if (get_id(cu, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context: looked up once per context (with
// the device current) and cached by the context's id.
la_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    set_thread_error("la_action_noalloc: no CUDA device");
    return LA_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = current_context_id();
  if (id != 0)
    for (int i = 0; i < kCacheSlots; ++i)
      if (g_cache[i].id == id) {
        *out = g_cache[i].addr;
        return LA_OK;
      }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    set_thread_error(e != cudaSuccess ? cudaGetErrorString(e) : "la_action_noalloc: null scratch address");
    return LA_ECUDA;
  }
  // the lookup makes the device's primary context current when none was
  if (id == 0) id = current_context_id();
  if (id != 0) {
    g_cache[g_cache_next] = CacheSlot{id, p};
    g_cache_next = (g_cache_next + 1) % kCacheSlots;
  }
  *out = p;
  return LA_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Variant of the residual kernel that forms f~ from psi0 on the fly instead of reading a stored
// right-hand side, and writes only the per-block partial sums of r~^dagger Wt r~.
__global__ void __launch_bounds__(kThreads) k_action_partials(FineOp g, const TimeMats* __restrict__ tm,
                                                              const double2* __restrict__ psi0,
                                                              const double2* __restrict__ c,
                                                              double* __restrict__ partials) {
  __shared__ double Qb[LA_KMAX * LA_KMAX], Ub[LA_KMAX * LA_KMAX], Eb[LA_KMAX * LA_KMAX], Wt[LA_KMAX * LA_KMAX];
  __shared__ double Ub0[LA_KMAX], Eb0[LA_KMAX];
  __shared__ double red[kThreads];
  const int K = tm->K;
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    Qb[i] = tm->Qb[i]; Ub[i] = tm->Ub[i]; Eb[i] = tm->Eb[i]; Wt[i] = tm->Wt[i];
  }
  for (int i = threadIdx.x; i < K; i += blockDim.x) { Ub0[i] = tm->Ub0[i]; Eb0[i] = tm->Eb0[i]; }
  __syncthreads();
  const int np = g.n[0] * g.n[1] * g.n[2];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double nsum = 0.0;
  if (p < np) {
    const int x = p % g.n[0], y = (p / g.n[0]) % g.n[1], z = p / (g.n[0] * g.n[1]);
    const int nb[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    const double dg = g.dsum + g.V0[p];
    double2 hpsi = make_double2(dg * psi0[p].x, dg * psi0[p].y);
    double2 cp[LA_KMAX], hc[LA_KMAX];
    for (int m = 0; m < K; ++m) {
      cp[m] = c[(long long)p * K + m];
      hc[m] = make_double2(dg * cp[m].x, dg * cp[m].y);
    }
    for (int t = 0; t < 2 * g.dim; ++t) {
      const int qx = x + nb[t][0], qy = y + nb[t][1], qz = z + nb[t][2];
      if (qx < 0 || qy < 0 || qz < 0 || qx >= g.n[0] || qy >= g.n[1] || qz >= g.n[2]) continue;
      const double w = -0.5 * g.ih2[t >> 1];
      const int q = (qz * g.n[1] + qy) * g.n[0] + qx;
      hpsi.x += w * psi0[q].x;
      hpsi.y += w * psi0[q].y;
      for (int m = 0; m < K; ++m) {
        const double2 a = c[(long long)q * K + m];
        hc[m].x += w * a.x;
        hc[m].y += w * a.y;
      }
    }
    const double xl = fine_x(g, x, y, z);
    const double2 ps = psi0[p];
    double2 r[LA_KMAX];
    for (int m = 0; m < K; ++m) {
      double qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
      for (int n = 0; n < K; ++n) {
        const double q = Qb[m * K + n], u = Ub[m * K + n], e = Eb[m * K + n];
        qr += q * cp[n].x; qi += q * cp[n].y;
        ur += u * hc[n].x; ui += u * hc[n].y;
        er += e * cp[n].x; ei += e * cp[n].y;
      }
      const double fr = Ub0[m] * hpsi.x + xl * Eb0[m] * ps.x;
      const double fi = Ub0[m] * hpsi.y + xl * Eb0[m] * ps.y;
      r[m].x = fr - (-qi - ur - xl * er);
      r[m].y = fi - (qr - ui - xl * ei);
    }
    for (int m = 0; m < K; ++m) {
      double zr = 0, zi = 0;
      for (int n = 0; n < K; ++n) { zr += Wt[m * K + n] * r[n].x; zi += Wt[m * K + n] * r[n].y; }
      nsum += r[m].x * zr + r[m].y * zi;
    }
  }
  red[threadIdx.x] = nsum;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

}  // namespace

extern "C" la_status la_action_noalloc(const la_config* cfg, const double* V0, const la_pulse* pulse,
                                       const void* psi0, double t0, const void* c, double* action,
                                       void* cuda_stream) {
  if (!cfg || !V0 || !psi0 || !c || !action) {
    set_thread_error("la_action_noalloc: null argument");
    return LA_EINVAL;
  }
  const la_config& k = *cfg;
  if (k.dim < 1 || k.dim > 3 || k.nt < 1 || k.nt > LA_KMAX || !(k.dt > 0) || k.weight < 0 || k.weight > 2 ||
      k.laser_axis < 0 || k.laser_axis >= k.dim) {
    set_thread_error("la_action_noalloc: invalid configuration");
    return LA_EINVAL;
  }
  long long np = 1;
  FineOp g{};
  g.dim = k.dim;
  double hd = 1.0;
  for (int a = 0; a < 3; ++a) {
    if (a < k.dim && (k.n[a] < 1 || !(k.h[a] > 0))) {
      set_thread_error("la_action_noalloc: invalid grid");
      return LA_EINVAL;
    }
    if (a >= k.dim && k.n[a] != 1) {
      set_thread_error("la_action_noalloc: unused axes must have n = 1");
      return LA_EINVAL;
    }
    g.n[a] = a < k.dim ? k.n[a] : 1;
    // each factor is checked before the product grows: three axes of up to 2^31 points would
    // overflow even a 64-bit count
    if (g.n[a] > kMaxPoints || np * g.n[a] > kMaxPoints) {
      set_thread_error("la_action_noalloc: the grid exceeds LA_NOALLOC_MAX_POINTS points");
      return LA_EINVAL;
    }
    g.h[a] = a < k.dim ? k.h[a] : 1.0;
    g.ih2[a] = a < k.dim ? 1.0 / (k.h[a] * k.h[a]) : 0.0;
    g.x0[a] = -0.5 * (g.n[a] - 1) * g.h[a];
    if (a < k.dim) {
      g.dsum += g.ih2[a];
      hd *= k.h[a];
    }
    np *= g.n[a];
  }
  if (!on_device(V0) || !on_device(psi0) || !on_device(c)) {
    set_thread_error("la_action_noalloc: V0, psi0 and c must be device pointers");
    return LA_EINVAL;
  }
  const int nc = pulse ? pulse->ncomp : 0;
  if (nc < 0 || nc > LA_NCOMP_MAX || (nc > 0 && (!pulse->amp || !pulse->omega || !pulse->t_center || !pulse->sigma))) {
    set_thread_error("la_action_noalloc: invalid pulse");
    return LA_EINVAL;
  }
  g.lax = k.laser_axis;
  g.V0 = V0;
  TimeMats htm;
  if (!time_constants_for(k, htm)) {
    set_thread_error("la_action_noalloc: singular time-basis Gram matrix");
    return LA_EINVAL;
  }
  htm.ncomp = nc;
  for (int i = 0; i < nc; ++i) {
    htm.amp[i] = pulse->amp[i];
    htm.omega[i] = pulse->omega[i];
    htm.tc[i] = pulse->t_center[i];
    htm.sigma[i] = pulse->sigma[i];
  }
  void* base = nullptr;
  la_status st = scratch_for_current_device(&base);
  if (st != LA_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  TimeMats* tm = reinterpret_cast<TimeMats*>(base);
  double* partials = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kTmBytes);
  const int nblocks = (int)((np + kThreads - 1) / kThreads);
  double* d_N = partials + kMaxBlocks;
  const double nscale = k.weight == 0 ? hd : (k.weight == 1 ? hd * hd * hd : hd * hd);
  cudaError_t e = cudaMemcpyAsync(tm, &htm, sizeof(TimeMats), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    launch_time_matrices(tm, t0, s);
    k_action_partials<<<nblocks, kThreads, 0, s>>>(g, tm, static_cast<const double2*>(psi0),
                                                   static_cast<const double2*>(c), partials);
    launch_norm_final(partials, nblocks, nscale, d_N, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(action, d_N, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return LA_ECUDA;
  }
  return LA_OK;
}
