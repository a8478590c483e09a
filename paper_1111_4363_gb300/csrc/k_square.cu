// Square-form subvolume relaxation on the finest level (Sec. II, the local problem in the
// preconditioner form): for every subvolume U of a colour,
//     M~_UU delta_U = (f~ - M~ c)_U,   c_U += delta_U,
// with delta = 0 outside U (the boundary values) and the initial condition already eliminated
// from M~.  M~ couples edge neighbours only, so the two-colour checkerboard of subvolumes
// (colour = parity of the sum of the block indices) makes same-colour updates independent.
// FP64 only.
//
// Factor store of one subvolume: the LU factors of P M~_UU (partial pivoting), column-major,
// NPAD x NPAD complex128: column k holds L below the diagonal (unit diagonal implied), U on and
// above it with the reciprocal of the pivot in place of U_kk; and the row permutation perm
// (NPAD ints) with (P r)_i = r_perm[i].  Padding rows and columns are identity.
#include "la_internal.cuh"

namespace la {
namespace {

constexpr int kSqFactorThreads = 256;
constexpr int kSqSweepThreads = 128;   // one thread per row of a subvolume system (NPAD <= 128)
constexpr int kSqPrefetch = 8;         // factor columns a sweep thread holds in flight

__device__ __forceinline__ double2 cmul(const double2 a, const double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc -= a * b
__device__ __forceinline__ void cfms(double2& acc, const double2 a, const double2 b) {
  acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ void sq_coords(int i, const int e[3], int& x, int& y, int& z) {
  x = i % e[0];
  const int r = i / e[0];
  y = r % e[1];
  z = r / e[1];
}

__device__ __forceinline__ int red_black(const LevelGeom& L, int b) {
  const int bx = b % L.nb[0], r = b / L.nb[0];
  return (bx + r % L.nb[1] + r / L.nb[1]) & 1;
}

// ------------------------------------------------------------------------------ factorisation
// One CTA per subvolume; the dense matrix lives in shared memory (row-major).  Right-looking LU
// with partial pivoting, per column: warp 0 finds the pivot (largest |a|^2, first index on ties),
// the CTA swaps the two rows in full, forms the multipliers, and applies the rank-1 update to the
// trailing block; the pivot's reciprocal replaces it on the diagonal.
template <int NPAD>
__global__ void __launch_bounds__(kSqFactorThreads, 1)
k_factor_square(LevelGeom L, FineOp g, const TimeMats* __restrict__ tm, double2* __restrict__ lu,
                int* __restrict__ perm, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  double2* A = reinterpret_cast<double2*>(smem);                  // [NPAD][NPAD]
  double2* sInvP = A + NPAD * NPAD;                                // reciprocal of the current pivot
  double* sQ = reinterpret_cast<double*>(sInvP + 1);               // [K][K]
  double* sU = sQ + LA_KMAX * LA_KMAX;
  double* sE = sU + LA_KMAX * LA_KMAX;
  int* sPerm = reinterpret_cast<int*>(sE + LA_KMAX * LA_KMAX);     // [NPAD]
  int* sPiv = sPerm + NPAD;                                        // [1]
  const int tid = threadIdx.x, b = blockIdx.x;
  const int K = tm->K, KK = K * K;
  int o[3], e[3];
  subvol_box(L, b, o, e);
  const int n = e[0] * e[1] * e[2] * K;
  for (int i = tid; i < KK; i += kSqFactorThreads) { sQ[i] = tm->Qb[i]; sU[i] = tm->Ub[i]; sE[i] = tm->Eb[i]; }
  for (int i = tid; i < NPAD; i += kSqFactorThreads) sPerm[i] = i;
  __syncthreads();
  // M~_(p m),(q nn) = i Qb[m][nn] d_pq - Ub[m][nn] H_pq - x_p Eb[m][nn] d_pq
  for (int t = tid; t < NPAD * NPAD; t += kSqFactorThreads) {
    const int i = t / NPAD, j = t % NPAD;
    double2 v = make_double2(i == j ? 1.0 : 0.0, 0.0);
    if (i < n && j < n) {
      const int p = i / K, m = i % K, q = j / K, nn = j % K;
      int px, py, pz, qx, qy, qz;
      sq_coords(p, e, px, py, pz);
      sq_coords(q, e, qx, qy, qz);
      px += o[0]; py += o[1]; pz += o[2];
      qx += o[0]; qy += o[1]; qz += o[2];
      const double Hpq = fine_H(g, px, py, pz, qx, qy, qz);
      const int mn = m * K + nn;
      v.x = -sU[mn] * Hpq;
      v.y = 0.0;
      if (p == q) {
        v.x -= fine_x(g, px, py, pz) * sE[mn];
        v.y = sQ[mn];
      }
    }
    A[t] = v;
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  for (int k = 0; k < NPAD; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < NPAD; i += 32) {
        const double2 a = A[i * NPAD + k];
        const double v = a.x * a.x + a.y * a.y;
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, s);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, s);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        if (!(best > 0.0)) { atomicOr(status, 1); bi = k; }
        *sPiv = bi;
        const int t = sPerm[k]; sPerm[k] = sPerm[bi]; sPerm[bi] = t;
        // one complex reciprocal per column, shared (an FP64 division per thread would cost as
        // much as the column's rank-1 update)
        const double2 d = A[bi * NPAD + k];
        const double sq = d.x * d.x + d.y * d.y;
        *sInvP = sq > 0.0 ? make_double2(d.x / sq, -d.y / sq) : make_double2(1.0, 0.0);
      }
    }
    __syncthreads();
    const int p = *sPiv;
    if (p != k)
      for (int j = tid; j < NPAD; j += kSqFactorThreads) {
        const double2 t = A[k * NPAD + j];
        A[k * NPAD + j] = A[p * NPAD + j];
        A[p * NPAD + j] = t;
      }
    __syncthreads();
    const double2 inv = *sInvP;
    for (int i = k + 1 + tid; i < NPAD; i += kSqFactorThreads) A[i * NPAD + k] = cmul(A[i * NPAD + k], inv);
    __syncthreads();
    for (int i = k + 1 + ty; i < NPAD; i += kSqFactorThreads / 16) {
      const double2 l = A[i * NPAD + k];
      for (int j = k + 1 + tx; j < NPAD; j += 16) cfms(A[i * NPAD + j], l, A[k * NPAD + j]);
    }
    if (tid == 0) A[k * NPAD + k] = inv;
    __syncthreads();
  }
  double2* F = lu + (size_t)b * NPAD * NPAD;
  for (int t = tid; t < NPAD * NPAD; t += kSqFactorThreads) {
    const int col = t / NPAD, row = t % NPAD;
    F[t] = A[row * NPAD + col];
  }
  for (int i = tid; i < NPAD; i += kSqFactorThreads) perm[(size_t)b * NPAD + i] = sPerm[i];
}

// ------------------------------------------------------------------------------ sweep
// One CTA per subvolume (those of the other colour return at once).  The residual rows of U,
// r = f~ - M~ c, are formed from c on U + 1 in shared memory; then thread i owns row i of the
// system: y = P r, forward substitution with unit L, backward substitution with U (pivot
// reciprocals on the diagonal), one barrier per column, the factor columns streamed from global
// memory kSqPrefetch columns ahead (coalesced: column k is contiguous).
template <int NPAD>
__global__ void __launch_bounds__(kSqSweepThreads)
k_sweep_square(LevelGeom L, FineOp g, const TimeMats* __restrict__ tm, const double2* __restrict__ f,
               double2* __restrict__ c, const double2* __restrict__ lu, const int* __restrict__ perm, int colour) {
  static_assert(NPAD <= kSqSweepThreads && NPAD % kSqPrefetch == 0, "one row per thread");
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x;
  if (red_black(L, b) != colour) return;
  const int tid = threadIdx.x, K = tm->K, KK = K * K;
  int o[3], e[3], eb[3], ob[3];
  subvol_box(L, b, o, e);
  for (int a = 0; a < 3; ++a) {
    const bool used = a < L.dim;
    eb[a] = used ? e[a] + 2 : 1;
    ob[a] = used ? o[a] - 1 : o[a];
  }
  const int npts = e[0] * e[1] * e[2], n = npts * K, nbox = eb[0] * eb[1] * eb[2];
  const int nbox_max = (L.sub[0] + 2) * (L.dim > 1 ? L.sub[1] + 2 : 1) * (L.dim > 2 ? L.sub[2] + 2 : 1);
  double* sQ = reinterpret_cast<double*>(smem);
  double* sU = sQ + LA_KMAX * LA_KMAX;
  double* sE = sU + LA_KMAX * LA_KMAX;
  double2* sC = reinterpret_cast<double2*>(sE + LA_KMAX * LA_KMAX);   // c on U + 1 [nbox_max * K]
  double2* sH = sC + (size_t)nbox_max * K;                            // H c on U [NPAD]
  double2* sY = sH + NPAD;                                            // r, then the broadcast entries [NPAD]

  // factor columns 0 .. kSqPrefetch-1 of this thread's row, issued first
  const double2* F = lu + (size_t)b * NPAD * NPAD;
  const int row = tid < NPAD ? tid : NPAD - 1;
  double2 pf[kSqPrefetch];
#pragma unroll
  for (int u = 0; u < kSqPrefetch; ++u) pf[u] = F[u * NPAD + row];
  const int pr = perm[(size_t)b * NPAD + row];

  for (int i = tid; i < KK; i += kSqSweepThreads) { sQ[i] = tm->Qb[i]; sU[i] = tm->Ub[i]; sE[i] = tm->Eb[i]; }
  for (int t = tid; t < nbox * K; t += kSqSweepThreads) {
    const int i = t / K, m = t % K;
    int lx, ly, lz;
    sq_coords(i, eb, lx, ly, lz);
    const int gx = ob[0] + lx, gy = ob[1] + ly, gz = ob[2] + lz;
    sC[t] = fine_in(g, gx, gy, gz) ? c[(size_t)((gz * g.n[1] + gy) * g.n[0] + gx) * K + m] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // box index of U point (lx, ly, lz): +1 on used axes
  const int sy = L.dim > 1 ? eb[0] : 0, sz = L.dim > 2 ? eb[0] * eb[1] : 0;
  const double wx = -0.5 * g.ih2[0], wy = -0.5 * g.ih2[1], wz = -0.5 * g.ih2[2];
  for (int t = tid; t < n; t += kSqSweepThreads) {
    const int i = t / K, m = t % K;
    int lx, ly, lz;
    sq_coords(i, e, lx, ly, lz);
    const int bi = (lx + 1) + (L.dim > 1 ? (ly + 1) * sy : 0) + (L.dim > 2 ? (lz + 1) * sz : 0);
    const int gx = o[0] + lx, gy = o[1] + ly, gz = o[2] + lz;
    const double dg = g.dsum + g.V0[(gz * g.n[1] + gy) * g.n[0] + gx];
    const double2 v = sC[bi * K + m];
    double2 h = make_double2(dg * v.x, dg * v.y);
    {
      const double2 a1 = sC[(bi + 1) * K + m], a2 = sC[(bi - 1) * K + m];
      h.x += wx * (a1.x + a2.x); h.y += wx * (a1.y + a2.y);
    }
    if (L.dim > 1) {
      const double2 a1 = sC[(bi + sy) * K + m], a2 = sC[(bi - sy) * K + m];
      h.x += wy * (a1.x + a2.x); h.y += wy * (a1.y + a2.y);
    }
    if (L.dim > 2) {
      const double2 a1 = sC[(bi + sz) * K + m], a2 = sC[(bi - sz) * K + m];
      h.x += wz * (a1.x + a2.x); h.y += wz * (a1.y + a2.y);
    }
    sH[t] = h;
  }
  __syncthreads();
  // r = f~ - (i Qb c - Ub H c - x Eb c) on the rows of U; padding 0
  for (int t = tid; t < NPAD; t += kSqSweepThreads) {
    double2 r = make_double2(0.0, 0.0);
    if (t < n) {
      const int i = t / K, m = t % K;
      int lx, ly, lz;
      sq_coords(i, e, lx, ly, lz);
      const int bi = (lx + 1) + (L.dim > 1 ? (ly + 1) * sy : 0) + (L.dim > 2 ? (lz + 1) * sz : 0);
      const int gx = o[0] + lx, gy = o[1] + ly, gz = o[2] + lz;
      const double xl = fine_x(g, gx, gy, gz);
      double qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
      for (int nn = 0; nn < K; ++nn) {
        const double2 cv = sC[bi * K + nn], hv = sH[i * K + nn];
        const double q = sQ[m * K + nn], u = sU[m * K + nn], ee = sE[m * K + nn];
        qr = fma(q, cv.x, qr); qi = fma(q, cv.y, qi);
        ur = fma(u, hv.x, ur); ui = fma(u, hv.y, ui);
        er = fma(ee, cv.x, er); ei = fma(ee, cv.y, ei);
      }
      const double2 fv = f ? f[(size_t)((gz * g.n[1] + gy) * g.n[0] + gx) * K + m] : make_double2(0.0, 0.0);
      r.x = fv.x - (-qi - ur - xl * er);
      r.y = fv.y - (qr - ui - xl * ei);
    }
    sY[t] = r;
  }
  __syncthreads();
  const bool own = tid < NPAD;
  double2 y = sY[pr];          // y = P r
  __syncthreads();
  // Only the warps that own rows take part, and each step's barrier (id 1) counts just the warps
  // that still have work in it: in the forward pass warp w is done after column 32 w + 31, in the
  // backward pass before column 32 w.  (A predicated update in finished warps would still occupy the
  // FP64 pipe.)  Id 2 separates the two passes.
  constexpr int NWo = (NPAD + 31) / 32;
  const int w = tid >> 5;
  if (w < NWo) {
    // forward: unit lower L, column k updates the rows below it
    for (int k0 = 0; k0 < NPAD; k0 += kSqPrefetch) {
      if (k0 >= 32 * (w + 1)) break;
      const unsigned cnt = 32u * (unsigned)(NWo - (k0 >> 5));
#pragma unroll
      for (int u = 0; u < kSqPrefetch; ++u) {
        const int k = k0 + u;
        const double2 lk = pf[u];
        if (k + kSqPrefetch < NPAD) pf[u] = F[(k + kSqPrefetch) * NPAD + row];
        if (tid == k) sY[k] = y;
        asm volatile("bar.sync 1, %0;" ::"r"(cnt) : "memory");
        if (own && tid > k) cfms(y, lk, sY[k]);
      }
    }
    asm volatile("bar.sync 2, %0;" ::"r"(32u * NWo) : "memory");
    // backward: columns of U from the last; x_k = y_k / U_kk
#pragma unroll
    for (int u = 0; u < kSqPrefetch; ++u) pf[u] = F[(NPAD - 1 - u) * NPAD + row];
    for (int k0 = NPAD - 1; k0 >= 0; k0 -= kSqPrefetch) {
      if (k0 < 32 * w) break;
      const unsigned cnt = 32u * (unsigned)((k0 >> 5) + 1);
#pragma unroll
      for (int u = 0; u < kSqPrefetch; ++u) {
        const int k = k0 - u;
        const double2 uk = pf[u];
        if (k - kSqPrefetch >= 0) pf[u] = F[(k - kSqPrefetch) * NPAD + row];
        if (tid == k) {
          y = cmul(y, uk);     // uk = 1 / U_kk on the diagonal
          sY[k] = y;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(cnt) : "memory");
        if (own && tid < k) cfms(y, uk, sY[k]);
      }
    }
  }
  if (own && tid < n) {
    const int i = tid / K, m = tid % K;
    int lx, ly, lz;
    sq_coords(i, e, lx, ly, lz);
    const size_t gi = (size_t)(((o[2] + lz) * g.n[1] + (o[1] + ly)) * g.n[0] + (o[0] + lx)) * K + m;
    double2 v = c[gi];
    v.x += y.x;
    v.y += y.y;
    c[gi] = v;
  }
}

template <int NPAD>
cudaError_t factor_square_n(const LevelGeom& L, const FineOp& g, const TimeMats* tm, double2* lu, int* perm,
                            int* status, cudaStream_t s) {
  const size_t smem = sizeof(double2) * (NPAD * NPAD + 1) + sizeof(double) * 3 * LA_KMAX * LA_KMAX +
                      sizeof(int) * (NPAD + 1);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_factor_square<NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           227 * 1024);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  k_factor_square<NPAD><<<L.nsub, kSqFactorThreads, smem, s>>>(L, g, tm, lu, perm, status);
  return cudaGetLastError();
}

template <int NPAD>
cudaError_t sweep_square_n(const LevelGeom& L, const FineOp& g, const TimeMats* tm, int K, const double2* f,
                           double2* c, const double2* lu, const int* perm, int colour, cudaStream_t s) {
  const int nbox = (L.sub[0] + 2) * (L.dim > 1 ? L.sub[1] + 2 : 1) * (L.dim > 2 ? L.sub[2] + 2 : 1);
  const size_t smem = sizeof(double) * 3 * LA_KMAX * LA_KMAX + sizeof(double2) * ((size_t)nbox * K + 2 * NPAD);
  k_sweep_square<NPAD><<<L.nsub, kSqSweepThreads, smem, s>>>(L, g, tm, f, c, lu, perm, colour);
  return cudaGetLastError();
}

}  // namespace

#define LA_SQ_DISPATCH(NPADV, CALL) \
  switch (NPADV) {                  \
    case 16: return CALL(16);       \
    case 32: return CALL(32);       \
    case 48: return CALL(48);       \
    case 64: return CALL(64);       \
    case 96: return CALL(96);       \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_factor_square(const LevelGeom& L, const FineOp& g, const TimeMats* tm, double2* lu, int* perm,
                                 int* status, cudaStream_t s) {
#define LA_CALL(N) factor_square_n<N>(L, g, tm, lu, perm, status, s)
  LA_SQ_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}

cudaError_t launch_sweep_square(const LevelGeom& L, const FineOp& g, const TimeMats* tm, int K, const double2* f,
                                double2* c, const double2* lu, const int* perm, int colour, cudaStream_t s) {
#define LA_CALL(N) sweep_square_n<N>(L, g, tm, K, f, c, lu, perm, colour, s)
  LA_SQ_DISPATCH(L.npad, LA_CALL)
#undef LA_CALL
}

}  // namespace la
