// Grid-wide kernels: per-step time matrices, right-hand side, action residual and residual
// norm, normal residual, Galerkin-level residual, intergrid transfers, step advance.
#include <algorithm>

#include "../../include/leastaction.h"
#include "la_internal.cuh"

namespace la {

// ------------------------------------------------------------------ complex helpers
template <typename T> struct CR;
template <> struct CR<double2> { typedef double R; };
template <> struct CR<float2> { typedef float R; };

template <typename CT> __device__ __forceinline__ CT cmk(typename CR<CT>::R a, typename CR<CT>::R b) {
  CT r; r.x = a; r.y = b; return r;
}

// ------------------------------------------------------------------ time matrices (Sec. I, IV)
// Eb[m,n] = (dt/2) sum_q w_q b_m(tau_q) b_n(tau_q) E(t_q), Eb0[m] = (dt/2) sum_q w_q b_m(tau_q) E(t_q),
// P_kk' = R_k^T Wt R_k' with R = (Qb, Ub, Eb).  One block.
__global__ void k_time_matrices(TimeMats* tm, double t0) {
  __shared__ double Eq[LA_NQ_MAX];
  __shared__ double R[3][LA_KMAX * LA_KMAX];
  __shared__ double Wt[LA_KMAX * LA_KMAX];
  const int K = tm->K, nq = tm->nq, KK = K * K;
  const double dt = tm->dt;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double t = t0 + 0.5 * (tm->tau[q] + 1.0) * dt;
    double e = 0.0;
    for (int k = 0; k < tm->ncomp; ++k) {
      double env = 1.0;
      if (tm->sigma[k] > 0.0) {
        double u = (t - tm->tc[k]) / tm->sigma[k];
        env = exp(-u * u);
      }
      e += tm->amp[k] * env * sin(tm->omega[k] * t);
    }
    Eq[q] = e;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < KK; i += blockDim.x) {
    int m = i / K, n = i % K;
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += tm->wq[q] * tm->bq[q * LA_KMAX + m] * tm->bq[q * LA_KMAX + n] * Eq[q];
    s *= 0.5 * dt;
    tm->Eb[i] = s;
    R[2][i] = s;
    R[0][i] = tm->Qb[i];
    R[1][i] = tm->Ub[i];
    Wt[i] = tm->Wt[i];
  }
  for (int m = threadIdx.x; m < K; m += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += tm->wq[q] * tm->bq[q * LA_KMAX + m] * Eq[q];
    tm->Eb0[m] = 0.5 * dt * s;
  }
  if (threadIdx.x == 0) tm->t0 = t0;
  __syncthreads();
  for (int i = threadIdx.x; i < LA_NPAIR * KK; i += blockDim.x) {
    int kk = i / KK, mn = i % KK, m = mn / K, n = mn % K;
    int k = kk / 3, kp = kk % 3;
    double s = 0.0;
    for (int a = 0; a < K; ++a) {
      double ra = R[k][a * K + m];
      if (ra == 0.0) continue;
      double t = 0.0;
      for (int b = 0; b < K; ++b) t += Wt[a * K + b] * R[kp][b * K + n];
      s += ra * t;
    }
    tm->P[kk][mn] = s;
  }
}

void launch_time_matrices(TimeMats* tm, double t0, cudaStream_t s) { k_time_matrices<<<1, 256, 0, s>>>(tm, t0); }

// ------------------------------------------------------------------ fine-level stencil helpers
__device__ __forceinline__ void pcoords(const FineOp& g, int p, int& x, int& y, int& z) {
  x = p % g.n[0];
  int r = p / g.n[0];
  y = r % g.n[1];
  z = r / g.n[1];
}

// K complex values of point p from a point-major field into registers (16-byte loads where the
// record allows: complex64 with even K pairs two values per load).
template <typename CT, int K>
__device__ __forceinline__ void load_k(const CT* __restrict__ v, long long p, CT (&out)[K]) {
  const CT* src = v + p * K;
  if constexpr (sizeof(CT) == 8 && K % 2 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int m = 0; m < K / 2; ++m) {
      const float4 q = s4[m];
      out[2 * m] = cmk<CT>(q.x, q.y);
      out[2 * m + 1] = cmk<CT>(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int m = 0; m < K; ++m) out[m] = src[m];
  }
}
template <typename CT, int K>
__device__ __forceinline__ void store_k(CT* __restrict__ v, long long p, const CT (&in)[K]) {
  CT* dst = v + p * K;
  if constexpr (sizeof(CT) == 8 && K % 2 == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int m = 0; m < K / 2; ++m) d4[m] = make_float4(in[2 * m].x, in[2 * m].y, in[2 * m + 1].x, in[2 * m + 1].y);
  } else {
#pragma unroll
    for (int m = 0; m < K; ++m) dst[m] = in[m];
  }
}
template <typename CT, typename RR, int K>
__device__ __forceinline__ void axpy_k(RR w, const CT (&a)[K], CT (&acc)[K]) {
#pragma unroll
  for (int m = 0; m < K; ++m) { acc[m].x += w * a[m].x; acc[m].y += w * a[m].y; }
}

// (H v)_p for a K-vector field v (point-major), Dirichlet zero outside the grid; also returns v_p.
// Neighbours in the order +x, -x, +y, -y, +z, -z.
template <typename CT, typename RR, int K>
__device__ __forceinline__ void apply_H(const FineOp& g, const CT* __restrict__ v, int p, int x, int y, int z,
                                        CT (&vp)[K], CT (&out)[K]) {
  const RR dg = (RR)(g.dsum + g.V0[p]);
  load_k<CT, K>(v, p, vp);
#pragma unroll
  for (int m = 0; m < K; ++m) out[m] = cmk<CT>(dg * vp[m].x, dg * vp[m].y);
  CT a[K];
  const RR wx = (RR)(-0.5 * g.ih2[0]);
  if (x + 1 < g.n[0]) { load_k<CT, K>(v, p + 1, a); axpy_k<CT, RR, K>(wx, a, out); }
  if (x > 0) { load_k<CT, K>(v, p - 1, a); axpy_k<CT, RR, K>(wx, a, out); }
  if (g.dim > 1) {
    const RR wy = (RR)(-0.5 * g.ih2[1]);
    const int sy = g.n[0];
    if (y + 1 < g.n[1]) { load_k<CT, K>(v, p + sy, a); axpy_k<CT, RR, K>(wy, a, out); }
    if (y > 0) { load_k<CT, K>(v, p - sy, a); axpy_k<CT, RR, K>(wy, a, out); }
  }
  if (g.dim > 2) {
    const RR wz = (RR)(-0.5 * g.ih2[2]);
    const int sz = g.n[0] * g.n[1];
    if (z + 1 < g.n[2]) { load_k<CT, K>(v, p + sz, a); axpy_k<CT, RR, K>(wz, a, out); }
    if (z > 0) { load_k<CT, K>(v, p - sz, a); axpy_k<CT, RR, K>(wz, a, out); }
  }
}

#define LA_K_DISPATCH(K, CALL)        \
  switch (K) {                        \
    case 1: CALL(1); break;           \
    case 2: CALL(2); break;           \
    case 3: CALL(3); break;           \
    case 4: CALL(4); break;           \
    case 5: CALL(5); break;           \
    case 6: CALL(6); break;           \
    case 7: CALL(7); break;           \
    case 8: CALL(8); break;           \
    default: break;                   \
  }

// f~[p, m] = Ub0[m] (H psi0)_p + x_p Eb0[m] psi0_p (the psi0 P_0 part moved to the right-hand side).
__global__ void k_rhs(FineOp g, const TimeMats* __restrict__ tm, const double2* __restrict__ psi0,
                      double2* __restrict__ f) {
  int np = g.n[0] * g.n[1] * g.n[2];
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  int x, y, z;
  pcoords(g, p, x, y, z);
  double2 hp[1], pv[1];
  apply_H<double2, double, 1>(g, psi0, p, x, y, z, pv, hp);
  const double xl = fine_x(g, x, y, z);
  const double2 ps = pv[0];
  const int K = tm->K;
  for (int m = 0; m < K; ++m) {
    double a = tm->Ub0[m], b = xl * tm->Eb0[m];
    f[(long long)p * K + m] = make_double2(a * hp[0].x + b * ps.x, a * hp[0].y + b * ps.y);
  }
}

void launch_rhs(const FineOp& g, const TimeMats* tm, const double2* psi0, double2* f, cudaStream_t s) {
  int np = g.n[0] * g.n[1] * g.n[2];
  k_rhs<<<(np + 255) / 256, 256, 0, s>>>(g, tm, psi0, f);
}

int norm_blocks(int np) { return (np + 255) / 256; }

// r = f~ - M~ c with (M~ c)_p = i Qb c_p - Ub (H c)_p - x_p Eb c_p; z = Wt r; partials of r^dagger Wt r.
// One thread per point, 256 threads per block, no grid stride (fixed block-to-point map so the
// norm reduction is deterministic).  f may be null (f = 0).  K is a template parameter so the
// per-point K-vectors live in registers.
template <typename CT, int K>
__global__ void __launch_bounds__(256) k_mresid(FineOp g, const TimeMats* __restrict__ tm,
                                                const CT* __restrict__ f, const CT* __restrict__ c,
                                                CT* __restrict__ rout, CT* __restrict__ zout,
                                                double* __restrict__ partials) {
  typedef typename CR<CT>::R RR;
  __shared__ RR Qb[K * K], Ub[K * K], Eb[K * K], Wt[K * K];
  __shared__ double red[256];
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    Qb[i] = (RR)tm->Qb[i]; Ub[i] = (RR)tm->Ub[i]; Eb[i] = (RR)tm->Eb[i]; Wt[i] = (RR)tm->Wt[i];
  }
  __syncthreads();
  const int np = g.n[0] * g.n[1] * g.n[2];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double nsum = 0.0;
  if (p < np) {
    int x, y, z;
    pcoords(g, p, x, y, z);
    CT r[K];
    if (f) load_k<CT, K>(f, p, r);
    else {
#pragma unroll
      for (int m = 0; m < K; ++m) r[m] = cmk<CT>(0, 0);
    }
    if (c) {   // c absent: c = 0 and r = f, with no stencil to apply
      CT cp[K], hc[K];
      apply_H<CT, RR, K>(g, c, p, x, y, z, cp, hc);
      const RR xl = (RR)fine_x(g, x, y, z);
#pragma unroll
      for (int m = 0; m < K; ++m) {
        RR qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
#pragma unroll
        for (int n = 0; n < K; ++n) {
          const RR q = Qb[m * K + n], u = Ub[m * K + n], e = Eb[m * K + n];
          qr += q * cp[n].x; qi += q * cp[n].y;
          ur += u * hc[n].x; ui += u * hc[n].y;
          er += e * cp[n].x; ei += e * cp[n].y;
        }
        // i (qr + i qi) = -qi + i qr
        r[m].x = r[m].x - (-qi - ur - xl * er);
        r[m].y = r[m].y - (qr - ui - xl * ei);
      }
    }
    CT zv[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      RR zr = 0, zi = 0;
#pragma unroll
      for (int n = 0; n < K; ++n) { zr += Wt[m * K + n] * r[n].x; zi += Wt[m * K + n] * r[n].y; }
      zv[m] = cmk<CT>(zr, zi);
      if (partials) nsum += (double)r[m].x * (double)zr + (double)r[m].y * (double)zi;
    }
    if (zout) store_k<CT, K>(zout, p, zv);
    if (rout) store_k<CT, K>(rout, p, r);
  }
  if (partials) {
    red[threadIdx.x] = nsum;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
  }
}

// ------------------------------------------------------------------ TMA-staged stencils (2D, 3D)
// complex64 V-cycle residual and normal residual on grids of dimension 2 and 3, for even K.  A CTA
// owns a kTX x kTY column tile and marches along z through a chunk of planes (chosen per launch so
// that the CTAs fill whole waves of the resident slots).  Each plane of the tile
// with a one-point halo in x and y is one TMA tensor load ({2K floats, x, y[, z]} box) into a
// ring of kNST shared-memory stages, completed on an mbarrier per stage; coordinates outside the
// grid read zeros, which is the Dirichlet wall in x, y and z.  Loads run kNST - 3 planes ahead of
// the plane being computed, issued by one thread, so the bytes in flight do not depend on the
// number of resident threads.
constexpr int kTX = 32, kTY = 8, kNST = 5;
constexpr int kPW = kTX + 2, kPH = kTY + 2, kPS = kPW * kPH;
// stage stride in float2 units: one plane box, rounded up to 128 bytes so every stage is aligned
__host__ __device__ constexpr int stage_f2(int K) { return ((kPS * K * 8 + 127) / 128) * 16; }

__device__ __forceinline__ void tma_plane(void* dst, const CUtensorMap* map, int dim, int x, int y, int z,
                                          unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  if (dim > 2)
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(0), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar)) : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(0), "r"(x), "r"(y), "r"(smem_addr(bar)) : "memory");
}

// K complex values of a staged point, two per 16-byte shared-memory load (K even).  For K = 4
// the records are 32 bytes apart, so lanes i and i + 4 of an 8-lane shared-memory wavefront would
// hit the same banks; lanes with bit 2 set read the two halves in the opposite order, which makes
// every wavefront touch each bank once (K = 6 records, 48 bytes apart, are conflict-free as is).
template <int K>
__device__ __forceinline__ void lds_k(const float2* src, float2 (&out)[K]) {
  const float4* q = reinterpret_cast<const float4*>(src);
  if constexpr (K == 4) {
    const bool sw = (threadIdx.x >> 2) & 1;
    const float4 a = q[sw ? 1 : 0], b = q[sw ? 0 : 1];
    const float4 lo = sw ? b : a, hi = sw ? a : b;
    out[0] = make_float2(lo.x, lo.y);
    out[1] = make_float2(lo.z, lo.w);
    out[2] = make_float2(hi.x, hi.y);
    out[3] = make_float2(hi.z, hi.w);
  } else {
#pragma unroll
    for (int m = 0; m < K / 2; ++m) {
      const float4 v = q[m];
      out[2 * m] = make_float2(v.x, v.y);
      out[2 * m + 1] = make_float2(v.z, v.w);
    }
  }
}

// NORMAL = false: out = Wt (f - M~ v) (f nullable).  NORMAL = true: out = M~^dagger v (+ yadd).
// Stage layout (as loaded): [y][x][K complex], point-major.
template <int K, bool NORMAL>
__global__ void __launch_bounds__(kTX * kTY, K <= 4 ? 4 : 2) k_stencil_tma(FineOp g, const __grid_constant__ CUtensorMap map,
                                                               const TimeMats* __restrict__ tm,
                                                               const float2* __restrict__ f, float2* __restrict__ out,
                                                               const float2* __restrict__ yadd, int* status, int zc) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr unsigned kPlaneBytes = kPS * K * 8;
  constexpr int kStage = stage_f2(K);
  float2* stage = reinterpret_cast<float2*>(smem);                                  // [kNST][kPS][K] (padded)
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + (size_t)kNST * kStage * 8);
  float* Qb = reinterpret_cast<float*>(bar + kNST);
  float* Ub = Qb + K * K;
  float* Eb = Ub + K * K;
  float* Wt = Eb + K * K;
  const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int nz = g.dim > 2 ? g.n[2] : 1;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  // planes j = 0 .. nplanes-1 hold z = zlo + j: z0-1 .. z1 in 3D, z = 0 alone in 2D
  const int zlo = g.dim > 2 ? z0 - 1 : 0;
  const int nplanes = g.dim > 2 ? z1 - z0 + 2 : 1;
  for (int i = tid; i < K * K; i += blockDim.x) {
    Qb[i] = (float)tm->Qb[i]; Ub[i] = (float)tm->Ub[i]; Eb[i] = (float)tm->Eb[i]; Wt[i] = (float)tm->Wt[i];
  }
  if (tid == 0) {
    for (int s = 0; s < kNST; ++s)
      mbar_init(bar + s, 1);
    mbar_init_fence();
  }
  __syncthreads();
  int issued = 0;   // planes issued so far (meaningful in thread 0)
  if (tid == 0)
    for (; issued < min(kNST, nplanes); ++issued)
      tma_plane(stage + (size_t)issued * kStage, &map, g.dim, x0 - 1, y0 - 1, zlo + issued, bar + issued, kPlaneBytes);
  const bool in = x0 + tx < g.n[0] && y0 + ty < g.n[1];
  const int x = x0 + tx, y = y0 + ty;
  const int c0 = (ty + 1) * kPW + tx + 1;
  const float wx = (float)(-0.5 * g.ih2[0]), wy = (float)(-0.5 * g.ih2[1]), wz = (float)(-0.5 * g.ih2[2]);
  const long long col = (long long)y * g.n[0] + x, plane = (long long)g.n[0] * g.n[1];
  // the point-wise inputs (f or yadd, and V0) are loaded before the plane wait, so their latency
  // overlaps it
  const float2* pin = NORMAL ? yadd : f;
  bool ok = true;
  // 3D: iteration z needs planes z-1, z, z+1 (indices jz-1, jz, jz+1 with jz = z - zlo); 2D: plane 0
  for (int z = z0; z < z1; ++z) {
    const int jz = z - zlo;
    float2 add[K];
    double v0 = 0.0;
#pragma unroll
    for (int m = 0; m < K; ++m) add[m] = make_float2(0.f, 0.f);
    if (in) {
      v0 = g.V0[(long long)z * plane + col];
      if (pin) load_k<float2, K>(pin, (long long)z * plane + col, add);
    }
    const int jfirst = g.dim > 2 ? (z == z0 ? jz - 1 : jz + 1) : 0, jlast = g.dim > 2 ? jz + 1 : 0;
    for (int j = jfirst; j <= jlast; ++j) ok = ok && mbar_wait(bar + j % kNST, (j / kNST) & 1, kMbarWaitLimit);
    if (__syncthreads_or(!ok)) {   // CTA-uniform: some thread gave up waiting
      ok = false;
      break;
    }
    if (in) {
      const float2* Pz = stage + (size_t)(jz % kNST) * kStage;
      const float2* own = Pz + (size_t)c0 * K;
      const long long p = (long long)z * plane + col;
      const float dg = (float)(g.dsum + v0);
      float2 cur[K], hv[K], a[K];
      lds_k<K>(own, cur);
#pragma unroll
      for (int m = 0; m < K; ++m) hv[m] = make_float2(dg * cur[m].x, dg * cur[m].y);
      // +x, -x, +y, -y, +z, -z, as in apply_H
      const float2* nb[6] = {own + K, own - K, own + kPW * K, own - kPW * K, nullptr, nullptr};
      const float wts[6] = {wx, wx, wy, wy, wz, wz};
      if (g.dim > 2) {
        nb[4] = stage + (size_t)((jz + 1) % kNST) * kStage + (size_t)c0 * K;
        nb[5] = stage + (size_t)((jz - 1) % kNST) * kStage + (size_t)c0 * K;
      }
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        if (t >= 4 && g.dim < 3) break;
        lds_k<K>(nb[t], a);
#pragma unroll
        for (int m = 0; m < K; ++m) { hv[m].x += wts[t] * a[m].x; hv[m].y += wts[t] * a[m].y; }
      }
      const float xl = (float)fine_x(g, x, y, z);
      float2 res[K];
#pragma unroll
      for (int m = 0; m < K; ++m) res[m] = add[m];   // f (zero when absent) or yadd
#pragma unroll
      for (int m = 0; m < K; ++m) {
        float qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
#pragma unroll
        for (int n = 0; n < K; ++n) {
          const float q = NORMAL ? Qb[n * K + m] : Qb[m * K + n], u = Ub[m * K + n], e = Eb[m * K + n];
          qr += q * cur[n].x; qi += q * cur[n].y;
          ur += u * hv[n].x; ui += u * hv[n].y;
          er += e * cur[n].x; ei += e * cur[n].y;
        }
        if (!NORMAL) {
          res[m].x = res[m].x - (-qi - ur - xl * er);   // r = f - (i Qb v - Ub H v - x Eb v)
          res[m].y = res[m].y - (qr - ui - xl * ei);
        } else {
          float2 w = make_float2(qi - ur - xl * er, -qr - ui - xl * ei);   // -i Qb^T v - Ub H v - x Eb v
          if (yadd) { w.x += res[m].x; w.y += res[m].y; }
          res[m] = w;
        }
      }
      if (!NORMAL) {
        float2 zv[K];
#pragma unroll
        for (int m = 0; m < K; ++m) {
          float zr = 0, zi = 0;
#pragma unroll
          for (int n = 0; n < K; ++n) { zr += Wt[m * K + n] * res[n].x; zi += Wt[m * K + n] * res[n].y; }
          zv[m] = make_float2(zr, zi);
        }
        store_k<float2, K>(out, p, zv);
      } else {
        store_k<float2, K>(out, p, res);
      }
    }
    // every thread is done with plane jz - 1: refill its stage with plane jz - 1 + kNST
    __syncthreads();
    const int jn = jz - 1 + kNST;
    if (g.dim > 2 && tid == 0 && jz >= 1 && jn < nplanes) {
      tma_plane(stage + (size_t)(jn % kNST) * kStage, &map, g.dim, x0 - 1, y0 - 1, zlo + jn, bar + jn % kNST,
                kPlaneBytes);
      issued = jn + 1;
    }
  }
  if (!ok) {
    // a plane did not arrive within the wait limit: flag it and give the copies in flight a last
    // bounded chance to land before the CTA exits
    if (tid == 0) {
      if (status) atomicOr(status, 4);
      for (int j = max(0, issued - kNST); j < issued; ++j) mbar_wait(bar + j % kNST, (j / kNST) & 1, kMbarWaitLimit);
    }
  }
}

// Resident CTAs of a stencil kernel on the whole GPU (SMs x CTAs per SM), queried once.
template <typename Kern>
static int stencil_slots(Kern kern, size_t smem) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTX * kTY, smem);
  return std::max(1, nsm * per_sm);
}
// Planes per CTA: among 4..16, the chunk whose CTA count fills the resident slots best (the last
// wave as full as possible), larger chunks on ties (fewer z-halo planes).
static int stencil_zchunk(int nz, int ncol, int slots) {
  if (nz <= 1) return 1;
  int best = 16;
  double best_eff = -1.0;
  for (int zc = 16; zc >= 4; --zc) {
    const long long ctas = (long long)ncol * ((nz + zc - 1) / zc);
    const long long waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots);
    if (eff > best_eff + 1e-9) { best_eff = eff; best = zc; }
  }
  return best;
}

size_t stencil_tma_smem(int K) {
  return (size_t)kNST * stage_f2(K) * 8 + kNST * sizeof(unsigned long long) + 4 * (size_t)K * K * sizeof(float);
}

// Tensor map of a complex64 point-major field for the TMA stencils: dims {2K floats, nx, ny[, nz]},
// box {2K, kTX + 2, kTY + 2[, 1]}, zero fill outside.  False when the field does not qualify (odd K,
// 1D grid) or the driver call fails; the per-point kernels are used then.
bool encode_stencil_map(const FineOp& g, int K, const float2* field, CUtensorMap* map) {
  if (g.dim < 2 || (K & 1) || !field) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint32_t rank = g.dim + 1;
  cuuint64_t dims[4] = {(cuuint64_t)(2 * K), (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
  cuuint64_t strides[3] = {(cuuint64_t)8 * K, (cuuint64_t)8 * K * g.n[0], (cuuint64_t)8 * K * g.n[0] * g.n[1]};
  cuuint32_t box[4] = {(cuuint32_t)(2 * K), (cuuint32_t)kPW, (cuuint32_t)kPH, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float2*>(field), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <bool NORMAL>
static bool launch_stencil_tma(const FineOp& g, const CUtensorMap* map, const TimeMats* tm, int K, const float2* f,
                               float2* out, const float2* yadd, int* status, cudaStream_t s) {
  if (!map || g.dim < 2 || (K & 1)) return false;
  const int nz = g.dim > 2 ? g.n[2] : 1;
  const size_t smem = stencil_tma_smem(K);
#define LA_CALL(KK)                                                                                  \
  {                                                                                                  \
    static bool attr = false;                                                                        \
    if (!attr) {                                                                                     \
      if (cudaFuncSetAttribute(k_stencil_tma<KK, NORMAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)smem) != cudaSuccess)                                            \
        return false;                                                                                \
      attr = true;                                                                                   \
    }                                                                                                \
    static int slots = 0;                                                                            \
    if (!slots) slots = stencil_slots(k_stencil_tma<KK, NORMAL>, smem);                              \
    const int ncol = ((g.n[0] + kTX - 1) / kTX) * ((g.n[1] + kTY - 1) / kTY);                       \
    const int zc = stencil_zchunk(nz, ncol, slots);                                                  \
    const dim3 grid((g.n[0] + kTX - 1) / kTX, (g.n[1] + kTY - 1) / kTY, (nz + zc - 1) / zc);         \
    k_stencil_tma<KK, NORMAL><<<grid, kTX * kTY, smem, s>>>(g, *map, tm, f, out, yadd, status, zc);  \
  }
  switch (K) {
    case 2: LA_CALL(2); break;
    case 4: LA_CALL(4); break;
    case 6: LA_CALL(6); break;
    case 8: LA_CALL(8); break;
    default: return false;
  }
#undef LA_CALL
  return true;
}

template <typename R>
void launch_mresid(const FineOp& g, const TimeMats* tm, int K, const typename C2<R>::T* f,
                   const typename C2<R>::T* c, typename C2<R>::T* r, typename C2<R>::T* z, double* partials, int nb,
                   cudaStream_t s, const CUtensorMap* cmap, int* status) {
  if constexpr (sizeof(R) == 4) {
    // the complex64 V-cycle residual (z out only) of a field with a tensor map takes the TMA kernel
    if (!r && !partials && z && launch_stencil_tma<false>(g, cmap, tm, K, f, z, nullptr, status, s)) return;
  } else {
    (void)cmap; (void)status;
  }
#define LA_CALL(KK) k_mresid<typename C2<R>::T, KK><<<nb, 256, 0, s>>>(g, tm, f, c, r, z, partials)
  LA_K_DISPATCH(K, LA_CALL)
#undef LA_CALL
}
template void launch_mresid<double>(const FineOp&, const TimeMats*, int, const double2*, const double2*, double2*,
                                    double2*, double*, int, cudaStream_t, const CUtensorMap*, int*);
template void launch_mresid<float>(const FineOp&, const TimeMats*, int, const float2*, const float2*, float2*,
                                   float2*, double*, int, cudaStream_t, const CUtensorMap*, int*);

// s = M~^dagger z: s_p = -i Qb^T z_p - Ub (H z)_p - x_p Eb z_p.
template <typename CT, int K>
__global__ void __launch_bounds__(256) k_mnormal(FineOp g, const TimeMats* __restrict__ tm,
                                                 const CT* __restrict__ zin, CT* __restrict__ out,
                                                 const CT* __restrict__ yadd) {
  typedef typename CR<CT>::R RR;
  __shared__ RR Qb[K * K], Ub[K * K], Eb[K * K];
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    Qb[i] = (RR)tm->Qb[i]; Ub[i] = (RR)tm->Ub[i]; Eb[i] = (RR)tm->Eb[i];
  }
  __syncthreads();
  const int np = g.n[0] * g.n[1] * g.n[2];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  int x, y, z;
  pcoords(g, p, x, y, z);
  CT zp[K], hz[K], v[K];
  apply_H<CT, RR, K>(g, zin, p, x, y, z, zp, hz);
  const RR xl = (RR)fine_x(g, x, y, z);
  if (yadd) load_k<CT, K>(yadd, p, v);
#pragma unroll
  for (int m = 0; m < K; ++m) {
    RR qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
#pragma unroll
    for (int n = 0; n < K; ++n) {
      const RR q = Qb[n * K + m], u = Ub[m * K + n], e = Eb[m * K + n];
      qr += q * zp[n].x; qi += q * zp[n].y;
      ur += u * hz[n].x; ui += u * hz[n].y;
      er += e * zp[n].x; ei += e * zp[n].y;
    }
    // -i (qr + i qi) = qi - i qr
    CT w = cmk<CT>(qi - ur - xl * er, -qr - ui - xl * ei);
    if (yadd) { w.x += v[m].x; w.y += v[m].y; }
    v[m] = w;
  }
  store_k<CT, K>(out, p, v);
}

template <typename R>
void launch_mnormal(const FineOp& g, const TimeMats* tm, int K, const typename C2<R>::T* z, typename C2<R>::T* out,
                    cudaStream_t s, const typename C2<R>::T* yadd, const CUtensorMap* zmap, int* status) {
  if constexpr (sizeof(R) == 4) {
    if (launch_stencil_tma<true>(g, zmap, tm, K, nullptr, out, yadd, status, s)) return;
  } else {
    (void)zmap; (void)status;
  }
  const int np = g.n[0] * g.n[1] * g.n[2];
#define LA_CALL(KK) k_mnormal<typename C2<R>::T, KK><<<(np + 255) / 256, 256, 0, s>>>(g, tm, z, out, yadd)
  LA_K_DISPATCH(K, LA_CALL)
#undef LA_CALL
}
template void launch_mnormal<double>(const FineOp&, const TimeMats*, int, const double2*, double2*, cudaStream_t,
                                     const double2*, const CUtensorMap*, int*);
template void launch_mnormal<float>(const FineOp&, const TimeMats*, int, const float2*, float2*, cudaStream_t,
                                    const float2*, const CUtensorMap*, int*);

// ------------------------------------------------------------------ Galerkin-level residual
// out_p = g_p - sum_{kk'} Theta_kk' sum_o Sigma[p][kk'][o] e_{p+o}  (coarse levels, all points)
__device__ __forceinline__ void lcoords(const LevelGeom& L, int p, int& x, int& y, int& z) {
  x = p % L.n[0];
  int r = p / L.n[0];
  y = r % L.n[1];
  z = r / L.n[1];
}

// ------------------------------------------------------------------ transfers (Sec. III)
// Cell-centred 2:1 interpolation per used axis: fine 2J <- 3/4 c_J + 1/4 c_{J-1},
// fine 2J+1 <- 3/4 c_J + 1/4 c_{J+1}; restriction is the transpose.
// Cell-centred 2:1 linear transfer weights along one axis.  Children of coarse J: fine 2J-1, 2J,
// 2J+1, 2J+2 with weights 1/4, 3/4, 3/4, 1/4 (those inside the grid).  Parents of fine a: a/2
// with 3/4 and the neighbour on a's side with 1/4 (if inside).  Unused axes map 1:1.
__device__ __forceinline__ bool child_1d(int J, int t, int nf, bool used, int& a, float& w) {
  if (!used) { a = J; w = 1.f; return t == 0; }
  a = 2 * J - 1 + t;
  w = (t == 1 || t == 2) ? 0.75f : 0.25f;
  return a >= 0 && a < nf;
}
__device__ __forceinline__ bool parent_1d(int a, int t, int nc, bool used, int& J, float& w) {
  if (!used) { J = a; w = 1.f; return t == 0; }
  const int j0 = a >> 1;
  if (t == 0) { J = j0; w = 0.75f; return true; }
  J = (a & 1) ? j0 + 1 : j0 - 1;
  w = 0.25f;
  return J >= 0 && J < nc;
}

template <typename CT, int K>
__global__ void k_restrict(LevelGeom F, LevelGeom C, const CT* __restrict__ sf, CT* __restrict__ gc) {
  typedef typename CR<CT>::R RR;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= C.np) return;
  int jx, jy, jz;
  lcoords(C, J, jx, jy, jz);
  CT acc[K], a[K];
#pragma unroll
  for (int m = 0; m < K; ++m) acc[m] = cmk<CT>(0, 0);
  for (int tz = 0; tz < 4; ++tz) {
    int az; float wz;
    if (!child_1d(jz, tz, F.n[2], F.dim > 2, az, wz)) continue;
    for (int ty = 0; ty < 4; ++ty) {
      int ay; float wy;
      if (!child_1d(jy, ty, F.n[1], F.dim > 1, ay, wy)) continue;
#pragma unroll
      for (int tx = 0; tx < 4; ++tx) {
        int ax; float wx;
        if (!child_1d(jx, tx, F.n[0], F.dim > 0, ax, wx)) continue;
        const RR w = (RR)(wx * wy * wz);
        load_k<CT, K>(sf, (long long)(az * F.n[1] + ay) * F.n[0] + ax, a);
        axpy_k<CT, RR, K>(w, a, acc);
      }
    }
  }
  store_k<CT, K>(gc, J, acc);
}

// Restriction I^T on 2D and 3D levels, one CTA per tile of kRx x kRy x kRz coarse points: the fine points the
// tile's children cover (2 kR + 2 per used axis, zero outside the grid) are loaded into shared memory with
// consecutive threads on consecutive complex entries, then each (coarse point, time function) sums its
// 4 x 4 (x 4) children there, in the same order and with the same weights as k_restrict.
constexpr int kRx = 8, kRy = 4, kRz = 2;
template <typename CT, int K>
__global__ void __launch_bounds__(256) k_restrict_tile(LevelGeom F, LevelGeom C, const CT* __restrict__ sf,
                                                       CT* __restrict__ gc) {
  typedef typename CR<CT>::R RR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* box = reinterpret_cast<CT*>(smem_raw);
  const bool uy = F.dim > 1, uz = F.dim > 2;
  const int tx = kRx, ty = uy ? kRy : 1, tz = uz ? kRz : 1;
  const int jx0 = blockIdx.x * tx, jy0 = blockIdx.y * ty, jz0 = blockIdx.z * tz;
  const int bx = 2 * tx + 2, by = uy ? 2 * ty + 2 : 1, bz = uz ? 2 * tz + 2 : 1;
  const int ox = 2 * jx0 - 1, oy = uy ? 2 * jy0 - 1 : 0, oz = uz ? 2 * jz0 - 1 : 0;
  const int nbox = bx * by * bz * K;
  for (int t = threadIdx.x; t < nbox; t += blockDim.x) {
    const int m = t % K, pnt = t / K;
    const int lx = pnt % bx, rest = pnt / bx, ly = rest % by, lz = rest / by;
    const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
    CT v = cmk<CT>(0, 0);
    if (gx >= 0 && gy >= 0 && gz >= 0 && gx < F.n[0] && gy < F.n[1] && gz < F.n[2])
      v = sf[((long long)(gz * F.n[1] + gy) * F.n[0] + gx) * K + m];
    box[t] = v;
  }
  __syncthreads();
  const int nitems = tx * ty * tz * K;
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    const int m = t % K, c = t / K;
    const int cx = c % tx, rest = c / tx, cy = rest % ty, cz = rest / ty;
    const int jx = jx0 + cx, jy = jy0 + cy, jz = jz0 + cz;
    if (jx >= C.n[0] || jy >= C.n[1] || jz >= C.n[2]) continue;
    CT acc = cmk<CT>(0, 0);
    for (int qz = 0; qz < 4; ++qz) {
      int az; float wz;
      if (!child_1d(jz, qz, F.n[2], uz, az, wz)) continue;
      for (int qy = 0; qy < 4; ++qy) {
        int ay; float wy;
        if (!child_1d(jy, qy, F.n[1], uy, ay, wy)) continue;
#pragma unroll
        for (int qx = 0; qx < 4; ++qx) {
          int ax; float wx;
          if (!child_1d(jx, qx, F.n[0], true, ax, wx)) continue;
          const RR w = (RR)(wx * wy * wz);
          const CT a = box[(((az - oz) * by + (ay - oy)) * bx + (ax - ox)) * K + m];
          acc.x += w * a.x;
          acc.y += w * a.y;
        }
      }
    }
    gc[((long long)(jz * C.n[1] + jy) * C.n[0] + jx) * K + m] = acc;
  }
}

template <typename CT, int K>
__global__ void k_prolong_add(LevelGeom F, LevelGeom C, const CT* __restrict__ ec, CT* __restrict__ ef) {
  typedef typename CR<CT>::R RR;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= F.np) return;
  int x, y, z;
  lcoords(F, p, x, y, z);
  CT acc[K], a[K];
  load_k<CT, K>(ef, p, acc);
  for (int tz = 0; tz < 2; ++tz) {
    int Jz; float wz;
    if (!parent_1d(z, tz, C.n[2], F.dim > 2, Jz, wz)) continue;
    for (int ty = 0; ty < 2; ++ty) {
      int Jy; float wy;
      if (!parent_1d(y, ty, C.n[1], F.dim > 1, Jy, wy)) continue;
#pragma unroll
      for (int tx = 0; tx < 2; ++tx) {
        int Jx; float wx;
        if (!parent_1d(x, tx, C.n[0], F.dim > 0, Jx, wx)) continue;
        const RR w = (RR)(wx * wy * wz);
        load_k<CT, K>(ec, (long long)(Jz * C.n[1] + Jy) * C.n[0] + Jx, a);
        axpy_k<CT, RR, K>(w, a, acc);
      }
    }
  }
  store_k<CT, K>(ef, p, acc);
}

template <typename R>
void launch_restrict(const LevelGeom& F, const LevelGeom& C, int K, const typename C2<R>::T* sf,
                     typename C2<R>::T* gc, cudaStream_t s) {
  typedef typename C2<R>::T CT;
  if (F.dim >= 2) {
    const int ty = kRy, tz = F.dim > 2 ? kRz : 1;
    const dim3 grid((C.n[0] + kRx - 1) / kRx, (C.n[1] + ty - 1) / ty, (C.n[2] + tz - 1) / tz);
    const size_t smem = sizeof(CT) * (size_t)(2 * kRx + 2) * (2 * ty + 2) * (F.dim > 2 ? 2 * tz + 2 : 1) * K;
#define LA_CALL(KK)                                                                                        \
  do {                                                                                                     \
    static bool attr = false;                                                                              \
    if (!attr) {                                                                                           \
      cudaFuncSetAttribute(k_restrict_tile<CT, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); \
      attr = true;                                                                                         \
    }                                                                                                      \
    k_restrict_tile<CT, KK><<<grid, 256, smem, s>>>(F, C, sf, gc);                                         \
  } while (0)
    switch (K) {
      case 1: LA_CALL(1); break;
      case 2: LA_CALL(2); break;
      case 3: LA_CALL(3); break;
      case 4: LA_CALL(4); break;
      case 5: LA_CALL(5); break;
      case 6: LA_CALL(6); break;
      case 7: LA_CALL(7); break;
      default: LA_CALL(8); break;
    }
#undef LA_CALL
    return;
  }
#define LA_CALL(KK) k_restrict<typename C2<R>::T, KK><<<(C.np + 127) / 128, 128, 0, s>>>(F, C, sf, gc)
  LA_K_DISPATCH(K, LA_CALL)
#undef LA_CALL
}
template <typename R>
void launch_prolong_add(const LevelGeom& F, const LevelGeom& C, int K, const typename C2<R>::T* ec,
                        typename C2<R>::T* ef, cudaStream_t s) {
#define LA_CALL(KK) k_prolong_add<typename C2<R>::T, KK><<<(F.np + 127) / 128, 128, 0, s>>>(F, C, ec, ef)
  LA_K_DISPATCH(K, LA_CALL)
#undef LA_CALL
}
template void launch_restrict<double>(const LevelGeom&, const LevelGeom&, int, const double2*, double2*, cudaStream_t);
template void launch_restrict<float>(const LevelGeom&, const LevelGeom&, int, const float2*, float2*, cudaStream_t);
template void launch_prolong_add<double>(const LevelGeom&, const LevelGeom&, int, const double2*, double2*,
                                         cudaStream_t);
template void launch_prolong_add<float>(const LevelGeom&, const LevelGeom&, int, const float2*, float2*, cudaStream_t);

// ------------------------------------------------------------------ norm, advance, conversions
// Deterministic final sum of the per-block partials (fixed order), times the weight scale.
__global__ void k_norm_final(const double* __restrict__ partials, int n, double scale, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}
void launch_norm_final(const double* partials, int n, double scale, double* out, cudaStream_t s) {
  k_norm_final<<<1, 256, 0, s>>>(partials, n, scale, out);
}

// ---------------------------------------------------------------- device-side relaxation loop
// Trial or zero start of a step's relaxation, decided on the device: the extrapolated trial is kept when
// its action is below N(0), else c = 0 and r = f (the residual of c = 0).
__global__ void k_seed_select(long long n, const double* __restrict__ Nslot, int tried, LoopState* st,
                              double2* __restrict__ c, double2* __restrict__ r, const double2* __restrict__ f) {
  const double Nt = Nslot[0], N0 = Nslot[1];
  const bool keep = tried && Nt < N0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->N0 = N0;
    st->N = keep ? Nt : N0;
    st->cyc = 0;
  }
  if (keep || !tried) return;   // without a trial c is already 0 and r = f
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    c[i] = make_double2(0.0, 0.0);
    r[i] = f[i];
  }
}
void launch_seed_select(long long n, const double* Nslot, int tried, LoopState* st, double2* c, double2* r,
                        const double2* f, cudaStream_t s) {
  const long long nb = std::min<long long>((n + 255) / 256, 4096);
  k_seed_select<<<(int)nb, 256, 0, s>>>(n, Nslot, tried, st, c, r, f);
}

// The loop's condition (one thread): after a cycle, take its action and count it; continue while the
// action is finite, fewer than max_cycles have run and (with a tolerance) N > tol N(0).
__global__ void k_loop_cond(LoopState* st, const double* __restrict__ Nnew, double tol, int max_cycles, int check,
                            int first, cudaGraphConditionalHandle h) {
  if (!first) {
    st->N = Nnew[0];
    st->cyc += 1;
  }
  const double N = st->N;
  const bool go = isfinite(N) && st->cyc < max_cycles && !(check && N <= tol * st->N0);
  cudaGraphSetConditional(h, go ? 1u : 0u);
}
void launch_loop_cond(LoopState* st, const double* Nnew, double tol, int max_cycles, int check, int first,
                      cudaGraphConditionalHandle h, cudaStream_t s) {
  k_loop_cond<<<1, 1, 0, s>>>(st, Nnew, tol, max_cycles, check, first, h);
}

__global__ void k_loop_record(const LoopState* st, LoopRecord* rec) {
  rec->N0 = st->N0;
  rec->N = st->N;
  rec->cycles = st->cyc;
  rec->pad = 0;
}
void launch_loop_record(const LoopState* st, LoopRecord* rec, cudaStream_t s) { k_loop_record<<<1, 1, 0, s>>>(st, rec); }

// psi(t0+dt)_p = psi0_p + sum_n b_n(+1) c_pn
__global__ void k_advance(int np, const TimeMats* __restrict__ tm, const double2* __restrict__ c,
                          double2* __restrict__ psi) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int K = tm->K;
  double2 v = psi[p];
  for (int n = 0; n < K; ++n) {
    double w = tm->endv[n];
    double2 a = c[(long long)p * K + n];
    v.x += w * a.x;
    v.y += w * a.y;
  }
  psi[p] = v;
}
void launch_advance(int np, const TimeMats* tm, const double2* c, double2* psi, cudaStream_t s) {
  k_advance<<<(np + 255) / 256, 256, 0, s>>>(np, tm, c, psi);
}

__global__ void k_axpy_c64_to_c128(long long n, const float2* __restrict__ x, double2* __restrict__ y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 v = y[i];
  float2 a = x[i];
  v.x += (double)a.x;
  v.y += (double)a.y;
  y[i] = v;
}
__global__ void k_c128_to_c64(long long n, const double2* __restrict__ x, float2* __restrict__ y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 a = x[i];
  y[i] = make_float2((float)a.x, (float)a.y);
}
void launch_axpy_c64_to_c128(long long n, const float2* x, double2* y, cudaStream_t s) {
  k_axpy_c64_to_c128<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y);
}
__global__ void k_scale_c128(long long n, double a, const double2* __restrict__ x, double2* __restrict__ y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 v = x[i];
  y[i] = make_double2(a * v.x, a * v.y);
}
void launch_scale_c128(long long n, double a, const double2* x, double2* y, cudaStream_t s) {
  k_scale_c128<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x, y);
}
// Trial coefficients c = a0 h0 + a1 h1 + a2 h2 (h1, h2 nullable), the extrapolation of the last
// converged coefficient vectors h0 (newest), h1, h2 of a propagation.
__global__ void k_trial(long long n, double a0, double a1, double a2, const double2* __restrict__ h0,
                        const double2* __restrict__ h1, const double2* __restrict__ h2, double2* __restrict__ c) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = h0[i];
    double re = a0 * v.x, im = a0 * v.y;
    if (h1) { const double2 u = h1[i]; re = fma(a1, u.x, re); im = fma(a1, u.y, im); }
    if (h2) { const double2 u = h2[i]; re = fma(a2, u.x, re); im = fma(a2, u.y, im); }
    c[i] = make_double2(re, im);
  }
}
void launch_trial(long long n, const double* a, const double2* h0, const double2* h1, const double2* h2, double2* c,
                  cudaStream_t s) {
  const long long nb = std::min<long long>((n + 255) / 256, 152LL * 8);
  k_trial<<<(unsigned)nb, 256, 0, s>>>(n, a[0], a[1], a[2], h0, h1, h2, c);
}
void launch_c128_to_c64(long long n, const double2* x, float2* y, cudaStream_t s) {
  k_c128_to_c64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y);
}
// y = (float) x, element by element (grid-stride)
__global__ void k_f64_to_f32(long long n, const double* __restrict__ x, float* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
void launch_f64_to_f32(long long n, const double* x, float* y, cudaStream_t s) {
  const long long nb = std::min<long long>((n + 255) / 256, 152LL * 8);
  k_f64_to_f32<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, s>>>(n, x, y);
}


// ------------------------------------------------------------------ bounded-wait self-test
// One CTA waits on an mbarrier that nothing completes, with the poll loop the staged kernels use,
// and on giving up sets flag 4 of the status word as they do.
__global__ void k_wait_selftest(unsigned polls, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, 4);
}

}  // namespace la

extern "C" la_status la_wait_selftest(int polls, int* status_out, void* cuda_stream) {
  if (polls < 1 || !status_out) return LA_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return LA_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    la::k_wait_selftest<<<1, 32, 0, s>>>((unsigned)polls, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(status_out, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  return e == cudaSuccess ? LA_OK : LA_ECUDA;
}
