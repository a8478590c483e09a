// Grid-wide kernels: per-step time matrices, right-hand side, action residual and residual
// norm, normal residual, Galerkin-level residual, intergrid transfers, step advance.
#include <algorithm>

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
    CT cp[K], hc[K], r[K];
    apply_H<CT, RR, K>(g, c, p, x, y, z, cp, hc);
    const RR xl = (RR)fine_x(g, x, y, z);
    if (f) load_k<CT, K>(f, p, r);
    else {
#pragma unroll
      for (int m = 0; m < K; ++m) r[m] = cmk<CT>(0, 0);
    }
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

template <typename R>
void launch_mresid(const FineOp& g, const TimeMats* tm, int K, const typename C2<R>::T* f,
                   const typename C2<R>::T* c, typename C2<R>::T* r, typename C2<R>::T* z, double* partials, int nb,
                   cudaStream_t s) {
#define LA_CALL(KK) k_mresid<typename C2<R>::T, KK><<<nb, 256, 0, s>>>(g, tm, f, c, r, z, partials)
  LA_K_DISPATCH(K, LA_CALL)
#undef LA_CALL
}
template void launch_mresid<double>(const FineOp&, const TimeMats*, int, const double2*, const double2*, double2*,
                                    double2*, double*, int, cudaStream_t);
template void launch_mresid<float>(const FineOp&, const TimeMats*, int, const float2*, const float2*, float2*,
                                   float2*, double*, int, cudaStream_t);

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
                    cudaStream_t s, const typename C2<R>::T* yadd) {
  const int np = g.n[0] * g.n[1] * g.n[2];
#define LA_CALL(KK) k_mnormal<typename C2<R>::T, KK><<<(np + 255) / 256, 256, 0, s>>>(g, tm, z, out, yadd)
  LA_K_DISPATCH(K, LA_CALL)
#undef LA_CALL
}
template void launch_mnormal<double>(const FineOp&, const TimeMats*, int, const double2*, double2*, cudaStream_t,
                                     const double2*);
template void launch_mnormal<float>(const FineOp&, const TimeMats*, int, const float2*, float2*, cudaStream_t,
                                    const float2*);

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

}  // namespace la
