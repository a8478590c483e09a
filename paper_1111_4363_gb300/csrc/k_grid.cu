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

// (H v)_p for a K-vector field v (point-major), Dirichlet zero outside the grid.
template <typename CT, typename RR>
__device__ __forceinline__ void apply_H(const FineOp& g, const CT* v, int K, int x, int y, int z, CT* out) {
  const int p = (z * g.n[1] + y) * g.n[0] + x;
  const RR dg = (RR)(g.dsum + g.V0[p]);
  for (int m = 0; m < K; ++m) {
    CT a = v[(long long)p * K + m];
    out[m] = cmk<CT>(dg * a.x, dg * a.y);
  }
  const int nb[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  for (int t = 0; t < 2 * g.dim; ++t) {
    int qx = x + nb[t][0], qy = y + nb[t][1], qz = z + nb[t][2];
    if (qx < 0 || qy < 0 || qz < 0 || qx >= g.n[0] || qy >= g.n[1] || qz >= g.n[2]) continue;
    const RR w = (RR)(-0.5 * g.ih2[t >> 1]);
    const long long q = (long long)((qz * g.n[1] + qy) * g.n[0] + qx) * K;
    for (int m = 0; m < K; ++m) {
      CT a = v[q + m];
      out[m].x += w * a.x;
      out[m].y += w * a.y;
    }
  }
}

// f~[p, m] = Ub0[m] (H psi0)_p + x_p Eb0[m] psi0_p (the psi0 P_0 part moved to the right-hand side).
__global__ void k_rhs(FineOp g, const TimeMats* __restrict__ tm, const double2* __restrict__ psi0,
                      double2* __restrict__ f) {
  int np = g.n[0] * g.n[1] * g.n[2];
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  int x, y, z;
  pcoords(g, p, x, y, z);
  double2 hp[1];
  apply_H<double2, double>(g, psi0, 1, x, y, z, hp);
  const double xl = fine_x(g, x, y, z);
  const double2 ps = psi0[p];
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
// norm reduction is deterministic).  f may be null (f = 0).
template <typename CT>
__global__ void __launch_bounds__(256) k_mresid(FineOp g, const TimeMats* __restrict__ tm,
                                                const CT* __restrict__ f, const CT* __restrict__ c,
                                                CT* __restrict__ rout, CT* __restrict__ zout,
                                                double* __restrict__ partials) {
  typedef typename CR<CT>::R RR;
  __shared__ RR Qb[LA_KMAX * LA_KMAX], Ub[LA_KMAX * LA_KMAX], Eb[LA_KMAX * LA_KMAX], Wt[LA_KMAX * LA_KMAX];
  __shared__ double red[256];
  const int K = tm->K;
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
    CT cp[LA_KMAX], hc[LA_KMAX], r[LA_KMAX];
    for (int m = 0; m < K; ++m) cp[m] = c[(long long)p * K + m];
    apply_H<CT, RR>(g, c, K, x, y, z, hc);
    const RR xl = (RR)fine_x(g, x, y, z);
    for (int m = 0; m < K; ++m) {
      RR qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
      for (int n = 0; n < K; ++n) {
        RR q = Qb[m * K + n], u = Ub[m * K + n], e = Eb[m * K + n];
        qr += q * cp[n].x; qi += q * cp[n].y;
        ur += u * hc[n].x; ui += u * hc[n].y;
        er += e * cp[n].x; ei += e * cp[n].y;
      }
      // i (qr + i qi) = -qi + i qr
      CT fv = f ? f[(long long)p * K + m] : cmk<CT>(0, 0);
      r[m].x = fv.x - (-qi - ur - xl * er);
      r[m].y = fv.y - (qr - ui - xl * ei);
    }
    for (int m = 0; m < K; ++m) {
      RR zr = 0, zi = 0;
      for (int n = 0; n < K; ++n) { zr += Wt[m * K + n] * r[n].x; zi += Wt[m * K + n] * r[n].y; }
      nsum += (double)r[m].x * (double)zr + (double)r[m].y * (double)zi;
      if (zout) zout[(long long)p * K + m] = cmk<CT>(zr, zi);
      if (rout) rout[(long long)p * K + m] = r[m];
    }
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
void launch_mresid(const FineOp& g, const TimeMats* tm, const typename C2<R>::T* f, const typename C2<R>::T* c,
                   typename C2<R>::T* r, typename C2<R>::T* z, double* partials, int nb, cudaStream_t s) {
  k_mresid<typename C2<R>::T><<<nb, 256, 0, s>>>(g, tm, f, c, r, z, partials);
}
template void launch_mresid<double>(const FineOp&, const TimeMats*, const double2*, const double2*, double2*,
                                    double2*, double*, int, cudaStream_t);
template void launch_mresid<float>(const FineOp&, const TimeMats*, const float2*, const float2*, float2*, float2*,
                                   double*, int, cudaStream_t);

// s = M~^dagger z: s_p = -i Qb^T z_p - Ub (H z)_p - x_p Eb z_p.
template <typename CT>
__global__ void __launch_bounds__(256) k_mnormal(FineOp g, const TimeMats* __restrict__ tm,
                                                 const CT* __restrict__ zin, CT* __restrict__ out,
                                                 const CT* __restrict__ yadd) {
  typedef typename CR<CT>::R RR;
  __shared__ RR Qb[LA_KMAX * LA_KMAX], Ub[LA_KMAX * LA_KMAX], Eb[LA_KMAX * LA_KMAX];
  const int K = tm->K;
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    Qb[i] = (RR)tm->Qb[i]; Ub[i] = (RR)tm->Ub[i]; Eb[i] = (RR)tm->Eb[i];
  }
  __syncthreads();
  const int np = g.n[0] * g.n[1] * g.n[2];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  int x, y, z;
  pcoords(g, p, x, y, z);
  CT zp[LA_KMAX], hz[LA_KMAX];
  for (int m = 0; m < K; ++m) zp[m] = zin[(long long)p * K + m];
  apply_H<CT, RR>(g, zin, K, x, y, z, hz);
  const RR xl = (RR)fine_x(g, x, y, z);
  for (int m = 0; m < K; ++m) {
    RR qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
    for (int n = 0; n < K; ++n) {
      RR q = Qb[n * K + m], u = Ub[m * K + n], e = Eb[m * K + n];
      qr += q * zp[n].x; qi += q * zp[n].y;
      ur += u * hz[n].x; ui += u * hz[n].y;
      er += e * zp[n].x; ei += e * zp[n].y;
    }
    // -i (qr + i qi) = qi - i qr
    CT v = cmk<CT>(qi - ur - xl * er, -qr - ui - xl * ei);
    if (yadd) {
      const CT ya = yadd[(long long)p * K + m];
      v.x += ya.x;
      v.y += ya.y;
    }
    out[(long long)p * K + m] = v;
  }
}

template <typename R>
void launch_mnormal(const FineOp& g, const TimeMats* tm, const typename C2<R>::T* z, typename C2<R>::T* out,
                    cudaStream_t s, const typename C2<R>::T* yadd) {
  int np = g.n[0] * g.n[1] * g.n[2];
  k_mnormal<typename C2<R>::T><<<(np + 255) / 256, 256, 0, s>>>(g, tm, z, out, yadd);
}
template void launch_mnormal<double>(const FineOp&, const TimeMats*, const double2*, double2*, cudaStream_t,
                                     const double2*);
template void launch_mnormal<float>(const FineOp&, const TimeMats*, const float2*, float2*, cudaStream_t,
                                    const float2*);

// ------------------------------------------------------------------ Galerkin-level residual
// out_p = g_p - sum_{kk'} Theta_kk' sum_o Sigma[p][kk'][o] e_{p+o}  (coarse levels, all points)
__device__ __forceinline__ void lcoords(const LevelGeom& L, int p, int& x, int& y, int& z) {
  x = p % L.n[0];
  int r = p / L.n[0];
  y = r % L.n[1];
  z = r / L.n[1];
}

template <typename CT>
__global__ void __launch_bounds__(128) k_gresid(LevelGeom L, const TimeMats* __restrict__ tm,
                                                const double* __restrict__ sigma, const CT* __restrict__ gvec,
                                                const CT* __restrict__ e, CT* __restrict__ out) {
  typedef typename CR<CT>::R RR;
  __shared__ RR P[LA_NPAIR][LA_KMAX * LA_KMAX];
  const int K = tm->K;
  for (int i = threadIdx.x; i < LA_NPAIR * K * K; i += blockDim.x) P[i / (K * K)][i % (K * K)] = (RR)tm->P[i / (K * K)][i % (K * K)];
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.np) return;
  int x, y, z;
  lcoords(L, p, x, y, z);
  const int nbox = box5_count(L.dim);
  const int rz = L.dim > 2 ? 2 : 0, ry = L.dim > 1 ? 2 : 0;
  CT acc[LA_KMAX];
  for (int m = 0; m < K; ++m) acc[m] = cmk<CT>(0, 0);
  for (int kk = 0; kk < LA_NPAIR; ++kk) {
    CT u[LA_KMAX];
    for (int m = 0; m < K; ++m) u[m] = cmk<CT>(0, 0);
    for (int oz = -rz; oz <= rz; ++oz)
      for (int oy = -ry; oy <= ry; ++oy)
        for (int ox = -2; ox <= 2; ++ox) {
          int qx = x + ox, qy = y + oy, qz = z + oz;
          if (qx < 0 || qy < 0 || qz < 0 || qx >= L.n[0] || qy >= L.n[1] || qz >= L.n[2]) continue;
          RR s = (RR)sigma[sigma_offset(p, kk, box5_index(L.dim, ox, oy, oz), nbox)];
          if (s == (RR)0) continue;
          const CT* eq = e + (long long)((qz * L.n[1] + qy) * L.n[0] + qx) * K;
          for (int m = 0; m < K; ++m) { u[m].x += s * eq[m].x; u[m].y += s * eq[m].y; }
        }
    const int ph = theta_phase(kk);
    for (int m = 0; m < K; ++m) {
      RR vr = 0, vi = 0;
      for (int n = 0; n < K; ++n) { RR pv = P[kk][m * K + n]; vr += pv * u[n].x; vi += pv * u[n].y; }
      if (ph == 0) { acc[m].x += vr; acc[m].y += vi; }
      else if (ph == 1) { acc[m].x -= vi; acc[m].y += vr; }   // i (vr + i vi)
      else { acc[m].x += vi; acc[m].y -= vr; }                // -i (vr + i vi)
    }
  }
  for (int m = 0; m < K; ++m) {
    CT gv = gvec[(long long)p * K + m];
    out[(long long)p * K + m] = cmk<CT>(gv.x - acc[m].x, gv.y - acc[m].y);
  }
}

template <typename R>
void launch_gresid(const LevelGeom& L, const TimeMats* tm, const double* sigma, const typename C2<R>::T* gvec,
                   const typename C2<R>::T* e, typename C2<R>::T* out, cudaStream_t s) {
  k_gresid<typename C2<R>::T><<<(L.np + 127) / 128, 128, 0, s>>>(L, tm, sigma, gvec, e, out);
}
template void launch_gresid<double>(const LevelGeom&, const TimeMats*, const double*, const double2*, const double2*,
                                    double2*, cudaStream_t);
template void launch_gresid<float>(const LevelGeom&, const TimeMats*, const double*, const float2*, const float2*,
                                   float2*, cudaStream_t);

// ------------------------------------------------------------------ transfers (Sec. III)
// Cell-centred 2:1 interpolation per used axis: fine 2J <- 3/4 c_J + 1/4 c_{J-1},
// fine 2J+1 <- 3/4 c_J + 1/4 c_{J+1}; restriction is the transpose.
__device__ __forceinline__ int parents_1d(int a, int nc, bool used, int J[2], float w[2]) {
  if (!used) { J[0] = a; w[0] = 1.f; return 1; }
  int j0 = a >> 1;
  int j1 = (a & 1) ? j0 + 1 : j0 - 1;
  J[0] = j0; w[0] = 0.75f;
  if (j1 >= 0 && j1 < nc) { J[1] = j1; w[1] = 0.25f; return 2; }
  return 1;
}
__device__ __forceinline__ int children_1d(int J, int nf, bool used, int a[4], float w[4]) {
  if (!used) { a[0] = J; w[0] = 1.f; return 1; }
  int cnt = 0;
  const int cand[4] = {2 * J - 1, 2 * J, 2 * J + 1, 2 * J + 2};
  const float wc[4] = {0.25f, 0.75f, 0.75f, 0.25f};
  for (int t = 0; t < 4; ++t)
    if (cand[t] >= 0 && cand[t] < nf) { a[cnt] = cand[t]; w[cnt] = wc[t]; ++cnt; }
  return cnt;
}

template <typename CT>
__global__ void k_restrict(LevelGeom F, LevelGeom C, int K, const CT* __restrict__ sf, CT* __restrict__ gc) {
  typedef typename CR<CT>::R RR;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= C.np) return;
  int jx, jy, jz;
  lcoords(C, J, jx, jy, jz);
  int ax[4], ay[4], az[4];
  float wx[4], wy[4], wz[4];
  int nx = children_1d(jx, F.n[0], F.dim > 0, ax, wx);
  int ny = children_1d(jy, F.n[1], F.dim > 1, ay, wy);
  int nz = children_1d(jz, F.n[2], F.dim > 2, az, wz);
  CT acc[LA_KMAX];
  for (int m = 0; m < K; ++m) acc[m] = cmk<CT>(0, 0);
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        RR w = (RR)(wx[ix] * wy[iy] * wz[iz]);
        const CT* s = sf + (long long)((az[iz] * F.n[1] + ay[iy]) * F.n[0] + ax[ix]) * K;
        for (int m = 0; m < K; ++m) { acc[m].x += w * s[m].x; acc[m].y += w * s[m].y; }
      }
  for (int m = 0; m < K; ++m) gc[(long long)J * K + m] = acc[m];
}

template <typename CT>
__global__ void k_prolong_add(LevelGeom F, LevelGeom C, int K, const CT* __restrict__ ec, CT* __restrict__ ef) {
  typedef typename CR<CT>::R RR;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= F.np) return;
  int x, y, z;
  lcoords(F, a, x, y, z);
  int Jx[2], Jy[2], Jz[2];
  float wx[2], wy[2], wz[2];
  int nx = parents_1d(x, C.n[0], F.dim > 0, Jx, wx);
  int ny = parents_1d(y, C.n[1], F.dim > 1, Jy, wy);
  int nz = parents_1d(z, C.n[2], F.dim > 2, Jz, wz);
  CT acc[LA_KMAX];
  for (int m = 0; m < K; ++m) acc[m] = ef[(long long)a * K + m];
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        RR w = (RR)(wx[ix] * wy[iy] * wz[iz]);
        const CT* s = ec + (long long)((Jz[iz] * C.n[1] + Jy[iy]) * C.n[0] + Jx[ix]) * K;
        for (int m = 0; m < K; ++m) { acc[m].x += w * s[m].x; acc[m].y += w * s[m].y; }
      }
  for (int m = 0; m < K; ++m) ef[(long long)a * K + m] = acc[m];
}

template <typename R>
void launch_restrict(const LevelGeom& F, const LevelGeom& C, int K, const typename C2<R>::T* sf,
                     typename C2<R>::T* gc, cudaStream_t s) {
  k_restrict<typename C2<R>::T><<<(C.np + 127) / 128, 128, 0, s>>>(F, C, K, sf, gc);
}
template <typename R>
void launch_prolong_add(const LevelGeom& F, const LevelGeom& C, int K, const typename C2<R>::T* ec,
                        typename C2<R>::T* ef, cudaStream_t s) {
  k_prolong_add<typename C2<R>::T><<<(F.np + 127) / 128, 128, 0, s>>>(F, C, K, ec, ef);
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
