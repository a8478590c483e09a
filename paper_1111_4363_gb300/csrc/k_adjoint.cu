// Kernels of the discrete adjoint (la_backward).
//
// Per step k, with lambda = dJ/dpsi_{k+1}^*:
//   y~ = B^T lambda / h^d                      (B^T lambda)_{p,m} = b_m(+1) lambda_p
//   G~ z = y~ by the same relaxation as the forward step (G~ = M~^dagger Wt M~), so that
//   mu = (I (x) Wt) M~ z = M^{-dagger} B^T lambda (the adjoint solve on the forward factors)
//   dJ/da_j += 2 h^d Re sum_p x_p sum_m conj(mu_pm) (Eb0^(j)_m psi_p + sum_n Eb^(j)_mn c_pn)
//   lambda  += h^d ( H (Ub0 . mu) + x Eb0 . mu )                    (F_k^T mu)
// The kernels below receive zneg = Wt (0 - M~ z) = -mu from the residual kernel.
#include "la_internal.cuh"

namespace la {

__global__ void k_bt_lambda(int np, const TimeMats* __restrict__ tm, double inv_hd, const double2* __restrict__ lam,
                            double2* __restrict__ y) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int K = tm->K;
  const double2 l = lam[p];
  for (int m = 0; m < K; ++m) {
    const double w = tm->endv[m] * inv_hd;
    y[(long long)p * K + m] = make_double2(w * l.x, w * l.y);
  }
}
void launch_bt_lambda(int np, const TimeMats* tm, double inv_hd, const double2* lam, double2* y, cudaStream_t s) {
  k_bt_lambda<<<(np + 255) / 256, 256, 0, s>>>(np, tm, inv_hd, lam, y);
}

// Euclidean norm^2 partials of a complex vector (fixed block-to-element map, deterministic).
__global__ void k_norm2_partials(long long n, const double2* __restrict__ v, double* __restrict__ partials) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const double2 a = v[i];
    s += a.x * a.x + a.y * a.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}
void launch_norm2_partials(long long n, const double2* v, double* partials, int nblocks, cudaStream_t s) {
  k_norm2_partials<<<nblocks, 256, 0, s>>>(n, v, partials);
}

// Z[m][n'] partial sums over 256-point blocks: sum_p x_p conj(mu_pm) w_{p,n'}, w_0 = psi_p,
// w_n = c_pn; mu = -zneg.  grid = (point blocks, K*(K+1) pairs).
__global__ void k_grad_partials(FineOp g, int K, const double2* __restrict__ zneg, const double2* __restrict__ psi,
                                const double2* __restrict__ c, double2* __restrict__ partials) {
  __shared__ double rr[256], ri[256];
  const int np = g.n[0] * g.n[1] * g.n[2];
  const int pair = blockIdx.y, m = pair / (K + 1), nn = pair % (K + 1);
  const int p = blockIdx.x * 256 + threadIdx.x;
  double sr = 0.0, si = 0.0;
  if (p < np) {
    const int x = p % g.n[0], y = (p / g.n[0]) % g.n[1], z = p / (g.n[0] * g.n[1]);
    const double xl = fine_x(g, x, y, z);
    const double2 mu = zneg[(long long)p * K + m];            // = -mu
    const double2 w = nn == 0 ? psi[p] : c[(long long)p * K + (nn - 1)];
    // conj(mu) w with mu = -zneg:  -(zneg.x - i zneg.y)(w.x + i w.y)
    sr = -xl * (mu.x * w.x + mu.y * w.y);
    si = -xl * (mu.x * w.y - mu.y * w.x);
  }
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) { rr[threadIdx.x] += rr[threadIdx.x + k]; ri[threadIdx.x] += ri[threadIdx.x + k]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(long long)pair * gridDim.x + blockIdx.x] = make_double2(rr[0], ri[0]);
}

// grad[j] += 2 h^d Re sum_{m,n'} E^(j)[m][n'] Z[m][n'], E^(j) = [Eb0^(j) | Eb^(j)] of the unit
// component j at t0 (Gauss-Legendre quadrature as in the time matrices).  One block.
__global__ void k_grad_final(const TimeMats* __restrict__ tm, double t0, double hd, const double2* __restrict__ partials,
                             int nblocks, double* __restrict__ grad) {
  __shared__ double2 Z[LA_KMAX * (LA_KMAX + 1)];
  const int K = tm->K, npair = K * (K + 1);
  for (int pr = threadIdx.x; pr < npair; pr += blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      const double2 v = partials[(long long)pr * nblocks + b];
      sx += v.x;
      sy += v.y;
    }
    Z[pr] = make_double2(sx, sy);
  }
  __syncthreads();
  const double dt = tm->dt;
  for (int j = threadIdx.x; j < tm->ncomp; j += blockDim.x) {
    double acc = 0.0;
    for (int m = 0; m < K; ++m) {
      for (int nn = 0; nn <= K; ++nn) {
        double e = 0.0;
        for (int q = 0; q < tm->nq; ++q) {
          const double t = t0 + 0.5 * (tm->tau[q] + 1.0) * dt;
          double env = 1.0;
          if (tm->sigma[j] > 0.0) {
            const double u = (t - tm->tc[j]) / tm->sigma[j];
            env = exp(-u * u);
          }
          const double fld = env * sin(tm->omega[j] * t);
          const double bn = nn == 0 ? 1.0 : tm->bq[q * LA_KMAX + (nn - 1)];
          e += tm->wq[q] * tm->bq[q * LA_KMAX + m] * bn * fld;
        }
        acc += 0.5 * dt * e * Z[m * (K + 1) + nn].x;
      }
    }
    grad[j] += 2.0 * hd * acc;
  }
}

void launch_grad_contract(const FineOp& g, const TimeMats* tm, int K, double t0, double hd, const double2* zneg,
                          const double2* psi, const double2* c, double2* partials, double* grad, cudaStream_t s) {
  const int np = g.n[0] * g.n[1] * g.n[2];
  dim3 grid((np + 255) / 256, K * (K + 1));
  k_grad_partials<<<grid, 256, 0, s>>>(g, K, zneg, psi, c, partials);
  k_grad_final<<<1, 64, 0, s>>>(tm, t0, hd, partials, grid.x, grad);
}

// lambda_p += h^d [ (H u)_p + x_p sum_m Eb0_m mu_pm ],  u_q = sum_m Ub0_m mu_qm, mu = -zneg
__global__ void k_lambda_update(FineOp g, const TimeMats* __restrict__ tm, double hd, const double2* __restrict__ zneg,
                                double2* __restrict__ lam) {
  const int np = g.n[0] * g.n[1] * g.n[2];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int K = tm->K;
  const int x = p % g.n[0], y = (p / g.n[0]) % g.n[1], z = p / (g.n[0] * g.n[1]);
  auto u_at = [&](int q) {
    double2 u = make_double2(0.0, 0.0);
    for (int m = 0; m < K; ++m) {
      const double2 v = zneg[(long long)q * K + m];
      u.x -= tm->Ub0[m] * v.x;
      u.y -= tm->Ub0[m] * v.y;
    }
    return u;
  };
  const double2 up = u_at(p);
  const double dg = g.dsum + g.V0[p];
  double2 hu = make_double2(dg * up.x, dg * up.y);
  const int nb[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  for (int t = 0; t < 2 * g.dim; ++t) {
    const int qx = x + nb[t][0], qy = y + nb[t][1], qz = z + nb[t][2];
    if (qx < 0 || qy < 0 || qz < 0 || qx >= g.n[0] || qy >= g.n[1] || qz >= g.n[2]) continue;
    const double2 uq = u_at((qz * g.n[1] + qy) * g.n[0] + qx);
    const double w = -0.5 * g.ih2[t >> 1];
    hu.x += w * uq.x;
    hu.y += w * uq.y;
  }
  double2 e = make_double2(0.0, 0.0);
  for (int m = 0; m < K; ++m) {
    const double2 v = zneg[(long long)p * K + m];
    e.x -= tm->Eb0[m] * v.x;
    e.y -= tm->Eb0[m] * v.y;
  }
  const double xl = fine_x(g, x, y, z);
  double2 l = lam[p];
  l.x += hd * (hu.x + xl * e.x);
  l.y += hd * (hu.y + xl * e.y);
  lam[p] = l;
}
void launch_lambda_update(const FineOp& g, const TimeMats* tm, double hd, const double2* zneg, double2* lam,
                          cudaStream_t s) {
  const int np = g.n[0] * g.n[1] * g.n[2];
  k_lambda_update<<<(np + 255) / 256, 256, 0, s>>>(g, tm, hd, zneg, lam);
}

}  // namespace la
