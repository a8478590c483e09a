// Galerkin coarse operators (Sec. III, P A P^T with P^T = I): the spatial factors of the
// Kronecker normal operator, Sigma^{l+1}_kk' = I^T Sigma^l_kk' I, as radius-2 box stencils.
// They depend only on the static potential and the grid, so they are built once per
// la_set_hamiltonian; the per-step time factors Theta_kk' are combined with them later.
#include "la_internal.cuh"

namespace la {

// children of coarse index J on one axis with interpolation weights (transpose of the
// cell-centred linear interpolation): fine {2J-1, 2J, 2J+1, 2J+2} with {1/4, 3/4, 3/4, 1/4}.
__device__ __forceinline__ int gal_children(int J, int nf, bool used, int a[4], double w[4]) {
  if (!used) { a[0] = J; w[0] = 1.0; return 1; }
  int cnt = 0;
  const int cand[4] = {2 * J - 1, 2 * J, 2 * J + 1, 2 * J + 2};
  const double wc[4] = {0.25, 0.75, 0.75, 0.25};
  for (int t = 0; t < 4; ++t)
    if (cand[t] >= 0 && cand[t] < nf) { a[cnt] = cand[t]; w[cnt] = wc[t]; ++cnt; }
  return cnt;
}

// Shared driver: thread per (coarse point J, coarse offset o').  For each fine pair (a in
// supp(J), b in supp(J+o')) with |a-b| <= 2 accumulate w_a w_b Sigma_f[a, b] (9 pairs).
template <bool FROM_FINE>
__global__ void k_galerkin(FineOp g, LevelGeom F, const double* __restrict__ sigma_f, LevelGeom C,
                           double* __restrict__ sigma_c) {
  const int nbox = box5_count(C.dim);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C.np * nbox) return;
  const int J = (int)(t / nbox), o = (int)(t % nbox);
  int ox = 0, oy = 0, oz = 0;
  if (C.dim == 1) { ox = o - 2; }
  else if (C.dim == 2) { ox = o % 5 - 2; oy = o / 5 - 2; }
  else { ox = o % 5 - 2; oy = (o / 5) % 5 - 2; oz = o / 25 - 2; }
  const int jx = J % C.n[0], jy = (J / C.n[0]) % C.n[1], jz = J / (C.n[0] * C.n[1]);
  const int kx = jx + ox, ky = jy + oy, kz = jz + oz;
  double acc[LA_NPAIR];
  for (int k = 0; k < LA_NPAIR; ++k) acc[k] = 0.0;
  if (kx >= 0 && ky >= 0 && kz >= 0 && kx < C.n[0] && ky < C.n[1] && kz < C.n[2]) {
    int ax[4], ay[4], az[4], bx[4], by[4], bz[4];
    double wax[4], way[4], waz[4], wbx[4], wby[4], wbz[4];
    const int nax = gal_children(jx, F.n[0], C.dim > 0, ax, wax), nbx = gal_children(kx, F.n[0], C.dim > 0, bx, wbx);
    const int nay = gal_children(jy, F.n[1], C.dim > 1, ay, way), nby = gal_children(ky, F.n[1], C.dim > 1, by, wby);
    const int naz = gal_children(jz, F.n[2], C.dim > 2, az, waz), nbz = gal_children(kz, F.n[2], C.dim > 2, bz, wbz);
    const int fnbox = box5_count(F.dim);
#pragma unroll 1
    for (int iaz = 0; iaz < naz; ++iaz)
#pragma unroll 1
      for (int iay = 0; iay < nay; ++iay)
#pragma unroll 1
        for (int iax = 0; iax < nax; ++iax) {
          const double wa = wax[iax] * way[iay] * waz[iaz];
          const int pa = (az[iaz] * F.n[1] + ay[iay]) * F.n[0] + ax[iax];
#pragma unroll 1
          for (int ibz = 0; ibz < nbz; ++ibz)
#pragma unroll 1
            for (int iby = 0; iby < nby; ++iby)
#pragma unroll 1
              for (int ibx = 0; ibx < nbx; ++ibx) {
                const int dx = bx[ibx] - ax[iax], dy = by[iby] - ay[iay], dz = bz[ibz] - az[iaz];
                if (abs(dx) > 2 || abs(dy) > 2 || abs(dz) > 2) continue;
                // the finest-level factors (I, H, X products) vanish beyond Manhattan distance 2
                if (FROM_FINE && abs(dx) + abs(dy) + abs(dz) > 2) continue;
                const double w = wa * wbx[ibx] * wby[iby] * wbz[ibz];
                if (FROM_FINE) {
                  double s[LA_NPAIR];
                  fine_sigma(g, ax[iax], ay[iay], az[iaz], bx[ibx], by[iby], bz[ibz], s);
                  for (int k = 0; k < LA_NPAIR; ++k) acc[k] += w * s[k];
                } else {
                  const int fo = box5_index(F.dim, dx, dy, dz);
                  for (int k = 0; k < LA_NPAIR; ++k) acc[k] += w * sigma_f[sigma_offset(pa, k, fo, fnbox)];
                }
              }
        }
  }
  for (int k = 0; k < LA_NPAIR; ++k) sigma_c[sigma_offset(J, k, o, nbox)] = acc[k];
}

void launch_galerkin_from_fine(const FineOp& g, const LevelGeom& coarse, double* sigma_c, cudaStream_t s) {
  LevelGeom F;
  F.dim = g.dim;
  for (int a = 0; a < 3; ++a) F.n[a] = g.n[a];
  F.np = g.n[0] * g.n[1] * g.n[2];
  long long nt = (long long)coarse.np * box5_count(coarse.dim);
  k_galerkin<true><<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(g, F, nullptr, coarse, sigma_c);
}

void launch_galerkin_coarse(const LevelGeom& fine, const double* sigma_f, const LevelGeom& coarse, double* sigma_c,
                            cudaStream_t s) {
  FineOp g{};
  long long nt = (long long)coarse.np * box5_count(coarse.dim);
  k_galerkin<false><<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(g, fine, sigma_f, coarse, sigma_c);
}

}  // namespace la
