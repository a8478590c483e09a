// Galerkin coarse operators (Sec. III, P A P^T with P^T = I): the spatial factors of the
// Kronecker normal operator, Sigma^{l+1}_kk' = I^T Sigma^l_kk' I, as radius-2 box stencils.
// They depend only on the static potential and the grid, so they are built once per
// la_set_hamiltonian; the per-step time factors Theta_kk' are combined with them later.
#include "la_internal.cuh"

namespace la {

// Children of coarse index J on one axis (transpose of the cell-centred linear interpolation):
// fine 2J-1 .. 2J+2 inside [0, nf) with weights 1/4, 3/4, 3/4, 1/4; an unused axis maps J to J.
__device__ __forceinline__ void gal_range(int J, int nf, bool used, int& lo, int& hi) {
  if (!used) { lo = hi = J; return; }
  lo = max(2 * J - 1, 0);
  hi = min(2 * J + 2, nf - 1);
}
__device__ __forceinline__ double gal_weight(int a, int J, bool used) {
  return !used ? 1.0 : ((a == 2 * J || a == 2 * J + 1) ? 0.75 : 0.25);
}

// Thread per (coarse point J, coarse offset o).  Sums w_a w_b Sigma_f[a, b] (9 pairs) over the fine
// pairs a in supp(J), b in supp(J + o) that can be nonzero: |a - b| <= 2 per axis on a Galerkin
// level (box stencils), and |a - b|_1 <= 2 on the finest level, where the factors are products of
// I, H (7-point) and X.  The b ranges are intersected with those limits axis by axis, so only
// contributing pairs are visited.
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
  const bool ux = C.dim > 0, uy = C.dim > 1, uz = C.dim > 2;
  double acc[LA_NPAIR];
#pragma unroll
  for (int k = 0; k < LA_NPAIR; ++k) acc[k] = 0.0;
  if (kx >= 0 && ky >= 0 && kz >= 0 && kx < C.n[0] && ky < C.n[1] && kz < C.n[2]) {
    int alx, ahx, aly, ahy, alz, ahz, blx, bhx, bly, bhy, blz, bhz;
    gal_range(jx, F.n[0], ux, alx, ahx); gal_range(kx, F.n[0], ux, blx, bhx);
    gal_range(jy, F.n[1], uy, aly, ahy); gal_range(ky, F.n[1], uy, bly, bhy);
    gal_range(jz, F.n[2], uz, alz, ahz); gal_range(kz, F.n[2], uz, blz, bhz);
    const int fnbox = box5_count(F.dim);
#pragma unroll 1
    for (int az = alz; az <= ahz; ++az)
#pragma unroll 1
      for (int ay = aly; ay <= ahy; ++ay)
#pragma unroll 1
        for (int ax = alx; ax <= ahx; ++ax) {
          const double wa = gal_weight(ax, jx, ux) * gal_weight(ay, jy, uy) * gal_weight(az, jz, uz);
          const int pa = (az * F.n[1] + ay) * F.n[0] + ax;
#pragma unroll 1
          for (int bz = max(blz, az - 2); bz <= min(bhz, az + 2); ++bz) {
            const int rz = FROM_FINE ? 2 - abs(bz - az) : 2;
#pragma unroll 1
            for (int by = max(bly, ay - rz); by <= min(bhy, ay + rz); ++by) {
              const int ry = FROM_FINE ? rz - abs(by - ay) : 2;
              const double wyz = wa * gal_weight(by, ky, uy) * gal_weight(bz, kz, uz);
#pragma unroll 1
              for (int bx = max(blx, ax - ry); bx <= min(bhx, ax + ry); ++bx) {
                const double w = wyz * gal_weight(bx, kx, ux);
                if (FROM_FINE) {
                  double s[LA_NPAIR];
                  fine_sigma(g, ax, ay, az, bx, by, bz, s);
#pragma unroll
                  for (int k = 0; k < LA_NPAIR; ++k) acc[k] += w * s[k];
                } else {
                  const int fo = box5_index(F.dim, bx - ax, by - ay, bz - az);
#pragma unroll
                  for (int k = 0; k < LA_NPAIR; ++k) acc[k] += w * sigma_f[sigma_offset(pa, k, fo, fnbox)];
                }
              }
            }
          }
        }
  }
#pragma unroll
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
