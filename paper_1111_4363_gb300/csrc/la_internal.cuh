// Internal declarations of the least-action CUDA library (not part of the C ABI).
//
// Notation (Walters, Secs. I-III).  One time step: unknowns c[p, n], p a grid point,
// n = 1..K the free Legendre time functions b_n = P_n - (-1)^n P_0.  Without the
// overlap factor h^d the least-action operator is the Kronecker sum
//     M~ = sum_k S_k (x) T_k,   S = (I, H, X),   T = (i Qb, -Ub, -Eb(t0)),
// H = T_kin + V0 (FD stencil), X = diag(x_laser).  The normal matrix of the
// residual norm is  G~ = M~^dagger (I (x) Wt) M~ = sum_{k,k'} (S_k S_k') (x) Theta_kk',
// Theta_kk' = T_k^dagger Wt T_k'.  Coarse levels keep this form with spatial
// factors Sigma^l_kk' = I^T Sigma^{l-1}_kk' I (Galerkin, Sec. III), stored as
// radius-2 box stencils.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#define LA_KMAX 8          // largest K (free time functions per point)
#define LA_NPAIR 9         // (k, k') pairs of the Kronecker normal operator
#define LA_BLK 16          // block size of the subvolume factor layout
#define LA_NPAD_MAX 128    // largest padded subvolume size (unknowns) factorised by one CTA in shared memory
#define LA_NPTS_MAX 32     // largest number of grid points in such a subvolume
#define LA_NPAD_WIDE 256   // largest padded size of a finest-level subvolume (factorised in global memory)
#define LA_NPTS_WIDE 64    // largest number of grid points in a finest-level subvolume
#define LA_NQ_MAX 32       // largest number of Gauss nodes per step
#define LA_NCOMP_MAX 64    // largest number of pulse components

namespace la {

// Per-context time-basis data, in device global memory.  Static parts are written by the
// host at init; Eb, Eb0 and Theta are rewritten by k_time_matrices for every step.
struct TimeMats {
  int K;
  int nq;
  double dt;
  double Qb[LA_KMAX * LA_KMAX];   // int b_m b_n'          (test m, trial n)
  double Ub[LA_KMAX * LA_KMAX];   // (dt/2) int b_m b_n
  double Wt[LA_KMAX * LA_KMAX];   // time part of the residual-norm weight
  double Ub0[LA_KMAX];            // (dt/2) int b_m P_0
  double endv[LA_KMAX];           // b_n(+1)
  double tau[LA_NQ_MAX], wq[LA_NQ_MAX];          // Gauss-Legendre rule on [-1, 1]
  double bq[LA_NQ_MAX * LA_KMAX];                // b_m(tau_q)
  int ncomp;
  double amp[LA_NCOMP_MAX], omega[LA_NCOMP_MAX], tc[LA_NCOMP_MAX], sigma[LA_NCOMP_MAX];
  // per step
  double t0;
  double Eb[LA_KMAX * LA_KMAX];
  double Eb0[LA_KMAX];
  double P[LA_NPAIR][LA_KMAX * LA_KMAX];  // R_k^T Wt R_k', R = (Qb, Ub, Eb)
};
// Theta_kk' = phase_kk' * P_kk' with phase = conj(alpha_k) alpha_k', alpha = (i, -1, -1):
// (0,0) -> 1, (0,1),(0,2) -> +i, (1,0),(2,0) -> -i, others 1.
__host__ __device__ inline int theta_phase(int kk) {  // 0: real +1, 1: +i, 2: -i
  int k = kk / 3, kp = kk % 3;
  if (k == 0 && kp != 0) return 1;
  if (kp == 0 && k != 0) return 2;
  return 0;
}

// ------------------------------------------------------------------ time-basis constants (host)
// Legendre P_0..P_n at y by the three-term recurrence.
__host__ inline void legendre_all(int n, double y, double* P) {
  P[0] = 1.0;
  if (n >= 1) P[1] = y;
  for (int k = 2; k <= n; ++k) P[k] = ((2.0 * k - 1.0) * y * P[k - 1] - (k - 1.0) * P[k - 2]) / k;
}
// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_q.
__host__ inline void gauss_legendre(int q, double* x, double* w) {
  std::vector<double> P(q + 1);
  for (int i = 0; i < q; ++i) {
    double y = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      legendre_all(q, y, P.data());
      double dp = q * (y * P[q] - P[q - 1]) / (y * y - 1.0);
      double dy = P[q] / dp;
      y -= dy;
      if (std::fabs(dy) < 1e-16) break;
    }
    legendre_all(q, y, P.data());
    double dp = q * (y * P[q] - P[q - 1]) / (y * y - 1.0);
    x[i] = y;
    w[i] = 2.0 / ((1.0 - y * y) * dp * dp);
  }
}
// Inverse of a small n x n matrix (n <= LA_KMAX) by Gauss-Jordan elimination with partial pivoting.
__host__ inline bool invert_small(int n, const double* A, double* Ainv) {
  double M[LA_KMAX][2 * LA_KMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    if (std::fabs(M[piv][col]) < 1e-300) return false;
    for (int j = 0; j < 2 * n; ++j) std::swap(M[col][j], M[piv][j]);
    double d = M[col][col];
    for (int j = 0; j < 2 * n; ++j) M[col][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = M[r][col];
      for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[col][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i][n + j];
  return true;
}
// The static part of TimeMats for K time functions, step dt and residual-norm weight (0 = Ub^{-1},
// 1 = Ub, 2 = identity), from the closed forms of Sec. IV (orthogonality 2 delta/(2n+1), Q_nm = 2 for
// n > m with n - m odd, P_n(+-1) = (+-1)^n) in the basis b_n = P_n - (-1)^n P_0, n = 1..K, and the
// K + 8-node Gauss rule the per-step field matrices use.  False when Ub cannot be inverted.
__host__ inline bool fill_time_constants(int K, double dt, int weight, TimeMats& t) {
  memset(&t, 0, sizeof t);
  t.K = K;
  t.dt = dt;
  for (int m = 1; m <= K; ++m) {
    const double sm = (m % 2) ? -1.0 : 1.0;
    t.Ub0[m - 1] = -sm * dt;
    t.endv[m - 1] = 1.0 - sm;
    for (int n = 1; n <= K; ++n) {
      const double sn = (n % 2) ? -1.0 : 1.0;
      t.Ub[(m - 1) * K + (n - 1)] = dt * ((m == n ? 1.0 / (2 * m + 1) : 0.0) + sm * sn);
      const double q = (n > m && ((n - m) % 2 == 1)) ? 2.0 : 0.0;
      t.Qb[(m - 1) * K + (n - 1)] = q - sm * (1.0 - sn);
    }
  }
  if (weight == 0) {
    if (!invert_small(K, t.Ub, t.Wt)) return false;
  } else if (weight == 1) {
    memcpy(t.Wt, t.Ub, sizeof(double) * K * K);
  } else {
    for (int i = 0; i < K; ++i) t.Wt[i * K + i] = 1.0;
  }
  t.nq = K + 8;
  gauss_legendre(t.nq, t.tau, t.wq);
  std::vector<double> P(K + 1);
  for (int q = 0; q < t.nq; ++q) {
    legendre_all(K, t.tau[q], P.data());
    for (int m = 1; m <= K; ++m) t.bq[q * LA_KMAX + (m - 1)] = P[m] - ((m % 2) ? -1.0 : 1.0);
  }
  return true;
}

// Geometry of one multigrid level.
// Division by a divisor fixed for a launch or a CTA: floor(x / d) = (x m) >> s for 0 <= x < 2^31, with
// s = 31 + ceil(log2 d) and m = floor(2^s / d) + 1 < 2^32 (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): one wide multiply and a shift instead of
// the instruction sequence of an integer division.
struct FastDiv {
  int d;
  unsigned m, s;
};
__host__ __device__ inline FastDiv make_fastdiv(int d) {
  unsigned l = 0;
  while ((1u << l) < (unsigned)d) ++l;
  FastDiv f;
  f.d = d;
  f.s = 31 + l;
  f.m = (unsigned)((1ull << f.s) / (unsigned long long)d + 1ull);
  return f;
}
__host__ __device__ __forceinline__ int fdiv(int x, const FastDiv& f) {
  return (int)(((unsigned long long)(unsigned)x * f.m) >> f.s);
}

struct LevelGeom {
  int dim;
  int n[3];        // points per axis (unused axes 1)
  int np;          // points
  int sub[3];      // subvolume extent per axis (unused axes 1)
  int nb[3];       // subvolumes per axis
  int nsub;        // subvolumes
  int npad;        // padded unknowns per subvolume, multiple of LA_BLK
  int nblk;        // npad / LA_BLK
  long long fsize; // complex entries per subvolume factor: nblk(nblk+1)/2 * LA_BLK^2
  // divisors of the finest-level sweep's index maps for a full (not ragged) subvolume: K, and the
  // x and y extents of U + 2 (c box), U + 1 (footprint) and U (1 on unused axes)
  FastDiv fd_K, fd_c[2], fd_f[2], fd_u[2];
  FastDiv fd_pair;   // Galerkin levels: stencil values per point, 9 pairs x the radius-2 box
  int one_per_cta;   // factorise one subvolume matrix per CTA (no packing of small matrices)
  // block bandwidth of the local factor: blocks (I, K) with I - K > band are exactly zero.  The
  // finest-level operator couples points at most two grid steps apart (H^2), so G_UU and its Cholesky
  // factor (no fill outside the envelope) vanish beyond the largest index distance of such a pair; the
  // wide (global-memory) factorisation and solves skip those blocks.  nblk - 1 where nothing is skipped.
  int band;
};

// Finest-level spatial operator: H = -1/2 Laplacian + V0, X = x along laser_axis.
struct FineOp {
  int dim;
  int n[3];
  double h[3];
  double ih2[3];   // 1/h^2 (0 on unused axes)
  double x0[3];    // coordinate of point 0: -(n-1)/2 h
  double dsum;     // diagonal of the kinetic stencil: sum_a 1/h_a^2
  int lax;         // laser axis
  const double* V0;
};

// index of offset (ox, oy, oz), each in [-2, 2] on used axes and 0 on unused ones, in a radius-2 box
__host__ __device__ inline int box5_index(int dim, int ox, int oy, int oz) {
  return dim == 1 ? ox + 2 : (dim == 2 ? (ox + 2) + 5 * (oy + 2) : (ox + 2) + 5 * (oy + 2) + 25 * (oz + 2));
}
__host__ __device__ inline int box5_count(int dim) { return dim == 1 ? 5 : (dim == 2 ? 25 : 125); }
// stencil storage of a coarse level: [point][pair][box5]
__host__ __device__ inline long long sigma_offset(int p, int kk, int o, int nbox) {
  return ((long long)p * LA_NPAIR + kk) * nbox + o;
}

__device__ inline double fine_H(const FineOp& g, int px, int py, int pz, int qx, int qy, int qz) {
  int dx = qx - px, dy = qy - py, dz = qz - pz;
  if (dx == 0 && dy == 0 && dz == 0) return g.dsum + g.V0[(pz * g.n[1] + py) * g.n[0] + px];
  int ad = abs(dx) + abs(dy) + abs(dz);
  if (ad != 1) return 0.0;
  if (dx) return -0.5 * g.ih2[0];
  if (dy) return -0.5 * g.ih2[1];
  return -0.5 * g.ih2[2];
}
// Selects instead of indexing the parameter arrays with g.lax: a runtime index into a by-value
// kernel parameter forces a local-memory copy of the struct.
__device__ inline double fine_x(const FineOp& g, int px, int py, int pz) {
  if (g.lax == 0) return g.x0[0] + px * g.h[0];
  if (g.lax == 1) return g.x0[1] + py * g.h[1];
  return g.x0[2] + pz * g.h[2];
}
__device__ inline bool fine_in(const FineOp& g, int x, int y, int z) {
  return x >= 0 && y >= 0 && z >= 0 && x < g.n[0] && y < g.n[1] && z < g.n[2];
}
// Sigma^0_kk'[p, q] = (S_k S_k')[p, q] for the 9 pairs, p and q inside the grid.
__device__ inline void fine_sigma(const FineOp& g, int px, int py, int pz, int qx, int qy, int qz, double s[9]) {
  double Hpq = fine_H(g, px, py, pz, qx, qy, qz);
  // (H^2)_pq = sum over r in {p, p +- e_a} inside the grid of H_pr H_rq
  double H2 = 0.0;
  int nofs = 1 + 2 * g.dim;
#pragma unroll 1
  for (int t = 0; t < nofs; ++t) {
    // r = p, then p + e_0, p - e_0, p + e_1, ... (offsets computed, not tabulated: a runtime-indexed
    // table would live in local memory)
    const int ax = (t - 1) >> 1, sg = (t & 1) ? 1 : -1;
    const int rx = px + (t > 0 && ax == 0 ? sg : 0), ry = py + (t > 0 && ax == 1 ? sg : 0),
              rz = pz + (t > 0 && ax == 2 ? sg : 0);
    if (!fine_in(g, rx, ry, rz)) continue;
    int ex = abs(qx - rx), ey = abs(qy - ry), ez = abs(qz - rz);
    if (ex + ey + ez > 1) continue;
    H2 += fine_H(g, px, py, pz, rx, ry, rz) * fine_H(g, rx, ry, rz, qx, qy, qz);
  }
  bool same = (px == qx && py == qy && pz == qz);
  double xp = fine_x(g, px, py, pz), xq = fine_x(g, qx, qy, qz);
  s[0] = same ? 1.0 : 0.0;      // (0,0) I
  s[1] = Hpq;                   // (0,1) H
  s[2] = same ? xp : 0.0;       // (0,2) X
  s[3] = Hpq;                   // (1,0) H
  s[4] = H2;                    // (1,1) H^2
  s[5] = Hpq * xq;              // (1,2) H X
  s[6] = same ? xp : 0.0;       // (2,0) X
  s[7] = xp * Hpq;              // (2,1) X H
  s[8] = same ? xp * xp : 0.0;  // (2,2) X^2
}

// Subvolume b (lexicographic, x fastest) of a level -> origin and extent.
__host__ __device__ inline void subvol_box(const LevelGeom& L, int b, int o[3], int e[3]) {
  int bx = b % L.nb[0];
  int rest = b / L.nb[0];
  int by = rest % L.nb[1];
  int bz = rest / L.nb[1];
  int bb[3] = {bx, by, bz};
  for (int a = 0; a < 3; ++a) {
    o[a] = bb[a] * L.sub[a];
    int r = L.n[a] - o[a];
    e[a] = r < L.sub[a] ? r : L.sub[a];
  }
}
// j-th subvolume of colour `colour` -> subvolume index.  colour bit a = parity of block index on axis a.
__host__ __device__ inline int colour_subvol(const LevelGeom& L, int colour, int j) {
  int cb[3] = {colour & 1, (colour >> 1) & 1, (colour >> 2) & 1};
  int cnt[3];
  for (int a = 0; a < 3; ++a) cnt[a] = (L.nb[a] - cb[a] + 1) / 2;
  int ix = j % cnt[0];
  int r = j / cnt[0];
  int iy = r % cnt[1];
  int iz = r / cnt[1];
  int bx = 2 * ix + cb[0], by = 2 * iy + cb[1], bz = 2 * iz + cb[2];
  return (bz * L.nb[1] + by) * L.nb[0] + bx;
}
__host__ inline int colour_count(const LevelGeom& L, int colour) {
  int c = 1;
  for (int a = 0; a < 3; ++a) {
    int cb = (colour >> a) & 1;
    if (a >= L.dim && cb) return 0;
    c *= (L.nb[a] - cb + 1) / 2;
  }
  return c;
}

// Block bandwidth of a finest-level subvolume factor (LevelGeom::band).  G_UU couples two unknowns only
// when their points are at most two grid steps apart (Manhattan), which in the subvolume's x-fastest
// point order means point indices at most d_max apart; the Cholesky factor keeps that envelope.  Block
// (I, J) holds the points floor(16 I / K) .. and .. floor((16 J + 15) / K), so it is zero when the
// nearest two are more than d_max apart; the band is the largest I - J of a block that may be nonzero,
// at least 1 (a wider band is exact too) and at most nblk - 1.
__host__ inline int fine_band_blocks(int dim, const int sub[3], int K, int nblk) {
  int maxd = 0;
  for (int dz = -2; dz <= 2; ++dz)
    for (int dy = -2; dy <= 2; ++dy)
      for (int dx = -2; dx <= 2; ++dx) {
        const int man = (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy) + (dz < 0 ? -dz : dz);
        if (man > 2 || (dim < 2 && dy != 0) || (dim < 3 && dz != 0)) continue;
        const int d = dx + sub[0] * dy + sub[0] * sub[1] * dz;
        if ((d < 0 ? -d : d) > maxd) maxd = d < 0 ? -d : d;
      }
  int band = 0;
  for (int d = 1; d < nblk; ++d)
    for (int J = 0; J + d < nblk; ++J)
      if ((LA_BLK * (J + d)) / K - (LA_BLK * J + LA_BLK - 1) / K <= maxd) band = d;
  if (band < 1) band = 1;
  return band < nblk - 1 ? band : nblk - 1;
}

template <typename R> struct C2;
template <> struct C2<double> { typedef double2 T; };
template <> struct C2<float> { typedef float2 T; };

// ---------------------------------------------------------------- launch wrappers
// time basis
void launch_time_matrices(TimeMats* tm, double t0, cudaStream_t s);
// grid kernels (FP64 unless noted)
void launch_rhs(const FineOp& g, const TimeMats* tm, const double2* psi0, double2* f, cudaStream_t s);
template <typename R>
void launch_mresid(const FineOp& g, const TimeMats* tm, int K, const typename C2<R>::T* f, const typename C2<R>::T* c,
                   typename C2<R>::T* r, typename C2<R>::T* z, double* partials, int nblocks_norm, cudaStream_t s,
                   const CUtensorMap* cmap = nullptr, int* status = nullptr);
template <typename R>
void launch_mnormal(const FineOp& g, const TimeMats* tm, int K, const typename C2<R>::T* z, typename C2<R>::T* out,
                    cudaStream_t s, const typename C2<R>::T* yadd = nullptr, const CUtensorMap* zmap = nullptr,
                    int* status = nullptr);
// Tensor map of a complex64 field for the TMA-staged stencils (false: field does not qualify).
bool encode_stencil_map(const FineOp& g, int K, const float2* field, CUtensorMap* map);
// adjoint
void launch_bt_lambda(int np, const TimeMats* tm, double inv_hd, const double2* lam, double2* y, cudaStream_t s);
void launch_norm2_partials(long long n, const double2* v, double* partials, int nblocks, cudaStream_t s);
void launch_grad_contract(const FineOp& g, const TimeMats* tm, int K, double t0, double hd, const double2* zneg,
                          const double2* psi, const double2* c, double2* partials, double* grad, cudaStream_t s);
void launch_lambda_update(const FineOp& g, const TimeMats* tm, double hd, const double2* zneg, double2* lam,
                          cudaStream_t s);
template <typename R>
void launch_restrict(const LevelGeom& fine, const LevelGeom& coarse, int K, const typename C2<R>::T* sf,
                     typename C2<R>::T* gc, cudaStream_t s);
template <typename R>
void launch_prolong_add(const LevelGeom& fine, const LevelGeom& coarse, int K, const typename C2<R>::T* ec,
                        typename C2<R>::T* ef, cudaStream_t s);
void launch_norm_final(const double* partials, int n, double scale, double* out, cudaStream_t s);
int norm_blocks(int np);
void launch_advance(int np, const TimeMats* tm, const double2* c, double2* psi, cudaStream_t s);
void launch_axpy_c64_to_c128(long long n, const float2* x, double2* y, cudaStream_t s);
void launch_c128_to_c64(long long n, const double2* x, float2* y, cudaStream_t s);
void launch_f64_to_f32(long long n, const double* x, float* y, cudaStream_t s);
void launch_scale_c128(long long n, double a, const double2* x, double2* y, cudaStream_t s);
void launch_trial(long long n, const double* a, const double2* h0, const double2* h1, const double2* h2, double2* c,
                  cudaStream_t s);
// device-side relaxation loop of one context (la_step_batch): state and per-step record
struct LoopState {
  double N0;   // N(0) = f^dagger W f of the step
  double N;    // N of the current iterate
  int cyc;     // cycles run in the step
  int pad;
};
struct LoopRecord {
  double N0, N;
  int cycles, pad;
};
// keep the trial (c from the extrapolation) when its action Nslot[0] is below N(0) = Nslot[1], else c = 0
// and r = f; initialises the loop state
void launch_seed_select(long long n, const double* Nslot, int tried, LoopState* st, double2* c, double2* r,
                        const double2* f, cudaStream_t s);
// sets the loop's condition: first = 1 before the first cycle, else after a cycle (N from Nnew[0], cycle
// counted); continue while N is finite, below max_cycles and (when check) above tol N(0)
void launch_loop_cond(LoopState* st, const double* Nnew, double tol, int max_cycles, int check, int first,
                      cudaGraphConditionalHandle h, cudaStream_t s);
void launch_loop_record(const LoopState* st, LoopRecord* rec, cudaStream_t s);
// Galerkin coarse stencils
void launch_galerkin_from_fine(const FineOp& g, const LevelGeom& coarse, double* sigma_c, cudaStream_t s);
void launch_galerkin_coarse(const LevelGeom& fine, const double* sigma_f, const LevelGeom& coarse, double* sigma_c,
                            cudaStream_t s);
// subvolume factorisation and sweeps (dispatch over the padded subvolume size)
template <typename R>
cudaError_t launch_factor(const LevelGeom& L, const FineOp* fine, const R* sigma, const TimeMats* tm,
                          typename C2<R>::T* factors, int* status, cudaStream_t s);
template <typename R>
cudaError_t launch_sweep_fine(const LevelGeom& L, const FineOp& g, const TimeMats* tm, int K,
                              const typename C2<R>::T* f, const typename C2<R>::T* yx, typename C2<R>::T* c,
                              const typename C2<R>::T* factors, int colour, int* status, cudaStream_t s);
template <typename R>
cudaError_t launch_gresid_tiles(const LevelGeom& L, const R* sigma, const TimeMats* tm, int K,
                                const typename C2<R>::T* gvec, const typename C2<R>::T* e, typename C2<R>::T* out,
                                cudaStream_t s);
// square local form (finest level, FP64): LU factors with row permutations, red-black sweeps
cudaError_t launch_factor_square(const LevelGeom& L, const FineOp& g, const TimeMats* tm, double2* lu, int* perm,
                                 int* status, cudaStream_t s);
cudaError_t launch_sweep_square(const LevelGeom& L, const FineOp& g, const TimeMats* tm, int K, const double2* f,
                                double2* c, const double2* lu, const int* perm, int colour, cudaStream_t s);
template <typename R>
cudaError_t launch_sweep_coarse(const LevelGeom& L, const R* sigma, const TimeMats* tm, int K,
                                const typename C2<R>::T* gvec, typename C2<R>::T* e,
                                const typename C2<R>::T* factors, int colour, int* status, cudaStream_t s);


// ------------------------------------------------------------------ mbarrier and bulk copies
// Every wait on an mbarrier polls a bounded number of times; a caller that gives up records a
// status bit instead of spinning on.
constexpr unsigned kMbarWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes initialised mbarriers visible to the asynchronous (copy) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Polls the phase of an mbarrier at most `limit` times; true when it completed.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace la
