// Subvolume relaxation kernels (Sec. II), templated on the arithmetic type R (double or float).
//
// A subvolume U is a block of grid points with all K time functions: n = |U| K unknowns,
// padded to NPAD (multiple of 16) with identity rows.  Its local least-squares problem
// (minimise the residual norm N over c_U, everything else fixed) has the Hermitian
// positive-definite matrix G_UU = sum_kk' Sigma_kk'[U, U] (x) Theta_kk' and right-hand side
// (M~^dagger Wt r)_U (finest level) or (g - G e)_U (Galerkin levels).
//
// Factor store of one subvolume: lower Cholesky factor L of G_UU in 16 x 16 blocks, block rows
// I = 0..NB-1 and block columns J <= I in the order (0,0), (1,0), (1,1), (2,0), ...; block
// (I, I) holds inv(L_II) instead of L_II so that every triangular-solve step is a mat-vec.
#pragma once
#include "la_internal.cuh"

namespace la {

template <typename CT> struct Re;
template <> struct Re<double2> { typedef double T; };
template <> struct Re<float2> { typedef float T; };

template <typename CT> __device__ __forceinline__ CT mkc(typename Re<CT>::T a, typename Re<CT>::T b) {
  CT r; r.x = a; r.y = b; return r;
}
// acc += a * b
template <typename CT> __device__ __forceinline__ void cfma(CT& acc, const CT a, const CT b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename CT> __device__ __forceinline__ void cfma_conj(CT& acc, const CT a, const CT b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

constexpr int kFactorThreads = 256;
constexpr int kSweepThreads = 128;

__device__ __forceinline__ void local_coords(int i, const int e[3], int& x, int& y, int& z) {
  x = i % e[0];
  int r = i / e[0];
  y = r % e[1];
  z = r / e[1];
}

// ======================================================================== factorisation
// One 256-thread CTA per subvolume of a level; two CTAs per SM.  The padded matrix lives in
// shared memory as a packed lower triangle (assembled tile-cyclically: thread (tid/16, tid%16)
// writes entries (16 I + tid/16, 16 J + tid%16)).  Right-looking Cholesky with two barriers per
// column: (A) column j is scaled by 1/L_jj and published, (B) the trailing triangle is updated
// with its entries spread linearly over the threads; the thread that updates the next pivot does
// it first and computes its reciprocal square root while the others are still updating
// (lookahead), so the pivot chain is off the critical path.
__host__ __device__ constexpr int tri_index(int r, int c) { return r * (r + 1) / 2 + c; }

// Small matrices leave most threads of a CTA idle in the later columns, so a CTA factorises
// factor_mpc(NPAD) matrices together: each phase's work is split over the entries of all of them and
// they share the two barriers per column.
__host__ __device__ constexpr int factor_mpc(int npad) { return npad <= 32 ? 8 : (npad <= 64 ? 2 : 1); }

template <typename R, int NPAD, int MPC>
__global__ void __launch_bounds__(kFactorThreads, 2)
k_factor(LevelGeom L, FineOp g, int is_fine, int nptsmax, const R* __restrict__ sigma,
         const TimeMats* __restrict__ tm, typename C2<R>::T* __restrict__ factors, int* __restrict__ status) {
  typedef typename C2<R>::T CT;
  constexpr int NTRI = NPAD * (NPAD + 1) / 2;
  constexpr int NB = NPAD / LA_BLK;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = tm->K, KK = K * K;
  const int npair_max = nptsmax * (nptsmax + 1) / 2;
  CT* sA = reinterpret_cast<CT*>(smem);                       // [MPC][NTRI] packed lower triangles
  CT* sCol = sA + MPC * NTRI;                                 // [MPC][NPAD] scaled column j
  R* sInv = reinterpret_cast<R*>(sCol + MPC * NPAD);          // [MPC][NPAD] 1/L_jj
  double* sP = reinterpret_cast<double*>(sInv + MPC * NPAD);  // [9][K*K]
  double* sPair = sP + LA_NPAIR * LA_KMAX * LA_KMAX;          // [MPC][npair_max][9], point pairs i >= j
  int* sMask = reinterpret_cast<int*>(sPair + (size_t)MPC * npair_max * LA_NPAIR);  // [MPC][npair_max]

  const int tid = threadIdx.x, ti = tid >> 4, tk = tid & 15;
  // the CTA's matrices; slots past the last subvolume factorise an identity and store nothing
  int bsv[MPC], nn_[MPC], npts_[MPC];
  int o_[MPC][3], e_[MPC][3];
#pragma unroll
  for (int mi = 0; mi < MPC; ++mi) {
    bsv[mi] = blockIdx.x * MPC + mi;
    if (bsv[mi] < L.nsub) {
      subvol_box(L, bsv[mi], o_[mi], e_[mi]);
      npts_[mi] = e_[mi][0] * e_[mi][1] * e_[mi][2];
    } else {
      o_[mi][0] = o_[mi][1] = o_[mi][2] = 0;
      e_[mi][0] = e_[mi][1] = e_[mi][2] = 1;
      npts_[mi] = 0;
    }
    nn_[mi] = npts_[mi] * K;
  }

  for (int i = tid; i < LA_NPAIR * KK; i += kFactorThreads) sP[i] = tm->P[i / KK][i % KK];
  // pair tables for point pairs i >= j: the nine spatial factors Sigma_kk'[p_i, p_j] and a bit mask
  // of the nonzero ones (most pairs of a subvolume are too far apart for most factors)
  const int nbox = box5_count(L.dim);
  for (int t = tid; t < MPC * npair_max; t += kFactorThreads) {
    const int mi = t / npair_max, q = t - mi * npair_max;
    int npts = 0, o[3] = {0, 0, 0}, e[3] = {1, 1, 1};
#pragma unroll
    for (int u = 0; u < MPC; ++u)
      if (u == mi) {
        npts = npts_[u];
        for (int a = 0; a < 3; ++a) { o[a] = o_[u][a]; e[a] = e_[u][a]; }
      }
    if (q >= npts * (npts + 1) / 2) continue;
    int i = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > q) --i;
    while ((i + 1) * (i + 2) / 2 <= q) ++i;
    const int j = q - i * (i + 1) / 2;
    int ix, iy, iz, jx, jy, jz;
    local_coords(i, e, ix, iy, iz);
    local_coords(j, e, jx, jy, jz);
    const int px = o[0] + ix, py = o[1] + iy, pz = o[2] + iz;
    const int qx = o[0] + jx, qy = o[1] + jy, qz = o[2] + jz;
    double s9[LA_NPAIR];
    if (is_fine) {
      fine_sigma(g, px, py, pz, qx, qy, qz, s9);
    } else {
      const int dx = qx - px, dy = qy - py, dz = qz - pz;
      const bool near = abs(dx) <= 2 && abs(dy) <= 2 && abs(dz) <= 2;
      const int p = (pz * L.n[1] + py) * L.n[0] + px;
      const int ofs = near ? box5_index(L.dim, dx, dy, dz) : 0;
      for (int k = 0; k < LA_NPAIR; ++k) s9[k] = near ? sigma[sigma_offset(p, k, ofs, nbox)] : 0.0;
    }
    int mask = 0;
    double* dst = sPair + ((size_t)mi * npair_max + q) * LA_NPAIR;
    for (int k = 0; k < LA_NPAIR; ++k) {
      dst[k] = s9[k];
      if (s9[k] != 0.0) mask |= 1 << k;
    }
    sMask[mi * npair_max + q] = mask;
  }
  // padding rows: identity
  for (int t = tid; t < MPC * NTRI; t += kFactorThreads) {
    const int mi = t / NTRI, u = t - mi * NTRI;
    int r = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > u) --r;
    while ((r + 1) * (r + 2) / 2 <= u) ++r;
    const int c = u - r * (r + 1) / 2;
    int n = 0;
#pragma unroll
    for (int w = 0; w < MPC; ++w) if (w == mi) n = nn_[w];
    if (r >= n) sA[t] = mkc<CT>((R)(r == c ? 1 : 0), (R)0);
  }
  __syncthreads();

  // ---- assemble pair-major: G_UU[(i,m),(j,n)] = sum_kk' Sigma_kk'[p_i, p_j] Theta_kk'[m, n].
  // Consecutive threads take the K*K entries of one point pair, so the skipped (zero) factors
  // are uniform across a warp except at pair boundaries.
  for (int t = tid; t < MPC * npair_max * KK; t += kFactorThreads) {
    const int mi = t / (npair_max * KK), tq = t - mi * npair_max * KK;
    const int q = tq / KK, mn = tq % KK, mm = mn / K, nn = mn % K;
    int npts = 0;
#pragma unroll
    for (int u = 0; u < MPC; ++u) if (u == mi) npts = npts_[u];
    if (q >= npts * (npts + 1) / 2) continue;
    int i = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > q) --i;
    while ((i + 1) * (i + 2) / 2 <= q) ++i;
    const int j = q - i * (i + 1) / 2;
    const int r = i * K + mm, c = j * K + nn;
    if (r < c) continue;
    const int mask = sMask[mi * npair_max + q];
    const double* pr = sPair + ((size_t)mi * npair_max + q) * LA_NPAIR;
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int kk = 0; kk < LA_NPAIR; ++kk) {
      if (!((mask >> kk) & 1)) continue;
      const double v = pr[kk] * sP[kk * KK + mm * K + nn];
      const int ph = theta_phase(kk);
      if (ph == 0) re += v; else if (ph == 1) im += v; else im -= v;
    }
    sA[mi * NTRI + tri_index(r, c)] = mkc<CT>((R)re, (R)im);
  }
  __syncthreads();
  if (tid < MPC) {
    CT* A = sA + tid * NTRI;
    R d2 = A[0].x;
    if (!(d2 > (R)0)) { atomicOr(status, 1); d2 = (R)1; }
    const R inv = rsqrt(d2);
    A[0] = mkc<CT>(d2 * inv, (R)0);
    sInv[tid * NPAD] = inv;
  }
  __syncthreads();

  // ---- right-looking Cholesky.  Work of each phase is spread linearly over exactly the active
  // entries of all the CTA's matrices (consecutive threads take consecutive entries of a row), so
  // every issued FP64 instruction has all lanes busy except in the last warp of a phase.
  for (int j = 0; j < NPAD; ++j) {
    // (A) scale and publish column j: rows j+1 .. NPAD-1 of every matrix
    {
      const int rows = NPAD - 1 - j;
      for (int t = tid; t < MPC * rows; t += kFactorThreads) {
        const int mi = t / rows, r = j + 1 + (t - mi * rows);
        const R inv = sInv[mi * NPAD + j];
        CT v = sA[mi * NTRI + tri_index(r, j)];
        v.x *= inv; v.y *= inv;
        sA[mi * NTRI + tri_index(r, j)] = v;
        sCol[mi * NPAD + r] = v;
      }
    }
    __syncthreads();
    // (B) trailing update of the entries (r, c), j < c <= r; entry e of a trailing triangle lies
    // in row r = j + m with (m-1) m / 2 <= e < m (m+1) / 2.  e = 0 is the next pivot: its thread
    // finishes it first and computes the reciprocal square root (lookahead).
    const int m1 = NPAD - 1 - j;
    const int T = m1 * (m1 + 1) / 2;
    for (int t = tid; t < MPC * T; t += kFactorThreads) {
      const int mi = t / T, e = t - mi * T;
      int m = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
      while ((m - 1) * m / 2 > e) --m;
      while (m * (m + 1) / 2 <= e) ++m;
      const int r = j + m, c = j + 1 + (e - (m - 1) * m / 2);
      const CT xr = sCol[mi * NPAD + r], y = sCol[mi * NPAD + c];
      CT a = sA[mi * NTRI + tri_index(r, c)];
      a.x = fma(-xr.x, y.x, a.x); a.x = fma(-xr.y, y.y, a.x);
      a.y = fma(-xr.y, y.x, a.y); a.y = fma(xr.x, y.y, a.y);
      if (e == 0) {
        R d2 = a.x;
        if (!(d2 > (R)0)) { atomicOr(status, 1); d2 = (R)1; }
        const R inv = rsqrt(d2);
        a = mkc<CT>(d2 * inv, (R)0);
        sInv[mi * NPAD + j + 1] = inv;
      }
      sA[mi * NTRI + tri_index(r, c)] = a;
    }
    __syncthreads();
  }

  // ---- store: off-diagonal blocks as they are, diagonal blocks inverted
#pragma unroll
  for (int mi = 0; mi < MPC; ++mi) {
    if (bsv[mi] >= L.nsub) continue;
    CT* F = factors + (size_t)bsv[mi] * L.fsize;
    const CT* A = sA + mi * NTRI;
#pragma unroll
    for (int I = 1; I < NB; ++I)
#pragma unroll
      for (int J = 0; J < I; ++J)
        F[(size_t)(I * (I + 1) / 2 + J) * 256 + ti * LA_BLK + tk] = A[tri_index(LA_BLK * I + ti, LA_BLK * J + tk)];
  }
  // inv(L_II): thread (matrix, I, column jj) solves L_II x = e_jj by forward substitution
  if (tid < MPC * NB * LA_BLK) {
    const int mi = tid / (NB * LA_BLK), rem = tid - mi * NB * LA_BLK;
    const int I = rem / LA_BLK, jj = rem % LA_BLK, base = LA_BLK * I;
    int bm = 0;
#pragma unroll
    for (int u = 0; u < MPC; ++u) if (u == mi) bm = bsv[u];
    if (bm < L.nsub) {
      const CT* A = sA + mi * NTRI;
      const R* Inv = sInv + mi * NPAD;
      CT x[LA_BLK];
#pragma unroll
      for (int i = 0; i < LA_BLK; ++i) {
        CT acc = mkc<CT>(0, 0);
#pragma unroll
        for (int k = 0; k < i; ++k)
          if (k >= jj) cfma(acc, A[tri_index(base + i, base + k)], x[k]);
        const R rinv = Inv[base + i];
        if (i < jj) x[i] = mkc<CT>(0, 0);
        else if (i == jj) x[i] = mkc<CT>(rinv, (R)0);
        else x[i] = mkc<CT>(-acc.x * rinv, -acc.y * rinv);
      }
      CT* D = factors + (size_t)bm * L.fsize + (size_t)(I * (I + 1) / 2 + I) * 256;
#pragma unroll
      for (int i = 0; i < LA_BLK; ++i) D[i * LA_BLK + jj] = x[i];
    }
  }
}

// ------------------------------------------------------------------------ complex64 variant
// For complex64 the whole factor fits in registers: thread (ti, tk) keeps its tile-cyclic entries
// (16 I + ti, 16 J + tk), J <= I, in registers with compile-time tile indices.  Blocked
// right-looking Cholesky: the 16 columns of a panel are eliminated one by one inside the panel's
// block column only (two barriers per column, pivot lookahead), the finished panel goes to shared
// memory k-major, and every trailing block then takes one rank-16 update from it (row reads are
// broadcasts, column reads are consecutive), so the per-entry bookkeeping is paid once per 16
// columns instead of once per column.
// Matrices per CTA of the blocked factorisation: small ones share the column barriers (their
// per-thread register tiles stay small: NT = 3 complex for NPAD 32, 6 for NPAD 48).
__host__ __device__ constexpr int factor_c64_mpc(int npad) { return npad <= 32 ? 4 : (npad <= 48 ? 2 : 1); }

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// The blocked factorisation, written for a precision R; the mixed path runs it in complex64 (two
// CTAs per SM).  In complex128 its register tiles allow one CTA per SM, and measured slower than the
// shared-memory factorisation above (NPAD 96 at 256 x 256: 9.4 ms against 5.7 ms), so the FP64
// path does not use it.
template <typename R, int NPAD, int MPC>
__global__ void __launch_bounds__(kFactorThreads, sizeof(R) == 4 ? (NPAD <= 96 ? 3 : 2) : 1)
k_factor_blk(LevelGeom L, FineOp g, int is_fine, int nptsmax, const R* __restrict__ sigma,
             const TimeMats* __restrict__ tm, typename C2<R>::T* __restrict__ factors, int* __restrict__ status) {
  typedef typename C2<R>::T CT;
  constexpr int NB = NPAD / LA_BLK;
  constexpr int NT = NB * (NB + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = tm->K, KK = K * K;
  const int nv = is_fine ? 2 : LA_NPAIR;
  const int pstride = nptsmax * nptsmax * nv;
  CT* sPan = reinterpret_cast<CT*>(smem);                          // [MPC][LA_BLK][NPAD] finished panel, k-major
  R* sInv = reinterpret_cast<R*>(sPan + MPC * LA_BLK * NPAD);     // [MPC][NPAD]
  CT* sDiag = reinterpret_cast<CT*>(sInv + MPC * NPAD);             // [MPC][NB][256]
  R* sP = reinterpret_cast<R*>(sDiag + MPC * NB * 256);             // [9][K*K]
  R* sPair = sP + LA_NPAIR * LA_KMAX * LA_KMAX;                     // [MPC][npts*npts][nv]
  R* sX = sPair + (size_t)MPC * pstride;                            // [MPC][npts] laser coordinate (finest)

  const int tid = threadIdx.x, ti = tid >> 4, tk = tid & 15;
  // the CTA's matrices; slots past the last subvolume factorise an identity and store nothing
  int bsv[MPC], npts_[MPC], o_[MPC][3], e_[MPC][3];
#pragma unroll
  for (int mi = 0; mi < MPC; ++mi) {
    bsv[mi] = blockIdx.x * MPC + mi;
    if (bsv[mi] < L.nsub) {
      subvol_box(L, bsv[mi], o_[mi], e_[mi]);
      npts_[mi] = e_[mi][0] * e_[mi][1] * e_[mi][2];
    } else {
      o_[mi][0] = o_[mi][1] = o_[mi][2] = 0;
      e_[mi][0] = e_[mi][1] = e_[mi][2] = 1;
      npts_[mi] = 0;
    }
  }
  for (int i = tid; i < LA_NPAIR * KK; i += kFactorThreads) sP[i] = (R)tm->P[i / KK][i % KK];
  for (int i = tid; i < MPC * NB * 256; i += kFactorThreads) sDiag[i] = mkc<CT>(0, 0);
  const int nbox = box5_count(L.dim);
#pragma unroll
  for (int mi = 0; mi < MPC; ++mi) {
    const int npts = npts_[mi];
    const int* o = o_[mi];
    const int* e = e_[mi];
    if (is_fine)
      for (int i = tid; i < npts; i += kFactorThreads) {
        int ix, iy, iz;
        local_coords(i, e, ix, iy, iz);
        sX[mi * nptsmax + i] = (R)fine_x(g, o[0] + ix, o[1] + iy, o[2] + iz);
      }
    for (int t = tid; t < npts * npts; t += kFactorThreads) {
      const int i = t / npts, j = t % npts;
      int ix, iy, iz, jx, jy, jz;
      local_coords(i, e, ix, iy, iz);
      local_coords(j, e, jx, jy, jz);
      const int px = o[0] + ix, py = o[1] + iy, pz = o[2] + iz;
      const int qx = o[0] + jx, qy = o[1] + jy, qz = o[2] + jz;
      R* dst = sPair + (size_t)mi * pstride + (size_t)t * nv;
      if (is_fine) {
        double s9[LA_NPAIR];
        fine_sigma(g, px, py, pz, qx, qy, qz, s9);
        dst[0] = (R)s9[1];
        dst[1] = (R)s9[4];
      } else {
        const int dx = qx - px, dy = qy - py, dz = qz - pz;
        const bool near = abs(dx) <= 2 && abs(dy) <= 2 && abs(dz) <= 2;
        const int p = (pz * L.n[1] + py) * L.n[0] + px;
        const int ofs = near ? box5_index(L.dim, dx, dy, dz) : 0;
        for (int k = 0; k < LA_NPAIR; ++k) dst[k] = near ? (R)sigma[sigma_offset(p, k, ofs, nbox)] : (R)0;
      }
    }
  }
  __syncthreads();

  CT a[MPC][NT];
#pragma unroll
  for (int mi = 0; mi < MPC; ++mi) {
    const int npts = npts_[mi], n = npts * K;
#pragma unroll
    for (int I = 0; I < NB; ++I) {
#pragma unroll
      for (int J = 0; J <= I; ++J) {
        const int r = LA_BLK * I + ti, c = LA_BLK * J + tk;
        // assembled in R (complex64: this factor only preconditions the FP64-refined iteration)
        R re = 0, im = 0;
        if (I == J && ti < tk) {
        } else if (r >= n || c >= n) {
          re = (r == c) ? (R)1 : (R)0;
        } else {
          const int i = r / K, mm = r % K, j = c / K, nn = c % K;
          R s9[LA_NPAIR];
          const R* pr = sPair + (size_t)mi * pstride + (size_t)(i * npts + j) * nv;
          if (is_fine) {
            const R xp = sX[mi * nptsmax + i], xq = sX[mi * nptsmax + j];
            const R same = (i == j) ? (R)1 : (R)0, Hpq = pr[0];
            s9[0] = same; s9[1] = Hpq; s9[2] = same * xp; s9[3] = Hpq; s9[4] = pr[1];
            s9[5] = Hpq * xq; s9[6] = same * xp; s9[7] = xp * Hpq; s9[8] = same * xp * xp;
          } else {
#pragma unroll
            for (int kk = 0; kk < LA_NPAIR; ++kk) s9[kk] = pr[kk];
          }
#pragma unroll
          for (int kk = 0; kk < LA_NPAIR; ++kk) {
            const R v = s9[kk] * sP[kk * KK + mm * K + nn];
            const int ph = theta_phase(kk);
            if (ph == 0) re += v; else if (ph == 1) im += v; else im -= v;
          }
        }
        a[mi][I * (I + 1) / 2 + J] = mkc<CT>(re, im);
      }
    }
  }
  if (tid == 0) {
#pragma unroll
    for (int mi = 0; mi < MPC; ++mi) {
      R d2 = a[mi][0].x;
      if (!(d2 > (R)0)) { atomicOr(status, 1); d2 = (R)1; }
      const R inv = rsq(d2);
      a[mi][0] = mkc<CT>(d2 * inv, 0);
      sInv[mi * NPAD] = inv;
    }
  }
  __syncthreads();

#pragma unroll
  for (int J0 = 0; J0 < NB; ++J0) {
    const int c0 = LA_BLK * J0 + tk;   // this thread's column inside the panel
    for (int jj = 0; jj < LA_BLK; ++jj) {
      const int j = LA_BLK * J0 + jj;
      // (A) owners of column j scale it and publish it
      if (tk == jj) {
#pragma unroll
        for (int mi = 0; mi < MPC; ++mi) {
          const R inv = sInv[mi * NPAD + j];
          CT* pan = sPan + (size_t)mi * LA_BLK * NPAD;
#pragma unroll
          for (int I = J0; I < NB; ++I) {
            const int r = LA_BLK * I + ti;
            if (r > j) {
              CT& v = a[mi][I * (I + 1) / 2 + J0];
              v.x *= inv;
              v.y *= inv;
              pan[jj * NPAD + r] = v;
            }
          }
        }
      }
      __syncthreads();
      if (jj == LA_BLK - 1) break;   // the panel's last column changes nothing inside the panel
      // (B) rank-1 update of the panel right of column j; the owner of entry (j+1, j+1) takes its rsqrt
      if (c0 > j) {
#pragma unroll
        for (int mi = 0; mi < MPC; ++mi) {
          const CT* pan = sPan + (size_t)mi * LA_BLK * NPAD;
          const CT y = pan[jj * NPAD + c0];
#pragma unroll
          for (int I = J0; I < NB; ++I) {
            const int r = LA_BLK * I + ti;
            if (r >= c0) {
              const CT xr = pan[jj * NPAD + r];
              CT& v = a[mi][I * (I + 1) / 2 + J0];
              v.x = fma(-xr.x, y.x, v.x); v.x = fma(-xr.y, y.y, v.x);
              v.y = fma(-xr.y, y.x, v.y); v.y = fma(xr.x, y.y, v.y);
            }
          }
          if (ti == jj + 1 && tk == jj + 1) {
            CT& v = a[mi][J0 * (J0 + 1) / 2 + J0];
            R d2 = v.x;
            if (!(d2 > (R)0)) { atomicOr(status, 1); d2 = (R)1; }
            const R inv = rsq(d2);
            v = mkc<CT>(d2 * inv, 0);
            sInv[mi * NPAD + j + 1] = inv;
          }
        }
      }
      __syncthreads();
    }
    if (J0 + 1 < NB) {
      // rank-16 update of the trailing blocks (I, J), J0 < J <= I (upper halves of diagonal blocks
      // are updated too and never read)
#pragma unroll
      for (int mi = 0; mi < MPC; ++mi) {
        const CT* pan = sPan + (size_t)mi * LA_BLK * NPAD;
        for (int k = 0; k < LA_BLK; ++k) {
          CT xr[NB], yc[NB];
#pragma unroll
          for (int I = J0 + 1; I < NB; ++I) {
            xr[I] = pan[k * NPAD + LA_BLK * I + ti];
            yc[I] = pan[k * NPAD + LA_BLK * I + tk];
          }
#pragma unroll
          for (int I = J0 + 1; I < NB; ++I)
#pragma unroll
            for (int J = J0 + 1; J <= I; ++J) {
              CT& v = a[mi][I * (I + 1) / 2 + J];
              v.x = fma(-xr[I].x, yc[J].x, v.x); v.x = fma(-xr[I].y, yc[J].y, v.x);
              v.y = fma(-xr[I].y, yc[J].x, v.y); v.y = fma(xr[I].x, yc[J].y, v.y);
            }
        }
      }
      if (tid == 0) {   // first pivot of the next panel
#pragma unroll
        for (int mi = 0; mi < MPC; ++mi) {
          CT& v = a[mi][(J0 + 1) * (J0 + 2) / 2 + J0 + 1];
          R d2 = v.x;
          if (!(d2 > (R)0)) { atomicOr(status, 1); d2 = (R)1; }
          const R inv = rsq(d2);
          v = mkc<CT>(d2 * inv, 0);
          sInv[mi * NPAD + LA_BLK * (J0 + 1)] = inv;
        }
      }
      __syncthreads();
    }
  }

#pragma unroll
  for (int mi = 0; mi < MPC; ++mi) {
    CT* F = factors + (size_t)bsv[mi] * L.fsize;
    const bool store = bsv[mi] < L.nsub;
#pragma unroll
    for (int I = 0; I < NB; ++I)
#pragma unroll
      for (int J = 0; J <= I; ++J) {
        if (I == J) {
          if (ti >= tk) sDiag[(mi * NB + I) * 256 + ti * LA_BLK + tk] = a[mi][I * (I + 1) / 2 + J];
        } else if (store) {
          F[(size_t)(I * (I + 1) / 2 + J) * 256 + ti * LA_BLK + tk] = a[mi][I * (I + 1) / 2 + J];
        }
      }
  }
  __syncthreads();
  if (tid < MPC * NB * LA_BLK) {
    const int mi = tid / (NB * LA_BLK), rem = tid - mi * NB * LA_BLK;
    const int I = rem / LA_BLK, jj = rem % LA_BLK, base = LA_BLK * I;
    int bm = 0;
#pragma unroll
    for (int u = 0; u < MPC; ++u) if (u == mi) bm = bsv[u];
    if (bm < L.nsub) {
      const CT* Ld = sDiag + (mi * NB + I) * 256;
      const R* Inv = sInv + mi * NPAD;
      CT x[LA_BLK];
#pragma unroll
      for (int i = 0; i < LA_BLK; ++i) {
        CT acc = mkc<CT>(0, 0);
#pragma unroll
        for (int k = 0; k < i; ++k)
          if (k >= jj) cfma(acc, Ld[i * LA_BLK + k], x[k]);
        const R rinv = Inv[base + i];
        if (i < jj) x[i] = mkc<CT>(0, 0);
        else if (i == jj) x[i] = mkc<CT>(rinv, 0);
        else x[i] = mkc<CT>(-acc.x * rinv, -acc.y * rinv);
      }
      CT* D = factors + (size_t)bm * L.fsize + (size_t)(I * (I + 1) / 2 + I) * 256;
#pragma unroll
      for (int i = 0; i < LA_BLK; ++i) D[i * LA_BLK + jj] = x[i];
    }
  }
}

// ======================================================================== wide subvolumes
// Finest-level subvolumes of up to 256 unknowns (4 x 4 x 4 points x K = 4 in 3D, 8 x 8 x 4 in 2D).
// Their factor (136 blocks: 557 KB complex128, 279 KB complex64) fits in no CTA's shared memory, so
// one 256-thread CTA per subvolume factorises left-looking by 16-column block columns directly in
// the factor store: block column J is assembled in registers, updated with the finished block
// columns 0..J-1 read back from global memory (recently written by the same CTA, so mostly L2
// hits), its diagonal block is factorised in shared memory, the blocks below it are divided by it,
// and the column is stored.  Entries of G_UU come from closed forms of H and H^2 on the grid, built
// once per subvolume into a shared-memory table of (H, H^2) over its point pairs.
constexpr int kWidePtsMax = 64;   // grid points of a wide subvolume
// row stride of the (H, H^2) pair table: odd, so that the rows of one column a warp reads spread over
// the banks
constexpr int kHHStride = kWidePtsMax + 1;

// Two consecutive complex entries (16-byte aligned), as one vector load where the type allows.
template <typename CT> struct CPair;
template <> struct CPair<float2> {
  float4 v;
  __device__ __forceinline__ void load(const float2* p) { v = __ldg(reinterpret_cast<const float4*>(p)); }
  __device__ __forceinline__ void load_zero() { v = make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ float2 a() const { return make_float2(v.x, v.y); }
  __device__ __forceinline__ float2 b() const { return make_float2(v.z, v.w); }
};
template <> struct CPair<double2> {
  double2 a_, b_;
  __device__ __forceinline__ void load(const double2* p) { a_ = __ldg(p); b_ = __ldg(p + 1); }
  __device__ __forceinline__ void load_zero() { a_ = make_double2(0.0, 0.0); b_ = a_; }
  __device__ __forceinline__ double2 a() const { return a_; }
  __device__ __forceinline__ double2 b() const { return b_; }
};
// the same pair from shared memory
__device__ __forceinline__ CPair<float2> lds_pair(const float2* p) {
  CPair<float2> r;
  r.v = *reinterpret_cast<const float4*>(p);
  return r;
}
__device__ __forceinline__ CPair<double2> lds_pair(const double2* p) {
  CPair<double2> r;
  r.a_ = p[0];
  r.b_ = p[1];
  return r;
}

// L2 eviction-priority policies and the loads that carry them.  The sweep reads each factor block
// twice, forward then backward; a launch's forward-read blocks outgrow L2 before the backward pass
// reaches them unless the single-use streams (the backward reads themselves, c and f) give way first.
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ldg_policy(const float4* p, unsigned long long pol) {
  float4 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float2 ldg_policy(const float2* p, unsigned long long pol) {
  float2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
// coherent loads (the array is written by the same launch elsewhere) with a policy
__device__ __forceinline__ float2 ld_policy(const float2* p, unsigned long long pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_policy(const double2* p, unsigned long long pol) {
  double2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}

// Asynchronous copy (cp.async) of one complex element global -> shared; cp_async_wait_all waits for the
// calling thread's copies.
__device__ __forceinline__ void cp_async_elem(float2* sdst, const float2* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* sdst, const double2* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// the same with zero fill (nothing read) where valid is false
__device__ __forceinline__ void cp_async_elem_zf(float2* sdst, const float2* gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
               "l"(gsrc), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_elem_zf(double2* sdst, const double2* gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
               "l"(gsrc), "r"(valid ? 16 : 0)
               : "memory");
}
// one real value
__device__ __forceinline__ void cp_async_real(float* sdst, const float* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_real(double* sdst, const double* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)), "l"(gsrc)
               : "memory");
}

// Shared-memory layout of the wide factorisation (bytes), for the padded size npad.
// Rows of the two shared-memory panels are padded so that the transposed stores of the block row and the
// column-wise accesses of the diagonal block spread over the banks: 17 entries for the block column,
// 18 for the block row (whose rows the update reads as 16-byte pairs, so they start 16-byte aligned).
constexpr int kWideStride = LA_BLK + 1;
constexpr int kRowStride = LA_BLK + 2;
__host__ __device__ constexpr size_t wide_factor_smem(int npad, size_t csize, size_t rsize) {
  return csize * ((size_t)(npad - LA_BLK) * kRowStride     // block row J+1, transposed (then the block (J+1, J))
                  + (size_t)npad * kWideStride             // the block column's rows at their absolute index
                  + 256)                                   // inv(L_JJ)^dagger, [k][c]
         + rsize * (LA_NPAIR * LA_KMAX * LA_KMAX + 3 * kWidePtsMax + LA_BLK) + sizeof(int) * kWidePtsMax
         + csize * (size_t)kWidePtsMax * kHHStride      // (H, H^2) of every point pair
         + rsize * 2 * LA_KMAX * LA_KMAX;               // P_HI - P_IH and P_XI - P_IX
}

// H_pq and (H^2)_pq of the finest-level operator H = -1/2 Laplacian + V0 for grid points p, q of one
// subvolume: D = dsum + V0 on the diagonal, -w_a = -1/(2 h_a^2) between neighbours along axis a,
// and H^2 by the paths of length two inside the grid (Dirichlet walls: the diagonal of H^2 counts
// only in-grid neighbours, nb2 = sum_a w_a^2 over them).
template <typename R>
__device__ __forceinline__ void wide_h_h2(int dx, int dy, int dz, R Dp, R Dq, R nb2p, R wx, R wy, R wz, R& H,
                                          R& H2) {
  const int ax = abs(dx), ay = abs(dy), az = abs(dz), a1 = ax + ay + az;
  H = 0;
  H2 = 0;
  if (a1 == 0) {
    H = Dp;
    H2 = Dp * Dp + nb2p;
  } else if (a1 == 1) {
    const R w = ax ? wx : (ay ? wy : wz);
    H = -w;
    H2 = -w * (Dp + Dq);
  } else if (a1 == 2) {
    if (ax == 2) H2 = wx * wx;
    else if (ay == 2) H2 = wy * wy;
    else if (az == 2) H2 = wz * wz;
    else H2 = 2 * (ax ? wx : wy) * (az ? wz : wy);
  }
}

// Shared-memory tables of the wide assembly: sHH[i * kHHStride + j] = (H_ij, (H^2)_ij) for the
// subvolume's points, sP the nine K x K products P_kk' = R_k^T Wt R_k' (Theta = phase x P) in the pair
// order (0,0) (0,1) (0,2) (1,0) (1,1) (1,2) (2,0) (2,1) (2,2) of (I, H, X), sPd = (P_01 - P_10, P_02 - P_20)
// (phases: (0,1), (0,2) +i; (1,0), (2,0) -i; the others real), sX the laser coordinate of each point.
template <typename R>
struct WideTables {
  typedef typename C2<R>::T CT;
  const CT* sHH;
  const R *sP, *sPd, *sX;
};
// The point and time function of one row of G_UU, decoded once per row.
template <typename R>
struct WideRow {
  int r, i, m;
  R xp;
};
template <typename R>
__device__ __forceinline__ WideRow<R> wide_row(int r, const FastDiv& dK, int K, const R* sX) {
  WideRow<R> w;
  w.r = r;
  w.i = fdiv(r, dK);
  w.m = r - w.i * K;
  w.xp = sX[w.i < kWidePtsMax ? w.i : 0];
  return w;
}

// Assembles G_UU[r, c] (r, c < npad; identity outside the n true unknowns).
template <typename R>
__device__ __forceinline__ typename C2<R>::T wide_entry(const WideRow<R>& w, int c, int n, const FastDiv& dK, int K,
                                                     const WideTables<R>& T) {
  typedef typename C2<R>::T CT;
  if (w.r >= n || c >= n) return mkc<CT>((R)(w.r == c ? 1 : 0), (R)0);
  const int j = fdiv(c, dK), nn = c - j * K;
  const CT hh = T.sHH[w.i * kHHStride + j];
  const R H = hh.x, H2 = hh.y;
  const int KK = K * K, mn = w.m * K + nn;
  const R xp = w.xp, xq = T.sX[j];
  R re = H2 * T.sP[4 * KK + mn] + H * (xq * T.sP[5 * KK + mn] + xp * T.sP[7 * KK + mn]);
  R im = H * T.sPd[mn];
  if (w.i == j) {
    re += T.sP[mn] + xp * xp * T.sP[8 * KK + mn];
    im += xp * T.sPd[KK + mn];
  }
  return mkc<CT>(re, im);
}

// Row r of block column Jc, columns c0 .. c0 + CPT - 1, assembled: acc[c] = G[r][16 Jc + c0 + c]
// (zero for a block beyond the band).  wide_partial_update then subtracts the finished block columns.
template <typename R, int CPT>
__device__ __forceinline__ void wide_assemble(int Jc, int band, int r, int c0, int n, const FastDiv& dK, int K,
                                              const WideTables<R>& T, typename C2<R>::T* acc) {
  typedef typename C2<R>::T CT;
  if ((r >> 4) - Jc > band) {
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[q] = mkc<CT>(0, 0);
    return;
  }
  const WideRow<R> w = wide_row<R>(r, dK, K, T.sX);
#pragma unroll
  for (int q = 0; q < CPT; ++q) acc[q] = wide_entry<R>(w, LA_BLK * Jc + c0 + q, n, dK, K, T);
}

// acc[c] -= sum_{k < 16 kb_end} L[r][k] conj(L[16 Jc + c0 + c][k]) over the finished block columns inside
// the band: row r's blocks read back from the factor store, block row Jc transposed in sRow.
template <typename R, int CPT>
__device__ __forceinline__ void wide_partial_update(int Jc, int kb_end, int band, int r, int c0,
                                                    const typename C2<R>::T* __restrict__ F,
                                                    const typename C2<R>::T* sRow, typename C2<R>::T* acc) {
  typedef typename C2<R>::T CT;
  const int I = r >> 4;
  if (I - Jc > band) return;   // a block beyond the band: zero, nothing to update
  // the blocks (I, Kb) with I - Kb > band are zero: the sum starts at Kb = I - band
  const int kb_begin = I - band > 0 ? I - band : 0;
  for (int h = 2 * kb_begin; h < 2 * kb_end; ++h) {   // half a finished block row (8 columns k) at a time
    const int Kb = h >> 1, k0 = (h & 1) * (LA_BLK / 2);
    const CT* src = F + (size_t)tri_index(I, Kb) * 256 + (r & 15) * LA_BLK + k0;
    CT v[LA_BLK / 2];
#pragma unroll
    for (int kk = 0; kk < LA_BLK / 2; ++kk) v[kk] = src[kk];
    const CT* rowk = sRow + ((size_t)Kb * LA_BLK + k0) * kRowStride + c0;
#pragma unroll
    for (int kk = 0; kk < LA_BLK / 2; ++kk) {
#pragma unroll
      for (int q = 0; q < CPT; q += (CPT > 1 ? 2 : 1)) {
        CT y[2];
        if (CPT > 1) {
          const CPair<CT> yp = lds_pair(rowk + kk * kRowStride + q);
          y[0] = yp.a();
          y[1] = yp.b();
        } else {
          y[0] = rowk[kk * kRowStride + q];
        }
#pragma unroll
        for (int u = 0; u < (CPT > 1 ? 2 : 1); ++u) {
          // acc -= v conj(y)
          acc[q + u].x = fma(-v[kk].x, y[u].x, acc[q + u].x); acc[q + u].x = fma(-v[kk].y, y[u].y, acc[q + u].x);
          acc[q + u].y = fma(-v[kk].y, y[u].x, acc[q + u].y); acc[q + u].y = fma(v[kk].x, y[u].y, acc[q + u].y);
        }
      }
    }
  }
}

// Shared state of the wide factorisation.
template <typename R>
struct WideSmem {
  typedef typename C2<R>::T CT;
  CT* sRow;   // [NPAD-16][18]: block row J' transposed, sRow[k][c] = L[16 J' + c][k]
  CT* sPan;   // [NPAD][17]: rows of the current block column at their absolute row index
  CT* sBT;    // [16][17]: sBT[k][c] = L[16 (J+1) + c][16 J + k] (the block (J+1, J)); in sRow's space
  CT* sInvT;  // [16][16]: sInvT[k][c] = conj(inv(L_JJ)[c][k])
  CT* sHH;    // [64][65]: (H, H^2) of the point pairs
  R *sP, *sPd, *sD, *sX, *sN, *sPiv;
  int* sXYZ;
  __device__ WideTables<R> tables() const { return WideTables<R>{sHH, sP, sPd, sX}; }
};

// Cholesky of the diagonal block of column J (rows 16 J .. 16 J + 15 of sPan) and its inverse in one
// sweep of 16 steps, by one warp.  Lane (i, h) = (lane % 16, lane / 16) updates row i's trailing entries of
// one column parity h and keeps the entries of parity h of row i of X = inv(L_JJ) in registers: X starts
// as the identity, and step j divides row j by L[j][j] and subtracts L[i][j] times it from the rows i > j
// (row j of X is final after step j), so the inverse costs no second chain of dependent steps.
template <typename R>
__device__ __forceinline__ void wide_diag(int J, const WideSmem<R>& S, typename C2<R>::T* F, int* status) {
  typedef typename C2<R>::T CT;
  const int lane = threadIdx.x & 31, ri = lane & 15, half = lane >> 4;
  CT* D = S.sPan + (size_t)LA_BLK * J * kWideStride;   // the diagonal block's rows
  CT x[LA_BLK / 2];                                     // X[ri][2 u + half]
#pragma unroll
  for (int u = 0; u < LA_BLK / 2; ++u) x[u] = mkc<CT>((R)(2 * u + half == ri ? 1 : 0), (R)0);
  for (int j = 0; j < LA_BLK; ++j) {
    R d2 = D[j * kWideStride + j].x;
    if (!(d2 > (R)0)) {
      if (lane == 0) atomicOr(status, 1);
      d2 = (R)1;
    }
    const R inv = rsq(d2);
    CT lij = mkc<CT>(0, 0);
    if (ri > j) {
      const CT v = D[ri * kWideStride + j];
      lij = mkc<CT>(v.x * inv, v.y * inv);
    }
    __syncwarp();
    if (ri > j && half == 0) D[ri * kWideStride + j] = lij;
    if (lane == j) D[j * kWideStride + j] = mkc<CT>(d2 * inv, (R)0);
    // X: row j /= L[j][j] (its lanes), then rows i > j -= L[i][j] X[j]; X[j][c] comes from lane (j, h)
#pragma unroll
    for (int u = 0; u < LA_BLK / 2; ++u) {
      if (ri == j) x[u] = mkc<CT>(x[u].x * inv, x[u].y * inv);
      CT xj;
      xj.x = __shfl_sync(0xffffffffu, x[u].x, j + 16 * half);
      xj.y = __shfl_sync(0xffffffffu, x[u].y, j + 16 * half);
      if (ri > j) {   // x -= L[i][j] X[j]
        x[u].x -= lij.x * xj.x - lij.y * xj.y;
        x[u].y -= lij.x * xj.y + lij.y * xj.x;
      }
    }
    __syncwarp();
    // trailing entries (i, k), j < k <= i: A[i][k] -= L[i][j] conj(L[k][j])
    if (ri > j) {
      for (int k = j + 1 + half; k <= ri; k += 2) {
        const CT lk = D[k * kWideStride + j];
        CT v = D[ri * kWideStride + k];
        v.x -= lij.x * lk.x + lij.y * lk.y;
        v.y -= lij.y * lk.x - lij.x * lk.y;
        D[ri * kWideStride + k] = v;
      }
    }
    __syncwarp();
  }
  // the inverse as the stored diagonal block (row ri, columns 2 u + half), and sInvT[k][c] = conj(X[c][k])
#pragma unroll
  for (int u = 0; u < LA_BLK / 2; ++u) {
    const int c = 2 * u + half;
    if (lane < 32) {
      F[(size_t)tri_index(J, J) * 256 + ri * LA_BLK + c] = x[u];
      S.sInvT[c * LA_BLK + ri] = mkc<CT>(x[u].x, -x[u].y);
    }
  }
}

// Named barrier of warps 1..7 (the lookahead update's threads).
__device__ __forceinline__ void wide_bar() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

// One block column J with lookahead: warp 0 factorises J's diagonal block while warps 1..7 assemble block
// column J+1 and update it with the finished block columns 0..J-1; then all threads divide J's rows below
// by L_JJ, and warps 1..7 add block column J's contribution to J+1 from shared memory.
template <typename R, int NPAD, int CPT>
__device__ __forceinline__ void wide_column_step(int J, int band, int n, const FastDiv& dK, int K,
                                                 typename C2<R>::T* F, const WideSmem<R>& S, int* status) {
  typedef typename C2<R>::T CT;
  constexpr int NB = NPAD / LA_BLK;
  constexpr int TPR = LA_BLK / CPT;
  const int tid = threadIdx.x;
  const bool next = J + 1 < NB;
  const int RJ1 = NPAD - LA_BLK * (J + 1);            // rows of block column J+1
  // warps 1..7 own rows q' = t' / TPR of block column J+1 (t' = tid - 32); rows beyond 224 / TPR
  // (block column 1 of a 256-unknown matrix has 240) fall to warp 0 after its diagonal work
  const int tl = tid - 32;
  const int q_own = tid >= 32 ? tl / TPR : 224 / TPR + (tid & 31);
  const int c0 = tid >= 32 ? (tl % TPR) * CPT : 0;
  const bool own = next && q_own < RJ1 && (tid >= 32 || (TPR == 1 && (tid & 31) < LA_BLK));
  const int r_own = LA_BLK * (J + 1) + q_own;
  CT acc[CPT];
  if (tid < 32) {
    wide_diag<R>(J, S, F, status);
  } else if (next) {
    // block row J+1's finished blocks (J+1, Kb < J) inside the band, transposed, every copy in flight at once
    const int kb0 = J + 1 - band > 0 ? J + 1 - band : 0;
    for (int t = kb0 * 256 + tl; t < J * 256; t += 224) {
      const int Kb = t >> 8, w = t & 255, c = w >> 4, kk = w & 15;
      cp_async_elem(S.sRow + (Kb * LA_BLK + kk) * kRowStride + c, F + (size_t)tri_index(J + 1, Kb) * 256 + w);
    }
    // the entries of G are assembled while the copies are in flight
    if (own) wide_assemble<R, CPT>(J + 1, band, r_own, c0, n, dK, K, S.tables(), acc);
    cp_async_wait_all();
    wide_bar();
    if (own) wide_partial_update<R, CPT>(J + 1, J, band, r_own, c0, F, S.sRow, acc);
  }
  __syncthreads();
  if (tid < 32 && own)   // warp 0's rows of block column 1 (no finished column before it)
    wide_assemble<R, CPT>(J + 1, band, r_own, c0, n, dK, K, S.tables(), acc);
  // rows below the diagonal block, one row per thread: L[r][c] = sum_{k <= c} A[r][k] conj(inv(L_JJ)[c][k])
  // (the row's entries in registers, sInvT's rows read as 16-byte pairs), written to the factor store and
  // back to the row in place; the rows of the block (J+1, J) also go to sBT for the update below
  // (rows beyond the band hold exact zeros, which stay zeros)
  for (int q = tid; q < RJ1 && q < LA_BLK * band; q += kFactorThreads) {
    const int rr = LA_BLK * (J + 1) + q;
    CT* row = S.sPan + (size_t)rr * kWideStride;
    CT a[LA_BLK], l[LA_BLK];
#pragma unroll
    for (int k = 0; k < LA_BLK; ++k) {
      a[k] = row[k];
      l[k] = mkc<CT>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < LA_BLK; ++k) {
#pragma unroll
      for (int c = k - (k & 1); c < LA_BLK; c += 2) {   // inv is lower triangular: only c >= k contribute
        const CPair<CT> ip = lds_pair(S.sInvT + k * LA_BLK + c);
        cfma(l[c], a[k], ip.a());
        cfma(l[c + 1], a[k], ip.b());
      }
    }
#pragma unroll
    for (int c = 0; c < LA_BLK; ++c) row[c] = l[c];
    if ((rr >> 4) == J + 1) {
#pragma unroll
      for (int c = 0; c < LA_BLK; ++c) S.sBT[c * kWideStride + (rr & 15)] = l[c];
    }
  }
  __syncthreads();
  // the divided rows to the factor store, consecutive threads on consecutive entries
  for (int e = tid; e < RJ1 * LA_BLK; e += kFactorThreads) {
    const int rr = LA_BLK * (J + 1) + (e >> 4), c = e & 15;
    F[(size_t)tri_index(rr >> 4, J) * 256 + (rr & 15) * LA_BLK + c] = S.sPan[(size_t)rr * kWideStride + c];
  }
  __syncthreads();   // the rows are overwritten below with block column J+1
  if (own && (r_own >> 4) - J <= band) {
    // block column J's contribution: acc[c] -= sum_k L[r][16 J + k] conj(L[16 (J+1) + c][16 J + k])
    // (zero for rows whose block (I, J) is beyond the band)
    const CT* a = S.sPan + (size_t)r_own * kWideStride;
#pragma unroll
    for (int k = 0; k < LA_BLK; ++k) {
      const CT lr = a[k];
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        const CT y = S.sBT[k * kWideStride + c0 + q];
        acc[q].x = fma(-lr.x, y.x, acc[q].x); acc[q].x = fma(-lr.y, y.y, acc[q].x);
        acc[q].y = fma(-lr.y, y.x, acc[q].y); acc[q].y = fma(lr.x, y.y, acc[q].y);
      }
    }
  }
  __syncwarp();
  if (own) {
#pragma unroll
    for (int q = 0; q < CPT; ++q) S.sPan[(size_t)r_own * kWideStride + c0 + q] = acc[q];
  }
  __syncthreads();
}

template <typename R, int NPAD>
__global__ void __launch_bounds__(kFactorThreads, sizeof(R) == 4 ? 2 : 1)
k_factor_wide(LevelGeom L, FineOp g, const TimeMats* __restrict__ tm, typename C2<R>::T* __restrict__ factors,
              int* __restrict__ status) {
  typedef typename C2<R>::T CT;
  constexpr int NB = NPAD / LA_BLK;
  extern __shared__ __align__(16) unsigned char smem[];
  WideSmem<R> S;
  S.sRow = reinterpret_cast<CT*>(smem);
  S.sBT = S.sRow;   // written after the lookahead update has read sRow, read before sRow is refilled
  S.sPan = S.sRow + (size_t)(NPAD - LA_BLK) * kRowStride;
  S.sInvT = S.sPan + (size_t)NPAD * kWideStride;
  S.sP = reinterpret_cast<R*>(S.sInvT + 256);
  S.sD = S.sP + LA_NPAIR * LA_KMAX * LA_KMAX;
  S.sX = S.sD + kWidePtsMax;
  S.sN = S.sX + kWidePtsMax;
  S.sPiv = S.sN + kWidePtsMax;
  S.sXYZ = reinterpret_cast<int*>(S.sPiv + LA_BLK);
  S.sHH = reinterpret_cast<CT*>(S.sXYZ + kWidePtsMax);
  S.sPd = reinterpret_cast<R*>(S.sHH + kWidePtsMax * kHHStride);

  const int tid = threadIdx.x;
  const int K = tm->K, KK = K * K;
  const int b = blockIdx.x;
  int o[3], e[3];
  subvol_box(L, b, o, e);
  const int npts = e[0] * e[1] * e[2], n = npts * K;
  CT* F = factors + (size_t)b * L.fsize;
  for (int i = tid; i < LA_NPAIR * KK; i += kFactorThreads) S.sP[i] = (R)tm->P[i / KK][i % KK];
  const R wx = (R)(0.5 * g.ih2[0]), wy = (R)(0.5 * g.ih2[1]), wz = (R)(0.5 * g.ih2[2]);
  for (int i = tid; i < npts; i += kFactorThreads) {
    int lx, ly, lz;
    local_coords(i, e, lx, ly, lz);
    const int px = o[0] + lx, py = o[1] + ly, pz = o[2] + lz;
    S.sD[i] = (R)(g.dsum + g.V0[(pz * g.n[1] + py) * g.n[0] + px]);
    S.sX[i] = (R)fine_x(g, px, py, pz);
    // unused axes have n = 1 and w = 0
    const int cx = (px > 0 ? 1 : 0) + (px + 1 < g.n[0] ? 1 : 0), cy = (py > 0 ? 1 : 0) + (py + 1 < g.n[1] ? 1 : 0),
              cz = (pz > 0 ? 1 : 0) + (pz + 1 < g.n[2] ? 1 : 0);
    S.sN[i] = wx * wx * (R)cx + wy * wy * (R)cy + wz * wz * (R)cz;
    S.sXYZ[i] = lx | (ly << 8) | (lz << 16);
  }
  __syncthreads();
  for (int p = tid; p < npts * npts; p += kFactorThreads) {
    const int i = p / npts, j = p - i * npts;
    const int pi = S.sXYZ[i], pj = S.sXYZ[j];
    const int dx = (pj & 255) - (pi & 255), dy = ((pj >> 8) & 255) - ((pi >> 8) & 255), dz = (pj >> 16) - (pi >> 16);
    R H, H2;
    wide_h_h2<R>(dx, dy, dz, S.sD[i], S.sD[j], S.sN[i], wx, wy, wz, H, H2);
    S.sHH[i * kHHStride + j] = mkc<CT>(H, H2);
  }
  for (int i = tid; i < KK; i += kFactorThreads) {
    S.sPd[i] = S.sP[1 * KK + i] - S.sP[3 * KK + i];
    S.sPd[KK + i] = S.sP[2 * KK + i] - S.sP[6 * KK + i];
  }
  __syncthreads();
  const FastDiv dK = L.fd_K;
  const WideTables<R> T = S.tables();
  // block column 0: assembled only, one row per thread
  if (tid < NPAD) {
    CT a0[LA_BLK];
    const WideRow<R> w = wide_row<R>(tid, dK, K, S.sX);
#pragma unroll
    for (int q = 0; q < LA_BLK; ++q) a0[q] = wide_entry<R>(w, q, n, dK, K, T);
#pragma unroll
    for (int q = 0; q < LA_BLK; ++q) S.sPan[(size_t)tid * kWideStride + q] = a0[q];
  }
  __syncthreads();
  for (int J = 0; J < NB; ++J) {
    // threads per row of block column J+1 over the 224 lookahead threads
    const int RJ1 = NPAD - LA_BLK * (J + 1);
    int tpr = 1;
    while (tpr < 8 && 2 * tpr * RJ1 <= 224) tpr *= 2;
    switch (tpr) {
      case 1: wide_column_step<R, NPAD, 16>(J, L.band, n, dK, K, F, S, status); break;
      case 2: wide_column_step<R, NPAD, 8>(J, L.band, n, dK, K, F, S, status); break;
      case 4: wide_column_step<R, NPAD, 4>(J, L.band, n, dK, K, F, S, status); break;
      default: wide_column_step<R, NPAD, 2>(J, L.band, n, dK, K, F, S, status); break;
    }
  }
}

// ======================================================================== triangular solves
// x = (L L^dagger)^{-1} rhs with the blocked factor F; rhs is overwritten by x.  Two warps (64
// threads, 4 lanes per row) do the block mat-vecs and synchronise with a named barrier; the other
// warps of the CTA skip the solve.  Four lanes per row keep the cross-lane reduction at two shuffle
// levels, which matters because every FP64 add issues on the slow FP64 pipe.  The caller
// synchronises the whole CTA before and after.
__device__ __forceinline__ void solve_bar() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

template <typename CT>
__device__ __forceinline__ CT reduce4(CT v) {
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 1); v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 2); v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
  return v;
}

template <typename CT, int NPAD>
__device__ __forceinline__ void subvol_solve(const CT* __restrict__ F, CT* rhs, CT* y, CT* tvec, CT* red) {
  constexpr int NB = NPAD / LA_BLK;
  (void)red;
  const int tid = threadIdx.x;
  if (tid >= 64) return;
  const int r = tid >> 2, l = tid & 3;
  // forward: y_I = inv(L_II) (rhs_I - sum_{J<I} L_IJ y_J)
  for (int I = 0; I < NB; ++I) {
    const CT* rowblk = F + (size_t)(I * (I + 1) / 2) * 256;
    CT acc0 = mkc<CT>(0, 0), acc1 = mkc<CT>(0, 0);
    for (int J = 0; J < I; ++J) {
      const CT* blk = rowblk + J * 256 + r * LA_BLK;
      const CT* yy = y + J * LA_BLK;
      cfma(acc0, blk[l], yy[l]);
      cfma(acc1, blk[l + 4], yy[l + 4]);
      cfma(acc0, blk[l + 8], yy[l + 8]);
      cfma(acc1, blk[l + 12], yy[l + 12]);
    }
    CT acc = reduce4(mkc<CT>(acc0.x + acc1.x, acc0.y + acc1.y));
    if (l == 0) tvec[r] = mkc<CT>(rhs[I * LA_BLK + r].x - acc.x, rhs[I * LA_BLK + r].y - acc.y);
    solve_bar();
    const CT* dblk = rowblk + I * 256 + r * LA_BLK;
    acc0 = mkc<CT>(0, 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = l + 4 * k;
      if (c <= r) cfma(acc0, dblk[c], tvec[c]);
    }
    acc = reduce4(acc0);
    if (l == 0) y[I * LA_BLK + r] = acc;
    solve_bar();
  }
  // backward: x_I = inv(L_II)^dagger (y_I - sum_{J>I} L_JI^dagger x_J), x stored in rhs
  for (int I = NB - 1; I >= 0; --I) {
    CT acc0 = mkc<CT>(0, 0), acc1 = mkc<CT>(0, 0);
    for (int J = I + 1; J < NB; ++J) {
      const CT* blk = F + (size_t)(J * (J + 1) / 2 + I) * 256;
      const CT* xx = rhs + J * LA_BLK;
      cfma_conj(acc0, blk[l * LA_BLK + r], xx[l]);
      cfma_conj(acc1, blk[(l + 4) * LA_BLK + r], xx[l + 4]);
      cfma_conj(acc0, blk[(l + 8) * LA_BLK + r], xx[l + 8]);
      cfma_conj(acc1, blk[(l + 12) * LA_BLK + r], xx[l + 12]);
    }
    CT acc = reduce4(mkc<CT>(acc0.x + acc1.x, acc0.y + acc1.y));
    if (l == 0) tvec[r] = mkc<CT>(y[I * LA_BLK + r].x - acc.x, y[I * LA_BLK + r].y - acc.y);
    solve_bar();
    const CT* dblk = F + (size_t)(I * (I + 1) / 2 + I) * 256;
    acc0 = mkc<CT>(0, 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int cc = l + 4 * k;
      if (cc >= r) cfma_conj(acc0, dblk[cc * LA_BLK + r], tvec[cc]);
    }
    acc = reduce4(acc0);
    if (l == 0) rhs[I * LA_BLK + r] = acc;
    solve_bar();
  }
}

// Triangular solves with a wide factor (more than eight block rows) by all 128 threads of the
// sweep's CTA: every load of a step (one block row forward, one block column backward) is issued
// together, and in complex64 the next step's blocks are loaded while the current step computes, so
// the 2 NB dependent steps wait on memory about once each instead of once per block.  Forward, thread
// (r, q) = (t / 8, t % 8) takes entries (r, 2q) and (r, 2q + 1) of each block of the row (coalesced
// 16-byte pairs); backward, thread (r, q) = (t % 16, t / 16) takes entries (2q, r) and (2q + 1, r) of
// each block of the column (two coalesced rows per warp).  x = (L L^dagger)^{-1} rhs; rhs is
// overwritten by x.  Called by all threads of the CTA, between barriers.
// the two complex entries (2q, r) and (2q + 1, r) of a block (a column pair, stride 16)
template <typename CT>
__device__ __forceinline__ CPair<CT> load_colpair(const CT* blk, int q, int r, unsigned long long pol);
template <>
__device__ __forceinline__ CPair<float2> load_colpair<float2>(const float2* blk, int q, int r, unsigned long long pol) {
  CPair<float2> p;
  const float2 x = ldg_policy(blk + (2 * q) * LA_BLK + r, pol), y = ldg_policy(blk + (2 * q + 1) * LA_BLK + r, pol);
  p.v = make_float4(x.x, x.y, y.x, y.y);
  return p;
}
template <>
__device__ __forceinline__ CPair<double2> load_colpair<double2>(const double2* blk, int q, int r, unsigned long long) {
  CPair<double2> p;
  p.a_ = __ldg(blk + (2 * q) * LA_BLK + r);
  p.b_ = __ldg(blk + (2 * q + 1) * LA_BLK + r);
  return p;
}

template <typename CT>
__device__ __forceinline__ CT reduce_xor(CT v, int m) {
  v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

// forward block loads of the solve: complex64 with the keep-for-the-backward-pass policy
template <typename CT>
__device__ __forceinline__ void load_fwd(CPair<CT>& p, const CT* a, unsigned long long pol) {
  p.load(a);
}
template <>
__device__ __forceinline__ void load_fwd<float2>(CPair<float2>& p, const float2* a, unsigned long long pol) {
  p.v = ldg_policy(reinterpret_cast<const float4*>(a), pol);
}
template <typename CT>
__device__ __forceinline__ CPair<CT> zero_pair() {
  CPair<CT> p;
  p.load_zero();
  return p;
}
// a block entry pair inside the band, else the zero it is known to be
template <typename CT>
__device__ __forceinline__ void load_fwd_band(CPair<CT>& p, const CT* a, bool in_band, unsigned long long pol) {
  if (in_band) load_fwd(p, a, pol);
  else p.load_zero();
}

template <typename CT, int NPAD>
__device__ __forceinline__ void subvol_solve_wide(const CT* __restrict__ F, int band, CT* rhs, CT* y, CT* tvec,
                                                  CT* part) {
  constexpr int NB = NPAD / LA_BLK;
  constexpr bool kPrefetch = sizeof(CT) == 8;   // complex64: next step's blocks in flight during this one
  const int t = threadIdx.x;
  const unsigned long long keep = l2_evict_last(), last_use = l2_evict_first();
  {
    const int r = t >> 3, q = t & 7;
    CPair<CT> cur[NB];
    load_fwd(cur[0], F + r * LA_BLK + 2 * q, keep);
#pragma unroll
    for (int I = 0; I < NB; ++I) {
      CPair<CT> nxt[NB];
      // blocks (I, J) with I - J > band are exact zeros: set, not loaded
      if (kPrefetch && I + 1 < NB) {
#pragma unroll
        for (int J = 0; J <= I + 1; ++J)
          load_fwd_band(nxt[J], F + (size_t)tri_index(I + 1, J) * 256 + r * LA_BLK + 2 * q, J >= I + 1 - band, keep);
      }
      if (!kPrefetch && I > 0) {
#pragma unroll
        for (int J = 0; J <= I; ++J)
          load_fwd_band(cur[J], F + (size_t)tri_index(I, J) * 256 + r * LA_BLK + 2 * q, J >= I - band, keep);
      }
      CT acc0 = mkc<CT>(0, 0), acc1 = mkc<CT>(0, 0);
#pragma unroll
      for (int J = 0; J < I; ++J) {
        cfma(acc0, cur[J].a(), y[J * LA_BLK + 2 * q]);
        cfma(acc1, cur[J].b(), y[J * LA_BLK + 2 * q + 1]);
      }
      CT acc = mkc<CT>(acc0.x + acc1.x, acc0.y + acc1.y);
      acc = reduce_xor(acc, 1);
      acc = reduce_xor(acc, 2);
      acc = reduce_xor(acc, 4);
      if (q == 0) tvec[r] = mkc<CT>(rhs[I * LA_BLK + r].x - acc.x, rhs[I * LA_BLK + r].y - acc.y);
      __syncthreads();
      CT d = mkc<CT>(0, 0);
      cfma(d, cur[I].a(), tvec[2 * q]);
      cfma(d, cur[I].b(), tvec[2 * q + 1]);
      d = reduce_xor(d, 1);
      d = reduce_xor(d, 2);
      d = reduce_xor(d, 4);
      if (q == 0) y[I * LA_BLK + r] = d;
      __syncthreads();
      if (kPrefetch) {
#pragma unroll
        for (int J = 0; J < NB; ++J) cur[J] = nxt[J];
      }
    }
  }
  {
    const int r = t & 15, q = t >> 4, w = t >> 5;
    CPair<CT> cur[NB];
    // step I uses blocks (J, I), J = I .. NB-1 ((I, I): the inverted diagonal block)
    if (kPrefetch) {
#pragma unroll
      for (int J = NB - 1; J < NB; ++J) cur[J] = load_colpair<CT>(F + (size_t)tri_index(J, NB - 1) * 256, q, r, last_use);
    }
#pragma unroll
    for (int I = NB - 1; I >= 0; --I) {
      CPair<CT> nxt[NB];
      if (kPrefetch && I > 0) {
#pragma unroll
        for (int J = I - 1; J < NB; ++J)
          nxt[J] = J <= I - 1 + band ? load_colpair<CT>(F + (size_t)tri_index(J, I - 1) * 256, q, r, last_use)
                                     : zero_pair<CT>();
      }
      if (!kPrefetch) {
#pragma unroll
        for (int J = I; J < NB; ++J)
          cur[J] = J <= I + band ? load_colpair<CT>(F + (size_t)tri_index(J, I) * 256, q, r, last_use) : zero_pair<CT>();
      }
      CT acc0 = mkc<CT>(0, 0), acc1 = mkc<CT>(0, 0);
#pragma unroll
      for (int J = I + 1; J < NB; ++J) {
        cfma_conj(acc0, cur[J].a(), rhs[J * LA_BLK + 2 * q]);
        cfma_conj(acc1, cur[J].b(), rhs[J * LA_BLK + 2 * q + 1]);
      }
      CT acc = reduce_xor(mkc<CT>(acc0.x + acc1.x, acc0.y + acc1.y), 16);
      if ((t & 16) == 0) part[w * LA_BLK + r] = acc;
      __syncthreads();
      if (t < LA_BLK) {
        CT s = part[r];
#pragma unroll
        for (int u = 1; u < 4; ++u) { s.x += part[u * LA_BLK + r].x; s.y += part[u * LA_BLK + r].y; }
        tvec[r] = mkc<CT>(y[I * LA_BLK + r].x - s.x, y[I * LA_BLK + r].y - s.y);
      }
      __syncthreads();
      CT d = mkc<CT>(0, 0);
      cfma_conj(d, cur[I].a(), tvec[2 * q]);
      cfma_conj(d, cur[I].b(), tvec[2 * q + 1]);
      d = reduce_xor(d, 16);
      if ((t & 16) == 0) part[w * LA_BLK + r] = d;
      __syncthreads();
      if (t < LA_BLK) {
        CT s = part[r];
#pragma unroll
        for (int u = 1; u < 4; ++u) { s.x += part[u * LA_BLK + r].x; s.y += part[u * LA_BLK + r].y; }
        rhs[I * LA_BLK + r] = s;
      }
      __syncthreads();
      if (kPrefetch) {
#pragma unroll
        for (int J = 0; J < NB; ++J) cur[J] = nxt[J];
      }
    }
  }
}

// The 128-thread solve (every step's blocks loaded together, the next step's in flight) serves every
// complex64 factor and the wide FP64 ones; shorter FP64 factors keep the two-warp solve, whose
// two-level reductions issue fewer adds on the slow FP64 pipe.
template <typename R, int NPAD>
__host__ __device__ constexpr bool use_wide_solve() {
  return sizeof(R) == 4 || NPAD > LA_NPAD_MAX;
}

// ======================================================================== finest-level sweep
// Matrix-free (M-form): residual r = f - M~ c on the footprint F = U + 1 from c on U + 2,
// z = Wt r, right-hand side (M~^dagger z)_U, solve, c_U += delta.
template <typename R, int NPAD>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep_fine(LevelGeom L, FineOp g, const TimeMats* __restrict__ tm, const typename C2<R>::T* __restrict__ f,
             const typename C2<R>::T* __restrict__ yx, typename C2<R>::T* __restrict__ c,
             const typename C2<R>::T* __restrict__ factors, int colour, int* __restrict__ status) {
  typedef typename C2<R>::T CT;
  extern __shared__ __align__(16) unsigned char smem[];
  (void)status;   // no bounded wait in this kernel
  const int K = tm->K, KK = K * K;
  const int tid = threadIdx.x;
  const int b = colour_subvol(L, colour, blockIdx.x);
  int o[3], e[3];
  subvol_box(L, b, o, e);
  int ec[3], ef[3], oc[3], of_[3];
  for (int a = 0; a < 3; ++a) {
    const bool used = a < L.dim;
    ec[a] = used ? e[a] + 4 : 1;  oc[a] = used ? o[a] - 2 : o[a];
    ef[a] = used ? e[a] + 2 : 1;  of_[a] = used ? o[a] - 1 : o[a];
  }
  const int nbc = ec[0] * ec[1] * ec[2], nbf = ef[0] * ef[1] * ef[2], npts = e[0] * e[1] * e[2];
  const int sx = L.sub[0] + 4, sy = L.dim > 1 ? L.sub[1] + 4 : 1, sz = L.dim > 2 ? L.sub[2] + 4 : 1;
  const int nbc_max = sx * sy * sz;
  const int nbf_max = (L.sub[0] + 2) * (L.dim > 1 ? L.sub[1] + 2 : 1) * (L.dim > 2 ? L.sub[2] + 2 : 1);
  // index maps item t -> (point i, time function m) and point -> (x, y, z) by multiply-shift
  // division: the level's divisors for a full subvolume, this CTA's own for a ragged one
  const bool full = e[0] == L.sub[0] && e[1] == L.sub[1] && e[2] == L.sub[2];
  const FastDiv dK = L.fd_K;
  const FastDiv dc0 = full ? L.fd_c[0] : make_fastdiv(ec[0]), dc1 = full ? L.fd_c[1] : make_fastdiv(ec[1]);
  const FastDiv df0 = full ? L.fd_f[0] : make_fastdiv(ef[0]), df1 = full ? L.fd_f[1] : make_fastdiv(ef[1]);
  const FastDiv du0 = full ? L.fd_u[0] : make_fastdiv(e[0]), du1 = full ? L.fd_u[1] : make_fastdiv(e[1]);
  auto item = [&](int t, int& i, int& m) {
    i = fdiv(t, dK);
    m = t - i * K;
  };
  auto coords = [](int i, const FastDiv& d0, const FastDiv& d1, int& x, int& y, int& z) {
    const int r = fdiv(i, d0);
    x = i - r * d0.d;
    z = fdiv(r, d1);
    y = r - z * d1.d;
  };

  R* sQ = reinterpret_cast<R*>(smem);
  R* sU = sQ + LA_KMAX * LA_KMAX;
  R* sW = sU + LA_KMAX * LA_KMAX;
  R* sE = sW + LA_KMAX * LA_KMAX;
  R* sV = sE + LA_KMAX * LA_KMAX;                     // dsum + V0 on the footprint F = U + 1 [nbf_max]
  R* sX = sV + ((nbf_max + 3) & ~3);                  // laser coordinate on the footprint [nbf_max]
  CT* sC = reinterpret_cast<CT*>(sX + ((nbf_max + 3) & ~3));  // c on U+2  [nbc_max * K]
  CT* sA = sC + (size_t)nbc_max * K;                  // Hc, then z, on the footprint   [nbf_max * K]
  CT* sB = sA + (size_t)nbf_max * K;                  // r, then Hz, on the footprint   [nbf_max * K]
  CT* sRhs = sB + (size_t)nbf_max * K;                // [NPAD]
  CT* sY = sRhs + NPAD;                               // [NPAD]
  CT* sT = sY + NPAD;                                 // [16]
  CT* sRed = sT + LA_BLK;                             // [128]

  for (int i = tid; i < KK; i += kSweepThreads) {
    sQ[i] = (R)tm->Qb[i]; sU[i] = (R)tm->Ub[i]; sW[i] = (R)tm->Wt[i]; sE[i] = (R)tm->Eb[i];
  }
  const unsigned long long stream = l2_evict_first();   // c and f: read once per launch
  for (int t = tid; t < nbc * K; t += kSweepThreads) {
    int i, m;
    item(t, i, m);
    int lx, ly, lz;
    coords(i, dc0, dc1, lx, ly, lz);
    const int gx = oc[0] + lx, gy = oc[1] + ly, gz = oc[2] + lz;
    CT v = mkc<CT>(0, 0);
    if (fine_in(g, gx, gy, gz)) v = ld_policy(c + (size_t)((gz * g.n[1] + gy) * g.n[0] + gx) * K + m, stream);
    sC[t] = v;
  }
  {
    // per footprint point, in the kernel's own precision (a complex64 sweep issues no FP64 work here)
    const R dsum = (R)g.dsum;
    const R xo = (R)(g.lax == 0 ? g.x0[0] : (g.lax == 1 ? g.x0[1] : g.x0[2]));
    const R xh = (R)(g.lax == 0 ? g.h[0] : (g.lax == 1 ? g.h[1] : g.h[2]));
    for (int i = tid; i < nbf; i += kSweepThreads) {
      int lx, ly, lz;
      coords(i, df0, df1, lx, ly, lz);
      const int gx = of_[0] + lx, gy = of_[1] + ly, gz = of_[2] + lz;
      sV[i] = fine_in(g, gx, gy, gz) ? dsum + (R)g.V0[(gz * g.n[1] + gy) * g.n[0] + gx] : (R)0;
      sX[i] = xo + (R)(g.lax == 0 ? gx : (g.lax == 1 ? gy : gz)) * xh;
    }
  }
  __syncthreads();
  // c-box index of footprint point (lx, ly, lz): (lx+1, ly+1, lz+1) on used axes
  const int dcx = 1, dcy = L.dim > 1 ? ec[0] : 0, dcz = L.dim > 2 ? ec[0] * ec[1] : 0;
  const R wx = (R)(-0.5 * g.ih2[0]), wy = (R)(-0.5 * g.ih2[1]), wz = (R)(-0.5 * g.ih2[2]);
  // stage 1: Hc on the footprint
  for (int t = tid; t < nbf * K; t += kSweepThreads) {
    int i, m;
    item(t, i, m);
    int lx, ly, lz;
    coords(i, df0, df1, lx, ly, lz);
    const int cx = L.dim > 0 ? lx + 1 : lx, cy = L.dim > 1 ? ly + 1 : ly, cz = L.dim > 2 ? lz + 1 : lz;
    const int ci = (cz * ec[1] + cy) * ec[0] + cx;
    const CT v = sC[ci * K + m];
    CT h = mkc<CT>(sV[i] * v.x, sV[i] * v.y);
    {
      const CT a1 = sC[(ci + dcx) * K + m], a2 = sC[(ci - dcx) * K + m];
      h.x += wx * (a1.x + a2.x); h.y += wx * (a1.y + a2.y);
    }
    if (L.dim > 1) {
      const CT a1 = sC[(ci + dcy) * K + m], a2 = sC[(ci - dcy) * K + m];
      h.x += wy * (a1.x + a2.x); h.y += wy * (a1.y + a2.y);
    }
    if (L.dim > 2) {
      const CT a1 = sC[(ci + dcz) * K + m], a2 = sC[(ci - dcz) * K + m];
      h.x += wz * (a1.x + a2.x); h.y += wz * (a1.y + a2.y);
    }
    sA[t] = h;
  }
  __syncthreads();
  // stage 2: r = f - (i Qb c - Ub Hc - x Eb c) on the footprint (0 outside the grid)
  for (int t = tid; t < nbf * K; t += kSweepThreads) {
    int i, m;
    item(t, i, m);
    int lx, ly, lz;
    coords(i, df0, df1, lx, ly, lz);
    const int gx = of_[0] + lx, gy = of_[1] + ly, gz = of_[2] + lz;
    CT r = mkc<CT>(0, 0);
    if (fine_in(g, gx, gy, gz)) {
      const int cx = L.dim > 0 ? lx + 1 : lx, cy = L.dim > 1 ? ly + 1 : ly, cz = L.dim > 2 ? lz + 1 : lz;
      const int ci = (cz * ec[1] + cy) * ec[0] + cx;
      const R xl = sX[i];
      R qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
      for (int nn = 0; nn < K; ++nn) {
        const CT cv = sC[ci * K + nn], hv = sA[i * K + nn];
        const R q = sQ[m * K + nn], u = sU[m * K + nn], ee = sE[m * K + nn];
        qr = fma(q, cv.x, qr); qi = fma(q, cv.y, qi);
        ur = fma(u, hv.x, ur); ui = fma(u, hv.y, ui);
        er = fma(ee, cv.x, er); ei = fma(ee, cv.y, ei);
      }
      const CT fv = f ? ld_policy(f + (size_t)((gz * g.n[1] + gy) * g.n[0] + gx) * K + m, stream) : mkc<CT>(0, 0);
      r.x = fv.x - (-qi - ur - xl * er);
      r.y = fv.y - (qr - ui - xl * ei);
    }
    sB[t] = r;
  }
  __syncthreads();
  // stage 3: z = Wt r
  for (int t = tid; t < nbf * K; t += kSweepThreads) {
    int i, m;
    item(t, i, m);
    R zr = 0, zi = 0;
    for (int nn = 0; nn < K; ++nn) {
      const R w = sW[m * K + nn];
      const CT rv = sB[i * K + nn];
      zr = fma(w, rv.x, zr); zi = fma(w, rv.y, zi);
    }
    sA[t] = mkc<CT>(zr, zi);
  }
  __syncthreads();
  // stage 4: Hz on U (footprint index of U point = local + 1 on used axes)
  const int dfy = L.dim > 1 ? ef[0] : 0, dfz = L.dim > 2 ? ef[0] * ef[1] : 0;
  for (int t = tid; t < npts * K; t += kSweepThreads) {
    int i, m;
    item(t, i, m);
    int lx, ly, lz;
    coords(i, du0, du1, lx, ly, lz);
    const int fx = L.dim > 0 ? lx + 1 : lx, fy = L.dim > 1 ? ly + 1 : ly, fz = L.dim > 2 ? lz + 1 : lz;
    const int fi = (fz * ef[1] + fy) * ef[0] + fx;
    const CT v = sA[fi * K + m];
    CT h = mkc<CT>(sV[fi] * v.x, sV[fi] * v.y);
    {
      const CT a1 = sA[(fi + 1) * K + m], a2 = sA[(fi - 1) * K + m];
      h.x += wx * (a1.x + a2.x); h.y += wx * (a1.y + a2.y);
    }
    if (L.dim > 1) {
      const CT a1 = sA[(fi + dfy) * K + m], a2 = sA[(fi - dfy) * K + m];
      h.x += wy * (a1.x + a2.x); h.y += wy * (a1.y + a2.y);
    }
    if (L.dim > 2) {
      const CT a1 = sA[(fi + dfz) * K + m], a2 = sA[(fi - dfz) * K + m];
      h.x += wz * (a1.x + a2.x); h.y += wz * (a1.y + a2.y);
    }
    sB[t] = h;
  }
  __syncthreads();
  // stage 5: rhs = -i Qb^T z - Ub Hz - x Eb z on U; padding 0
  for (int t = tid; t < NPAD; t += kSweepThreads) {
    CT out = mkc<CT>(0, 0);
    if (t < npts * K) {
      int i, m;
      item(t, i, m);
      int lx, ly, lz;
      coords(i, du0, du1, lx, ly, lz);
      const int fx = L.dim > 0 ? lx + 1 : lx, fy = L.dim > 1 ? ly + 1 : ly, fz = L.dim > 2 ? lz + 1 : lz;
      const int fi = (fz * ef[1] + fy) * ef[0] + fx;
      const R xl = sX[fi];
      R qr = 0, qi = 0, ur = 0, ui = 0, er = 0, ei = 0;
      for (int nn = 0; nn < K; ++nn) {
        const CT zv = sA[fi * K + nn], hv = sB[i * K + nn];
        const R q = sQ[nn * K + m], u = sU[m * K + nn], ee = sE[m * K + nn];
        qr = fma(q, zv.x, qr); qi = fma(q, zv.y, qi);
        ur = fma(u, hv.x, ur); ui = fma(u, hv.y, ui);
        er = fma(ee, zv.x, er); ei = fma(ee, zv.y, ei);
      }
      out.x = qi - ur - xl * er;
      out.y = -qr - ui - xl * ei;
      if (yx) {  // additive right-hand side (adjoint relaxation of G z = y)
        const CT yv = yx[(size_t)(((o[2] + lz) * g.n[1] + (o[1] + ly)) * g.n[0] + (o[0] + lx)) * K + m];
        out.x += yv.x;
        out.y += yv.y;
      }
    }
    sRhs[t] = out;
  }
  __syncthreads();
  if (use_wide_solve<R, NPAD>())
    subvol_solve_wide<CT, NPAD>(factors + (size_t)b * L.fsize, L.band, sRhs, sY, sT, sRed);
  else
    subvol_solve<CT, NPAD>(factors + (size_t)b * L.fsize, sRhs, sY, sT, sRed);
  __syncthreads();
  for (int t = tid; t < npts * K; t += kSweepThreads) {
    int i, m;
    item(t, i, m);
    int lx, ly, lz;
    coords(i, du0, du1, lx, ly, lz);
    const size_t gi = (size_t)(((o[2] + lz) * g.n[1] + (o[1] + ly)) * g.n[0] + (o[0] + lx)) * K + m;
    CT v = c[gi];
    v.x += sRhs[t].x;
    v.y += sRhs[t].y;
    c[gi] = v;
  }
}

// ======================================================================== Galerkin-level sweep
// rhs = (g - G e)_U with G = sum_kk' Sigma_kk' (x) Theta_kk' from the stored stencils.  The
// subvolume's stencils (|U| x 9 x box) and e on U + 2 are staged in shared memory with
// coalesced loads first, so the stencil sums run from shared memory with short dependency
// chains: (i, kk', n) tasks form u = Sigma_kk' e, then (i, m) tasks combine the nine pairs.
template <typename R>
struct CoarseSmem {
  typedef typename C2<R>::T CT;
  R* P; CT* E; R* Sg; CT* U; CT* Rhs; CT* Y; CT* T; CT* Red;
};
__host__ __device__ inline size_t coarse_sg_count(const LevelGeom& L) {
  const size_t nptsmax = (size_t)L.sub[0] * L.sub[1] * L.sub[2];
  return (nptsmax * LA_NPAIR * box5_count(L.dim) + 3) & ~(size_t)3;
}
__host__ __device__ inline size_t coarse_box_count(const LevelGeom& L) {
  const int sx = L.sub[0] + 4, sy = L.dim > 1 ? L.sub[1] + 4 : 1, sz = L.dim > 2 ? L.sub[2] + 4 : 1;
  return (size_t)sx * sy * sz;
}
template <typename R>
__device__ inline CoarseSmem<R> coarse_smem_layout(unsigned char* smem, const LevelGeom& L, int K, int npad) {
  typedef typename C2<R>::T CT;
  CoarseSmem<R> m;
  const size_t nptsmax = (size_t)L.sub[0] * L.sub[1] * L.sub[2];
  m.P = reinterpret_cast<R*>(smem);
  m.E = reinterpret_cast<CT*>(m.P + LA_NPAIR * LA_KMAX * LA_KMAX);
  m.Sg = reinterpret_cast<R*>(m.E + coarse_box_count(L) * K);
  m.U = reinterpret_cast<CT*>(m.Sg + coarse_sg_count(L));
  m.Rhs = m.U + nptsmax * LA_NPAIR * K;
  m.Y = m.Rhs + npad;
  m.T = m.Y + npad;
  m.Red = m.T + LA_BLK;
  return m;
}

// Multiply-shift index maps of one subvolume: item -> (point, time function), point -> (x, y, z) in U
// and in U + 2 (the level's divisors for a full subvolume, the CTA's own for a ragged one).
struct SubvolDiv {
  FastDiv K, c0, c1, u0, u1;
  __device__ SubvolDiv(const LevelGeom& L, const int e[3]) {
    const bool full = e[0] == L.sub[0] && e[1] == L.sub[1] && e[2] == L.sub[2];
    K = L.fd_K;
    c0 = full ? L.fd_c[0] : make_fastdiv(e[0] + 4);
    c1 = full ? L.fd_c[1] : make_fastdiv(L.dim > 1 ? e[1] + 4 : 1);
    u0 = full ? L.fd_u[0] : make_fastdiv(e[0]);
    u1 = full ? L.fd_u[1] : make_fastdiv(e[1]);
  }
  __device__ __forceinline__ void item(int t, int& i, int& m) const {
    i = fdiv(t, K);
    m = t - i * K.d;
  }
  __device__ __forceinline__ static void coords(int i, const FastDiv& d0, const FastDiv& d1, int& x, int& y,
                                                int& z) {
    const int r = fdiv(i, d0);
    x = i - r * d0.d;
    z = fdiv(r, d1);
    y = r - z * d1.d;
  }
};

// Fills S.Rhs[0..npad) with (g - G e) on the subvolume with origin o and extent e (0 in padding).
template <typename R>
__device__ inline void coarse_rhs(const LevelGeom& L, const R* __restrict__ sigma,
                                  const TimeMats* __restrict__ tm, const typename C2<R>::T* __restrict__ gvec,
                                  const typename C2<R>::T* __restrict__ ev, const int o[3], const int e[3], int npad,
                                  const CoarseSmem<R>& S) {
  typedef typename C2<R>::T CT;
  const int K = tm->K, KK = K * K;
  const int tid = threadIdx.x, nthr = blockDim.x;
  int ec[3], oc[3];
  for (int a = 0; a < 3; ++a) {
    const bool used = a < L.dim;
    ec[a] = used ? e[a] + 4 : 1;  oc[a] = used ? o[a] - 2 : o[a];
  }
  const int nbc = ec[0] * ec[1] * ec[2], npts = e[0] * e[1] * e[2];
  const int nbox = box5_count(L.dim);
  const SubvolDiv dv(L, e);
  for (int i = tid; i < LA_NPAIR * KK; i += nthr) S.P[i] = (R)tm->P[i / KK][i % KK];
  // e on U + 2 (zero outside the grid) and the stencils of U's points reach shared memory by cp.async,
  // every copy of a thread in flight at once instead of one dependent load per loop trip
  for (int t = tid; t < nbc * K; t += nthr) {
    int i, m;
    dv.item(t, i, m);
    int lx, ly, lz;
    SubvolDiv::coords(i, dv.c0, dv.c1, lx, ly, lz);
    const int gx = oc[0] + lx, gy = oc[1] + ly, gz = oc[2] + lz;
    const bool in = gx >= 0 && gy >= 0 && gz >= 0 && gx < L.n[0] && gy < L.n[1] && gz < L.n[2];
    cp_async_elem_zf(S.E + t, in ? ev + (size_t)((gz * L.n[1] + gy) * L.n[0] + gx) * K + m : ev, in);
  }
  const int per_pt = LA_NPAIR * nbox;
  for (int t = tid; t < npts * per_pt; t += nthr) {
    const int i = fdiv(t, L.fd_pair), w = t - i * per_pt;
    int lx, ly, lz;
    SubvolDiv::coords(i, dv.u0, dv.u1, lx, ly, lz);
    const int p = ((o[2] + lz) * L.n[1] + (o[1] + ly)) * L.n[0] + (o[0] + lx);
    cp_async_real(S.Sg + t, sigma + (size_t)p * per_pt + w);
  }
  cp_async_wait_all();
  __syncthreads();
  // u[i][kk][n] = sum_o Sigma_kk[p_i][o] e[p_i + o][n]
  const int ry = L.dim > 1 ? 2 : 0, rz = L.dim > 2 ? 2 : 0;
  for (int t = tid; t < npts * LA_NPAIR * K; t += nthr) {
    int ikk, n;
    dv.item(t, ikk, n);
    const int i = ikk / LA_NPAIR;
    int lx, ly, lz;
    SubvolDiv::coords(i, dv.u0, dv.u1, lx, ly, lz);
    const int cx = lx + 2, cy = L.dim > 1 ? ly + 2 : ly, cz = L.dim > 2 ? lz + 2 : lz;
    const R* sg = S.Sg + (size_t)ikk * nbox;
    R ur0 = 0, ui0 = 0, ur1 = 0, ui1 = 0;
    int q = 0;
    for (int oz = -rz; oz <= rz; ++oz)
      for (int oy = -ry; oy <= ry; ++oy) {
        const CT* ep = S.E + (size_t)(((cz + oz) * ec[1] + (cy + oy)) * ec[0] + (cx - 2)) * K + n;
#pragma unroll
        for (int ox = 0; ox < 5; ++ox, ++q) {
          const R sv = sg[q];
          const CT v = ep[ox * K];
          if (ox & 1) { ur1 = fma(sv, v.x, ur1); ui1 = fma(sv, v.y, ui1); }
          else { ur0 = fma(sv, v.x, ur0); ui0 = fma(sv, v.y, ui0); }
        }
      }
    S.U[t] = mkc<CT>(ur0 + ur1, ui0 + ui1);
  }
  __syncthreads();
  // rhs[i, m] = g - sum_kk phase_kk sum_n P_kk[m][n] u[i][kk][n]   (pairs in fixed order)
  for (int t = tid; t < npad; t += nthr) {
    CT out = mkc<CT>(0, 0);
    if (t < npts * K) {
      int i, m;
      dv.item(t, i, m);
      int lx, ly, lz;
      SubvolDiv::coords(i, dv.u0, dv.u1, lx, ly, lz);
      const int p = ((o[2] + lz) * L.n[1] + (o[1] + ly)) * L.n[0] + (o[0] + lx);
      out = gvec[(size_t)p * K + m];
#pragma unroll
      for (int kk = 0; kk < LA_NPAIR; ++kk) {
        const CT* u = S.U + ((size_t)i * LA_NPAIR + kk) * K;
        const R* pr = S.P + kk * KK + m * K;
        R vr = 0, vi = 0;
        for (int nn = 0; nn < K; ++nn) { vr = fma(pr[nn], u[nn].x, vr); vi = fma(pr[nn], u[nn].y, vi); }
        const int ph = theta_phase(kk);
        if (ph == 0) { out.x -= vr; out.y -= vi; }
        else if (ph == 1) { out.x += vi; out.y -= vr; }   // -(i v)
        else { out.x -= vi; out.y += vr; }                // -(-i v)
      }
    }
    S.Rhs[t] = out;
  }
  __syncthreads();
}

template <typename R, int NPAD>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep_coarse(LevelGeom L, const R* __restrict__ sigma, const TimeMats* __restrict__ tm,
               const typename C2<R>::T* __restrict__ gvec, typename C2<R>::T* __restrict__ ev,
               const typename C2<R>::T* __restrict__ factors, int colour, int* __restrict__ status) {
  typedef typename C2<R>::T CT;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = tm->K;
  const int b = colour_subvol(L, colour, blockIdx.x);
  int o[3], e[3];
  subvol_box(L, b, o, e);
  const int npts = e[0] * e[1] * e[2];
  CoarseSmem<R> S = coarse_smem_layout<R>(smem, L, K, NPAD);
  coarse_rhs<R>(L, sigma, tm, gvec, ev, o, e, NPAD, S);
  subvol_solve<CT, NPAD>(factors + (size_t)b * L.fsize, S.Rhs, S.Y, S.T, S.Red);
  __syncthreads();
  const SubvolDiv dv(L, e);
  for (int t = threadIdx.x; t < npts * K; t += kSweepThreads) {
    int i, m;
    dv.item(t, i, m);
    int lx, ly, lz;
    SubvolDiv::coords(i, dv.u0, dv.u1, lx, ly, lz);
    const size_t gi = (size_t)(((o[2] + lz) * L.n[1] + (o[1] + ly)) * L.n[0] + (o[0] + lx)) * K + m;
    CT v = ev[gi];
    v.x += S.Rhs[t].x;
    v.y += S.Rhs[t].y;
    ev[gi] = v;
  }
}

// s = g - G e on every point of a Galerkin level, one CTA per subvolume (all colours at once).
template <typename R>
__global__ void __launch_bounds__(kSweepThreads)
k_gresid_tiles(LevelGeom L, const R* __restrict__ sigma, const TimeMats* __restrict__ tm,
               const typename C2<R>::T* __restrict__ gvec, const typename C2<R>::T* __restrict__ ev,
               typename C2<R>::T* __restrict__ out, int npad) {
  typedef typename C2<R>::T CT;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = tm->K;
  int o[3], e[3];
  subvol_box(L, blockIdx.x, o, e);
  const int npts = e[0] * e[1] * e[2];
  CoarseSmem<R> S = coarse_smem_layout<R>(smem, L, K, npad);
  coarse_rhs<R>(L, sigma, tm, gvec, ev, o, e, npad, S);
  const SubvolDiv dv(L, e);
  for (int t = threadIdx.x; t < npts * K; t += kSweepThreads) {
    int i, m;
    dv.item(t, i, m);
    int lx, ly, lz;
    SubvolDiv::coords(i, dv.u0, dv.u1, lx, ly, lz);
    out[(size_t)(((o[2] + lz) * L.n[1] + (o[1] + ly)) * L.n[0] + (o[0] + lx)) * K + m] = S.Rhs[t];
  }
}

// ======================================================================== host dispatch
// Several matrices per CTA only on levels of at least 512 subvolumes; a level with fewer (a small
// grid such as the 1D workload's 8) runs one matrix per CTA, so that its few matrices are
// factorised side by side instead of one after another in a single CTA.  (Per context: the
// batched workload's grids of 512 and more subvolumes, running concurrently, keep the grouping.)
constexpr int kFactorMultiMin = 512;
inline int factor_grid_mpc(const LevelGeom& L, int mpc) {
  return (L.nsub >= kFactorMultiMin && !L.one_per_cta) ? mpc : 1;
}

inline size_t factor_smem(const LevelGeom& L, int nptsmax, size_t csize, int mpc_) {
  const size_t ntri = (size_t)L.npad * (L.npad + 1) / 2;
  const size_t npair = (size_t)nptsmax * (nptsmax + 1) / 2;
  const size_t mpc = (size_t)mpc_;
  return mpc * (csize * (ntri + L.npad) + (size_t)L.npad * (csize / 2)) +
         sizeof(double) * (LA_NPAIR * LA_KMAX * LA_KMAX + mpc * npair * LA_NPAIR) + sizeof(int) * (mpc * npair + 1);
}
inline size_t sweep_fine_smem(const LevelGeom& L, int K, size_t rsize, size_t csize) {
  const int sx = L.sub[0] + 4, sy = L.dim > 1 ? L.sub[1] + 4 : 1, sz = L.dim > 2 ? L.sub[2] + 4 : 1;
  const size_t nbc = (size_t)sx * sy * sz;
  const size_t nbf = (size_t)(L.sub[0] + 2) * (L.dim > 1 ? L.sub[1] + 2 : 1) * (L.dim > 2 ? L.sub[2] + 2 : 1);
  return rsize * (4 * LA_KMAX * LA_KMAX + 2 * ((nbf + 3) & ~(size_t)3)) +
         csize * (nbc * K + 2 * nbf * K + 2 * (size_t)L.npad + LA_BLK + 128);
}
inline size_t sweep_coarse_smem(const LevelGeom& L, int K, size_t rsize, size_t csize) {
  const size_t nptsmax = (size_t)L.sub[0] * L.sub[1] * L.sub[2];
  return rsize * (LA_NPAIR * LA_KMAX * LA_KMAX + coarse_sg_count(L)) +
         csize * (coarse_box_count(L) * K + nptsmax * LA_NPAIR * K + 2 * (size_t)L.npad + LA_BLK + 128);
}

template <typename R, int NPAD, int mpc>
cudaError_t launch_factor_blk_m(const LevelGeom& L, const FineOp* fine, const R* sigma, const TimeMats* tm,
                                typename C2<R>::T* factors, int* status, cudaStream_t s) {
  typedef typename C2<R>::T CT;
  const int nptsmax = L.sub[0] * L.sub[1] * L.sub[2];
  const size_t smem = mpc * (sizeof(CT) * ((size_t)LA_BLK * NPAD + (size_t)(NPAD / LA_BLK) * 256) + sizeof(R) * NPAD) +
                      sizeof(R) * (LA_NPAIR * LA_KMAX * LA_KMAX +
                                   mpc * ((size_t)nptsmax * nptsmax * (fine ? 2 : LA_NPAIR) + nptsmax));
  auto kern = k_factor_blk<R, NPAD, mpc>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  FineOp g = fine ? *fine : FineOp{};
  kern<<<(L.nsub + mpc - 1) / mpc, kFactorThreads, smem, s>>>(L, g, fine ? 1 : 0, nptsmax, sigma, tm, factors, status);
  return cudaGetLastError();
}

template <typename R, int NPAD>
cudaError_t launch_factor_blk_n(const LevelGeom& L, const FineOp* fine, const R* sigma, const TimeMats* tm,
                                typename C2<R>::T* factors, int* status, cudaStream_t s) {
  constexpr int mpc = factor_c64_mpc(NPAD);
  if (mpc > 1 && factor_grid_mpc(L, mpc) == 1)
    return launch_factor_blk_m<R, NPAD, 1>(L, fine, sigma, tm, factors, status, s);
  return launch_factor_blk_m<R, NPAD, mpc>(L, fine, sigma, tm, factors, status, s);
}

// Wide subvolumes (more than LA_NPAD_MAX unknowns) exist on the finest level only.
template <typename R, int NPAD>
cudaError_t launch_factor_wide_n(const LevelGeom& L, const FineOp* fine, const TimeMats* tm,
                                 typename C2<R>::T* factors, int* status, cudaStream_t s) {
  typedef typename C2<R>::T CT;
  if (!fine) return cudaErrorInvalidValue;
  const size_t smem = wide_factor_smem(NPAD, sizeof(CT), sizeof(R));
  auto kern = k_factor_wide<R, NPAD>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  kern<<<L.nsub, kFactorThreads, smem, s>>>(L, *fine, tm, factors, status);
  return cudaGetLastError();
}

template <typename R, int NPAD, int mpc>
cudaError_t launch_factor_m(const LevelGeom& L, const FineOp* fine, const R* sigma, const TimeMats* tm,
                            typename C2<R>::T* factors, int* status, cudaStream_t s) {
  const int nptsmax = L.sub[0] * L.sub[1] * L.sub[2];
  const size_t smem = factor_smem(L, nptsmax, sizeof(typename C2<R>::T), mpc);
  auto kern = k_factor<R, NPAD, mpc>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  FineOp g = fine ? *fine : FineOp{};
  kern<<<(L.nsub + mpc - 1) / mpc, kFactorThreads, smem, s>>>(L, g, fine ? 1 : 0, nptsmax, sigma, tm, factors, status);
  return cudaGetLastError();
}
template <typename R, int NPAD>
cudaError_t launch_factor_n(const LevelGeom& L, const FineOp* fine, const R* sigma, const TimeMats* tm,
                            typename C2<R>::T* factors, int* status, cudaStream_t s) {
  constexpr int mpc = factor_mpc(NPAD);
  if (mpc > 1 && factor_grid_mpc(L, mpc) == 1)
    return launch_factor_m<R, NPAD, 1>(L, fine, sigma, tm, factors, status, s);
  return launch_factor_m<R, NPAD, mpc>(L, fine, sigma, tm, factors, status, s);
}
template <typename R, int NPAD>
cudaError_t launch_sweep_fine_n(const LevelGeom& L, const FineOp& g, const TimeMats* tm, int K,
                                const typename C2<R>::T* f, const typename C2<R>::T* yx, typename C2<R>::T* c,
                                const typename C2<R>::T* factors, int colour, int* status, cudaStream_t s) {
  const int nblocks = colour_count(L, colour);
  if (nblocks == 0) return cudaSuccess;
  const size_t smem = sweep_fine_smem(L, K, sizeof(R), sizeof(typename C2<R>::T));
  auto kern = k_sweep_fine<R, NPAD>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  kern<<<nblocks, kSweepThreads, smem, s>>>(L, g, tm, f, yx, c, factors, colour, status);
  return cudaGetLastError();
}
template <typename R, int NPAD>
cudaError_t launch_sweep_coarse_n(const LevelGeom& L, const R* sigma, const TimeMats* tm, int K,
                                  const typename C2<R>::T* gvec, typename C2<R>::T* e,
                                  const typename C2<R>::T* factors, int colour, int* status, cudaStream_t s) {
  const int nblocks = colour_count(L, colour);
  if (nblocks == 0) return cudaSuccess;
  const size_t smem = sweep_coarse_smem(L, K, sizeof(R), sizeof(typename C2<R>::T));
  auto kern = k_sweep_coarse<R, NPAD>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  kern<<<nblocks, kSweepThreads, smem, s>>>(L, sigma, tm, gvec, e, factors, colour, status);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gresid_tiles_r(const LevelGeom& L, const R* sigma, const TimeMats* tm, int K,
                                  const typename C2<R>::T* gvec, const typename C2<R>::T* e, typename C2<R>::T* out,
                                  cudaStream_t s) {
  const size_t smem = sweep_coarse_smem(L, K, sizeof(R), sizeof(typename C2<R>::T));
  auto kern = k_gresid_tiles<R>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  kern<<<L.nsub, kSweepThreads, smem, s>>>(L, sigma, tm, gvec, e, out, L.npad);
  return cudaGetLastError();
}

// finest-level sweeps and factorisations also take the wide sizes
#define LA_NPAD_DISPATCH_WIDE(NPADV, CALL) \
  switch (NPADV) {                    \
    case 192: return CALL(192);       \
    case 256: return CALL(256);       \
    default: break;                   \
  }

#define LA_NPAD_DISPATCH(NPADV, CALL) \
  switch (NPADV) {                    \
    case 16: return CALL(16);         \
    case 32: return CALL(32);         \
    case 48: return CALL(48);         \
    case 64: return CALL(64);         \
    case 96: return CALL(96);         \
    case 128: return CALL(128);       \
    default: return cudaErrorInvalidValue; \
  }

}  // namespace la
