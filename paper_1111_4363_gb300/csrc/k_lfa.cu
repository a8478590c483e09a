// Convergence maps of one relaxation step in the paper's Legendre-element basis (Secs. IV-V):
// for every case (method, Nx, Nt, kappa, nu) and every (w, k) of a grid, the trial function
// exp(i (k x + w t)) on x, t in [-1, 1] is projected onto the element basis and relaxed once; the
// maps hold log10 of the residual norm N (Eq. residnorm) and of |S| (the action) after over before.
//
// Element rows (Eq. leastaction_dimensionless), test (j, m), trial (i, n), index i*Nt + n:
//   A = i O (x) Qt - 2 kappa K (x) U - nu O (x) U,
// O_ii = U_ii = 2/(2i+1), Qt[m][n] = 2 for n > m with n - m odd (int P_m P_n'), and
// K[j][i] = (j(j+1) - i(i+1))/2 for i > j with i - j even (Eq. Tmatelt's closed form, row = test).
// A relaxation solves A delta + B^T lambda = r, B delta = 0 (r = -A C; the constraints B fix the
// initial time, the ends of the relaxation volume and continuity between its elements) on the
// null space Z of B: delta = Z (Z^T A Z)^{-1} Z^T r.  The whole step is linear in C, so it is one
// matrix R per case, and the trial coefficients are linear in the element overlaps
// fhat = a(k) (x) b(w): C = Pi fhat.  With the four matrices (built once per case on the host,
// small dense algebra, n <= 128)
//   M0 = A Pi (= -r),  M1 = A R Pi (= -r after),  M2 = Pi (= C),  M3 = R Pi (= C after),
// N = |M0 fhat|_W^2 before and |M1 fhat|_W^2 after, S = (M2 fhat)^H (M0 fhat) before and
// (M3 fhat)^H (M1 fhat) after.  The residuals are formed as vectors, so a strong reduction of N
// costs no more digits than the residual itself (a precomputed quadratic form would square the
// cancellation).  On the GPU the matrices are contracted with b(w) over the time index once per
// (case, w); every k then needs four (n x Nel Nx) mat-vecs, accumulated row by row.
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/leastaction.h"
#include "la_internal.cuh"

namespace la {
void set_thread_error(const char* msg);
void gauss_legendre_rule(int q, double* x, double* w);

namespace {

typedef std::complex<double> cx;
constexpr int kLfaQuad = 48;     // quadrature nodes of the plane-wave overlaps
constexpr int kLfaMaxP = 16;     // (elements x Nx) at most

// ------------------------------------------------------------------ host dense algebra
struct Mat {
  int r = 0, c = 0;
  std::vector<cx> v;
  Mat() = default;
  Mat(int r_, int c_) : r(r_), c(c_), v((size_t)r_ * c_) {}
  cx& operator()(int i, int j) { return v[(size_t)i * c + j]; }
  cx operator()(int i, int j) const { return v[(size_t)i * c + j]; }
};
Mat mul(const Mat& a, const Mat& b) {
  Mat o(a.r, b.c);
  for (int i = 0; i < a.r; ++i)
    for (int k = 0; k < a.c; ++k) {
      const cx x = a(i, k);
      if (x == cx(0.0)) continue;
      for (int j = 0; j < b.c; ++j) o(i, j) += x * b(k, j);
    }
  return o;
}
Mat adj(const Mat& a) {   // conjugate transpose
  Mat o(a.c, a.r);
  for (int i = 0; i < a.r; ++i)
    for (int j = 0; j < a.c; ++j) o(j, i) = std::conj(a(i, j));
  return o;
}
Mat eye(int n) {
  Mat o(n, n);
  for (int i = 0; i < n; ++i) o(i, i) = 1.0;
  return o;
}
// X = M^{-1} Y by Gaussian elimination with partial pivoting; false when M is singular
bool solve(Mat M, Mat Y, Mat& X) {
  const int n = M.r;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(M(i, k)) > std::abs(M(p, k))) p = i;
    if (!(std::abs(M(p, k)) > 1e-300)) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(M(k, j), M(p, j));
      for (int j = 0; j < Y.c; ++j) std::swap(Y(k, j), Y(p, j));
    }
    const cx inv = 1.0 / M(k, k);
    for (int i = k + 1; i < n; ++i) {
      const cx l = M(i, k) * inv;
      if (l == cx(0.0)) continue;
      for (int j = k; j < n; ++j) M(i, j) -= l * M(k, j);
      for (int j = 0; j < Y.c; ++j) Y(i, j) -= l * Y(k, j);
    }
  }
  X = Mat(n, Y.c);
  for (int i = n - 1; i >= 0; --i)
    for (int j = 0; j < Y.c; ++j) {
      cx s = Y(i, j);
      for (int k = i + 1; k < n; ++k) s -= M(i, k) * X(k, j);
      X(i, j) = s / M(i, i);
    }
  return true;
}
// Orthonormal basis (columns) of the null space of the real rows B: Gram-Schmidt of B's rows,
// then of the unit vectors against them; repeated conditions drop out.
Mat null_space(const std::vector<std::vector<double>>& B, int n) {
  std::vector<std::vector<double>> basis;
  auto orth = [&](std::vector<double> v) -> std::vector<double> {
    for (int pass = 0; pass < 2; ++pass)
      for (const auto& q : basis) {
        double d = 0.0;
        for (int i = 0; i < n; ++i) d += q[i] * v[i];
        for (int i = 0; i < n; ++i) v[i] -= d * q[i];
      }
    return v;
  };
  auto nrm = [&](const std::vector<double>& v) {
    double s = 0.0;
    for (double x : v) s += x * x;
    return std::sqrt(s);
  };
  for (const auto& row : B) {
    const double n0 = nrm(row);
    std::vector<double> v = orth(row);
    const double n1 = nrm(v);
    if (n1 > 1e-10 * n0) {
      for (double& x : v) x /= n1;
      basis.push_back(v);
    }
  }
  const size_t rank = basis.size();
  for (int e = 0; e < n; ++e) {
    std::vector<double> v(n, 0.0);
    v[e] = 1.0;
    v = orth(v);
    const double n1 = nrm(v);
    if (n1 > 1e-6) {
      for (double& x : v) x /= n1;
      basis.push_back(v);
    }
  }
  Mat Z(n, (int)(basis.size() - rank));
  for (size_t k = rank; k < basis.size(); ++k)
    for (int i = 0; i < n; ++i) Z(i, (int)(k - rank)) = basis[k][i];
  return Z;
}

// ------------------------------------------------------------------ element operators
double leg(int n, double y) {
  double p0 = 1.0, p1 = y;
  if (n == 0) return p0;
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * y * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}
Mat element_operator(int nx, int nt, double kappa, double nu) {
  const int n = nx * nt;
  Mat A(n, n);
  for (int j = 0; j < nx; ++j)
    for (int m = 0; m < nt; ++m)
      for (int i = 0; i < nx; ++i)
        for (int q = 0; q < nt; ++q) {
          const double O = i == j ? 2.0 / (2 * i + 1) : 0.0;
          const double U = q == m ? 2.0 / (2 * q + 1) : 0.0;
          const double Qt = (q > m && (q - m) % 2 == 1) ? 2.0 : 0.0;
          const double K = (i > j && (i - j) % 2 == 0) ? 0.5 * (j * (j + 1) - i * (i + 1)) : 0.0;
          A(j * nt + m, i * nt + q) = cx(-2.0 * kappa * K * U - nu * O * U, O * Qt);
        }
  return A;
}
Mat block2(const Mat& a) {   // diag(a, a)
  Mat o(2 * a.r, 2 * a.c);
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < a.r; ++i)
      for (int j = 0; j < a.c; ++j) o(b * a.r + i, b * a.c + j) = a(i, j);
  return o;
}
// initial time in every element, the ends of the volume, continuity between its elements
std::vector<std::vector<double>> conditions(int nx, int nt, int nel, bool ends, bool initial) {
  const int n = nx * nt, N = nel * n;
  std::vector<std::vector<double>> B;
  if (initial)
    for (int e = 0; e < nel; ++e)
      for (int i = 0; i < nx; ++i) {
        std::vector<double> r(N, 0.0);
        for (int q = 0; q < nt; ++q) r[e * n + i * nt + q] = (q & 1) ? -1.0 : 1.0;   // P_q(-1)
        B.push_back(r);
      }
  for (int q = 0; q < nt; ++q) {
    if (ends) {
      std::vector<double> l(N, 0.0), rr(N, 0.0);
      for (int i = 0; i < nx; ++i) {
        l[i * nt + q] = (i & 1) ? -1.0 : 1.0;          // P_i(-1) at the left end of element 0
        rr[(nel - 1) * n + i * nt + q] = 1.0;          // P_i(+1) at the right end of the last one
      }
      B.push_back(l);
      B.push_back(rr);
    }
    for (int e = 0; e + 1 < nel; ++e) {
      std::vector<double> r(N, 0.0);
      for (int i = 0; i < nx; ++i) {
        r[e * n + i * nt + q] = 1.0;
        r[(e + 1) * n + i * nt + q] = (i & 1) ? 1.0 : -1.0;
      }
      B.push_back(r);
    }
  }
  return B;
}
Mat rowsT(const Mat& Z) { return adj(Z); }   // Z is real: Z^T
// R = I - Z (Z^T A Z)^{-1} Z^T A for the conditions B
bool relax_map(const Mat& A, const std::vector<std::vector<double>>& B, Mat& R) {
  const Mat Z = null_space(B, A.r);
  const Mat ZtA = mul(rowsT(Z), A);
  Mat X;
  if (!solve(mul(ZtA, Z), ZtA, X)) return false;
  const Mat ZX = mul(Z, X);
  R = eye(A.r);
  for (size_t t = 0; t < R.v.size(); ++t) R.v[t] -= ZX.v[t];
  return true;
}
// child coefficients of the parent's spatial functions (2 Nx x Nx) and the projection back
// (Nx x 2 Nx), P = (E^T Of E)^{-1} E^T Of, each extended over the time index
void transfers(int nx, int nt, Mat& I, Mat& P) {
  double y[kLfaQuad], w[kLfaQuad];
  gauss_legendre_rule(kLfaQuad, y, w);
  Mat E(2 * nx, nx);
  for (int s = 0; s < 2; ++s)
    for (int j = 0; j < nx; ++j)
      for (int i = 0; i < nx; ++i) {
        double acc = 0.0;
        for (int q = 0; q < kLfaQuad; ++q) acc += w[q] * leg(i, 0.5 * (y[q] + (s ? 1.0 : -1.0))) * leg(j, y[q]);
        E(s * nx + j, i) = acc * (2 * j + 1) / 2.0;
      }
  Mat EtOf(nx, 2 * nx);
  for (int i = 0; i < nx; ++i)
    for (int s = 0; s < 2; ++s)
      for (int j = 0; j < nx; ++j) EtOf(i, s * nx + j) = E(s * nx + j, i) * (2.0 / (2 * j + 1));
  Mat Ps;
  solve(mul(EtOf, E), EtOf, Ps);
  I = Mat(2 * nx * nt, nx * nt);
  P = Mat(nx * nt, 2 * nx * nt);
  for (int a = 0; a < 2 * nx; ++a)
    for (int b = 0; b < nx; ++b)
      for (int q = 0; q < nt; ++q) {
        I(a * nt + q, b * nt + q) = E(a, b);
        P(b * nt + q, a * nt + q) = Ps(b, a);
      }
}

struct CaseMats {
  int nel, nx, nt, n;
  std::vector<double2> G;   // [4][n][n]: the step matrices M0 .. M3
  std::vector<double> W;    // [n]: the diagonal weight O (x) U per element
};

bool build_case(const la_lfa_case& cs, CaseMats& out, std::string& why) {
  const int nx = cs.nx, nt = cs.nt;
  const int nel = cs.method == 0 ? 1 : 2, n = nel * nx * nt;
  const Mat A1 = element_operator(nx, nt, cs.kappa, cs.nu);
  const Mat A = nel == 1 ? A1 : block2(A1);
  Mat R;
  if (cs.method <= 1) {
    if (!relax_map(A, conditions(nx, nt, nel, true, true), R)) { why = "singular relaxation system"; return false; }
  } else {
    Mat I, P, R1, Rc;
    transfers(nx, nt, I, P);
    // coarse correction: delta = I Z (Z^T Ac Z)^{-1} Z^T P r, Ac = P A I, r = -A C
    const Mat Ac = mul(mul(P, A), I);
    const Mat Z = null_space(conditions(nx, nt, 1, true, true), nx * nt);
    const Mat ZtAc = mul(rowsT(Z), Ac);
    Mat X;
    if (!solve(mul(ZtAc, Z), mul(mul(rowsT(Z), P), A), X)) { why = "singular coarse system"; return false; }
    const Mat IZX = mul(mul(I, Z), X);
    Rc = eye(n);
    for (size_t t = 0; t < Rc.v.size(); ++t) Rc.v[t] -= IZX.v[t];
    if (!relax_map(A1, conditions(nx, nt, 1, true, true), R1)) { why = "singular relaxation system"; return false; }
    R = mul(block2(R1), Rc);
  }
  // trial projection Pi (real): W^{-1} on one element; continuity-constrained on two
  Mat Pi(n, n);
  std::vector<double> winv(n);
  for (int e = 0; e < nel; ++e)
    for (int i = 0; i < nx; ++i)
      for (int q = 0; q < nt; ++q) winv[(e * nx + i) * nt + q] = (2 * i + 1) * (2 * q + 1) / 4.0;
  if (nel == 1) {
    for (int t = 0; t < n; ++t) Pi(t, t) = winv[t];
  } else {
    // Pi = W^-1 - W^-1 Bc^T (Bc W^-1 Bc^T)^-1 Bc W^-1
    const auto Bc = conditions(nx, nt, 2, false, false);
    const int nc = (int)Bc.size();
    Mat BW(nc, n), S(nc, nc);
    for (int a = 0; a < nc; ++a)
      for (int t = 0; t < n; ++t) BW(a, t) = Bc[a][t] * winv[t];
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b) {
        double s = 0.0;
        for (int t = 0; t < n; ++t) s += Bc[a][t] * winv[t] * Bc[b][t];
        S(a, b) = s;
      }
    Mat Y;
    if (!solve(S, BW, Y)) { why = "singular continuity projection"; return false; }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        cx s = i == j ? cx(winv[i]) : cx(0.0);
        for (int a = 0; a < nc; ++a) s -= BW(a, i) * Y(a, j);
        Pi(i, j) = s;
      }
  }
  const Mat RPi = mul(R, Pi);
  const Mat mats[4] = {mul(A, Pi), mul(A, RPi), Pi, RPi};
  out.nel = nel;
  out.nx = nx;
  out.nt = nt;
  out.n = n;
  out.W.resize(n);
  for (int t = 0; t < n; ++t) out.W[t] = 1.0 / winv[t];
  out.G.resize((size_t)4 * n * n);
  for (int f = 0; f < 4; ++f)
    for (size_t t = 0; t < (size_t)n * n; ++t)
      out.G[(size_t)f * n * n + t] = make_double2(mats[f].v[t].real(), mats[f].v[t].imag());
  return true;
}

// ------------------------------------------------------------------ kernels
// overlaps a[k][e][i] = int exp(i k x_e(y)) P_i(y) dy (x_0 = y for one element; x_e = (y - 1)/2 + e
// for two) and b[w][n] = int exp(i w y) P_n(y) dy, by a Gauss-Legendre rule
__global__ void k_lfa_overlaps(const double* __restrict__ k, int nk, const double* __restrict__ w, int nw,
                               const double* __restrict__ qy, const double* __restrict__ qw, int nel, int nx, int nt,
                               double2* __restrict__ a, double2* __restrict__ b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nk + nw) return;
  const bool space = t < nk;
  const double kk = space ? k[t] : w[t - nk];
  const int nf = space ? nx : nt, ne = space ? nel : 1;
  for (int e = 0; e < ne; ++e) {
    double2 acc[8];
    for (int i = 0; i < 8; ++i) acc[i] = make_double2(0.0, 0.0);
    for (int q = 0; q < kLfaQuad; ++q) {
      const double y = qy[q];
      const double x = (space && nel == 2) ? 0.5 * (y - 1.0) + e : y;
      double s, c;
      sincos(kk * x, &s, &c);
      double p0 = 1.0, p1 = y;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        double p;
        if (i == 0) p = p0;
        else if (i == 1) p = p1;
        else {
          p = ((2.0 * i - 1.0) * y * p1 - (i - 1.0) * p0) / i;
          p0 = p1;
          p1 = p;
        }
        if (i < nf) { acc[i].x += qw[q] * p * c; acc[i].y += qw[q] * p * s; }
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < nf) {
        if (space) a[((size_t)t * nel + e) * nx + i] = acc[i];
        else b[(size_t)(t - nk) * nt + i] = acc[i];
      }
  }
}

// Mb[w][f][t][p] = sum_q M_f[t][(p, q)] b_q(w), p = e*Nx + i
__global__ void k_lfa_time(const double2* __restrict__ M, const double2* __restrict__ b, int n, int np, int nt,
                           double2* __restrict__ Mb) {
  const int wi = blockIdx.x;
  const double2* bw = b + (size_t)wi * nt;
  double2* out = Mb + (size_t)wi * 4 * n * np;
  for (int o = threadIdx.x; o < 4 * n * np; o += blockDim.x) {
    const int f = o / (n * np), tp = o % (n * np), t = tp / np, p = tp % np;
    const double2* row = M + ((size_t)f * n + t) * n + p * nt;
    double re = 0.0, im = 0.0;
    for (int q = 0; q < nt; ++q) {
      const double2 m = row[q], bq = bw[q];
      re += m.x * bq.x - m.y * bq.y;
      im += m.x * bq.y + m.y * bq.x;
    }
    out[o] = make_double2(re, im);
  }
}

// out[q][w][k]: log10 of N after / before (q = 0) and of |S| after / before (q = 1).  One CTA per
// (w, block of k); the contracted matrices of w and the weight sit in shared memory.
__global__ void k_lfa_eval(const double2* __restrict__ Mb, const double* __restrict__ W, const double2* __restrict__ a,
                           int nk, int nw, int n, int np, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  double2* sM = reinterpret_cast<double2*>(smem);              // [4][n][np]
  double* sW = reinterpret_cast<double*>(sM + (size_t)4 * n * np);
  const int wi = blockIdx.y;
  for (int t = threadIdx.x; t < 4 * n * np; t += blockDim.x) sM[t] = Mb[(size_t)wi * 4 * n * np + t];
  for (int t = threadIdx.x; t < n; t += blockDim.x) sW[t] = W[t];
  __syncthreads();
  const int ki = blockIdx.x * blockDim.x + threadIdx.x;
  if (ki >= nk) return;
  double2 av[kLfaMaxP];
#pragma unroll
  for (int p = 0; p < kLfaMaxP; ++p) av[p] = p < np ? a[(size_t)ki * np + p] : make_double2(0.0, 0.0);
  double N0 = 0.0, N1 = 0.0, S0r = 0.0, S0i = 0.0, S1r = 0.0, S1i = 0.0;
  for (int t = 0; t < n; ++t) {
    double2 v[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const double2* row = sM + ((size_t)f * n + t) * np;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int p = 0; p < kLfaMaxP; ++p) {
        if (p >= np) break;
        const double2 m = row[p];
        re += m.x * av[p].x - m.y * av[p].y;
        im += m.x * av[p].y + m.y * av[p].x;
      }
      v[f] = make_double2(re, im);
    }
    N0 += sW[t] * (v[0].x * v[0].x + v[0].y * v[0].y);
    N1 += sW[t] * (v[1].x * v[1].x + v[1].y * v[1].y);
    S0r += v[2].x * v[0].x + v[2].y * v[0].y;   // conj(C_t) (A C)_t
    S0i += v[2].x * v[0].y - v[2].y * v[0].x;
    S1r += v[3].x * v[1].x + v[3].y * v[1].y;
    S1i += v[3].x * v[1].y - v[3].y * v[1].x;
  }
  out[(size_t)wi * nk + ki] = log10(N1 / N0);
  out[((size_t)nw + wi) * nk + ki] = log10(hypot(S1r, S1i) / hypot(S0r, S0i));
}

}  // namespace
}  // namespace la

using namespace la;

extern "C" la_status la_lfa_maps(const la_lfa_case* cases, int ncases, const double* k, int nk, const double* w,
                                 int nw, void* out, void* cuda_stream) {
  if (!cases || ncases < 1 || !k || nk < 1 || !w || nw < 1 || !out) {
    set_thread_error("la_lfa_maps: null argument or empty grid");
    return LA_EINVAL;
  }
  for (int c = 0; c < ncases; ++c) {
    const la_lfa_case& cs = cases[c];
    if (cs.method < 0 || cs.method > 2 || cs.nx < 2 || cs.nx > 8 || cs.nt < 2 || cs.nt > 8) {
      set_thread_error("la_lfa_maps: method must be 0..2 and nx, nt in [2, 8]");
      return LA_EINVAL;
    }
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  static bool attr_set = false;
  if (!attr_set) {   // up to 4 x 128 x 16 complex128 (128 KB) of contracted matrices per CTA
    if (cudaFuncSetAttribute(k_lfa_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) != cudaSuccess) {
      cudaGetLastError();
      set_thread_error("la_lfa_maps: shared-memory attribute refused");
      return LA_ECUDA;
    }
    attr_set = true;
  }
  const size_t map_doubles = (size_t)2 * nw * nk;
  cudaPointerAttributes pa;
  const bool out_dev = cudaPointerGetAttributes(&pa, out) == cudaSuccess &&
                       (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  double qy[kLfaQuad], qw[kLfaQuad];
  gauss_legendre_rule(kLfaQuad, qy, qw);
  // the cases' step matrices, built on host threads (independent dense algebra per case)
  std::vector<CaseMats> mats(ncases);
  std::vector<std::string> why(ncases);
  std::vector<char> ok(ncases, 0);
  {
    const int nth = std::max(1, std::min(ncases, std::min(32, (int)std::thread::hardware_concurrency())));
    std::vector<std::thread> pool;
    for (int t = 0; t < nth; ++t)
      pool.emplace_back([&, t]() {
        for (int c = t; c < ncases; c += nth) ok[c] = build_case(cases[c], mats[c], why[c]) ? 1 : 0;
      });
    for (auto& th : pool) th.join();
  }
  for (int c = 0; c < ncases; ++c)
    if (!ok[c]) {
      set_thread_error(("la_lfa_maps: case " + std::to_string(c) + ": " + why[c]).c_str());
      return LA_EINVAL;
    }
  // all cases' matrices and weights in one upload (offsets in elements, 256-byte aligned)
  std::vector<size_t> goff(ncases), woff(ncases);
  size_t gtot = 0, wtot = 0;
  for (int c = 0; c < ncases; ++c) {
    goff[c] = gtot;
    gtot += (mats[c].G.size() + 15) & ~(size_t)15;
    woff[c] = wtot;
    wtot += (mats[c].W.size() + 31) & ~(size_t)31;
  }
  std::vector<double2> Gall(gtot);
  std::vector<double> Wall(wtot);
  for (int c = 0; c < ncases; ++c) {
    std::copy(mats[c].G.begin(), mats[c].G.end(), Gall.begin() + goff[c]);
    std::copy(mats[c].W.begin(), mats[c].W.end(), Wall.begin() + woff[c]);
  }
  void* buf = nullptr;
  // every sub-array starts on a 256-byte boundary (double2 accesses need 16-byte alignment)
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t off_k = 0, off_w = up(off_k + nk * sizeof(double)), off_qy = up(off_w + nw * sizeof(double));
  const size_t off_qw = up(off_qy + kLfaQuad * sizeof(double)), off_a = up(off_qw + kLfaQuad * sizeof(double));
  const size_t off_b = up(off_a + (size_t)nk * kLfaMaxP * sizeof(double2));
  const size_t off_g = up(off_b + (size_t)nw * 8 * sizeof(double2));
  const size_t off_wt = up(off_g + gtot * sizeof(double2));
  const size_t off_h = up(off_wt + wtot * sizeof(double));
  const size_t off_o = up(off_h + (size_t)nw * 4 * 128 * kLfaMaxP * sizeof(double2));
  const size_t total = off_o + (out_dev ? 0 : map_doubles * ncases * sizeof(double));
  if (cudaMalloc(&buf, total) != cudaSuccess) {
    cudaGetLastError();
    set_thread_error("la_lfa_maps: device allocation failed");
    return LA_ENOMEM;
  }
  unsigned char* B = static_cast<unsigned char*>(buf);
  cudaError_t e = cudaMemcpyAsync(B + off_k, k, nk * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B + off_w, w, nw * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B + off_qy, qy, sizeof(qy), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B + off_qw, qw, sizeof(qw), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B + off_g, Gall.data(), gtot * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B + off_wt, Wall.data(), wtot * sizeof(double), cudaMemcpyHostToDevice, s);
  double* maps = out_dev ? static_cast<double*>(out) : reinterpret_cast<double*>(B + off_o);
  double2* a = reinterpret_cast<double2*>(B + off_a);
  double2* b = reinterpret_cast<double2*>(B + off_b);
  double2* H = reinterpret_cast<double2*>(B + off_h);
  // the overlap tables and the contracted matrices are reused case after case in stream order
  int tab_nel = 0, tab_nx = 0, tab_nt = 0;
  for (int c = 0; c < ncases && e == cudaSuccess; ++c) {
    const CaseMats& F = mats[c];
    const int np = F.nel * F.nx;
    const double2* G = reinterpret_cast<const double2*>(B + off_g) + goff[c];
    const double* Wt = reinterpret_cast<const double*>(B + off_wt) + woff[c];
    if (F.nel != tab_nel || F.nx != tab_nx || F.nt != tab_nt) {
      k_lfa_overlaps<<<(nk + nw + 127) / 128, 128, 0, s>>>(reinterpret_cast<double*>(B + off_k), nk,
                                                           reinterpret_cast<double*>(B + off_w), nw,
                                                           reinterpret_cast<double*>(B + off_qy),
                                                           reinterpret_cast<double*>(B + off_qw), F.nel, F.nx, F.nt,
                                                           a, b);
      tab_nel = F.nel;
      tab_nx = F.nx;
      tab_nt = F.nt;
    }
    k_lfa_time<<<nw, 256, 0, s>>>(G, b, F.n, np, F.nt, H);
    const size_t smem = (size_t)4 * F.n * np * sizeof(double2) + F.n * sizeof(double);
    k_lfa_eval<<<dim3((nk + 127) / 128, nw), 128, smem, s>>>(H, Wt, a, nk, nw, F.n, np,
                                                            maps + (size_t)c * map_doubles);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !out_dev)
    e = cudaMemcpyAsync(out, maps, map_doubles * ncases * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return LA_ECUDA;
  }
  return LA_OK;
}
