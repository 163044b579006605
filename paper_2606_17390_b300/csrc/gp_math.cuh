// Device math shared by the sweep and adjoint kernels (internal): Mandel index helpers,
// the symmetric 3x3 Jacobi eigen-decomposition, the Mandel rotation, divided differences of
// 1/2 ln, and the FP64 hardening law.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "../../include/hfe.h"

namespace hfe {
namespace gpm {

constexpr double kSq23 = 0.81649658092772603273;   // sqrt(2/3)
constexpr double kSq2 = 1.41421356237309504880;
constexpr double kISq2 = 0.70710678118654752440;

// Mandel pair index helpers: p -> (i, j) and (i, j) -> p for the order 11,22,33,12,23,13.
__host__ __device__ constexpr int pI(int p) { return p < 3 ? p : (p == 4 ? 1 : 0); }
__host__ __device__ constexpr int pJ(int p) { return p < 3 ? p : (p == 3 ? 1 : 2); }
__host__ __device__ constexpr int pidx(int i, int j) {
  return i == j ? i : (i + j == 1 ? 3 : (i + j == 3 ? 4 : 5));
}

// packed index of the major-symmetric A_PQ (P = 3i + J, Q = 3k + L), upper triangle P <= Q
__host__ __device__ constexpr int asym(int P, int Q) {
  return P <= Q ? P * 9 - (P * (P - 1)) / 2 + (Q - P) : Q * 9 - (Q * (Q - 1)) / 2 + (P - Q);
}

template <typename R> struct Num;
template <> struct Num<float> {
  static constexpr float jac_eps2 = 1e-14f;   // Jacobi stop: off^2 <= eps2 * diag^2
  static constexpr float dd1_series = 1e-3f;  // |x| below which log1p(x)/x uses its series
  static constexpr float dd2_tau = 1e-2f;     // relative spread below which f2 uses f''(m)/2
  __device__ static float log1p_(float x) { return log1pf(x); }
  __device__ static float expm1_(float x) { return expm1f(x); }
  __device__ static float sqrt_(float x) { return sqrtf(x); }
  __device__ static float rsqrt_(float x) { return rsqrtf(x); }
  // FP32 quotients of the mixed path: the hardware reciprocal times a (within 2 ulp for the
  // normal-range divisors met here), far inside the mixed tolerances, instead of the
  // correctly rounded division with its slow-path branch
  __device__ static float div(float a, float b) { return __fdividef(a, b); }
};
template <> struct Num<double> {
  static constexpr double jac_eps2 = 1e-30;
  static constexpr double dd1_series = 1e-4;
  static constexpr double dd2_tau = 1e-5;
  __device__ static double log1p_(double x) { return log1p(x); }
  __device__ static double expm1_(double x) { return expm1(x); }
  __device__ static double sqrt_(double x) { return sqrt(x); }
  __device__ static double rsqrt_(double x) { return rsqrt(x); }
  __device__ static double div(double a, double b) { return a / b; }
};

// ----------------------------------------------------------------------------------------
// Symmetric 3x3 eigen-decomposition by the cyclic Jacobi method (Jacobi 1846, in the
// rotation form of Rutishauser): each rotation annihilates one off-diagonal entry; the
// off-diagonal norm falls quadratically.  Bounded to 10 sweeps.  Columns of V = eigenvectors.
template <typename R>
__device__ __forceinline__ void jacobi3(R A[3][3], R w[3], R V[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? R(1) : R(0);
  for (int sweep = 0; sweep < 10; ++sweep) {
    R off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    R dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= Num<R>::jac_eps2 * dia || off == R(0)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = (pq == 2) ? 1 : 0;
      const int q = (pq == 0) ? 1 : 2;
      const int r = 3 - p - q;
      R apq = A[p][q];
      if (apq != R(0)) {
        R theta = Num<R>::div(A[q][q] - A[p][p], R(2) * apq);
        R at = fabs(theta);
        R t = (at > R(1e15)) ? Num<R>::div(R(0.5), theta)
                             : Num<R>::div(theta >= R(0) ? R(1) : R(-1), at + Num<R>::sqrt_(theta * theta + R(1)));
        R c = Num<R>::rsqrt_(t * t + R(1));
        R s = t * c;
        A[p][p] -= t * apq;
        A[q][q] += t * apq;
        A[p][q] = A[q][p] = R(0);
        R arp = A[r][p], arq = A[r][q];
        A[r][p] = A[p][r] = c * arp - s * arq;
        A[r][q] = A[q][r] = s * arp + c * arq;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          R vp = V[k][p], vq = V[k][q];
          V[k][p] = c * vp - s * vq;
          V[k][q] = s * vp + c * vq;
        }
      }
    }
  }
  w[0] = A[0][0];
  w[1] = A[1][1];
  w[2] = A[2][2];
}

template <typename R>
__device__ __forceinline__ void swap_pair(R w[3], R V[3][3], int a, int b) {
  if (w[b] < w[a]) {
    R t = w[a]; w[a] = w[b]; w[b] = t;
#pragma unroll
    for (int k = 0; k < 3; ++k) { R v = V[k][a]; V[k][a] = V[k][b]; V[k][b] = v; }
  }
}

// Mandel rotation: for a symmetric X, (Q^T X Q)_M = Rm X_M with Mandel vectors
// (X11, X22, X33, sqrt2 X12, sqrt2 X23, sqrt2 X13).  Rm is orthogonal.
template <typename R>
__device__ __forceinline__ void mandel_rotation(const R Q[3][3], R Rm[6][6]) {
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int a = pI(p), b = pJ(p);
    const R so = (a != b) ? R(kSq2) : R(1);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int i = pI(q), j = pJ(q);
      if (i == j) Rm[p][q] = so * Q[i][a] * Q[i][b];
      else Rm[p][q] = so * R(kISq2) * (Q[i][a] * Q[j][b] + Q[j][a] * Q[i][b]);
    }
  }
}

// First divided difference of f(l) = 1/2 ln l at l_a = 1 + 2 e_a, l_b = 1 + 2 e_b, written as
// log1p(x) / (2 l_b x) with x = (l_a - l_b) / l_b, which has no cancellation; the limit is
// f'(l) = 1 / (2 l).
template <typename R>
__device__ __forceinline__ R dd1(R ea, R eb) {
  R lb = R(1) + R(2) * eb;
  R x = Num<R>::div(R(2) * (ea - eb), lb);
  R L;
  if (fabs(x) < Num<R>::dd1_series) L = R(1) + x * (R(-0.5) + x * (R(1) / R(3) + x * R(-0.25)));
  else L = Num<R>::div(Num<R>::log1p_(x), x);
  return Num<R>::div(L, R(2) * lb);
}

// Second divided difference of f(l) = 1/2 ln l on the sorted multiset l_i <= l_j <= l_k:
// (f[l_k, l_j] - f[l_j, l_i]) / (l_k - l_i); when the spread is below tau * l_j the value at
// the mean m, f''(m)/2 = -1/(4 m^2), which is exact to second order in the spread.
template <typename R>
__device__ __forceinline__ R dd2(R ei, R ej, R ek, R f_kj, R f_ji) {
  R li = R(1) + R(2) * ei, lj = R(1) + R(2) * ej;
  R den = R(2) * (ek - ei);
  if (den > Num<R>::dd2_tau * lj) return Num<R>::div(f_kj - f_ji, den);
  R m = lj + (R(2) / R(3)) * (ei + ek - R(2) * ej);
  (void)li;
  return Num<R>::div(R(-0.25), m * m);
}

// ----------------------------------------------------------------------------------------
// Small value types: the helpers below receive copies, never addresses, of material data
// (a uniform material record is a kernel parameter, whose address must not be taken).
struct Hard3 { double p0, p1, p2; };
struct Vec6d { double v[6]; };
struct Vec6f { float v[6]; };

// Hardening.  Plain FP64 evaluation (library pow / exp).
__device__ __forceinline__ void sigy64(int type, Hard3 hp, double a, double& sy, double& dsy) {
  if (type == HFE_HARDENING_SWIFT) {
    double z = hp.p1 + a;
    sy = hp.p0 * pow(z, hp.p2);
    dsy = hp.p2 * sy / z;
  } else {
    double e = exp(-hp.p2 * a);
    sy = hp.p0 + hp.p1 * (1.0 - e);
    dsy = hp.p1 * hp.p2 * e;
  }
}


// Scalar form of the closest-point projection.  With isotropic E and a deviatoric Hill
// tensor, E : H = 2 mu H, so the first row of Eq. local_cpp at the solution reads
// (I + (2 mu dgamma / phi_y) H) : T = T_tr with phi(T) = phi_y = sqrt(2/3) sigma_y(alpha_n+1);
// in the eigenbasis of H this is T_i = t_i / (1 + s h_i), s = 2 mu dgamma / phi_y, and the
// remaining unknown dgamma solves r(dgamma) = sqrt(sum h_i T_i^2) - phi_y(dgamma) = 0, which
// is strictly decreasing from r(0) = f_tr > 0; its root lies in (0, f_tr / (2 mu h_min)].
// Safeguarded Newton: a step that leaves the bracket is replaced by bisection.
struct RM {
  double dgamma;   // plastic multiplier
  double syn1;     // sigma_y(alpha_{n+1})
  float dsy;       // d sigma_y / d alpha at alpha_{n+1}
  int iters;
  bool ok;
};

// Plain FP64 form (every operation in FP64).
__device__ __forceinline__ RM return_map_fp64(const double t[6], const Vec6d hv, double mu, double hmin,
                              int type, Hard3 hp, double alpn, double ftr, int maxit,
                              double tol) {
  RM out;
  double dg = 0.0, lo = 0.0, hi = ftr / (2.0 * mu * hmin);
  double sy = 0.0, dsy = 0.0;
  int k = 0;
  bool ok = false;
  for (; k < maxit; ++k) {
    sigy64(type, hp, alpn + kSq23 * dg, sy, dsy);
    double phy = kSq23 * sy, dphy = (2.0 / 3.0) * dsy;
    double s = 2.0 * mu * dg / phy;
    double ds = 2.0 * mu * (phy - dg * dphy) / (phy * phy);
    double phi2 = 0.0, acc = 0.0;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
      double d = 1.0 + s * hv.v[i];
      double Ti = t[i] / d;
      double hT = hv.v[i] * Ti;
      phi2 += hT * Ti;
      acc += hT * hT / d;
    }
    double phi = sqrt(phi2);
    double r = phi - phy;
    if (fabs(r) <= tol * phy) { ok = true; break; }
    double dr = -(acc / phi) * ds - dphy;
    if (r > 0.0) lo = dg; else hi = dg;
    double dgn = dg - r / dr;
    if (!(dgn > lo && dgn < hi)) dgn = 0.5 * (lo + hi);
    if (fabs(dgn - dg) <= 1e-15 * dg) { dg = dgn; ok = true; break; }
    dg = dgn;
  }
  sigy64(type, hp, alpn + kSq23 * dg, sy, dsy);
  out.dgamma = dg;
  out.syn1 = sy;
  out.dsy = (float)dsy;
  out.iters = k + 1;
  out.ok = ok;
  return out;
}

}  // namespace gpm
}  // namespace hfe
