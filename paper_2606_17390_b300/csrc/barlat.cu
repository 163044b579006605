// Barlat Yld2004-18p material points: the yield function (Eq. Phi_barlat, App. A.2) and the
// closest-point projection on y = [T, alpha, dgamma] (Eq. local_cpp, Eq. local_solver) with the
// line search of App. B, for a batch of trial stresses.  One thread per material point.
//
// phi(T) = [1/4 sum_ij |a_i - b_j|^m]^(1/m), a_i and b_j the eigenvalues of s' = C' : P : T_l and
// s'' = C'' : P : T_l, T_l = Theta^T T Theta.  Both maps are linear in the six stress components,
// so the host folds Theta, P and C', C'' into two 6x6 tables LA, LB (component p of s' for a unit
// component b of T).  On the device:
// * s' and s'' are shifted by the same multiple of I (the sum only sees differences a_i - b_j)
//   and diagonalised by cyclic Jacobi; the differences are divided by D = max |a_i - b_j|, so S
//   stays in [1, 9] for any m and stress scale;
// * dphi/dT from dS/dA = sum_i g(a_i) n_i n_i, g(x) = m sum_j (x - b_j)^(m-1) (and likewise for
//   B), contracted with the tables;
// * the Hessian of phi from the Daleckii-Krein form of d(dS/dA): in the eigenbasis of A the
//   entry (i, k) is scaled by the divided difference g[a_i, a_k], which for a polynomial g is
//   the exact sum m sum_j sum_r (a_i - b_j)^r (a_k - b_j)^(m-2-r) (no cancellation, smooth
//   through repeated eigenvalues), plus the cross term -m(m-1) (a_i - b_j)^(m-2) between the
//   eigenvalue perturbations of A and B;
// * the 8x8 Newton system is reduced by block elimination (G_alpha is linear) to a 6x6 LU
//   with partial pivoting and two right-hand sides.
// The convergence test, the line search (Goldstein test, quadratic step model, eta safeguard,
// first model step tested before it is updated, last step taken when j_max is exhausted) and
// the iteration count follow App. B and App. C step by step.
//
// Precision.  FP64 runs every iteration in double.  B300 issues FP64 at a small fraction of
// the FP32 rate, so the mixed path runs the same iteration (line search included) in FP32 down
// to a scaled residual of 1e-5, about ten times the FP32 rounding floor, and finishes with at
// most six iterations from there whose residual, test and line search are FP64 and whose
// Newton matrix is formed in FP32; the elastic test is taken in FP32 outside a
// band of 1e-5 s around f_tr = 0 and in FP64 inside it.  The tangent is always formed in FP64
// at the returned state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "gp_math.cuh"
#include "hfe.h"
#include "hfe_internal.h"

namespace {

using hfe::gpm::jacobi3;
using hfe::gpm::pI;
using hfe::gpm::pJ;

constexpr int kThreads = 128;
// mixed precision: the FP32 phase runs until the scaled residual is below kTolSwitch (about
// ten times its FP32 rounding floor), then at most kPolishMax FP64 Newton iterations finish;
// an elastic test with |f_tr| <= kElasticBand * s is taken again in FP64
constexpr float kTolSwitch = 1e-5f;
constexpr float kElasticBand = 1e-5f;
constexpr int kPolishMax = 6;

// phase outcomes (the first five are the HFE_CPP_* codes)
constexpr int kConverged = HFE_CPP_CONVERGED, kElastic = HFE_CPP_ELASTIC, kMaxit = HFE_CPP_MAXIT,
              kSingular = HFE_CPP_SINGULAR, kNonfinite = HFE_CPP_NONFINITE, kAmbiguous = 6;

// X : Y = sum_p w(p) X_p Y_p over the six components
template <typename R>
__host__ __device__ constexpr R kWf(int p) { return p < 3 ? R(1) : R(2); }

template <typename R>
struct Scal {
  R lam, mu;        // Lame constants of the isotropic log-space elasticity
  R h0, h1, h2;     // hardening parameters
  R beta, eta;      // line-search constants
};

struct BarlatDev {
  double LA[6][6];  // LA[b][p]: component p of s' for a unit component b of the global stress
  double LB[6][6];  // the same for s''
  double EE[6][6];  // orthotropic E on components: (E : X)_p = sum_q EE[p][q] X_q
  float LAf[6][6], LBf[6][6], EEf[6][6];
  Scal<double> sd;
  Scal<float> sf;
  double tol;
  int m, hardening, kmax, jmax, line_search, precision, ortho;
};

template <typename R>
__device__ __forceinline__ R tabA(const BarlatDev& P, int b, int p) {
  if constexpr (sizeof(R) == 4) return P.LAf[b][p];
  else return P.LA[b][p];
}
template <typename R>
__device__ __forceinline__ R tabB(const BarlatDev& P, int b, int p) {
  if constexpr (sizeof(R) == 4) return P.LBf[b][p];
  else return P.LB[b][p];
}
template <typename R>
__device__ __forceinline__ R tabE(const BarlatDev& P, int p, int q) {
  if constexpr (sizeof(R) == 4) return P.EEf[p][q];
  else return P.EE[p][q];
}
template <typename R>
__device__ __forceinline__ const Scal<R>& scal(const BarlatDev& P) {
  if constexpr (sizeof(R) == 4) return P.sf;
  else return P.sd;
}

template <typename R>
__device__ __forceinline__ R sigma_y(const BarlatDev& P, R a, R* dsig) {
  const Scal<R>& c = scal<R>(P);
  if (P.hardening == HFE_HARDENING_SWIFT) {
    const R base = c.h1 + a;
    const R s = c.h0 * pow(base, c.h2);
    *dsig = c.h2 * s / base;
    return s;
  }
  const R e = exp(-c.h2 * a);
  *dsig = c.h1 * c.h2 * e;
  return c.h0 + c.h1 * (R(1) - e);
}

// x^k for a small non-negative integer k
template <typename R>
__device__ __forceinline__ R ipow(R x, int k) {
  R r = R(1);
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

// sum_{r=0}^{n} x^r y^(n-r)
template <typename R>
__device__ __forceinline__ R dd_sum(R x, R y, int n) {
  R p = R(1), yp = R(1);
  for (int k = 1; k <= n; ++k) {
    yp *= y;
    p = x * p + yp;
  }
  return p;
}

// Eigen data of one stress state.
template <typename R>
struct Spec {
  R a[3], b[3];
  R VA[3][3], VB[3][3];
  R D;     // max |a_i - b_j|
  R Sh;    // sum_ij ((a_i - b_j) / D)^m
  R phi;
};

// phi, and dphi/dT_b (component derivative: a shear component moves both symmetric entries).
// Returns false when phi = 0 (no deviatoric stress: N is undefined) or a value is not finite.
template <typename R>
__device__ __forceinline__ bool phi_grad(const BarlatDev& P, const R T[6], Spec<R>& s, R dphi[6]) {
  R sa[6], sb[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    R xa = R(0), xb = R(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      xa = fma(T[q], tabA<R>(P, q, p), xa);
      xb = fma(T[q], tabB<R>(P, q, p), xb);
    }
    sa[p] = xa;
    sb[p] = xb;
  }
  const R c = (sa[0] + sa[1] + sa[2] + sb[0] + sb[1] + sb[2]) * (R(1) / R(6));
  R A[3][3] = {{sa[0] - c, sa[3], sa[5]}, {sa[3], sa[1] - c, sa[4]}, {sa[5], sa[4], sa[2] - c}};
  R B[3][3] = {{sb[0] - c, sb[3], sb[5]}, {sb[3], sb[1] - c, sb[4]}, {sb[5], sb[4], sb[2] - c}};
  jacobi3<R>(A, s.a, s.VA);
  jacobi3<R>(B, s.b, s.VB);
  R D = R(0);
  bool nan = false;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R x = fabs(s.a[i] - s.b[j]);
      nan = nan || !(x == x);
      D = fmax(D, x);
    }
  s.D = D;
  if (nan || !(D > R(0)) || !isfinite(D)) {   // no deviatoric stress (phi = 0), or not finite
    const R v = (nan || !isfinite(D)) ? R(NAN) : R(0);
    s.Sh = v;
    s.phi = v;
#pragma unroll
    for (int p = 0; p < 6; ++p) dphi[p] = v;
    return false;
  }
  const int m = P.m;
  const R iD = R(1) / D;
  R Sh = R(0), ga[3] = {R(0), R(0), R(0)}, gb[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R t = (s.a[i] - s.b[j]) * iD;
      const R t1 = ipow<R>(t, m - 1);
      Sh = fma(t1, t, Sh);
      ga[i] += t1;
      gb[j] -= t1;
    }
  s.Sh = Sh;
  s.phi = D * pow(R(0.25) * Sh, R(1) / R(m));
  // (dS/da_i) / S = m ga_i / (D Sh); dphi = phi / m * dS / S
  const R f = s.phi * iD / Sh;
  R GA[6], GB[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int i = pI(p), j = pJ(p);
    GA[p] = ga[0] * s.VA[i][0] * s.VA[j][0] + ga[1] * s.VA[i][1] * s.VA[j][1] + ga[2] * s.VA[i][2] * s.VA[j][2];
    GB[p] = gb[0] * s.VB[i][0] * s.VB[j][0] + gb[1] * s.VB[i][1] * s.VB[j][1] + gb[2] * s.VB[i][2] * s.VB[j][2];
  }
#pragma unroll
  for (int b = 0; b < 6; ++b) {
    R x = R(0);
#pragma unroll
    for (int p = 0; p < 6; ++p) x += kWf<R>(p) * (GA[p] * tabA<R>(P, b, p) + GB[p] * tabB<R>(P, b, p));
    dphi[b] = f * x;
  }
  return true;
}

// (V^T X V) as 6 components for the symmetric X given by row b of a table
template <typename R, bool TAB_B>
__device__ __forceinline__ void rotate_row(const BarlatDev& P, int b, const R V[3][3], R out[6]) {
  R x[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) x[p] = TAB_B ? tabB<R>(P, b, p) : tabA<R>(P, b, p);
  const R X[3][3] = {{x[0], x[3], x[5]}, {x[3], x[1], x[4]}, {x[5], x[4], x[2]}};
  R XV[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) XV[r][k] = X[r][0] * V[0][k] + X[r][1] * V[1][k] + X[r][2] * V[2][k];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int i = pI(p), k = pJ(p);
    out[p] = V[0][i] * XV[0][k] + V[1][i] * XV[1][k] + V[2][i] * XV[2][k];
  }
}

// Hessian of phi in component space, H[b][c] = d^2 phi / dT_b dT_c, at a state with phi > 0.
template <typename R>
__device__ __forceinline__ void phi_hessian(const BarlatDev& P, const Spec<R>& s, const R dphi[6], R H[6][6]) {
  const int m = P.m;
  const R iD = R(1) / s.D;
  const R sc = R(m) * iD * iD / s.Sh;   // 1/S times the D^(m-2) of the sums below
  R t[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) t[i][j] = (s.a[i] - s.b[j]) * iD;
  // divided differences (over S) in the eigenbases, as 6 components (i, k)
  R HAA[6], HBB[6], HAB[3][3];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int i = pI(p), k = pJ(p);
    R xa = R(0), xb = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      xa += dd_sum<R>(t[i][j], t[k][j], m - 2);
      xb += dd_sum<R>(t[j][i], t[j][k], m - 2);
    }
    HAA[p] = sc * xa;
    HBB[p] = sc * xb;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) HAB[i][j] = -sc * R(m - 1) * ipow<R>(t[i][j], m - 2);
  // unit-component images in the eigenbases
  R XA[6][6], XB[6][6];
#pragma unroll
  for (int b = 0; b < 6; ++b) {
    rotate_row<R, false>(P, b, s.VA, XA[b]);
    rotate_row<R, true>(P, b, s.VB, XB[b]);
  }
  const R f = s.phi / R(m);
  R g[6];   // (dS/dT_b) / S
#pragma unroll
  for (int b = 0; b < 6; ++b) g[b] = dphi[b] / f;
  const R cm = R(1) / R(m) - R(1);
#pragma unroll
  for (int b = 0; b < 6; ++b)
#pragma unroll
    for (int c = b; c < 6; ++c) {
      R x = R(0);
#pragma unroll
      for (int p = 0; p < 6; ++p) x += kWf<R>(p) * (HAA[p] * XA[b][p] * XA[c][p] + HBB[p] * XB[b][p] * XB[c][p]);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) x += HAB[i][j] * (XA[b][i] * XB[c][j] + XA[c][i] * XB[b][j]);
      const R v = f * (x + cm * g[b] * g[c]);
      H[b][c] = v;
      H[c][b] = v;
    }
}

// E : X on components (isotropic lambda tr(X) I + 2 mu X, or the orthotropic table)
template <typename R>
__device__ __forceinline__ void elastic(const BarlatDev& P, const R X[6], R out[6]) {
  if (P.ortho) {
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      R v = R(0);
#pragma unroll
      for (int q = 0; q < 6; ++q) v = fma(tabE<R>(P, p, q), X[q], v);
      out[p] = v;
    }
    return;
  }
  const Scal<R>& c = scal<R>(P);
  const R tr = c.lam * (X[0] + X[1] + X[2]);
#pragma unroll
  for (int p = 0; p < 6; ++p) out[p] = R(2) * c.mu * X[p] + (p < 3 ? tr : R(0));
}

// G(y) of Eq. local_cpp; returns false if phi = 0 or a value is not finite.
template <typename R>
__device__ __forceinline__ bool residual(const BarlatDev& P, const R y[8], const R Ttr[6], R alpn, R G[8],
                                         Spec<R>& s, R dphi[6]) {
  const bool ok = phi_grad<R>(P, y, s, dphi);
  R N[6], EN[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) N[p] = dphi[p] / kWf<R>(p);
  elastic<R>(P, N, EN);
#pragma unroll
  for (int p = 0; p < 6; ++p) G[p] = y[p] - Ttr[p] + y[7] * EN[p];
  G[6] = y[6] - alpn - y[7];
  R ds;
  G[7] = s.phi - sigma_y<R>(P, y[6], &ds);
  bool fin = ok;
#pragma unroll
  for (int p = 0; p < 8; ++p) fin = fin && isfinite(G[p]);
  return fin;
}

// Gaussian elimination with partial pivoting on A (6x6) for NR right-hand sides X (6 x NR);
// returns false on a zero pivot.
template <typename R, int NR>
__device__ __forceinline__ bool lu_solve6(R A[6][6], R X[6][NR]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    int piv = k;
    R best = fabs(A[k][k]);
#pragma unroll
    for (int r = k + 1; r < 6; ++r)
      if (fabs(A[r][k]) > best) { best = fabs(A[r][k]); piv = r; }
    if (!(best > R(0))) return false;
    // row exchange with compile-time indices only (keeps A and X in registers)
#pragma unroll
    for (int r = k + 1; r < 6; ++r) {
      if (r == piv) {
#pragma unroll
        for (int c = 0; c < 6; ++c) { const R t = A[k][c]; A[k][c] = A[r][c]; A[r][c] = t; }
#pragma unroll
        for (int c = 0; c < NR; ++c) { const R t = X[k][c]; X[k][c] = X[r][c]; X[r][c] = t; }
      }
    }
    const R inv = R(1) / A[k][k];
#pragma unroll
    for (int r = k + 1; r < 6; ++r) {
      const R l = A[r][k] * inv;
#pragma unroll
      for (int c = k + 1; c < 6; ++c) A[r][c] -= l * A[k][c];
#pragma unroll
      for (int c = 0; c < NR; ++c) X[r][c] -= l * X[k][c];
    }
  }
#pragma unroll
  for (int k = 5; k >= 0; --k) {
    const R inv = R(1) / A[k][k];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      R v = X[k][c];
#pragma unroll
      for (int q = k + 1; q < 6; ++q) v -= A[k][q] * X[q][c];
      X[k][c] = v * inv;
    }
  }
  return true;
}

// A6 = dG_T/dT = I + dgamma E : dN/dT with dN_a/dT_c = H[a][c] / w_a
template <typename R>
__device__ __forceinline__ void build_A6(const BarlatDev& P, const R H[6][6], R dg, R A6[6][6]) {
  const Scal<R>& cs = scal<R>(P);
  if (P.ortho) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      R dN[6], EdN[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) dN[q] = H[q][c] / kWf<R>(q);
      elastic<R>(P, dN, EdN);
#pragma unroll
      for (int a = 0; a < 6; ++a) A6[a][c] = (a == c ? R(1) : R(0)) + dg * EdN[a];
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const R tr = cs.lam * (H[0][c] + H[1][c] + H[2][c]);
#pragma unroll
    for (int a = 0; a < 6; ++a)
      A6[a][c] = (a == c ? R(1) : R(0)) + dg * (R(2) * cs.mu * H[a][c] / kWf<R>(a) + (a < 3 ? tr : R(0)));
  }
}

template <typename R>
__device__ __forceinline__ R psi_of(const R G[8]) {
  R s = R(0);
#pragma unroll
  for (int p = 0; p < 8; ++p) s = fma(G[p], G[p], s);
  return R(0.5) * s;
}

// One precision phase of the closest-point projection: Newton on G(y) = 0 from y (updated in
// place) with the App. B line search, until the scaled residual is <= tol, or k reaches kend.
// elastic_test: 0 none, 1 f_tr <= 0 is elastic (the exact test, taken at the first
// evaluation), 2 banded (f_tr < -band elastic, |f_tr| <= band undecided: kAmbiguous).
//
// Every pass of the loop evaluates G at one trial point, so that the lanes of a warp, which
// sit at different stages of their own iterations, share that evaluation; a lane whose trial
// is accepted (or that starts) goes on, in the same pass, to its convergence test and its
// next Newton direction.  With the full step accepted, one Newton iteration is one pass.
// RJ: arithmetic of the Newton matrix (R, or float for the FP64 finish of the mixed path,
// where a Jacobian good to ~1e-7 still takes the residual from 1e-5 to the tolerance in the
// same two iterations; the residual, its test and the line search stay in R).
template <typename R, typename RJ = R>
__device__ __forceinline__ int cpp_phase(const BarlatDev& P, R y[8], const R Ttr[6], R alpn, R isref, R tol,
                                         int kend, int& k, int elastic_test) {
  const Scal<R>& cs = scal<R>(P);
  R dy[8];
  // trial of this pass: y itself (kAt), the full step (kFull), a line-search step (kLine)
  constexpr int kAt = 0, kFull = 1, kLine = 2;
  int mode = kAt;
  int j = 0;
  R z = R(1), psi0 = R(0);
#pragma unroll
  for (int p = 0; p < 8; ++p) dy[p] = R(0);
  const int guard = (kend - k + 1) * (P.jmax + 3) + 2;
  for (int it = 0; it < guard; ++it) {
    R yt[8], G[8], dphi[6];
    Spec<R> s;
    const R zt = (mode == kAt) ? R(0) : z;
#pragma unroll
    for (int p = 0; p < 8; ++p) yt[p] = fma(zt, dy[p], y[p]);
    const bool fin = residual<R>(P, yt, Ttr, alpn, G, s, dphi);
    if (mode != kAt) {
      const R psit = fin ? psi_of<R>(G) : R(INFINITY);
      const R zc = (mode == kFull) ? R(1) : z;
      if (!(psit < (R(1) - R(2) * cs.beta * zc) * psi0)) {   // Eq. goldstein_full fails
        if (mode == kFull) {
          z = psi0 / (psi0 + psit);                          // Eq. alpha_init
          mode = kLine;
          j = 0;
        } else {
          z = fmax(cs.eta * z, psi0 / (psi0 + psit));        // Eq. alpha_update_ls, Eq. alpha_safeguard
          if (++j > P.jmax) {                                // j_max exhausted: take the last step untested
#pragma unroll
            for (int p = 0; p < 8; ++p) y[p] = fma(z, dy[p], y[p]);
            mode = kAt;
          }
        }
        continue;
      }
      // the tested step is accepted: its residual is the new iterate's
#pragma unroll
      for (int p = 0; p < 8; ++p) y[p] = yt[p];
      mode = kAt;
    }
    if (elastic_test != 0) {   // elastic predictor test (App. C): f_tr = phi(T_tr) - sigma_y(alpha_n)
      const R f = G[7];
      const int et = elastic_test;
      elastic_test = 0;
      if (isfinite(f)) {
        if (et == 1 && f <= R(0)) return kElastic;
        if (et == 2) {
          const R band = R(kElasticBand) / isref;
          if (f < -band) return kElastic;
          if (f <= band) return kAmbiguous;
        }
      }
    }
    if (!fin) return kNonfinite;
    R r2 = R(0);
#pragma unroll
    for (int p = 0; p < 6; ++p) r2 += (G[p] * isref) * (G[p] * isref);
    r2 += G[6] * G[6] + (G[7] * isref) * (G[7] * isref);
    if (sqrt(r2) <= tol) return kConverged;
    if (k >= kend) return kMaxit;
    // Newton direction: J dy = -G by block elimination (G_alpha is linear in y)
    RJ H[6][6], A6[6][6], X[6][2], EN[6], N[6], dj[6];
    Spec<RJ> sj;
    if constexpr (sizeof(RJ) == sizeof(R)) {
      phi_hessian<RJ>(P, s, dphi, H);
#pragma unroll
      for (int p = 0; p < 6; ++p) dj[p] = dphi[p];
    } else {
      RJ yj[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) yj[p] = (RJ)y[p];
      if (!phi_grad<RJ>(P, yj, sj, dj)) return kSingular;
      phi_hessian<RJ>(P, sj, dj, H);
    }
    build_A6<RJ>(P, H, (RJ)y[7], A6);
#pragma unroll
    for (int p = 0; p < 6; ++p) N[p] = dj[p] / kWf<RJ>(p);
    elastic<RJ>(P, N, EN);
#pragma unroll
    for (int p = 0; p < 6; ++p) { X[p][0] = (RJ)G[p]; X[p][1] = EN[p]; }
    RJ hs;
    sigma_y<RJ>(P, (RJ)y[6], &hs);
    bool okj = lu_solve6<RJ, 2>(A6, X);
    RJ nx1 = RJ(0), nx2 = RJ(0);
#pragma unroll
    for (int p = 0; p < 6; ++p) { nx1 += dj[p] * X[p][0]; nx2 += dj[p] * X[p][1]; }
    const RJ den = nx2 + hs;
    okj = okj && den != RJ(0) && isfinite(den);
    if (!okj) return kSingular;
    const RJ ddg = ((RJ)G[7] + hs * (RJ)G[6] - nx1) / den;
#pragma unroll
    for (int p = 0; p < 6; ++p) dy[p] = (R)(-X[p][0] - X[p][1] * ddg);
    dy[6] = (R)ddg - G[6];
    dy[7] = (R)ddg;
    ++k;
    if (!P.line_search) {
#pragma unroll
      for (int p = 0; p < 8; ++p) y[p] += dy[p];
      continue;   // mode stays kAt: the next pass evaluates the new iterate
    }
    psi0 = psi_of<R>(G);
    z = R(1);
    mode = kFull;
  }
  return kMaxit;
}

// Per-point inputs shared by the kernels: the trial stress, alpha_n, whether they are finite,
// and 1/s of the convergence test, s = max(sigma_y(alpha_n), |T_tr|).
struct PointIn {
  double Ttr[6];
  double alpn;
  double isref;
  bool finite;
};

__device__ __forceinline__ void load_point(const BarlatDev& P, const double* __restrict__ Ttr_g,
                                           const double* __restrict__ alpn_g, int64_t pt, PointIn& q) {
#pragma unroll
  for (int p = 0; p < 6; ++p) q.Ttr[p] = Ttr_g[pt * 6 + p];
  q.alpn = alpn_g[pt];
  bool fin = isfinite(q.alpn);
#pragma unroll
  for (int p = 0; p < 6; ++p) fin = fin && isfinite(q.Ttr[p]);
  q.finite = fin;
  double ds0;
  double sref = sigma_y<double>(P, q.alpn, &ds0);
  double nt = 0.0;
#pragma unroll
  for (int p = 0; p < 6; ++p) nt = fma(q.Ttr[p], q.Ttr[p], nt);
  q.isref = 1.0 / fmax(sref, sqrt(nt));
}

__device__ __forceinline__ void store_point(int64_t pt, const double y[8], int k, int status,
                                            double* __restrict__ T_out, double* __restrict__ alpha_out,
                                            double* __restrict__ dg_out, int32_t* __restrict__ it_out,
                                            int8_t* __restrict__ st_out) {
#pragma unroll
  for (int p = 0; p < 6; ++p) T_out[pt * 6 + p] = y[p];
  alpha_out[pt] = y[6];
  dg_out[pt] = y[7];
  it_out[pt] = k;
  st_out[pt] = (int8_t)status;
}

// Persistent lane scheduling.  The grid holds as many threads as the GPU keeps resident;
// warp w owns the points [n w / W, n (w + 1) / W).  Each lane works on one point at a time
// for at most `chunk` Newton iterations per turn; a lane whose point is finished takes the
// next unclaimed point of its warp (ranked by a ballot), so that the lanes of a warp are not
// held by the slowest point of a fixed group.  A turn ends at a Newton iterate (cpp_phase
// returns kMaxit there when k reaches its bound), and the next turn starts from that iterate
// with the same state, so the result does not depend on `chunk`.
struct LaneSched {
  int64_t cursor, hi;
  int lane;
};

__device__ __forceinline__ LaneSched lane_sched(int64_t n) {
  const int64_t wid = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * kThreads) >> 5;
  LaneSched L;
  L.cursor = n * wid / W;
  L.hi = n * (wid + 1) / W;
  L.lane = threadIdx.x & 31;
  return L;
}

// Claims points for the lanes with pt == -1 (in lane order); pt = -2 once the warp's range
// is exhausted.  Returns false when every lane of the warp is done.  All 32 lanes call it.
__device__ __forceinline__ bool lane_claim(LaneSched& L, int64_t& pt) {
  const unsigned need = __ballot_sync(0xffffffffu, pt == -1);
  if (pt == -1) {
    const int64_t c = L.cursor + __popc(need & ((1u << L.lane) - 1u));
    pt = (c < L.hi) ? c : -2;
  }
  L.cursor += __popc(need);
  return !__all_sync(0xffffffffu, pt == -2);
}

// Mixed precision, first kernel: the FP32 phase (registers bounded for 5 resident blocks per
// SM: the spills cost less than the latency hidden by the extra warps, measured on the
// 16,000-point map and on a 64 times larger batch).  Its results go to the output arrays:
// kConverged (the scaled residual reached kTolSwitch; the FP64 finish follows), kElastic,
// kMaxit and kNonfinite (final), or kRestart (an undecided elastic test or an FP32 failure:
// the FP64 kernel starts this point again).
constexpr int kRestart = 5;

__global__ void __launch_bounds__(kThreads, 5) barlat_fp32_kernel(BarlatDev prm, const double* __restrict__ Ttr_g,
                                                               const double* __restrict__ alpn_g, int64_t n,
                                                               int chunk, double* __restrict__ T_out,
                                                               double* __restrict__ alpha_out,
                                                               double* __restrict__ dg_out,
                                                               int32_t* __restrict__ it_out,
                                                               int8_t* __restrict__ st_out) {
  __shared__ BarlatDev P;
  if (threadIdx.x == 0) P = prm;
  __syncthreads();
  LaneSched L = lane_sched(n);
  int64_t pt = -1;
  float yf[8], Tf[6], alf = 0.f, isf = 0.f;
  int k = 0, test = 0;
  bool fresh = true;   // the lane's point has not started a turn yet
  while (lane_claim(L, pt)) {
    if (pt < 0) continue;
    if (fresh) {
      PointIn q;
      load_point(P, Ttr_g, alpn_g, pt, q);
      if (!q.finite) {
        double y0[8];
#pragma unroll
        for (int p = 0; p < 6; ++p) y0[p] = q.Ttr[p];
        y0[6] = q.alpn;
        y0[7] = 0.0;
        store_point(pt, y0, 0, kNonfinite, T_out, alpha_out, dg_out, it_out, st_out);
        pt = -1;
        continue;
      }
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        Tf[p] = (float)q.Ttr[p];
        yf[p] = Tf[p];
      }
      alf = (float)q.alpn;
      yf[6] = alf;
      yf[7] = 0.f;
      isf = (float)q.isref;
      k = 0;
      test = 2;
      fresh = false;
    }
    const int k0 = k;
    const int r = cpp_phase<float>(P, yf, Tf, alf, isf, kTolSwitch, min(k + chunk, P.kmax), k, test);
    test = 0;
    if (r == kMaxit && k < P.kmax && k > k0) continue;   // end of a turn: the point goes on
    double y[8];
    int status;
    if (r == kConverged || r == kMaxit) {
#pragma unroll
      for (int p = 0; p < 8; ++p) y[p] = (double)yf[p];
      status = r;
    } else {
      PointIn q;
      load_point(P, Ttr_g, alpn_g, pt, q);
#pragma unroll
      for (int p = 0; p < 6; ++p) y[p] = q.Ttr[p];
      y[6] = q.alpn;
      y[7] = 0.0;
      status = (r == kElastic) ? kElastic : kRestart;
    }
    store_point(pt, y, k, status, T_out, alpha_out, dg_out, it_out, st_out);
    pt = -1;
    fresh = true;
  }
}

// FP64 kernel: the whole projection (full != 0: precision FP64), or the finish of the mixed
// path from the FP32 results in the output arrays (full == 0).  Elastic points get T = T_tr.
// Same lane scheduling as the FP32 kernel.  MINB: resident blocks per SM the register
// allocation is bounded for (3 for the whole FP64 projection, 1 for the short finish; both
// measured on the 16,000-point map and on a 64 times larger batch).  RJ: arithmetic of the
// Newton matrix (double for the FP64 projection, float for the finish of the mixed path).
template <int MINB, typename RJ>
__global__ void __launch_bounds__(kThreads, MINB) barlat_fp64_kernel(BarlatDev prm, const double* __restrict__ Ttr_g,
                                                               const double* __restrict__ alpn_g, int64_t n,
                                                               int full, int chunk, double* __restrict__ T_out,
                                                               double* __restrict__ alpha_out,
                                                               double* __restrict__ dg_out,
                                                               int32_t* __restrict__ it_out,
                                                               int8_t* __restrict__ st_out) {
  __shared__ BarlatDev P;
  if (threadIdx.x == 0) P = prm;
  __syncthreads();
  LaneSched L = lane_sched(n);
  int64_t pt = -1;
  PointIn q;
  double y[8];
  int k = 0, kend_pt = 0, test = 0;
  bool fresh = true;   // the lane's point has not started a turn yet
  while (lane_claim(L, pt)) {
    if (pt < 0) continue;
    if (fresh) {
      const int code = full ? kRestart : (int)st_out[pt];
      if (code == kMaxit || code == kNonfinite) {   // final after the FP32 phase
        pt = -1;
        continue;
      }
      load_point(P, Ttr_g, alpn_g, pt, q);
      if (code == kConverged) {   // FP64 Newton finish from the FP32 iterate
#pragma unroll
        for (int p = 0; p < 6; ++p) y[p] = T_out[pt * 6 + p];
        y[6] = alpha_out[pt];
        y[7] = dg_out[pt];
        k = it_out[pt];
        kend_pt = k + kPolishMax;
        test = 0;
      } else {
#pragma unroll
        for (int p = 0; p < 6; ++p) y[p] = q.Ttr[p];
        y[6] = q.alpn;
        y[7] = 0.0;
        k = 0;
        kend_pt = P.kmax;
        test = 1;
      }
      if (code == kElastic || !q.finite) {
        store_point(pt, y, 0, code == kElastic ? kElastic : kNonfinite, T_out, alpha_out, dg_out, it_out, st_out);
        pt = -1;
        continue;
      }
      fresh = false;
    }
    const int k0 = k;
    int status = cpp_phase<double, RJ>(P, y, q.Ttr, q.alpn, q.isref, P.tol, min(k + chunk, kend_pt), k, test);
    test = 0;
    if (status == kMaxit && k < kend_pt && k > k0) continue;   // end of a turn: the point goes on
    if (status == kElastic) {
#pragma unroll
      for (int p = 0; p < 6; ++p) y[p] = q.Ttr[p];
      y[6] = q.alpn;
      y[7] = 0.0;
    }
    store_point(pt, y, k, status, T_out, alpha_out, dg_out, it_out, st_out);
    pt = -1;
    fresh = true;
  }
}

// dT/dT_tr (App. D) at the state y, in FP64: J z = [e_c; 0; 0] for each component c (a shear
// component moving both symmetric entries).  Also returns N = dphi/dT (tensor components) at
// y.  False if phi = 0 or the system is singular.
__device__ __forceinline__ bool cpp_tangent(const BarlatDev& P, const double y[8], const double Ttr[6], double alpn,
                                            double Tg[6][6], double N[6]) {
  double G[8], dphi[6];
  Spec<double> s;
  if (!residual<double>(P, y, Ttr, alpn, G, s, dphi)) return false;
  double H[6][6], A6[6][6], X[6][7], EN[6];
  phi_hessian<double>(P, s, dphi, H);
  build_A6<double>(P, H, y[7], A6);
#pragma unroll
  for (int p = 0; p < 6; ++p) N[p] = dphi[p] / kWf<double>(p);
  elastic<double>(P, N, EN);
#pragma unroll
  for (int p = 0; p < 6; ++p) {
#pragma unroll
    for (int c = 0; c < 6; ++c) X[p][c] = (p == c) ? 1.0 : 0.0;
    X[p][6] = EN[p];
  }
  double hs;
  sigma_y<double>(P, y[6], &hs);
  if (!lu_solve6<double, 7>(A6, X)) return false;
  double nx2 = 0.0;
#pragma unroll
  for (int p = 0; p < 6; ++p) nx2 += dphi[p] * X[p][6];
  const double den = nx2 + hs;
  if (!(den != 0.0 && isfinite(den))) return false;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double nz = 0.0;
#pragma unroll
    for (int p = 0; p < 6; ++p) nz += dphi[p] * X[p][c];
    const double zg = nz / den;
#pragma unroll
    for (int a = 0; a < 6; ++a) Tg[a][c] = X[a][c] - X[a][6] * zg;
  }
  return true;
}

// dT/dT_tr at the returned state; the identity for elastic and failed points.
__global__ void __launch_bounds__(kThreads) barlat_tangent_kernel(BarlatDev prm, const double* __restrict__ Ttr_g,
                                                                  const double* __restrict__ alpn_g, int64_t n,
                                                                  const double* __restrict__ T_out,
                                                                  const double* __restrict__ alpha_out,
                                                                  const double* __restrict__ dg_out,
                                                                  const int8_t* __restrict__ st_out,
                                                                  double* __restrict__ tan_out) {
  __shared__ BarlatDev P;
  if (threadIdx.x == 0) P = prm;
  __syncthreads();
  const int64_t pt = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (pt >= n) return;
  const int status = st_out[pt];
  double Tg[6][6];
  bool okt = status == kConverged || status == kMaxit;
  if (okt) {
    PointIn q;
    load_point(P, Ttr_g, alpn_g, pt, q);
    double y[8], N[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) y[p] = T_out[pt * 6 + p];
    y[6] = alpha_out[pt];
    y[7] = dg_out[pt];
    okt = cpp_tangent(P, y, q.Ttr, q.alpn, Tg, N);
  }
  if (!okt) {
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = 0; c < 6; ++c) Tg[a][c] = (a == c) ? 1.0 : 0.0;
  }
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int c = 0; c < 6; ++c) tan_out[pt * 36 + a * 6 + c] = Tg[a][c];
}

// The strain-driven update of a hex8 sweep's Gauss points (App. C, Algorithm
// global_stress_update steps 2-6): a prep kernel forms T_tr = E : (eps - eps_p,n) and alpha_n
// from the Mandel log strain and the FP64 history [8][n_gp] (eps_p tensor components, alpha,
// sigma_y cache); the projection kernels of the batch run on them (FP32 phase and FP64 finish,
// or FP64, with lane refill); a post kernel recovers eps_p,n+1 = eps_p,n + dgamma N(T) and
// T = E : (eps - eps_p,n+1), and writes the trial history, the Mandel stress, the plastic
// flag and (tangent != 0) D = dT/deps = (dT/dT_tr) E in Mandel form.  Projections that end
// without convergence are counted in status->local_fail.
constexpr double kISq2d = 0.70710678118654752440, kSq2d = 1.41421356237309504880;

// history component c of Gauss point i in the handle's layout (H = double: [8][n_gp] with the
// sigma_y cache at row 7; H = float: [7][n_gp] and the FP64 cache after it, at byte 28 n_gp)
template <typename H>
__device__ __forceinline__ double* hist_cache(void* h, int64_t ng) {
  if constexpr (sizeof(H) == 8) return reinterpret_cast<double*>(h) + 7 * ng;
  else return reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(h) + 28 * ng);
}

template <typename H>
__global__ void __launch_bounds__(kThreads) barlat_gp_prep_kernel(BarlatDev prm, const double* __restrict__ eps_M,
                                                                  const H* __restrict__ hist, int64_t ng,
                                                                  double* __restrict__ Ttr_out,
                                                                  double* __restrict__ alpn_out) {
  __shared__ BarlatDev P;
  if (threadIdx.x == 0) P = prm;
  __syncthreads();
  const int64_t pt = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (pt >= ng) return;
  double ee[6], Ttr[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) ee[p] = eps_M[pt * 6 + p] * (p < 3 ? 1.0 : kISq2d) - (double)hist[p * ng + pt];
  elastic<double>(P, ee, Ttr);
#pragma unroll
  for (int p = 0; p < 6; ++p) Ttr_out[pt * 6 + p] = Ttr[p];
  alpn_out[pt] = (double)hist[6 * ng + pt];
}

template <typename H>
__global__ void __launch_bounds__(kThreads) barlat_gp_post_kernel(
    BarlatDev prm, const double* __restrict__ eps_M, const H* __restrict__ hist,
    const double* __restrict__ Ttr_g, const double* __restrict__ alpn_g, const double* __restrict__ Ty,
    const double* __restrict__ aly, const double* __restrict__ dgy, const int8_t* __restrict__ st_g, int64_t ng,
    H* __restrict__ hist_trial, double* __restrict__ T_M, double* __restrict__ D_M, uint8_t* __restrict__ pl,
    int tangent, hfe::DevStatus* __restrict__ status) {
  __shared__ BarlatDev P;
  if (threadIdx.x == 0) P = prm;
  __syncthreads();
  const int64_t pt = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (pt >= ng) return;
  double eps[6], epn[6], Ttr[6], ee[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    eps[p] = eps_M[pt * 6 + p] * (p < 3 ? 1.0 : kISq2d);
    epn[p] = (double)hist[p * ng + pt];
    Ttr[p] = Ttr_g[pt * 6 + p];
  }
  const double alpn = alpn_g[pt];
  const int st = st_g[pt];
  double T[6], epnew[6], alpha = alpn, Dc[6][6];
  bool plastic = false, ok = false;
  double Tg[6][6];
  if (st == kElastic) {
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      T[p] = Ttr[p];
      epnew[p] = epn[p];
    }
  } else {
    plastic = true;
    if (st != kConverged) atomicAdd(&status->local_fail, 1);
    double y[8], N[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) y[p] = Ty[pt * 6 + p];
    y[6] = aly[pt];
    y[7] = dgy[pt];
    ok = st != kNonfinite && cpp_tangent(P, y, Ttr, alpn, Tg, N);
    if (!ok) {
      atomicAdd(&status->nonfinite, 1);
#pragma unroll
      for (int p = 0; p < 6; ++p) N[p] = 0.0;
    }
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      epnew[p] = epn[p] + y[7] * N[p];
      ee[p] = eps[p] - epnew[p];
    }
    elastic<double>(P, ee, T);
    alpha = y[6];
  }
  if (tangent) {
    // D = Tg E (E alone when elastic): column q of E is E applied to the unit component q
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double eq[6], Eq[6];
#pragma unroll
      for (int p = 0; p < 6; ++p) eq[p] = (p == q) ? 1.0 : 0.0;
      elastic<double>(P, eq, Eq);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        double v = Eq[a];
        if (ok) {
          v = 0.0;
#pragma unroll
          for (int c = 0; c < 6; ++c) v += Tg[a][c] * Eq[c];
        }
        Dc[a][q] = v;
      }
    }
    // Mandel: D_M[p][q] = s_p Dc[p][q] / s_q, s = (1, 1, 1, sqrt2, sqrt2, sqrt2)
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int q = 0; q < 6; ++q)
        D_M[pt * 36 + a * 6 + q] = Dc[a][q] * (a < 3 ? 1.0 : kSq2d) * (q < 3 ? 1.0 : kISq2d);
  }
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    T_M[pt * 6 + p] = T[p] * (p < 3 ? 1.0 : kSq2d);
    hist_trial[p * ng + pt] = (H)epnew[p];
  }
  hist_trial[6 * ng + pt] = (H)alpha;
  double dsy;
  hist_cache<H>(hist_trial, ng)[pt] = sigma_y<double>(P, alpha, &dsy);
  pl[pt] = plastic ? 1 : 0;
}

__global__ void __launch_bounds__(kThreads) barlat_phi_kernel(BarlatDev prm, const double* __restrict__ T_g,
                                                              int64_t n, double* __restrict__ phi_out,
                                                              double* __restrict__ N_out) {
  __shared__ BarlatDev P;
  if (threadIdx.x == 0) P = prm;
  __syncthreads();
  const int64_t pt = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (pt >= n) return;
  double T[6], dphi[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) T[p] = T_g[pt * 6 + p];
  Spec<double> s;
  phi_grad<double>(P, T, s, dphi);
  phi_out[pt] = s.phi;
  if (N_out != nullptr) {
#pragma unroll
    for (int p = 0; p < 6; ++p) N_out[pt * 6 + p] = dphi[p] / kWf<double>(p);
  }
}

// ------------------------------------------------------------------------------ host side
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// The 6x6 matrix of App. A.2 on components (11, 22, 33, 12, 23, 13).
void transform6(const double c[9], double C[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 6; ++k) C[i][k] = 0.0;
  C[0][1] = -c[0]; C[0][2] = -c[1];
  C[1][0] = -c[2]; C[1][2] = -c[3];
  C[2][0] = -c[4]; C[2][1] = -c[5];
  C[3][3] = c[6]; C[4][4] = c[7]; C[5][5] = c[8];
}

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

constexpr int I6[6] = {0, 1, 2, 0, 1, 0}, J6[6] = {0, 1, 2, 1, 2, 2};   // component p -> (i, j)

hfe_status make_params(const hfe_barlat_material* mat, BarlatDev* P) {
  if (mat == nullptr) return HFE_EINVAL;
  if (mat->m < 2 || mat->m > HFE_BARLAT_MAX_M || (mat->m % 2) != 0) return HFE_EINVAL;
  if (!(mat->E > 0.0) || !(mat->nu > -1.0 && mat->nu < 0.5)) return HFE_EINVAL;
  if (mat->hardening != HFE_HARDENING_SWIFT && mat->hardening != HFE_HARDENING_VOCE) return HFE_EINVAL;
  if (!finite_all(mat->c1, 9) || !finite_all(mat->c2, 9) || !finite_all(mat->h, 3) || !finite_all(mat->Theta, 9))
    return HFE_EINVAL;
  if (mat->orthotropic != 0) {
    if (!finite_all(mat->d, 9)) return HFE_EINVAL;
    const int diag[6] = {0, 1, 2, 6, 7, 8};
    for (int t : diag)
      if (!(mat->d[t] > 0.0)) return HFE_EINVAL;
  }
  // Theta must be orthonormal (columns = material axes)
  const double* Q = mat->Theta;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double d = 0.0;
      for (int k = 0; k < 3; ++k) d += Q[k * 3 + a] * Q[k * 3 + b];
      if (std::fabs(d - (a == b ? 1.0 : 0.0)) > 1e-10) return HFE_EINVAL;
    }
  double C1[6][6], C2[6][6];
  transform6(mat->c1, C1);
  transform6(mat->c2, C2);
  for (int b = 0; b < 6; ++b) {
    // unit component b of the global stress (both symmetric entries for a shear component)
    double E[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    E[I6[b]][J6[b]] = 1.0;
    E[J6[b]][I6[b]] = 1.0;
    // T_l = Theta^T E Theta
    double Tl[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double v = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) v += Q[k * 3 + i] * E[k][l] * Q[l * 3 + j];
        Tl[i][j] = v;
      }
    double v6[6], s6[6];
    for (int p = 0; p < 6; ++p) v6[p] = Tl[I6[p]][J6[p]];
    const double mean = (v6[0] + v6[1] + v6[2]) / 3.0;
    for (int p = 0; p < 6; ++p) s6[p] = v6[p] - (p < 3 ? mean : 0.0);   // P : T_l
    for (int p = 0; p < 6; ++p) {
      double xa = 0.0, xb = 0.0;
      for (int q = 0; q < 6; ++q) {
        xa += C1[p][q] * s6[q];
        xb += C2[p][q] * s6[q];
      }
      P->LA[b][p] = xa;
      P->LB[b][p] = xb;
    }
  }
  for (int b = 0; b < 6; ++b)
    for (int p = 0; p < 6; ++p) {
      P->LAf[b][p] = (float)P->LA[b][p];
      P->LBf[b][p] = (float)P->LB[b][p];
    }
  P->sd.lam = mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu));
  P->sd.mu = mat->E / (2.0 * (1.0 + mat->nu));
  P->ortho = mat->orthotropic != 0;
  if (P->ortho) {
    // E_l from the nine coefficients (E1111, E2222, E3333, E1122, E1133, E2233, E1212, E2323,
    // E1313) with the minor and major symmetries; E_g,ijkl = Q_ia Q_jb Q_kc Q_ld E_l,abcd
    const double* d = mat->d;
    double El[3][3][3][3] = {};
    El[0][0][0][0] = d[0];
    El[1][1][1][1] = d[1];
    El[2][2][2][2] = d[2];
    const int na[3] = {0, 0, 1}, nb[3] = {1, 2, 2};
    const double dn[3] = {d[3], d[4], d[5]};
    const int sa[3] = {0, 1, 0}, sb[3] = {1, 2, 2};
    const double ds[3] = {d[6], d[7], d[8]};
    for (int t = 0; t < 3; ++t) {
      El[na[t]][na[t]][nb[t]][nb[t]] = El[nb[t]][nb[t]][na[t]][na[t]] = dn[t];
      const int a = sa[t], b = sb[t];
      El[a][b][a][b] = El[a][b][b][a] = El[b][a][a][b] = El[b][a][b][a] = ds[t];
    }
    for (int p = 0; p < 6; ++p)
      for (int q = 0; q < 6; ++q) {
        const int i = I6[p], j = J6[p], k = I6[q], l = J6[q];
        double v = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c)
              for (int e = 0; e < 3; ++e)
                v += Q[i * 3 + a] * Q[j * 3 + b] * Q[k * 3 + c] * Q[l * 3 + e] * El[a][b][c][e];
        // acting on components: the kl and lk entries of X both equal X_q
        P->EE[p][q] = v * (k == l ? 1.0 : 2.0);
        P->EEf[p][q] = (float)P->EE[p][q];
      }
  }
  P->sd.h0 = mat->h[0];
  // Voce as Eq. Hard prints it for this model: sigma0 + sqrt(2/3) Q (1 - exp(-b alpha))
  P->sd.h1 = mat->hardening == HFE_HARDENING_VOCE ? 0.81649658092772603273 * mat->h[1] : mat->h[1];
  P->sd.h2 = mat->h[2];
  P->m = mat->m;
  P->hardening = mat->hardening;
  return HFE_OK;
}

constexpr int kChunk = 8;   // Newton iterations per turn of the persistent kernels
constexpr int kMaxDevices = 64;
std::mutex g_occ_mutex;
int g_occ32[kMaxDevices] = {}, g_occ64[kMaxDevices] = {}, g_occ64f[kMaxDevices] = {};

// Blocks of the persistent kernels that the device keeps resident at once (SM count x
// blocks per SM), looked up once per device.
cudaError_t resident_blocks(int dev, int* g32, int* g64, int* g64f) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_occ_mutex);
  if (g_occ32[dev] == 0) {
    int sms = 0, b32 = 0, b64 = 0, b64f = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, barlat_fp32_kernel, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, barlat_fp64_kernel<3, double>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64f, barlat_fp64_kernel<1, float>, kThreads, 0);
    if (e != cudaSuccess) return e;
    g_occ32[dev] = std::max(1, sms * b32);
    g_occ64[dev] = std::max(1, sms * b64);
    g_occ64f[dev] = std::max(1, sms * b64f);
  }
  *g32 = g_occ32[dev];
  *g64 = g_occ64[dev];
  *g64f = g_occ64f[dev];
  return cudaSuccess;
}

hfe_status apply_options(const hfe_cpp_options* opt, BarlatDev* P) {
  hfe_cpp_options o;
  if (opt != nullptr) o = *opt;
  else hfe_default_cpp_options(&o);
  if (o.kmax < 0 || o.kmax > 100000 || o.jmax < 0 || o.jmax > 1000) return HFE_EINVAL;
  if (!(o.beta > 0.0 && o.beta < 0.5) || !(o.eta > 0.0 && o.eta < 1.0) || !(o.tol > 0.0)) return HFE_EINVAL;
  if (o.precision != HFE_PRECISION_FP64 && o.precision != HFE_PRECISION_MIXED) return HFE_EINVAL;
  P->kmax = o.kmax;
  P->jmax = o.jmax;
  P->line_search = o.line_search != 0;
  P->precision = o.precision;
  P->sd.beta = o.beta;
  P->sd.eta = o.eta;
  P->tol = o.tol;
  P->sf = Scal<float>{(float)P->sd.lam, (float)P->sd.mu, (float)P->sd.h0, (float)P->sd.h1,
                      (float)P->sd.h2, (float)P->sd.beta, (float)P->sd.eta};
  return HFE_OK;
}

// The projection of n trial states (FP32 phase and FP64 finish, or FP64) with lane refill
// once the batch exceeds the resident threads.
cudaError_t launch_projection(const BarlatDev& P, const double* Ttr, const double* alpn, int64_t n, double* T_out,
                              double* alpha_out, double* dg_out, int32_t* it_out, int8_t* st_out, cudaStream_t s) {
  const int64_t blocks = (n + kThreads - 1) / kThreads;
  int dev = 0, g32 = 0, g64 = 0, g64f = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = resident_blocks(dev, &g32, &g64, &g64f);
  if (e != cudaSuccess) return e;
  auto grid = [&](int resident) { return (unsigned)std::min<int64_t>(blocks, resident); };
  auto chunk = [&](int resident) { return blocks > resident ? kChunk : (1 << 30); };
  if (P.precision == HFE_PRECISION_MIXED) {
    barlat_fp32_kernel<<<grid(g32), kThreads, 0, s>>>(P, Ttr, alpn, n, chunk(g32), T_out, alpha_out, dg_out, it_out,
                                                      st_out);
    barlat_fp64_kernel<1, float><<<grid(g64f), kThreads, 0, s>>>(P, Ttr, alpn, n, 0, chunk(g64f), T_out, alpha_out, dg_out,
                                                          it_out, st_out);
  } else {
    barlat_fp64_kernel<3, double><<<grid(g64), kThreads, 0, s>>>(P, Ttr, alpn, n, 1, chunk(g64), T_out, alpha_out, dg_out,
                                                         it_out, st_out);
  }
  return cudaGetLastError();
}

}  // namespace

// ---- the Barlat material of a hex8 handle (internal interface, hfe_internal.h)
namespace hfe {
struct BarlatModel {
  BarlatDev P;
};

BarlatModel* barlat_model_new(const hfe_barlat_material* mat, const hfe_cpp_options* opt, hfe_status* st) {
  BarlatModel* m = new BarlatModel();
  *st = make_params(mat, &m->P);
  if (*st == HFE_OK) *st = apply_options(opt, &m->P);
  if (*st != HFE_OK) {
    delete m;
    return nullptr;
  }
  return m;
}

void barlat_model_free(BarlatModel* m) { delete m; }

void launch_barlat_gp(const BarlatModel* m, bool fp64_hist, const double* eps_M, const void* hist,
                      void* hist_trial, int64_t n_gp, double* T_M, double* D_M, uint8_t* plastic, int tangent,
                      DevStatus* status, double* work, int32_t* iters, int8_t* st, cudaStream_t s) {
  const unsigned blocks = (unsigned)((n_gp + kThreads - 1) / kThreads);
  if (blocks == 0) return;
  double* Ttr = work;                 // [n_gp*6]
  double* alpn = work + 6 * n_gp;     // [n_gp]
  double* Ty = work + 7 * n_gp;       // [n_gp*6]
  double* aly = work + 13 * n_gp;     // [n_gp]
  double* dgy = work + 14 * n_gp;     // [n_gp]
  if (fp64_hist)
    barlat_gp_prep_kernel<double><<<blocks, kThreads, 0, s>>>(m->P, eps_M, (const double*)hist, n_gp, Ttr, alpn);
  else
    barlat_gp_prep_kernel<float><<<blocks, kThreads, 0, s>>>(m->P, eps_M, (const float*)hist, n_gp, Ttr, alpn);
  launch_projection(m->P, Ttr, alpn, n_gp, Ty, aly, dgy, iters, st, s);
  if (fp64_hist)
    barlat_gp_post_kernel<double><<<blocks, kThreads, 0, s>>>(m->P, eps_M, (const double*)hist, Ttr, alpn, Ty, aly,
                                                              dgy, st, n_gp, (double*)hist_trial, T_M, D_M, plastic,
                                                              tangent, status);
  else
    barlat_gp_post_kernel<float><<<blocks, kThreads, 0, s>>>(m->P, eps_M, (const float*)hist, Ttr, alpn, Ty, aly, dgy,
                                                             st, n_gp, (float*)hist_trial, T_M, D_M, plastic, tangent,
                                                             status);
}
}  // namespace hfe

extern "C" void hfe_default_cpp_options(hfe_cpp_options* o) {
  if (o == nullptr) return;
  o->kmax = 40;
  o->line_search = 1;
  o->jmax = 10;
  o->beta = 1e-4;
  o->eta = 0.1;
  o->tol = 1e-13;
  o->precision = HFE_PRECISION_FP64;
}

extern "C" hfe_status hfe_barlat_phi(const hfe_barlat_material* mat, const double* T, int64_t n, double* phi_out,
                                     double* N_out, void* cuda_stream) {
  BarlatDev P{};
  hfe_status st = make_params(mat, &P);
  if (st != HFE_OK) return st;
  if (n < 0) return HFE_EINVAL;
  if (n == 0) return HFE_OK;
  if (T == nullptr || phi_out == nullptr) return HFE_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HFE_ECUDA;
  if (!on_device(T, dev) || !on_device(phi_out, dev) || (N_out != nullptr && !on_device(N_out, dev)))
    return HFE_EINVAL;
  const int64_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 0x7fffffffLL) return HFE_EINVAL;
  barlat_phi_kernel<<<(unsigned)blocks, kThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(P, T, n, phi_out,
                                                                                              N_out);
  return cudaGetLastError() == cudaSuccess ? HFE_OK : HFE_ECUDA;
}

extern "C" hfe_status hfe_barlat_return_map(const hfe_barlat_material* mat, const hfe_cpp_options* opt,
                                            const double* T_trial, const double* alpha_n, int64_t n,
                                            double* T_out, double* alpha_out, double* dgamma_out,
                                            int32_t* iters_out, int8_t* status_out, double* tangent_out,
                                            void* cuda_stream) {
  BarlatDev P{};
  hfe_status st = make_params(mat, &P);
  if (st != HFE_OK) return st;
  st = apply_options(opt, &P);
  if (st != HFE_OK) return st;
  if (n < 0) return HFE_EINVAL;
  if (n == 0) return HFE_OK;
  if (!T_trial || !alpha_n || !T_out || !alpha_out || !dgamma_out || !iters_out || !status_out) return HFE_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HFE_ECUDA;
  const void* ptrs[7] = {T_trial, alpha_n, T_out, alpha_out, dgamma_out, iters_out, status_out};
  for (const void* p : ptrs)
    if (!on_device(p, dev)) return HFE_EINVAL;
  if (tangent_out != nullptr && !on_device(tangent_out, dev)) return HFE_EINVAL;
  const int64_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 0x7fffffffLL) return HFE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (launch_projection(P, T_trial, alpha_n, n, T_out, alpha_out, dgamma_out, iters_out, status_out, s) !=
      cudaSuccess)
    return HFE_ECUDA;
  if (tangent_out != nullptr)
    barlat_tangent_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(P, T_trial, alpha_n, n, T_out, alpha_out,
                                                               dgamma_out, status_out, tangent_out);
  return cudaGetLastError() == cudaSuccess ? HFE_OK : HFE_ECUDA;
}
