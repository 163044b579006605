// Discrete adjoint of the load-step solve (paper Sec. 2.3: Lagrangian Eq. Lagrangian, adjoint
// equation Eq. dR_u, gradient Eq. main_grad, Algorithm adjoint_ad) with the history written out:
// states (u^n, h^n), R^n(u^n, h^{n-1}, theta) = 0 and h^n = H(u^n, h^{n-1}, theta).  With
// mu^N = 0, for n = N..1:
//   ubar   = dJ^n/du^n + (dH^n/du^n)^T mu^n                        (pass A)
//   K_n^T lambda^n = -ubar   (free dofs; FP64 CG, K_n symmetric; with the F-bar element
//                             K_n is not, and BiCGSTAB solves with its transposed blocks)
//   mu^{n-1} = (dR^n/dh^{n-1})^T lambda^n + (dH^n/dh^{n-1})^T mu^n  (passes A and B)
//   g += (dR^n/dtheta)^T lambda^n + (dH^n/dtheta)^T mu^n
// All per-Gauss-point partials are vector-Jacobian products of (P, h_new) with respect to
// (F, h_old, theta): the converged local return mapping is differentiated by the implicit
// function theorem on its 8-unknown system y = [T, alpha, dgamma] (App. D, applied in reverse:
// J_y^T w = (dz/dy)^T zbar, pbar = (dz/dp)^T zbar - (dG/dp)^T w), then through the geometric
// post-processor (first and second divided differences) and C = F^T F.  Everything in FP64.
//
// The forward pass runs in the handle's precision; on the mixed path each step ends with an
// FP64 Newton iteration (FP64 tangent, FP64 CG) and the FP64 history at the polished
// displacement, so that the linearisation point of the adjoint is FP64-accurate.
// History checkpoints are kept every ckpt_every steps and recomputed in between (one FP64
// residual sweep per step, no linear solve, since h^n = H(u^n, h^{n-1}, theta)).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "gp_math.cuh"
#include "handle.h"

namespace hfe {
namespace {

using namespace gpm;

constexpr int kAdjEl = 8;          // elements per CTA
constexpr int kAdjThreads = 64;    // 8 elements x 8 Gauss points
constexpr int kGpW = 44;           // shared doubles per Gauss point: Fbar 9, g 24, thetabar 11

struct VjpArgs {
  const double* X;
  const int32_t* conn;
  const double* u;
  const double* hist;        // FP64 history [8][n_gp] at t_{n-1}
  const MatRec* mat;
  int mat_per_element;
  int hardening;
  const double* theta;       // [n_mat][11]
  const double* Theta;       // [n_mat][9] or nullptr
  const int32_t* elems;
  const int32_t* slot;
  const double* lam;         // pass B: adjoint solution [n_dof]
  const double* mu;          // pass A: history cotangent [7][n_gp]
  double* ubar;              // pass A: nodal cotangent (first launch stores, later launches add)
  double* hbar;              // [7][n_gp]: pass A writes, pass B adds
  double* thbar;             // [n_el][11], accumulated
  DevStatus* status;
  int64_t n_gp;
  int local_maxit;
  double local_tol;
  int fbar;                  // F-bar element (Eq. Fbar)
};

// d sigma_y / d(h1, h2, h3) at alpha: Swift (K, eps0, n), Voce (sigma0, Q, b)
__device__ __forceinline__ void sigy_dtheta(int type, Hard3 hp, double a, double d[3]) {
  if (type == HFE_HARDENING_SWIFT) {
    const double z = hp.p1 + a, zn = pow(z, hp.p2);
    d[0] = zn;
    d[1] = hp.p0 * hp.p2 * zn / z;
    d[2] = hp.p0 * zn * log(z);
  } else {
    const double e = exp(-hp.p2 * a);
    d[0] = 1.0;
    d[1] = 1.0 - e;
    d[2] = hp.p1 * a * e;
  }
}

// E v for the isotropic Mandel elasticity E = lambda m m^T + 2 mu I
__device__ __forceinline__ void iso_apply(double lam, double mu, const double v[6], double o[6]) {
  const double tr = v[0] + v[1] + v[2];
#pragma unroll
  for (int p = 0; p < 6; ++p) o[p] = 2.0 * mu * v[p] + (p < 3 ? lam * tr : 0.0);
}

// symmetric 3x3 (tensor components) <-> Mandel vector
__device__ __forceinline__ void to_mandel(const double A[3][3], double v[6]) {
#pragma unroll
  for (int p = 0; p < 6; ++p) v[p] = (pI(p) == pJ(p)) ? A[pI(p)][pJ(p)] : kSq2 * A[pI(p)][pJ(p)];
}
__device__ __forceinline__ void from_mandel(const double v[6], double A[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[i][j] = (i == j) ? v[pidx(i, j)] : kISq2 * v[pidx(i, j)];
}
// B = Q^T A Q and A = Q B Q^T for symmetric A
__device__ __forceinline__ void rot_in(const double Q[3][3], const double A[3][3], double B[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) s += Q[i][a] * A[i][j] * Q[j][b];
      B[a][b] = s;
    }
}
__device__ __forceinline__ void rot_out(const double Q[3][3], const double B[3][3], double A[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) s += Q[i][a] * B[a][b] * Q[j][b];
      A[i][j] = s;
    }
}

// Gaussian elimination with partial pivoting: solves M x = b in place (n = 8)
__device__ __forceinline__ bool solve8(double M[8][8], double b[8]) {
  for (int k = 0; k < 8; ++k) {
    int piv = k;
    double best = fabs(M[k][k]);
    for (int r = k + 1; r < 8; ++r)
      if (fabs(M[r][k]) > best) { best = fabs(M[r][k]); piv = r; }
    if (!(best > 0.0)) return false;
    if (piv != k) {
      for (int c = 0; c < 8; ++c) { double t = M[k][c]; M[k][c] = M[piv][c]; M[piv][c] = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    const double inv = 1.0 / M[k][k];
    for (int r = k + 1; r < 8; ++r) {
      const double f = M[r][k] * inv;
      if (f != 0.0) {
        for (int c = k; c < 8; ++c) M[r][c] -= f * M[k][c];
        b[r] -= f * b[k];
      }
    }
  }
  for (int k = 7; k >= 0; --k) {
    double s = b[k];
    for (int c = k + 1; c < 8; ++c) s -= M[k][c] * b[c];
    b[k] = s / M[k][k];
  }
  return true;
}

template <bool PASS_A>
__global__ void __launch_bounds__(kAdjThreads) gp_vjp_kernel(VjpArgs a, int64_t cbeg, int64_t ccount) {
  __shared__ double sNode[kAdjEl][8][9];        // dX(3), du(3), lambda(3) per node
  __shared__ double sGp[kAdjEl][8][kGpW];       // Fbar(9), g(24), thetabar(11) per Gauss point
  const int tid = threadIdx.x, le = tid >> 3, g = tid & 7;
  const int64_t li = (int64_t)blockIdx.x * kAdjEl + le;
  const bool valid = li < ccount;
  const int e = valid ? a.elems[cbeg + li] : 0;
  const unsigned lane = tid & 31, gmask = 0xffu << (lane & 24);
  const int64_t ng = a.n_gp, gpi = (int64_t)e * 8 + g;
  {
    const int node = valid ? a.conn[(int64_t)e * 8 + g] : 0;
    double x[3], u[3], l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c] = a.X[3 * (int64_t)node + c];
      u[c] = a.u[3 * (int64_t)node + c];
      l[c] = PASS_A ? 0.0 : a.lam[3 * (int64_t)node + c];
    }
    const int src = lane & 24;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x0 = __shfl_sync(gmask, x[c], src), u0 = __shfl_sync(gmask, u[c], src);
      sNode[le][g][c] = x[c] - x0;
      sNode[le][g][3 + c] = u[c] - u0;
      sNode[le][g][6 + c] = l[c];
    }
  }
  __syncwarp(gmask);
  int flag_local = 0;
  if (valid) {
    const double(*nd)[9] = sNode[le];
    // kinematics (as in the sweep, FP64)
    const double c3 = 0.57735026918962576451;
    const double xg = (g & 1) ? c3 : -c3, yg = (g & 2) ? c3 : -c3, zg = (g & 4) ? c3 : -c3;
    double dN[8][3];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const double xa = (n == 1 || n == 2 || n == 5 || n == 6) ? 1.0 : -1.0;
      const double ya = (n == 2 || n == 3 || n == 6 || n == 7) ? 1.0 : -1.0;
      const double za = (n >= 4) ? 1.0 : -1.0;
      const double fx = 1.0 + xa * xg, fy = 1.0 + ya * yg, fz = 1.0 + za * zg;
      dN[n][0] = 0.125 * xa * fy * fz;
      dN[n][1] = 0.125 * ya * fx * fz;
      dN[n][2] = 0.125 * za * fx * fy;
    }
    double J0[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
#pragma unroll
        for (int n = 1; n < 8; ++n) s += nd[n][i] * dN[n][j];
        J0[i][j] = s;
      }
    const double c00 = J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1];
    const double c01 = J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2];
    const double c02 = J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0];
    const double det0 = J0[0][0] * c00 + J0[0][1] * c01 + J0[0][2] * c02;
    const double id = 1.0 / det0;
    double Ji[3][3];
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2]) * id;
    Ji[1][1] = (J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0]) * id;
    Ji[2][1] = (J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1]) * id;
    Ji[0][2] = (J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1]) * id;
    Ji[1][2] = (J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2]) * id;
    Ji[2][2] = (J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0]) * id;
    double gN[8][3];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int k = 0; k < 3; ++k) gN[n][k] = dN[n][0] * Ji[0][k] + dN[n][1] * Ji[1][k] + dN[n][2] * Ji[2][k];
    double H[3][3], F[3][3], Em[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
#pragma unroll
        for (int n = 1; n < 8; ++n) s += nd[n][3 + i] * gN[n][j];
        H[i][j] = s;
        F[i][j] = s + (i == j ? 1.0 : 0.0);
      }
    // F-bar element (Eq. Fbar), as in the sweep: Jbar - 1 = sum_q det J0_q (J_q - 1) / V_e over
    // the element's 8 threads, s = (Jbar / J)^(1/3), and the constitutive chain below runs on
    // s F.  The standard F, J and the element sums are kept for the pull-back in pass A.
    double F0[3][3], fb_s = 1.0, fb_jbar = 1.0, fb_j = 1.0, fb_det0 = det0, fb_vol = 1.0;
    if (a.fbar) {
      const double I1 = H[0][0] + H[1][1] + H[2][2];
      const double I2 = H[0][0] * H[1][1] + H[1][1] * H[2][2] + H[0][0] * H[2][2] - H[0][1] * H[1][0] -
                        H[1][2] * H[2][1] - H[0][2] * H[2][0];
      const double I3 = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                        H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                        H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
      const double jm1 = I1 + I2 + I3;
      double wj = det0 * jm1, wv = det0;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        wj += __shfl_xor_sync(gmask, wj, o);
        wv += __shfl_xor_sync(gmask, wv, o);
      }
      const double jbm1 = wj / wv;
      const double sm1 = expm1((log1p(jbm1) - log1p(jm1)) * (1.0 / 3.0));
      fb_s = 1.0 + sm1;
      fb_jbar = 1.0 + jbm1;
      fb_j = 1.0 + jm1;
      fb_vol = wv;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          F0[i][j] = F[i][j];
          H[i][j] += sm1 * F[i][j];
          F[i][j] *= fb_s;
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        double s = H[i][j] + H[j][i];
#pragma unroll
        for (int k = 0; k < 3; ++k) s += H[k][i] * H[k][j];
        Em[i][j] = Em[j][i] = 0.5 * s;
      }
    double ev[3], Q[3][3];
    jacobi3<double>(Em, ev, Q);
    swap_pair<double>(ev, Q, 0, 1);
    swap_pair<double>(ev, Q, 1, 2);
    swap_pair<double>(ev, Q, 0, 1);
    double epsM[6];
    {
      double epa[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) epa[k] = 0.5 * log1p(2.0 * ev[k]);
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int i = pI(p), j = pJ(p);
        const double s = Q[i][0] * epa[0] * Q[j][0] + Q[i][1] * epa[1] * Q[j][1] + Q[i][2] * epa[2] * Q[j][2];
        epsM[p] = (i == j) ? s : kSq2 * s;
      }
    }
    // return mapping (FP64, as the FP64 sweep)
    const int mi = a.mat_per_element ? e : 0;
    const MatRec& m = a.mat[mi];
    const double* th = a.theta + (int64_t)mi * 11;
    double epn[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) epn[c] = a.hist[c * ng + gpi];
    const double alpn = a.hist[6 * ng + gpi];
    double ee[6], Ttr[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) ee[p] = epsM[p] - (p < 3 ? epn[p] : kSq2 * epn[p]);
    iso_apply(m.lam, m.mu, ee, Ttr);
    double t[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < 6; ++i) s += m.QH[i * 6 + j] * Ttr[i];
      t[j] = s;
    }
    const Hard3 hp3{m.hard[0], m.hard[1], m.hard[2]};
    Vec6d hv;
#pragma unroll
    for (int i = 0; i < 6; ++i) hv.v[i] = m.h[i];
    double syn, dsyn;
    sigy64(a.hardening, hp3, alpn, syn, dsyn);
    double phi2 = 0.0;
#pragma unroll
    for (int i = 1; i < 6; ++i) phi2 += hv.v[i] * t[i] * t[i];
    const double ftr = sqrt(phi2) - kSq23 * syn;
    const bool plastic = ftr > 0.0;
    RM rm;
    rm.dgamma = 0.0; rm.syn1 = syn; rm.dsy = (float)dsyn; rm.iters = 0; rm.ok = true;
    double dsy1 = dsyn;
    if (plastic) {
      rm = return_map_fp64(t, hv, m.mu, m.hmin, a.hardening, hp3, alpn, ftr, a.local_maxit, a.local_tol);
      double sy_tmp;
      sigy64(a.hardening, hp3, alpn + kSq23 * rm.dgamma, sy_tmp, dsy1);
    }
    flag_local = rm.ok ? 0 : 1;
    const double dg = rm.dgamma;
    const double alpha1 = alpn + kSq23 * dg;
    const double phy = kSq23 * rm.syn1;
    double TM[6], NM[6];
    {
      double Teig[6], neig[6];
      const double s_pl = plastic ? 2.0 * m.mu * dg / phy : 0.0;
      Teig[0] = t[0];
      neig[0] = 0.0;
#pragma unroll
      for (int i = 1; i < 6; ++i) {
        Teig[i] = t[i] / (1.0 + s_pl * hv.v[i]);
        neig[i] = hv.v[i] * Teig[i] / phy;
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        double s1 = 0.0, s2 = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) { s1 += m.QH[i * 6 + j] * Teig[j]; s2 += m.QH[i * 6 + j] * neig[j]; }
        TM[i] = s1;
        NM[i] = s2;
      }
    }
    // post-processor: Shat = 2 f1 o That, S = Q Shat Q^T, P = F S
    double f1[3][3], f2[3][3][3];
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
      for (int bb = aa; bb < 3; ++bb) {
        const double v = (aa == bb) ? 0.5 / (1.0 + 2.0 * ev[aa]) : dd1<double>(ev[bb], ev[aa]);
        f1[aa][bb] = f1[bb][aa] = v;
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
#pragma unroll
        for (int k = j; k < 3; ++k) {
          const double v = dd2<double>(ev[i], ev[j], ev[k], f1[k][j], f1[j][i]);
          f2[i][j][k] = f2[i][k][j] = f2[j][i][k] = f2[j][k][i] = f2[k][i][j] = f2[k][j][i] = v;
        }
    double Tt[3][3], That[3][3], Shat[3][3], S[3][3];
    from_mandel(TM, Tt);
    rot_in(Q, Tt, That);
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) Shat[aa][bb] = 2.0 * f1[aa][bb] * That[aa][bb];
    rot_out(Q, Shat, S);

    // ---------------- reverse sweep of one Gauss point ----------------
    double Pbar[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (!PASS_A) {   // R_a = w detJ0 P g_a  ->  Pbar = w detJ0 sum_a lambda_a (x) g_a
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J) {
          double s = 0.0;
#pragma unroll
          for (int n = 0; n < 8; ++n) s += nd[n][6 + i] * gN[n][J];
          Pbar[i][J] = det0 * s;
        }
    }
    double mu_ep[6] = {0, 0, 0, 0, 0, 0}, mu_al = 0.0;
    if (PASS_A) {
#pragma unroll
      for (int c = 0; c < 6; ++c) mu_ep[c] = a.mu[c * ng + gpi] * (c < 3 ? 1.0 : kISq2);   // Mandel cotangent
      mu_al = a.mu[6 * ng + gpi];
    }
    // P = F S: Fbar = Pbar S, Sbar = sym(F^T Pbar)
    double Fbar[3][3], Sbar[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double s = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          s += Pbar[i][k] * S[k][j];
          s2 += F[k][i] * Pbar[k][j];
          s3 += F[k][j] * Pbar[k][i];
        }
        Fbar[i][j] = s;
        Sbar[i][j] = 0.5 * (s2 + s3);
      }
    // S = 2 Deps(C)[T]: Tbar = 2 Deps[Sbar]; Cbar = 2 D2eps[T, Sbar] (eigenbasis of C)
    double Sbh[3][3], Tbh[3][3], Cbh[3][3], Tbar[3][3], TbarM[6];
    rot_in(Q, Sbar, Sbh);
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        Tbh[aa][bb] = 2.0 * f1[aa][bb] * Sbh[aa][bb];
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) s += f2[aa][c][bb] * (That[aa][c] * Sbh[c][bb] + Sbh[aa][c] * That[c][bb]);
        Cbh[aa][bb] = 2.0 * s;
      }
    rot_out(Q, Tbh, Tbar);
    to_mandel(Tbar, TbarM);
    // local return mapping, reverse
    double ebarM[6], epnbarM[6], anbar;
    double thb[11];
#pragma unroll
    for (int q = 0; q < 11; ++q) thb[q] = 0.0;
    const double E = th[0], nu = th[1];
    const double dl_dE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), dm_dE = 1.0 / (2.0 * (1.0 + nu));
    const double Dn = (1.0 + nu) * (1.0 - 2.0 * nu);
    const double dl_dnu = E * (1.0 + 2.0 * nu * nu) / (Dn * Dn), dm_dnu = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
    if (!plastic) {
      iso_apply(m.lam, m.mu, TbarM, ebarM);
#pragma unroll
      for (int p = 0; p < 6; ++p) epnbarM[p] = mu_ep[p] - ebarM[p];
      anbar = mu_al;
      const double trw = TbarM[0] + TbarM[1] + TbarM[2], tre = ee[0] + ee[1] + ee[2];
      double we = 0.0;
#pragma unroll
      for (int p = 0; p < 6; ++p) we += TbarM[p] * ee[p];
      thb[0] = dl_dE * trw * tre + 2.0 * dm_dE * we;
      thb[1] = dl_dnu * trw * tre + 2.0 * dm_dnu * we;
    } else {
      const double phi = phy;
      // Hill matrix in global Mandel components
      double Hm[6][6];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) {
          double s = 0.0;
#pragma unroll
          for (int k = 1; k < 6; ++k) s += m.QH[i * 6 + k] * hv.v[k] * m.QH[j * 6 + k];
          Hm[i][j] = Hm[j][i] = s;
        }
      double EN[6];
      iso_apply(m.lam, m.mu, NM, EN);
      // J_y (rows: G_T, G_alpha, G_f; columns: T, alpha, dgamma), transposed into Mt
      double Mt[8][8];
      const double cf = dg / phi;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          double col[6];   // (H - N N^T) column c
#pragma unroll
          for (int k = 0; k < 6; ++k) col[k] = Hm[k][c] - NM[k] * NM[c];
          const double trc = col[0] + col[1] + col[2];
          const double Jrc = (r == c ? 1.0 : 0.0) + cf * (2.0 * m.mu * col[r] + (r < 3 ? m.lam * trc : 0.0));
          Mt[c][r] = Jrc;
        }
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        Mt[6][r] = 0.0;          // dG_T/dalpha
        Mt[7][r] = EN[r];        // dG_T/ddgamma
        Mt[r][6] = 0.0;          // dG_alpha/dT
        Mt[r][7] = NM[r];        // dG_f/dT
      }
      Mt[6][6] = 1.0;
      Mt[7][6] = -kSq23;
      Mt[6][7] = -kSq23 * dsy1;
      Mt[7][7] = 0.0;
      // ybar = (dz/dy)^T zbar: z = (T, eps_p,new = eps_p,n + dgamma N(T), alpha)
      double w[8];
      double HNep[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) s += (Hm[i][k] - NM[i] * NM[k]) * mu_ep[k];
        HNep[i] = s;
      }
      double Nep = 0.0;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        w[i] = TbarM[i] + cf * HNep[i];
        Nep += NM[i] * mu_ep[i];
      }
      w[6] = mu_al;
      w[7] = Nep;
      if (!solve8(Mt, w)) flag_local = 1;
      double wT[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) wT[i] = w[i];
      iso_apply(m.lam, m.mu, wT, ebarM);                 // ebar = E w_T
#pragma unroll
      for (int p = 0; p < 6; ++p) epnbarM[p] = mu_ep[p] - ebarM[p];
      anbar = w[6];
      // theta: elastic constants through E (eps - eps_p,n - dgamma N)
      double eef[6];
#pragma unroll
      for (int p = 0; p < 6; ++p) eef[p] = ee[p] - dg * NM[p];
      {
        const double trw = wT[0] + wT[1] + wT[2], tre = eef[0] + eef[1] + eef[2];
        double we = 0.0;
#pragma unroll
        for (int p = 0; p < 6; ++p) we += wT[p] * eef[p];
        thb[0] = dl_dE * trw * tre + 2.0 * dm_dE * we;
        thb[1] = dl_dnu * trw * tre + 2.0 * dm_dnu * we;
      }
      // Hill constants: H_q T and T.H_q.T through the local frame (Theta)
      double Rt[6][6];
      bool rot = a.Theta != nullptr;
      if (rot) {
        double Th[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) Th[i][j] = a.Theta[(int64_t)mi * 9 + i * 3 + j];
        mandel_rotation<double>(Th, Rt);
      }
      double Tl[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (rot) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < 6; ++k) s += Rt[i][k] * TM[k];
          Tl[i] = s;
        } else {
          Tl[i] = TM[i];
        }
      }
      double dmix[6];   // eps_p,bar - E w_T
#pragma unroll
      for (int p = 0; p < 6; ++p) dmix[p] = mu_ep[p] - ebarM[p];
      const double c23 = 2.0 / 3.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) {   // theta index 2 + q: F, G, H, L, M, N
        double hl[6] = {0, 0, 0, 0, 0, 0};
        if (q == 0) { hl[1] = c23 * (Tl[1] - Tl[2]); hl[2] = c23 * (Tl[2] - Tl[1]); }
        if (q == 1) { hl[0] = c23 * (Tl[0] - Tl[2]); hl[2] = c23 * (Tl[2] - Tl[0]); }
        if (q == 2) { hl[0] = c23 * (Tl[0] - Tl[1]); hl[1] = c23 * (Tl[1] - Tl[0]); }
        if (q == 3) hl[4] = c23 * Tl[4];
        if (q == 4) hl[5] = c23 * Tl[5];
        if (q == 5) hl[3] = c23 * Tl[3];
        double sq = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) sq += Tl[i] * hl[i];
        double hg[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          if (rot) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) s += Rt[k][i] * hl[k];
            hg[i] = s;
          } else {
            hg[i] = hl[i];
          }
        }
        double dNd = 0.0;   // (dN/dq) . dmix with dN/dq = H_q T / phi - N (T.H_q.T) / (2 phi^2)
#pragma unroll
        for (int i = 0; i < 6; ++i) dNd += (hg[i] / phi - NM[i] * sq / (2.0 * phi * phi)) * dmix[i];
        thb[2 + q] = dg * dNd - w[7] * sq / (2.0 * phi);
      }
      double dsd[3];
      sigy_dtheta(a.hardening, hp3, alpha1, dsd);
#pragma unroll
      for (int q = 0; q < 3; ++q) thb[8 + q] = w[7] * kSq23 * dsd[q];
    }
    // eps = eps(C): Cbar += Deps[ebar]
    {
      double eb[3][3], ebh[3][3];
      from_mandel(ebarM, eb);
      // Mandel cotangent -> tensor cotangent: shear components carry 1/sqrt2 twice (from_mandel
      // gives X_ij = v/sqrt2 for the cotangent too, since <ebar, deps> is the Mandel dot product)
      rot_in(Q, eb, ebh);
#pragma unroll
      for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) Cbh[aa][bb] += f1[aa][bb] * ebh[aa][bb];
    }
    double Cbar[3][3];
    rot_out(Q, Cbh, Cbar);
    // C = F^T F: Fbar += 2 F Cbar
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) s += F[i][k] * Cbar[k][j];
        Fbar[i][j] += 2.0 * s;
      }
    // history cotangent (stored tensor components): hbar = D epnbar_M
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double v = epnbarM[c] * (c < 3 ? 1.0 : kSq2);
      if (PASS_A) a.hbar[c * ng + gpi] = v;
      else a.hbar[c * ng + gpi] += v;
    }
    if (PASS_A) a.hbar[6 * ng + gpi] = anbar;
    else a.hbar[6 * ng + gpi] += anbar;
    if (PASS_A && a.fbar) {
      // pull the cotangent of s F back to F (the element's 8 threads): with c_q = G_q : F_q,
      // Fbar_q = s_q G_q - c_q s_q / (3 J_q) cof(F_q) + (sum_r c_r s_r) / (3 Jbar) det J0_q / V cof(F_q)
      double cof[3][3];
      cof[0][0] = F0[1][1] * F0[2][2] - F0[1][2] * F0[2][1];
      cof[0][1] = F0[1][2] * F0[2][0] - F0[1][0] * F0[2][2];
      cof[0][2] = F0[1][0] * F0[2][1] - F0[1][1] * F0[2][0];
      cof[1][0] = F0[0][2] * F0[2][1] - F0[0][1] * F0[2][2];
      cof[1][1] = F0[0][0] * F0[2][2] - F0[0][2] * F0[2][0];
      cof[1][2] = F0[0][1] * F0[2][0] - F0[0][0] * F0[2][1];
      cof[2][0] = F0[0][1] * F0[1][2] - F0[0][2] * F0[1][1];
      cof[2][1] = F0[0][2] * F0[1][0] - F0[0][0] * F0[1][2];
      cof[2][2] = F0[0][0] * F0[1][1] - F0[0][1] * F0[1][0];
      double c = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c += Fbar[i][j] * F0[i][j];
      const double cs = c * fb_s;
      double sum = cs;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) sum += __shfl_xor_sync(gmask, sum, o);
      const double k = -cs / (3.0 * fb_j) + sum / (3.0 * fb_jbar) * fb_det0 / fb_vol;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Fbar[i][j] = fb_s * Fbar[i][j] + k * cof[i][j];
    }
    double* sg = sGp[le][g];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) sg[i * 3 + j] = Fbar[i][j];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int k = 0; k < 3; ++k) sg[9 + n * 3 + k] = gN[n][k];
#pragma unroll
    for (int q = 0; q < 11; ++q) sg[33 + q] = thb[q];
  }
  {
    const unsigned bl = __ballot_sync(0xffffffffu, flag_local);
    if (lane == 0 && bl) atomicAdd(&a.status->local_fail, __popc(bl));
  }
  __syncthreads();
  if (!valid) return;
  if (PASS_A) {   // ubar_a = sum_gp Fbar^gp g_a^gp (F = I + sum_a u_a (x) g_a)
    double ub[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      const double* sg = sGp[le][q];
#pragma unroll
      for (int k = 0; k < 3; ++k) ub[k] += sg[k * 3 + 0] * sg[9 + g * 3] + sg[k * 3 + 1] * sg[9 + g * 3 + 1] +
                                           sg[k * 3 + 2] * sg[9 + g * 3 + 2];
    }
    const int node = a.conn[(int64_t)e * 8 + g];
    const bool store = a.slot[(int64_t)e * 64 + g * 9] < 0;
    double* dst = a.ubar + 3 * (int64_t)node;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (store) dst[k] = ub[k];
      else atomicAdd(dst + k, ub[k]);
    }
  }
  if (g == 0) {
#pragma unroll 1
    for (int q = 0; q < 11; ++q) {
      double s = 0.0;
#pragma unroll
      for (int p = 0; p < 8; ++p) s += sGp[le][p][33 + q];
      a.thbar[(int64_t)e * 11 + q] += s;
    }
  }
}

// KT = K^T in the (structurally symmetric) block pattern: block (i, j) transposed goes to the
// slot of block (j, i)
__global__ void transpose_blocks_kernel(const double* __restrict__ K, const int64_t* __restrict__ tslot,
                                        double* __restrict__ KT, int64_t n_blocks) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blocks) return;
  const int64_t t = tslot[b];
  const double* src = K + 9 * b;
  double* dst = KT + 9 * t;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) dst[3 * i + j] = src[3 * j + i];
}

// J^n = w ||u - ugt||^2 (all dofs) and rhs = -2 w (u - ugt) on free dofs; deterministic sum
__global__ void misfit_kernel(const double* __restrict__ u, const double* __restrict__ ugt, const uint8_t* freem,
                              double w, double* rhs, int64_t n_dof, double* part, unsigned* ticket, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n_dof; d += (int64_t)gridDim.x * blockDim.x) {
    const double r = u[d] - ugt[d];
    s += r * r;
    rhs[d] = freem[d] ? -2.0 * w * r : 0.0;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
    *out = w * t;
    *ticket = 0u;
  }
}

// rhs -= ubar on free dofs
__global__ void sub_free_kernel(double* rhs, const double* ubar, const uint8_t* freem, int64_t n) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d < n && freem[d]) rhs[d] -= ubar[d];
}

// r = b - K x on the free dofs, 0 on the fixed ones (the FP64 residual of iterative refinement)
__global__ void refine_residual_kernel(double* r, const double* b, const double* Kx, const uint8_t* freem, int64_t n) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d < n) r[d] = freem[d] ? b[d] - Kx[d] : 0.0;
}

// FP64 history [8][n_gp] -> mixed history (float [7][n_gp] + double cache)
__global__ void hist64_to_mixed_kernel(const double* h64, void* hm, int64_t n_gp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * n_gp) return;
  if (i < 7 * n_gp) reinterpret_cast<float*>(hm)[i] = (float)h64[i];
  else reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(hm) + 28 * n_gp)[i - 7 * n_gp] = h64[i];
}

}  // namespace

struct AdjointWork {
  int n_steps = 0, n_ckpt = 0, k = 1;
  // the forward pass's accepted (sub)steps: load factors, the requested step each one reaches
  // (-1 for an intermediate substep of adaptive stepping), and the capacity of u_all / ckpt
  std::vector<double> t_sub;
  std::vector<int> mark;
  int cap_sub = 0;
  LinSys ls;                 // FP64 system (K, CG vectors)
  std::vector<void*> mem;
  double *u_all = nullptr, *ckpt = nullptr, *h_prev = nullptr, *h_trial = nullptr, *h_tmp = nullptr;
  double *mu = nullptr, *hbar = nullptr, *thbar = nullptr, *ubar = nullptr, *rhs = nullptr, *R64 = nullptr;
  double *ugt = nullptr, *Jn = nullptr, *part = nullptr;
  unsigned* ticket = nullptr;
  // F-bar element: K is not symmetric; K^T (values in the same block pattern) and the map
  // from each block (i, j) to the slot of block (j, i)
  double* KT = nullptr;
  int64_t* tslot = nullptr;
  ~AdjointWork() {
    for (void* p : mem) cudaFree(p);
    if (ls.graph) cudaGraphExecDestroy(ls.graph);
  }
};

void adjoint_free(AdjointWork* w) { delete w; }

namespace {

// Mixed path: K lambda = rhs (K the FP64 tangent in w->ls.K, symmetric) by iterative
// refinement in the precision of the handle's own system: lambda = 0, then repeatedly the
// FP64 residual r = rhs - K lambda, its correction solved with the FP32 copy of K in FP32 CG
// (to kInnerRtol, BiCGSTAB if indefinite), lambda += correction, until |r| <= 0.3 pcg_rtol
// |rhs| in FP64.  Each pass contracts the error
// by about max(kInnerRtol, kappa eps_32), at the FP32 iteration's cost; a system that stalls
// is handed to FP64 CG.  lambda is left in w->ls.vx (FP64), the iterations added to *iters.
hfe_status refined_reverse_solve(hfe_handle* h, AdjointWork* w, int64_t* iters) {
  constexpr double kInnerRtol = 1e-3;
  constexpr int kMaxPasses = 8;
  const int64_t ndof = h->n_dof;
  const unsigned blocks = (unsigned)((ndof + 255) / 256);
  double* lam = reinterpret_cast<double*>(w->ls.vx);
  double* Kx = reinterpret_cast<double*>(w->ls.vq);
  to_float(reinterpret_cast<const double*>(w->ls.K), reinterpret_cast<float*>(h->K), 9 * h->P.n_blocks, h->s);
  HFE_TRY(cuda_check(h, cudaMemsetAsync(lam, 0, ndof * sizeof(double), h->s), "memset"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(w->R64, w->rhs, ndof * sizeof(double), cudaMemcpyDeviceToDevice, h->s),
                     "copy"));
  const Csr K = csr_of(h);
  double target = -1.0;
  for (int pass = 0;; ++pass) {
    free_norm(w->R64, h->freem, ndof, h->sc, h->part, h->s, nullptr);
    HFE_TRY(read_status(h));
    const double rn = std::sqrt(h->h_sc->norm2);
    if (!std::isfinite(rn)) return fail(h, HFE_ENONFINITE, "adjoint: non-finite residual");
    // a third of the solve tolerance: the gradient carries the reverse residual's relative
    // error, and is to meet 1e-6 of the FP64 adjoint with a margin (measured on the 4x2x1
    // Voce box: per-component 8.8e-7 at pcg_rtol, 1e-8 at a third of it)
    if (target < 0.0) target = 0.3 * h->opt.pcg_rtol * rn;
    if (rn <= target) return HFE_OK;
    if (pass == kMaxPasses) break;
    int64_t it = 0;
    h->pcg_rtol_now = kInnerRtol;
    const hfe_status st = solve_sys(h, h->ls, w->R64, 1.0, &it);
    h->pcg_rtol_now = 0.0;
    HFE_TRY(st);
    *iters += h->h_sc->iters;
    add_update<float>(lam, reinterpret_cast<const float*>(h->ls.vx), h->freem, ndof, h->s);
    spmv<double>(K, reinterpret_cast<const double*>(w->ls.K), h->freem, lam, Kx, nullptr, nullptr, h->s);
    refine_residual_kernel<<<blocks, 256, 0, h->s>>>(w->R64, w->rhs, Kx, h->freem, ndof);
    HFE_TRY(cuda_check(h, cudaGetLastError(), "refinement residual"));
  }
  // refinement stalled (kappa eps_32 near one): FP64 CG on the whole system
  const hfe_status st = solve_sys(h, w->ls, w->rhs, 1.0, nullptr);
  HFE_TRY(st);
  *iters += h->h_sc->iters;
  return HFE_OK;
}

}  // namespace

namespace {

template <typename T>
hfe_status aalloc(hfe_handle* h, AdjointWork* w, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, HFE_ENOMEM, "adjoint workspace allocation failed");
  }
  w->mem.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return HFE_OK;
}

hfe_status ensure_work(hfe_handle* h, int n_steps) {
  const int k = std::max(1, h->opt.ckpt_every);
  const int n_ckpt = (n_steps + k - 1) / k;    // h^j for j = 0, k, 2k, ... (grows with substeps)
  AdjointWork* w = h->adj;
  if (w != nullptr && w->n_steps == n_steps && w->k == k) return HFE_OK;
  delete w;
  w = new AdjointWork();
  h->adj = w;
  w->n_steps = n_steps;
  w->k = k;
  w->n_ckpt = n_ckpt;
  const size_t ndof = h->n_dof, ngp = h->n_gp;
  if (h->fp64) {
    w->ls = h->ls;             // share the handle's FP64 system
    w->ls.graph = nullptr;
    w->ls.graph_len = 0;
  } else {
    double* b;
    HFE_TRY(aalloc(h, w, &b, 9 * (size_t)h->P.n_blocks + kKPad)); w->ls.K = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vx = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vr = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vz = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vp = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vq = b;
    HFE_TRY(aalloc(h, w, &b, 9 * (size_t)h->n_nodes)); w->ls.vminv = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vp2 = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vrh = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vy = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vt = b;
    HFE_TRY(aalloc(h, w, &b, ndof)); w->ls.vxt = b;
    w->ls.fp64 = true;
  }
  HFE_TRY(aalloc(h, w, &w->u_all, ndof * n_steps));
  HFE_TRY(aalloc(h, w, &w->ckpt, 8 * ngp * (n_ckpt + 1)));
  w->cap_sub = n_steps;
  HFE_TRY(aalloc(h, w, &w->h_prev, 8 * ngp));
  HFE_TRY(aalloc(h, w, &w->h_trial, 8 * ngp));
  HFE_TRY(aalloc(h, w, &w->h_tmp, 8 * ngp));
  HFE_TRY(aalloc(h, w, &w->mu, 7 * ngp));
  HFE_TRY(aalloc(h, w, &w->hbar, 7 * ngp));
  HFE_TRY(aalloc(h, w, &w->thbar, 11 * (size_t)h->n_el));
  HFE_TRY(aalloc(h, w, &w->ubar, ndof));
  HFE_TRY(aalloc(h, w, &w->rhs, ndof));
  HFE_TRY(aalloc(h, w, &w->R64, ndof));
  HFE_TRY(aalloc(h, w, &w->ugt, ndof * n_steps));
  HFE_TRY(aalloc(h, w, &w->Jn, n_steps));
  HFE_TRY(aalloc(h, w, &w->part, 1024));
  HFE_TRY(aalloc(h, w, &w->ticket, 1));
  HFE_TRY(cuda_check(h, cudaMemsetAsync(w->ticket, 0, sizeof(unsigned), h->s), "memset"));
  return HFE_OK;
}

// Room for m substeps in u_all and their checkpoints (adaptive stepping adds substeps):
// the buffers double, the stored part is copied over.
template <typename T>
hfe_status regrow(hfe_handle* h, AdjointWork* w, T** p, size_t keep, size_t n_new) {
  T* q = nullptr;
  HFE_TRY(aalloc(h, w, &q, n_new));
  if (keep) HFE_TRY(cuda_check(h, cudaMemcpyAsync(q, *p, sizeof(T) * keep, cudaMemcpyDeviceToDevice, h->s), "copy"));
  HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "copy"));
  for (auto& x : w->mem)
    if (x == *p) {
      cudaFree(x);
      x = w->mem.back();
      w->mem.pop_back();
      break;
    }
  *p = q;
  return HFE_OK;
}

hfe_status ensure_substeps(hfe_handle* h, AdjointWork* w, int m) {
  if (m <= w->cap_sub) return HFE_OK;
  const int cap = std::max(m, 2 * w->cap_sub);
  const size_t ndof = h->n_dof, ngp = h->n_gp;
  HFE_TRY(regrow(h, w, &w->u_all, ndof * (size_t)w->t_sub.size(), ndof * (size_t)cap));
  const int nck = cap / w->k + 1;
  HFE_TRY(regrow(h, w, &w->ckpt, 8 * ngp * (size_t)(w->n_ckpt + 1), 8 * ngp * (size_t)(nck + 1)));
  w->n_ckpt = nck;
  w->cap_sub = cap;
  return HFE_OK;
}

// FP64 history h^j: copy of the checkpoint at or below j, then one FP64 residual sweep per
// step (h^{i+1} = H(u^{i+1}, h^i)); dst must differ from the scratch buffers used here.
hfe_status history_at(hfe_handle* h, AdjointWork* w, int j, double* dst) {
  const double* t = w->t_sub.data();
  const size_t ngp = h->n_gp;
  const int j0 = (j / w->k) * w->k;
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(dst, w->ckpt + 8 * ngp * (j0 / w->k), 8 * ngp * sizeof(double),
                                        cudaMemcpyDeviceToDevice, h->s), "copy"));
  for (int i = j0; i < j; ++i) {   // step i (0-based) maps h^i to h^{i+1}
    HFE_TRY(sweep_ex(h, w->u_all + (size_t)i * h->n_dof, t[i], HFE_SWEEP_RESIDUAL, w->R64, nullptr, w->ls.K, dst,
                     w->h_tmp, true));
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(dst, w->h_tmp, 8 * ngp * sizeof(double), cudaMemcpyDeviceToDevice, h->s),
                       "copy"));
  }
  return HFE_OK;
}

// Forward-pass hook: stores u^n and the FP64 history checkpoints; on the mixed path it first
// takes one FP64 Newton iteration at the converged mixed state and installs the FP64 history.
struct AdjHook : StepHook {
  AdjointWork* w;
  int64_t pcg_iters = 0;
  hfe_status before_commit(hfe_handle* h, double t_new) override {
    if (h->fp64) return HFE_OK;
    const size_t ngp = h->n_gp;
    // FP64 refinement of the mixed-converged state: the FP64 residual (FP64 sweep with the FP64
    // history), corrected with the mixed tangent of the last Newton iteration (still in the
    // handle) solved to 1e-2 in FP32; each pass contracts the error by about
    // max(1e-2, kappa eps_32).  Stops once the FP64 residual is 1e-3 of its first value (the
    // accuracy one FP64 Newton iteration would reach) or after kPolishPasses passes.
    constexpr int kPolishPasses = 4;
    double r0 = -1.0;
    for (int pass = 0;; ++pass) {
      HFE_TRY(sweep_ex(h, h->u, t_new, HFE_SWEEP_RESIDUAL, w->R64, nullptr, w->ls.K, w->h_prev, w->h_trial, true));
      free_norm(w->R64, h->freem, h->n_dof, h->sc, h->part, h->s, nullptr);
      HFE_TRY(read_status(h));
      HFE_TRY(check_sweep_status(h));
      const double rn = std::sqrt(h->h_sc->norm2);
      if (r0 < 0.0) r0 = rn;
      if (!(rn > 1e-3 * r0) || pass == kPolishPasses) break;
      int64_t it = 0;
      h->allow_indefinite = true;   // an indefinite tangent is solved by BiCGSTAB
      h->pcg_rtol_now = 1e-2;
      const hfe_status pst = solve_sys(h, h->ls, w->R64, -1.0, &it);
      h->allow_indefinite = false;
      h->pcg_rtol_now = 0.0;
      HFE_TRY(pst);
      pcg_iters += h->h_sc->iters;
      add_update<float>(h->u, (const float*)h->ls.vx, h->freem, h->n_dof, h->s);
    }
    const unsigned blocks = (unsigned)((8 * ngp + 255) / 256);
    hist64_to_mixed_kernel<<<blocks, 256, 0, h->s>>>(w->h_trial, h->hist_trial, (int64_t)ngp);
    return HFE_OK;
  }
  hfe_status after_commit(hfe_handle* h, double t_new, int marker) override {
    const size_t ngp = h->n_gp;
    const int m = (int)w->t_sub.size();   // index of this substep
    HFE_TRY(ensure_substeps(h, w, m + 1));
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(w->u_all + (size_t)m * h->n_dof, h->u, h->n_dof * sizeof(double),
                                          cudaMemcpyDeviceToDevice, h->s), "copy"));
    w->t_sub.push_back(t_new);
    w->mark.push_back(marker);
    const double* hn = h->fp64 ? reinterpret_cast<const double*>(h->hist) : w->h_trial;   // h^{m+1}
    if (!h->fp64) std::swap(w->h_prev, w->h_trial);
    const int j = m + 1;   // history index after this substep
    if (j % w->k == 0)
      HFE_TRY(cuda_check(h, cudaMemcpyAsync(w->ckpt + 8 * ngp * (j / w->k), h->fp64 ? hn : w->h_prev,
                                            8 * ngp * sizeof(double), cudaMemcpyDeviceToDevice, h->s), "copy"));
    return HFE_OK;
  }
};

void launch_vjp(hfe_handle* h, AdjointWork* w, bool pass_a, const double* u, const double* hist, const double* lam) {
  VjpArgs a;
  a.X = h->X;
  a.conn = h->conn;
  a.u = u;
  a.hist = hist;
  a.mat = h->mat64;
  a.mat_per_element = h->n_mat > 1 ? 1 : 0;
  a.hardening = h->hardening;
  a.theta = h->theta;
  a.Theta = h->Theta;
  a.elems = h->elems;
  a.slot = h->slot;
  a.lam = lam;
  a.mu = w->mu;
  a.ubar = w->ubar;
  a.hbar = w->hbar;
  a.thbar = w->thbar;
  a.status = h->status;
  a.n_gp = h->n_gp;
  a.local_maxit = h->opt.local_maxit;
  a.local_tol = h->opt.local_tol;
  a.fbar = h->opt.fbar != 0;
  const auto& off = h->P.launch_off;
  for (size_t c = 0; c + 1 < off.size(); ++c) {
    const int64_t cnt = off[c + 1] - off[c];
    if (cnt <= 0) continue;
    const unsigned blocks = (unsigned)((cnt + kAdjEl - 1) / kAdjEl);
    if (pass_a) gp_vjp_kernel<true><<<blocks, kAdjThreads, 0, h->s>>>(a, off[c], cnt);
    else gp_vjp_kernel<false><<<blocks, kAdjThreads, 0, h->s>>>(a, off[c], cnt);
  }
}

}  // namespace

// The transpose map of the block pattern (host, once per work area) and room for K^T.
hfe_status ensure_transpose(hfe_handle* h, AdjointWork* w) {
  if (w->tslot != nullptr) return HFE_OK;
  const Pattern& P = h->P;
  std::vector<int64_t> ts((size_t)P.n_blocks, -1);
  for (int64_t i = 0; i < h->n_nodes; ++i)
    for (int64_t b = P.rowptr[i]; b < P.rowptr[i + 1]; ++b) {
      const int64_t j = P.cols[b];
      for (int64_t c = P.rowptr[j]; c < P.rowptr[j + 1]; ++c)
        if (P.cols[c] == i) {
          ts[b] = c;
          break;
        }
      if (ts[b] < 0) return fail(h, HFE_EINVAL, "adjoint: the block pattern is not structurally symmetric");
    }
  HFE_TRY(aalloc(h, w, &w->tslot, (size_t)P.n_blocks));
  HFE_TRY(aalloc(h, w, &w->KT, 9 * (size_t)P.n_blocks + kKPad));
  return cuda_check(h, cudaMemcpy(w->tslot, ts.data(), ts.size() * sizeof(int64_t), cudaMemcpyHostToDevice),
                    "copy");
}

hfe_status adjoint_run(hfe_handle* h, int n_steps, const double* t_in, const double* u_target, double wgt,
                       double* J_out, double* grad_out, hfe_stats* stats) {
  auto w0 = std::chrono::steady_clock::now();
  if (h->barlat != nullptr) return fail(h, HFE_EINVAL, "adjoint: the Hill-48 parameters only (Barlat material set)");
  std::vector<double> t(t_in, t_in + n_steps);
  HFE_TRY(ensure_work(h, n_steps));
  AdjointWork* w = h->adj;
  if (h->opt.fbar) HFE_TRY(ensure_transpose(h, w));
  const size_t ndof = h->n_dof, ngp = h->n_gp;
  // forward pass from the zero state
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->u, 0, ndof * sizeof(double), h->s), "memset"));
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->hist, 0, hist_bytes(h->n_gp, h->fp64 != 0), h->s), "memset"));
  launch_sigma_cache(h->hist, h->fp64 != 0, h->mat64, h->n_mat > 1, h->hardening, h->n_gp, h->s);
  HFE_TRY(cuda_check(h, cudaMemsetAsync(w->h_prev, 0, 8 * ngp * sizeof(double), h->s), "memset"));
  launch_sigma_cache(w->h_prev, true, h->mat64, h->n_mat > 1, h->hardening, h->n_gp, h->s);
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(w->ckpt, w->h_prev, 8 * ngp * sizeof(double), cudaMemcpyDeviceToDevice, h->s),
                     "copy"));
  h->t_state = 0.0;
  h->pred_valid = false;
  h->extrap_n = 0;
  w->t_sub.clear();
  w->mark.clear();
  HFE_TRY(copy_in(h, w->ugt, u_target, ndof * n_steps * sizeof(double)));
  AdjHook hook;
  hook.w = w;
  hfe_stats fst;
  std::memset(&fst, 0, sizeof(fst));
  cudaEvent_t ta, tb, tc;
  cudaEventCreate(&ta);
  cudaEventCreate(&tb);
  cudaEventCreate(&tc);
  cudaEventRecord(ta, h->s);
  HFE_TRY(newton_steps(h, n_steps, t.data(), nullptr, nullptr, nullptr, &fst, &hook));
  cudaEventRecord(tb, h->s);
  // misfit at the requested load factors (substeps in between do not enter J)
  const int M = (int)w->t_sub.size();
  for (int m = 0; m < M; ++m)
    if (w->mark[m] >= 0)
      misfit_kernel<<<256, 256, 0, h->s>>>(w->u_all + (size_t)m * ndof, w->ugt + (size_t)w->mark[m] * ndof, h->freem,
                                           wgt, w->rhs, (int64_t)ndof, w->part, w->ticket, w->Jn + w->mark[m]);
  // reverse pass over the accepted (sub)steps
  HFE_TRY(cuda_check(h, cudaMemsetAsync(w->mu, 0, 7 * ngp * sizeof(double), h->s), "memset"));
  HFE_TRY(cuda_check(h, cudaMemsetAsync(w->thbar, 0, 11 * (size_t)h->n_el * sizeof(double), h->s), "memset"));
  int64_t adj_pcg = 0;
  for (int n = M - 1; n >= 0; --n) {
    const double* un = w->u_all + (size_t)n * ndof;
    HFE_TRY(history_at(h, w, n, w->h_prev));           // h^n: history before substep n
    HFE_TRY(sweep_ex(h, un, w->t_sub[n], HFE_SWEEP_TANGENT, w->R64, nullptr, w->ls.K, w->h_prev, w->h_trial, true));
    if (w->mark[n] >= 0)                                // rhs = -dJ^n/du^n (R64 as scratch)
      misfit_kernel<<<256, 256, 0, h->s>>>(un, w->ugt + (size_t)w->mark[n] * ndof, h->freem, wgt, w->rhs,
                                           (int64_t)ndof, w->part, w->ticket, w->R64);
    else
      HFE_TRY(cuda_check(h, cudaMemsetAsync(w->rhs, 0, ndof * sizeof(double), h->s), "memset"));
    HFE_TRY(cuda_check(h, cudaMemsetAsync(w->hbar, 0, 7 * ngp * sizeof(double), h->s), "memset"));
    if (n < M - 1) {   // pass A: history cotangent mu^{n+1} of h^{n+1} = H(u^n, h^n)
      launch_vjp(h, w, true, un, w->h_prev, nullptr);
      sub_free_kernel<<<(unsigned)((ndof + 255) / 256), 256, 0, h->s>>>(w->rhs, w->ubar, h->freem, (int64_t)ndof);
    }
    HFE_TRY(read_status(h));
    HFE_TRY(check_sweep_status(h));
    h->allow_indefinite = true;   // K^T lambda = rhs (K symmetric; BiCGSTAB if indefinite)
    void* Kn = w->ls.K;
    if (h->opt.fbar) {            // F-bar: K is not symmetric, BiCGSTAB on the transposed blocks
      const int64_t nb = h->P.n_blocks;
      transpose_blocks_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, h->s>>>((const double*)Kn, w->tslot, w->KT, nb);
      w->ls.K = w->KT;
    }
    hfe_status ast;
    if (!h->fp64 && !h->opt.fbar) {   // mixed: FP32 solves inside FP64 iterative refinement
      ast = refined_reverse_solve(h, w, &adj_pcg);
    } else {
      ast = solve_sys(h, w->ls, w->rhs, 1.0, nullptr);
      if (ast == HFE_OK) adj_pcg += h->h_sc->iters;
    }
    w->ls.K = Kn;
    h->allow_indefinite = false;
    HFE_TRY(ast);
    launch_vjp(h, w, false, un, w->h_prev, reinterpret_cast<const double*>(w->ls.vx));   // pass B
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(w->mu, w->hbar, 7 * ngp * sizeof(double), cudaMemcpyDeviceToDevice, h->s),
                       "copy"));
  }
  cudaEventRecord(tc, h->s);
  h->pred_valid = false;   // the reverse pass reassembled K (FP64 handles share it)
  HFE_TRY(read_status(h));
  if (h->h_status->local_fail > 0) return fail(h, HFE_ELOCAL, "adjoint: local system failures");
  // J and gradient
  std::vector<double> Jn(n_steps);
  HFE_TRY(cuda_check(h, cudaMemcpy(Jn.data(), w->Jn, n_steps * sizeof(double), cudaMemcpyDeviceToHost), "copy"));
  double J = 0.0;
  for (double v : Jn) J += v;
  if (J_out) *J_out = J;
  std::vector<double> tb_h(11 * (size_t)h->n_el);
  HFE_TRY(cuda_check(h, cudaMemcpy(tb_h.data(), w->thbar, tb_h.size() * sizeof(double), cudaMemcpyDeviceToHost), "copy"));
  std::vector<double> g(11 * (size_t)h->n_mat, 0.0);
  if (h->n_mat == 1) {
    for (int64_t e = 0; e < h->n_el; ++e)
      for (int q = 0; q < 11; ++q) g[q] += tb_h[e * 11 + q];
  } else {
    g = tb_h;
  }
  if (grad_out != nullptr) {
    if (is_device_ptr(grad_out)) {
      HFE_TRY(cuda_check(h, cudaMemcpy(grad_out, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice), "copy"));
    } else {
      std::memcpy(grad_out, g.data(), g.size() * sizeof(double));
    }
  }
  if (stats) {
    *stats = fst;
    stats->pcg_iters = fst.pcg_iters + hook.pcg_iters + adj_pcg;
    stats->refine_pcg_iters = hook.pcg_iters;
    stats->reverse_pcg_iters = adj_pcg;
    float fms = 0.f, bms = 0.f;
    cudaEventElapsedTime(&fms, ta, tb);
    cudaEventElapsedTime(&bms, tb, tc);
    stats->sweep_ms = fms;   // forward pass (device time)
    stats->solve_ms = bms;   // reverse pass (device time)
    stats->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  }
  cudaEventDestroy(ta);
  cudaEventDestroy(tb);
  cudaEventDestroy(tc);
  return HFE_OK;
}

}  // namespace hfe
