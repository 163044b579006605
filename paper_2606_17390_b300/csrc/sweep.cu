// Gauss-point sweep: kinematics, log strain, Hill-48 return mapping, consistent tangent,
// geometric post-processing, hex8 element contraction and conflict-free block-CSR scatter.
//
// Paper references: geometric pre-processor Eq. c_decomp; log-space elasticity Eq. T;
// Hill-48 Eq. Phi_hill with App. A.1; hardening Eq. Hard; flow rule Eq. ep_evol and the
// Kuhn-Tucker conditions Eq. KT; elastic predictor Eq. Tr_stress; closest-point projection
// Eq. local_cpp (solved here in its scalar form, see return_map_*); implicit-function
// tangent App. D; post-processor Eq. proj_lagrange / Eq. pk_stress with P_L and L_L applied
// through first and second divided differences (Sec. 2.2.5); element residual and stiffness
// Sec. 2.2.4 / Eq. Stiffness_mat.
//
// Thread layout: a CTA of 128 threads holds 16 elements x 8 Gauss points.  Phase 1: one
// thread per Gauss point runs the constitutive update and stages the per-point tangent
// A = dP/dF (rotated into the eigenbasis of C), the rotated shape-function gradients and the
// rotated first Piola-Kirchhoff stress in shared memory.  Phase 2: one thread per
// (element, node row a) contracts the eight Gauss points into the 3x24 row block of K^e
// and the 3 entries of R^e; the warp stages its element matrices in shared memory and
// writes them through the element-to-block slot map with consecutive lanes on consecutive
// entries.  Elements of one launch share no node (one colour of one slab of the launch
// order), so every block has one writer per launch: the first launch that touches a block
// stores, later launches add (bit 31 of the slot), in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "gp_math.cuh"
#include "hfe_internal.h"

namespace hfe {
namespace {

constexpr int kElemsPerCta = 16;
constexpr int kThreads = 128;
// shared words per Gauss point: A 45 (major-symmetric) + pad 3, P 9 + pad 3, g 24; every
// section starts on a 16-byte boundary, so phase 1 stores and phase 2 loads A and P as
// 4-vectors.  The F-bar element adds M = A : Fbar (9 + pad 3) and the vectors v_b (24) of
// its rank-one tangent terms.
constexpr int kOffP = 48;
constexpr int kOffG = 60;
constexpr int kOffM = 84;
constexpr int kOffV = 96;
// per element 8 * stride + 8 = 8 mod 32 words: the 4 elements of a warp read g from banks
// offset by 0, 8, 16, 24 in phase 2 (conflict-free scalar loads); the 8 Gauss points of one
// element (one quarter-warp phase of a 16-byte store) start at 20 g (84) or 28 g (124) mod 32
// words: distinct bank quads
template <bool FBAR> struct Lay {
  static constexpr int kGpStride = FBAR ? 124 : 84;
  static constexpr int kElStride = 8 * kGpStride + 8;
};


// 4-vector shared-memory stores and loads of R values (16-byte aligned addresses)
template <typename R> struct V4;
template <> struct V4<float> {
  __device__ static void st(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  }
  __device__ static void ld(const float* p, float* v) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
};
template <> struct V4<double> {
  __device__ static void st(double* p, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
  }
  __device__ static void ld(const double* p, double* v) {
    const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
};

using namespace gpm;

// Streamed per-point data (the history and the slot map, each read or written once per
// sweep) carries an L2 evict-first policy, so that it displaces the K rows the assembly adds
// into last (createpolicy + .L2::cache_hint).
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
template <typename T> struct Stream;
template <> struct Stream<float> {
  __device__ static float ld(const float* p, uint64_t pol) {
    float v;
    asm("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
  }
  __device__ static void st(float* p, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
  }
};
template <> struct Stream<double> {
  __device__ static double ld(const double* p, uint64_t pol) {
    double v;
    asm("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
  }
  __device__ static void st(double* p, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
  }
};
template <> struct Stream<int32_t> {
  __device__ static int32_t ld(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
  }
};

// Mixed path: sigma_y(alpha_n + da) = sigma_y(alpha_n) + inc(da) with the FP64 cache
// sigma_y(alpha_n) and the increment in FP32 (relative error ~1e-7 of the increment only).
// Swift: inc = sy_n (exp(n log1p(da / (eps0 + alpha_n))) - 1); Voce: inc = A (1 - exp(-b da))
// with A = sigma0 + Q - sy_n = Q exp(-b alpha_n).
struct HardInc {
  int type;
  float p2, z_or_A, syn;   // Swift: n, eps0 + alpha_n, sy_n ; Voce: b, A, sy_n
  __device__ __forceinline__ void eval(float da, float& inc, float& dsy) const {
    if (type == HFE_HARDENING_SWIFT) {
      float g = expm1f(p2 * log1pf(__fdividef(da, z_or_A)));
      inc = syn * g;
      dsy = __fdividef(p2 * (syn + inc), z_or_A + da);
    } else {
      float em = expm1f(-p2 * da);
      inc = -z_or_A * em;
      dsy = p2 * z_or_A * (1.0f + em);
    }
  }
};

// Mixed form: the Newton iterations in FP32 to ~1e-6, then one FP64 Newton step on the yield
// residual (written as phi^2 - phi_y^2 to avoid a square root) with FP64 reciprocals.
__device__ __forceinline__ RM return_map_mixed(const float t[6], const Vec6d hv, const Vec6f hfv, float mu,
                               float hmin, const HardInc& inc, double syn64, float ftr, int maxit) {
  RM out;
  const float sq23 = (float)kSq23;
  float dg = 0.0f, lo = 0.0f, hi = __fdividef(ftr, 2.0f * mu * hmin);
  float dr = -1.0f;
  int k = 0;
  bool ok = false;
  for (; k < maxit; ++k) {
    float incv, dsy;
    inc.eval(sq23 * dg, incv, dsy);
    float phy = sq23 * (inc.syn + incv), dphy = (2.0f / 3.0f) * dsy;
    const float iphy = __fdividef(1.0f, phy);
    float s = 2.0f * mu * dg * iphy;
    float ds = 2.0f * mu * (phy - dg * dphy) * iphy * iphy;
    float phi2 = 0.0f, acc = 0.0f;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
      const float rd = __fdividef(1.0f, 1.0f + s * hfv.v[i]);
      float Ti = t[i] * rd;
      float hT = hfv.v[i] * Ti;
      phi2 += hT * Ti;
      acc += hT * hT * rd;
    }
    float phi = sqrtf(phi2);
    float r = phi - phy;
    dr = -__fdividef(acc, phi) * ds - dphy;
    if (fabsf(r) <= 1e-6f * phy) { ok = true; break; }
    if (r > 0.0f) lo = dg; else hi = dg;
    float dgn = dg - __fdividef(r, dr);
    if (!(dgn > lo && dgn < hi)) dgn = 0.5f * (lo + hi);
    if (fabsf(dgn - dg) <= 1e-7f * dg) { dg = dgn; ok = true; break; }
    dg = dgn;
  }
  // FP64 polish: one Newton step on rho(dgamma) = sum_i h_i (t_i / D_i)^2 - 1, the yield
  // residual phi^2 - phi_y^2 divided by phi_y^2, with D_i = phi_y + 2 mu dgamma h_i (so that
  // t_i / D_i = T_i / phi_y).  Each quotient is formed in FP32, q_i ~ t_i / D_i, and its FP64
  // residual t_i - D_i q_i = D_i d_i gives the exact square (t_i / D_i)^2 = q_i^2 +
  // d_i (2 q_i + d_i): q_i^2 is exact in FP64 and carries the sum, the correction (~1e-7 of
  // it) needs FP32 only.  Four FP64 operations per component (the FP64 pipe of this part is
  // 1/64 of its FP32 rate); the derivative 2 phi_y r' comes from the FP32 iteration.
  float incv, dsy;
  inc.eval(sq23 * dg, incv, dsy);
  const double phy = kSq23 * (syn64 + (double)incv);
  const float tmu = 2.0f * mu;                       // exact
  const double k2 = (double)tmu * (double)dg;        // 2 mu dgamma, exact in FP64
  const float phyf = (float)phy, k2f = tmu * dg;
  double rho = -1.0;
  float cor = 0.0f;
#pragma unroll
  for (int i = 1; i < 6; ++i) {
    const float rD = __frcp_rn(fmaf(k2f, hfv.v[i], phyf));
    const float qf = t[i] * rD;
    const double qd = (double)qf;
    const double Di = fma(k2, hv.v[i], phy);
    const float del = (float)fma(-Di, qd, (double)t[i]) * rD;
    rho = fma(hv.v[i], qd * qd, rho);
    cor = fmaf(hfv.v[i] * del, fmaf(2.0f, qf, del), cor);
  }
  rho += (double)cor;
  // Newton: d(phi^2 - phi_y^2) / d dgamma = 2 phi_y r', so the step is phi_y rho / (2 r')
  const float corr = __fdividef((float)rho * phyf, 2.0f * dr);
  double dg64 = (double)dg - (double)corr;
  float dgf = dg - corr;
  if (corr > dg) {   // dgamma < 0: none
    dg64 = 0.0;
    dgf = 0.0f;
  }
  inc.eval(sq23 * dgf, incv, dsy);
  out.dgamma = dg64;
  out.syn1 = syn64 + (double)incv;
  out.dsy = dsy;
  out.iters = k + 1;
  out.ok = ok;
  return out;
}

template <typename R> struct Hist {
  // component c of Gauss point i, and the FP64 sigma_y(alpha) cache
  __device__ static R* comp(void* b, int c, int64_t ng) { return reinterpret_cast<R*>(b) + c * ng; }
  __device__ static double* cache(void* b, int64_t ng) {
    return sizeof(R) == 8 ? reinterpret_cast<double*>(b) + 7 * ng
                          : reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(b) + 28 * ng);
  }
};

template <typename R> struct MatOf;
template <> struct MatOf<float> { using T = MatRecF; };
template <> struct MatOf<double> { using T = MatRec; };

// ----------------------------------------------------------------------------------------
// Phase 2 of the tangent sweep: thread (element le, node row a = g) contracts the eight Gauss-point records into the blocks (a, a + d mod 8), d = 0..3 (and
// d = 4 for a < 4) — each unordered block pair once, as K^e is symmetric (A is stored with
// its major symmetry) — and into R_a.  The blocks and their transposes are then staged in the
// warp's own (already consumed) record area, row-major [a][b][3x3] per element, and the warp
// writes its four elements out with consecutive lanes on consecutive entries: a block's nine
// values are contiguous in K and an element row's blocks lie close together, so each warp
// store covers a few 32-byte sectors.  The first launch that touches a block stores (bit 31 of
// the slot), later launches add: one writer per block per launch, launches in a fixed order,
// so the sums are deterministic.  The F-bar element (FBAR) adds its non-symmetric rank-one part
// K_ab += sum_q (M_q g_a,q) (x) v_b,q to the staged row a before the write-out; its staging
// stays inside the element's own record area (words 0..71 of each Gauss-point record, entry r
// at record r / 72), clear of the M and v_b sections the rank-one part reads afterwards.
constexpr int kStageEl = 584;   // staging words per element: 576 used; 584 = 8 mod 32 spreads
                                // the four elements of a warp over the banks

template <typename R, bool FBAR>
__device__ __forceinline__ void phase2_staged(const SweepArgs& a, R* sGp, int le, int g, int e, unsigned lane,
                                              bool valid, int node, unsigned cta, int64_t ccount, uint64_t pol) {
  constexpr int kGpStride = Lay<FBAR>::kGpStride;
  constexpr int kElStride = Lay<FBAR>::kElStride;
  static_assert(4 * kStageEl <= 4 * kElStride, "staging must fit in the warp's records");
  static_assert(!FBAR || 72 <= kOffM, "F-bar staging must leave M and v_b in place");
  // staging word of entry r ([a][b][3x3] row-major) relative to the element's staging base
  auto sw = [](int r) { return FBAR ? (r / 72) * kGpStride + (r - 72 * (r / 72)) : r; };
  const int arow = g;
  // the element's slot-map row is read during the write-out: start bringing it into L1
  if (valid && g < 2) asm volatile("prefetch.global.L1 [%0];\n" ::"l"(a.slot + (int64_t)e * 64 + 32 * g));
  constexpr int kNb = 5;
  const int nb = (arow < 4) ? 5 : 4;
  R Kr[kNb][9];
#pragma unroll
  for (int d = 0; d < kNb; ++d)
#pragma unroll
    for (int c = 0; c < 9; ++c) Kr[d][c] = R(0);
  R Ra[3] = {R(0), R(0), R(0)};
  if (valid) {
    const R* G = sGp + (size_t)le * kElStride;
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      const R* Aq = G + q * kGpStride;
      const R* gt = Aq + kOffG;
      const R ga0 = gt[arow * 3], ga1 = gt[arow * 3 + 1], ga2 = gt[arow * 3 + 2];
      R A[48];
#pragma unroll
      for (int k = 0; k < 12; ++k) V4<R>::ld(Aq + 4 * k, A + 4 * k);
      R U[3][3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int L = 0; L < 3; ++L)
            U[i][k][L] = ga0 * A[asym(i * 3 + 0, k * 3 + L)] + ga1 * A[asym(i * 3 + 1, k * 3 + L)] +
                         ga2 * A[asym(i * 3 + 2, k * 3 + L)];
#pragma unroll
      for (int d = 0; d < kNb; ++d) {
        if (d < nb) {
          const int b = (arow + d) & 7;
          const R gb0 = gt[b * 3], gb1 = gt[b * 3 + 1], gb2 = gt[b * 3 + 2];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) Kr[d][i * 3 + k] += U[i][k][0] * gb0 + U[i][k][1] * gb1 + U[i][k][2] * gb2;
        }
      }
      R P[12];
#pragma unroll
      for (int k = 0; k < 3; ++k) V4<R>::ld(Aq + kOffP + 4 * k, P + 4 * k);
#pragma unroll
      for (int i = 0; i < 3; ++i) Ra[i] += P[i * 3] * ga0 + P[i * 3 + 1] * ga1 + P[i * 3 + 2] * ga2;
    }
  }
  // F-bar: M_q g_a,q for the eight points, read before the staging overwrites g
  R ua[FBAR ? 8 : 1][3];
  if constexpr (FBAR) {
#pragma unroll
    for (int q = 0; q < 8; ++q) ua[q][0] = ua[q][1] = ua[q][2] = R(0);
    if (valid) {
      const R* G = sGp + (size_t)le * kElStride;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const R* Aq = G + q * kGpStride;
        const R ga0 = Aq[kOffG + arow * 3], ga1 = Aq[kOffG + arow * 3 + 1], ga2 = Aq[kOffG + arow * 3 + 2];
        R mv[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) V4<R>::ld(Aq + kOffM + 4 * k, mv + 4 * k);
        ua[q][0] = mv[0] * ga0 + mv[1] * ga1 + mv[2] * ga2;
        ua[q][1] = mv[3] * ga0 + mv[4] * ga1 + mv[5] * ga2;
        ua[q][2] = mv[6] * ga0 + mv[7] * ga1 + mv[8] * ga2;
      }
    }
  }
  // every lane of the warp has read its records: the record areas become staging
  __syncwarp();
  R* stage = sGp + (size_t)(le & ~3) * kElStride;
  R* se = FBAR ? sGp + (size_t)le * kElStride : stage + (le & 3) * kStageEl;
  if (valid) {
#pragma unroll
    for (int d = 0; d < kNb; ++d) {
      if (d < nb) {
        const int b = (arow + d) & 7;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            se[sw((arow * 8 + b) * 9 + i * 3 + k)] = Kr[d][i * 3 + k];
            if (d != 0) se[sw((b * 8 + arow) * 9 + k * 3 + i)] = Kr[d][i * 3 + k];
          }
      }
    }
  }
  __syncwarp();
  if constexpr (FBAR) {
    // the rank-one part of row a (only this thread writes row a now)
    if (valid) {
      const R* G = sGp + (size_t)le * kElStride;
#pragma unroll 1
      for (int b = 0; b < 8; ++b) {
        R C[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) C[c] = R(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const R* vb = G + q * kGpStride + kOffV + b * 3;
          const R v0 = vb[0], v1 = vb[1], v2 = vb[2];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            C[i * 3] += ua[q][i] * v0;
            C[i * 3 + 1] += ua[q][i] * v1;
            C[i * 3 + 2] += ua[q][i] * v2;
          }
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) se[sw((arow * 8 + b) * 9 + c)] += C[c];
      }
    }
    __syncwarp();
  }
  R* Kv = reinterpret_cast<R*>(a.K);
  const int w0 = le & ~3;
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    const int ej = __shfl_sync(0xffffffffu, e, 8 * j);             // element of lanes 8j..8j+7
    if ((int64_t)cta * kElemsPerCta + w0 + j >= ccount) break;   // the same for every lane
    const R* sej = FBAR ? sGp + (size_t)(w0 + j) * kElStride : stage + j * kStageEl;
    const int32_t* slj = a.slot + (int64_t)ej * 64;
    // lane l writes entries l + 32 i (i < 18) of the 576: all 18 slot loads are issued
    // before the first write so that their latencies overlap
    int32_t sv[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) sv[i] = Stream<int32_t>::ld(slj + ((int)lane + 32 * i) / 9, pol);
#pragma unroll
    for (int i = 0; i < 18; ++i) {
      const int r = (int)lane + 32 * i;
      const int c = r - 9 * (r / 9);
      R* dst = Kv + (int64_t)(sv[i] & 0x7fffffff) * 9 + c;
      const R v = sej[sw(r)];
      if (sv[i] < 0) *dst = v;
      else atomicAdd(dst, v);
    }
  }
  if (!valid) return;
  // node of row a = g is the node this thread gathered in phase 1
  const bool store = Stream<int32_t>::ld(a.slot + (int64_t)e * 64 + arow * 9, pol) < 0;   // diagonal block (a, a)
  double* Rg = a.R + 3 * (int64_t)node;
  if (!(isfinite(Ra[0]) && isfinite(Ra[1]) && isfinite(Ra[2])))
    atomicAdd(&a.status->nonfinite, 1);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double v = (double)Ra[i];
    if (store) Rg[i] = v - (a.f_ext ? a.load * a.f_ext[3 * (int64_t)node + i] : 0.0);
    else atomicAdd(Rg + i, v);
  }
}

// ----------------------------------------------------------------------------------------
// UNIF: one material for all elements, passed by value so that its entries are kernel-
// parameter (constant-bank) operands rather than loads.
// MAT: 0 the Hill-48 update in the kernel; 1 the strain pass of an external material model
// (the Mandel log strain of every Gauss point out, nothing assembled); 2 the external model's
// stress, plastic flag and tangent dT/deps in (S4 and S5 replaced, S6-S8 as for Hill).
// Occupancy: the mixed uniform-material Hill-48 sweeps run five CTAs per SM (96 registers; the
// tangent form spills a few values, measured 3.42 -> 3.33 ms at 100^3 against four CTAs at
// 128 registers; the residual form spills none), the other mixed forms four, F-bar three.
template <typename R, bool TANGENT, bool UNIF, bool FBAR, int MAT = 0>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? (FBAR ? 3 : (UNIF && MAT == 0 ? 5 : 4)) : 1)
    gp_sweep_kernel(SweepArgs a, const typename MatOf<R>::T mrec, int64_t cbeg, int64_t ccount) {
  constexpr int kGpStride = Lay<FBAR>::kGpStride;
  constexpr int kElStride = Lay<FBAR>::kElStride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [16][kElStride] Gauss-point records; an element's first 48 words hold its nodal data
  // [8][6] (dX, du) until the kinematics have read them
  R* sGp = reinterpret_cast<R*>(smem_raw);
  // the next launch may start its CTAs once every CTA of this one has started: its phase 1
  // reads nothing this launch writes, and its phase 2 waits for this launch below
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");

  const int tid = threadIdx.x;
  const int le = tid >> 3;
  const int g = tid & 7;
  const int64_t li = (int64_t)blockIdx.x * kElemsPerCta + le;
  const bool valid = li < ccount;
  const int e = valid ? a.elems[cbeg + li] : 0;
  const unsigned lane = tid & 31;
  const unsigned gmask = 0xffu << (lane & 24);
  const uint64_t pol = l2_evict_first();

  using MR = typename MatOf<R>::T;
  const MR* matR = reinterpret_cast<const MR*>(a.mat);
  const int mi = a.mat_per_element ? e : 0;

  // the element's 64 slot-map entries (256 B, read in phase 2): into L2 while phase 1 runs
  if (valid && g < 2) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.slot + (int64_t)e * 64 + 32 * g));

  // history of this Gauss point, loaded first so that it arrives during the kinematics
  const int64_t ng = a.n_gp;
  const int64_t gpi = (int64_t)e * 8 + g;   // global Gauss-point index
  R epn[6];
  R alpn_r = R(0);
  double syn_cache = 0.0;
  if (valid) {
    void* hb = const_cast<void*>(a.hist);
#pragma unroll
    for (int c = 0; c < 6; ++c) epn[c] = Stream<R>::ld(Hist<R>::comp(hb, c, ng) + gpi, pol);
    alpn_r = Stream<R>::ld(Hist<R>::comp(hb, 6, ng) + gpi, pol);
    if (sizeof(R) == 4) syn_cache = Stream<double>::ld(Hist<R>::cache(hb, ng) + gpi, pol);
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) epn[c] = R(0);
  }

  int node;   // node g of element e (also row a = g of phase 2)
  // ---- S1 gather: node g of element e; coordinates and displacements relative to node 0
  // (displacement differences taken in FP64, then rounded to R; the mixed path reads the
  // element's coordinate differences, rounded once at set-up)
  {
    node = valid ? a.conn[(int64_t)e * 8 + g] : 0;
    double u0 = a.u[3 * (int64_t)node], u1 = a.u[3 * (int64_t)node + 1], u2 = a.u[3 * (int64_t)node + 2];
    const int src = lane & 24;
    double bu0 = __shfl_sync(gmask, u0, src), bu1 = __shfl_sync(gmask, u1, src), bu2 = __shfl_sync(gmask, u2, src);
    R* dst = sGp + (size_t)le * kElStride + g * 6;
    if constexpr (sizeof(R) == 8) {
      double x0 = a.X[3 * (int64_t)node], x1 = a.X[3 * (int64_t)node + 1], x2 = a.X[3 * (int64_t)node + 2];
      double bx0 = __shfl_sync(gmask, x0, src), bx1 = __shfl_sync(gmask, x1, src), bx2 = __shfl_sync(gmask, x2, src);
      dst[0] = (R)(x0 - bx0); dst[1] = (R)(x1 - bx1); dst[2] = (R)(x2 - bx2);
    } else {
      const float* dx = a.dX32 + (int64_t)e * 21 + (g - 1) * 3;
      dst[0] = (g > 0 && valid) ? dx[0] : 0.0f;
      dst[1] = (g > 0 && valid) ? dx[1] : 0.0f;
      dst[2] = (g > 0 && valid) ? dx[2] : 0.0f;
    }
    dst[3] = (R)(u0 - bu0); dst[4] = (R)(u1 - bu1); dst[5] = (R)(u2 - bu2);
  }
  __syncwarp(gmask);

  int flag_detj = 0, flag_local = 0, flag_plastic = 0, local_iters = 0;

  if (valid) {
    const R* nd = sGp + (size_t)le * kElStride;
    // ---- S2 kinematics: dN/dxi at Gauss point g, J0 = dX/dxi, g_a = J0^{-T} dN_a
    const R c3 = R(0.57735026918962576451);
    const R xg = (g & 1) ? c3 : -c3, yg = (g & 2) ? c3 : -c3, zg = (g & 4) ? c3 : -c3;
    R dN[8][3];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const R xa = (n == 1 || n == 2 || n == 5 || n == 6) ? R(1) : R(-1);
      const R ya = (n == 2 || n == 3 || n == 6 || n == 7) ? R(1) : R(-1);
      const R za = (n >= 4) ? R(1) : R(-1);
      const R fx = R(1) + xa * xg, fy = R(1) + ya * yg, fz = R(1) + za * zg;
      dN[n][0] = R(0.125) * xa * fy * fz;
      dN[n][1] = R(0.125) * ya * fx * fz;
      dN[n][2] = R(0.125) * za * fx * fy;
    }
    R J0[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        R s = R(0);
#pragma unroll
        for (int n = 1; n < 8; ++n) s += nd[n * 6 + i] * dN[n][j];
        J0[i][j] = s;
      }
    R c00 = J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1];
    R c01 = J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2];
    R c02 = J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0];
    R det0 = J0[0][0] * c00 + J0[0][1] * c01 + J0[0][2] * c02;
    if (!(det0 > R(0))) flag_detj = 1;
    R id = Num<R>::div(R(1), det0);
    R Ji[3][3];   // inverse of J0: Ji[j][k] = d xi_j / d X_k
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2]) * id;
    Ji[1][1] = (J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0]) * id;
    Ji[2][1] = (J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1]) * id;
    Ji[0][2] = (J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1]) * id;
    Ji[1][2] = (J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2]) * id;
    Ji[2][2] = (J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0]) * id;
    R gN[8][3];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int k = 0; k < 3; ++k) gN[n][k] = dN[n][0] * Ji[0][k] + dN[n][1] * Ji[1][k] + dN[n][2] * Ji[2][k];
    // H = grad u = sum_a du_a (x) g_a ; F = I + H ; E = (H + H^T + H^T H) / 2
    R H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        R s = R(0);
#pragma unroll
        for (int n = 1; n < 8; ++n) s += nd[n * 6 + 3 + i] * gN[n][j];
        H[i][j] = s;
      }
    // the nodal data share the element's record area: every thread of the element has read
    // them before any writes its record
    __syncwarp(gmask);
    R F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? R(1) : R(0));
    R* gp = sGp + (size_t)le * kElStride + g * kGpStride;
    R fb_s = R(1);      // F-bar: (Jbar / J)^(1/3)
    R fb_jbar = R(1);   // F-bar: det Fbar = Jbar
    if constexpr (FBAR) {
      // J - 1 from the invariants of H (no cancellation at small strain); the element average
      // Jbar - 1 = sum_q w det J0_q (J_q - 1) / V_e over the element's 8 threads (Eq. Fbar)
      const R I1 = H[0][0] + H[1][1] + H[2][2];
      const R I2 = H[0][0] * H[1][1] + H[1][1] * H[2][2] + H[0][0] * H[2][2] - H[0][1] * H[1][0] -
                   H[1][2] * H[2][1] - H[0][2] * H[2][0];
      const R I3 = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) - H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                   H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
      const R jm1 = I1 + I2 + I3;
      R wj = det0 * jm1, wv = det0;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        wj += __shfl_xor_sync(gmask, wj, o);
        wv += __shfl_xor_sync(gmask, wv, o);
      }
      const R jbm1 = Num<R>::div(wj, wv);
      const R sm1 = Num<R>::expm1_((Num<R>::log1p_(jbm1) - Num<R>::log1p_(jm1)) * R(1.0 / 3.0));
      fb_s = R(1) + sm1;
      fb_jbar = R(1) + jbm1;
      if constexpr (TANGENT) {
        // v_b = dJbar/du_b / (3 Jbar) - (1/3) F^-T g_b, with dJbar/du_b = (1/V) sum_q w det J0_q
        // J_q F_q^-T g_b,q and J F^-T = cof(F): the non-symmetric rank-one part of K^e
        R cof[3][3];
        cof[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
        cof[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
        cof[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
        cof[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
        cof[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
        cof[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
        cof[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
        cof[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
        cof[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
        const R iJ = Num<R>::div(R(1), R(1) + jm1);
        const R iV = Num<R>::div(R(1), wv);
        const R i3jb = Num<R>::div(R(1), R(3) * fb_jbar);
        R vv[24];
#pragma unroll
        for (int n = 0; n < 8; ++n)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const R cg = cof[k][0] * gN[n][0] + cof[k][1] * gN[n][1] + cof[k][2] * gN[n][2];   // (J F^-T g_n)_k
            R b = det0 * cg;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) b += __shfl_xor_sync(gmask, b, o);
            vv[n * 3 + k] = b * iV * i3jb - R(1.0 / 3.0) * cg * iJ;
          }
#pragma unroll
        for (int k = 0; k < 6; ++k) V4<R>::st(gp + kOffV + 4 * k, vv[4 * k], vv[4 * k + 1], vv[4 * k + 2], vv[4 * k + 3]);
      }
      // Fbar = s F enters the constitutive model: H <- Fbar - I = H + (s - 1) F
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          H[i][j] += sm1 * F[i][j];
          F[i][j] *= fb_s;
        }
    }
    R Em[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        R s = H[i][j] + H[j][i];
#pragma unroll
        for (int k = 0; k < 3; ++k) s += H[k][i] * H[k][j];
        Em[i][j] = Em[j][i] = R(0.5) * s;
      }
    R detF = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
             F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
    if (!(detF > R(0))) flag_detj = 1;
    if constexpr (FBAR) {
      if (!(fb_jbar > R(0))) flag_detj = 1;
    }

    // ---- S3 log strain: E = Q diag(e) Q^T, C = I + 2E, eps = sum_a 1/2 log1p(2 e_a) n_a (x) n_a
    R ev[3], Q[3][3];
    jacobi3<R>(Em, ev, Q);
    swap_pair<R>(ev, Q, 0, 1);
    swap_pair<R>(ev, Q, 1, 2);
    swap_pair<R>(ev, Q, 0, 1);
    if (!(R(1) + R(2) * ev[0] > R(0))) flag_detj = 1;
    R epa[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) epa[k] = R(0.5) * Num<R>::log1p_(R(2) * ev[k]);
    R epsM[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const int i = pI(p), j = pJ(p);
      R s = Q[i][0] * epa[0] * Q[j][0] + Q[i][1] * epa[1] * Q[j][1] + Q[i][2] * epa[2] * Q[j][2];
      epsM[p] = (i == j) ? s : R(kSq2) * s;
    }

    if constexpr (MAT == 1) {
      // strain pass of an external material: the Mandel log strain out, nothing else
#pragma unroll
      for (int p = 0; p < 6; ++p) a.ext_eps[gpi * 6 + p] = (double)epsM[p];
    } else {
    // ---- S4 elastic predictor (Eq. Tr_stress) and return mapping in the Hill eigenbasis
    const double alpn = (double)alpn_r;
    const MR& m = UNIF ? mrec : matR[mi];
    const R lam = m.lam, mu = m.mu;
    bool plastic = false;
    RM rm;
    rm.dgamma = 0.0; rm.dsy = 0.0f; rm.iters = 0; rm.ok = true; rm.syn1 = 0.0;
    R Teig[6];
    R s_pl = R(0), phy = R(1);
    R TM[6];
    if constexpr (MAT == 2) {
      // external material (its own kernel ran S4 and wrote the trial history): the Mandel
      // stress and the plastic flag of this Gauss point
#pragma unroll
      for (int p = 0; p < 6; ++p) TM[p] = (R)a.ext_T[gpi * 6 + p];
      plastic = a.ext_plastic[gpi] != 0;
      flag_plastic = plastic ? 1 : 0;
#pragma unroll
      for (int p = 0; p < 6; ++p) Teig[p] = R(0);
      (void)alpn;
    } else {
    R ee[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) ee[p] = epsM[p] - (p < 3 ? epn[p] : R(kSq2) * epn[p]);
    R tre = ee[0] + ee[1] + ee[2];
    R Ttr[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) Ttr[p] = R(2) * mu * ee[p] + (p < 3 ? lam * tre : R(0));
    R t[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      R s = R(0);
#pragma unroll
      for (int i = 0; i < 6; ++i) s += m.QH[i * 6 + j] * Ttr[i];
      t[j] = s;
    }
    double syn64;
    if constexpr (sizeof(R) == 8) {
      const MR& m64 = m;
      double dsy0;
      const Hard3 hp3{m64.hard[0], m64.hard[1], m64.hard[2]};
      Vec6d hv;
#pragma unroll
      for (int i = 0; i < 6; ++i) hv.v[i] = m64.h[i];
      sigy64(a.hardening, hp3, alpn, syn64, dsy0);
      double phi2 = 0.0;
#pragma unroll
      for (int i = 1; i < 6; ++i) phi2 += m64.h[i] * (double)t[i] * (double)t[i];
      double ftr = sqrt(phi2) - kSq23 * syn64;
      if (ftr > 0.0) {
        plastic = true;
        double td[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) td[i] = (double)t[i];
        rm = return_map_fp64(td, hv, m64.mu, m64.hmin, a.hardening, hp3, alpn, ftr, a.local_maxit,
                             a.local_tol);
      } else {
        rm.syn1 = syn64;
        rm.dsy = (float)dsy0;
      }
    } else {
      syn64 = syn_cache;
      const MR& mf = m;
      float phi2 = 0.0f;
#pragma unroll
      for (int i = 1; i < 6; ++i) phi2 += mf.h[i] * (float)t[i] * (float)t[i];
      const float synf = (float)syn64;
      // the band below (1e-5) is far wider than the FP32 rounding of phi_y^2
      const float phyn2 = (2.0f / 3.0f) * synf * synf;
      bool pl;
      if (phi2 > phyn2 * 1.00001f) pl = true;
      else if (phi2 < phyn2 * 0.99999f) pl = false;
      else {   // near the yield surface: decide in FP64
        double p2 = 0.0;
#pragma unroll
        for (int i = 1; i < 6; ++i) p2 += mf.h64[i] * (double)t[i] * (double)t[i];
        pl = p2 > (2.0 / 3.0) * syn64 * syn64;
      }
      HardInc inc;
      inc.type = a.hardening;
      inc.p2 = mf.hard[2];
      inc.syn = synf;
      // Swift: eps0 + alpha_n (FP32 sum of FP32 values); Voce: Q exp(-b alpha_n) by a
      // difference that cancels, in FP64
      if (a.hardening == HFE_HARDENING_SWIFT) inc.z_or_A = mf.hard[1] + alpn_r;
      else inc.z_or_A = (float)(mf.hard64[0] + mf.hard64[1] - syn64);
      if (pl) {
        plastic = true;
        float ftr = sqrtf(phi2) - (float)kSq23 * inc.syn;
        if (!(ftr > 0.0f)) ftr = 1e-30f;
        float tf[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) tf[i] = (float)t[i];
        Vec6d hv;
        Vec6f hfv;
#pragma unroll
        for (int i = 0; i < 6; ++i) { hv.v[i] = mf.h64[i]; hfv.v[i] = mf.h[i]; }
        rm = return_map_mixed(tf, hv, hfv, mf.mu, mf.hmin, inc, syn64, ftr, a.local_maxit);
      } else {
        float incv, dsy;
        inc.eval(0.0f, incv, dsy);
        rm.syn1 = syn64;
        rm.dsy = dsy;
      }
    }
    flag_plastic = plastic ? 1 : 0;
    flag_local = rm.ok ? 0 : 1;
    local_iters = rm.iters;

    // stress T and plastic update in the Hill eigenbasis, then back to Mandel components
    const R dgR = (R)rm.dgamma;
    if (plastic) {
      phy = (R)(kSq23 * rm.syn1);
      s_pl = Num<R>::div(R(2) * mu * dgR, phy);
    }
    Teig[0] = t[0];
#pragma unroll
    for (int i = 1; i < 6; ++i) Teig[i] = plastic ? Num<R>::div(t[i], R(1) + s_pl * (R)m.h[i]) : t[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      R s = R(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) s += m.QH[i * 6 + j] * Teig[j];
      TM[i] = s;
    }
    {
      void* hb = a.hist_trial;
      if (plastic) {
        R neig[6];
        neig[0] = R(0);
#pragma unroll
        for (int i = 1; i < 6; ++i) neig[i] = Num<R>::div((R)m.h[i] * Teig[i], phy);
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          R s = R(0);
#pragma unroll
          for (int j = 1; j < 6; ++j) s += m.QH[p * 6 + j] * neig[j];
          Stream<R>::st(Hist<R>::comp(hb, p, ng) + gpi, epn[p] + dgR * s * (p < 3 ? R(1) : R(kISq2)), pol);
        }
        Stream<R>::st(Hist<R>::comp(hb, 6, ng) + gpi, (R)(alpn + kSq23 * rm.dgamma), pol);
      } else {
#pragma unroll
        for (int p = 0; p < 6; ++p) Stream<R>::st(Hist<R>::comp(hb, p, ng) + gpi, epn[p], pol);
        Stream<R>::st(Hist<R>::comp(hb, 6, ng) + gpi, alpn_r, pol);
      }
      // the FP64 path keeps sigma_y(alpha_n+1) with the history; the mixed path's cache is
      // recomputed from alpha when a step is committed, so the trial cache is not written
      if constexpr (sizeof(R) == 8) Stream<double>::st(Hist<R>::cache(hb, ng) + gpi, rm.syn1, pol);
    }
    }   // MAT == 0

    // ---- S6 post-processor in the eigenbasis of C: That = Q^T T Q, Shat_ab = 2 f1_ab That_ab
    R Tt[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int p = pidx(i, j);
        Tt[i][j] = (i == j) ? TM[p] : R(kISq2) * TM[p];
      }
    R That[3][3];
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
      for (int bb = aa; bb < 3; ++bb) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          R qi = Q[i][aa];
#pragma unroll
          for (int j = 0; j < 3; ++j) s += qi * Tt[i][j] * Q[j][bb];
        }
        That[aa][bb] = That[bb][aa] = s;
      }
    R f1[3][3];
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
      for (int bb = aa; bb < 3; ++bb) {
        R v = (aa == bb) ? Num<R>::div(R(0.5), R(1) + R(2) * ev[aa]) : dd1<R>(ev[bb], ev[aa]);
        f1[aa][bb] = f1[bb][aa] = v;
      }
    R Sh[3][3];
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) Sh[aa][bb] = R(2) * f1[aa][bb] * That[aa][bb];
    // Ftilde = F Q ; Ptilde = Ftilde Shat ; gtilde_a = Q^T g_a ; weight w det J0 (w = 1)
    R Ft[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ft[i][j] = F[i][0] * Q[0][j] + F[i][1] * Q[1][j] + F[i][2] * Q[2][j];
    const R wd = det0;
    {
      R gq[24];
#pragma unroll
      for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int j = 0; j < 3; ++j) gq[n * 3 + j] = gN[n][0] * Q[0][j] + gN[n][1] * Q[1][j] + gN[n][2] * Q[2][j];
#pragma unroll
      for (int k = 0; k < 6; ++k) V4<R>::st(gp + kOffG + 4 * k, gq[4 * k], gq[4 * k + 1], gq[4 * k + 2], gq[4 * k + 3]);
      R pq[12];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) pq[i * 3 + j] = wd * (Ft[i][0] * Sh[0][j] + Ft[i][1] * Sh[1][j] + Ft[i][2] * Sh[2][j]);
      pq[9] = pq[10] = pq[11] = R(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) V4<R>::st(gp + kOffP + 4 * k, pq[4 * k], pq[4 * k + 1], pq[4 * k + 2], pq[4 * k + 3]);
    }
    if (a.sigma != nullptr) {   // Cauchy stress sigma = P F^T / J, P = Ftilde Shat Q^T
      R P[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          R s = R(0);
#pragma unroll
          for (int j = 0; j < 3; ++j) s += (Ft[i][0] * Sh[0][j] + Ft[i][1] * Sh[1][j] + Ft[i][2] * Sh[2][j]) * Q[k][j];
          P[i][k] = s;
        }
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int i = pI(p), j = pJ(p);
        R s = P[i][0] * F[j][0] + P[i][1] * F[j][1] + P[i][2] * F[j][2];
        a.sigma[gpi * 6 + p] = (double)Num<R>::div(s, FBAR ? fb_jbar : detF);
      }
    }

    if constexpr (TANGENT) {
      // ---- S5 algorithmic tangent D = dT/deps (Mandel), rotated into the eigenbasis of C
      R Dh[6][6];
      R Rq[6][6];
      mandel_rotation<R>(Q, Rq);
      if constexpr (MAT == 2) {
        // external material: D = dT/deps (Mandel) from its kernel, rotated, Dh = Rq D Rq^T
        R RD[6][6];
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            R v = R(0);
#pragma unroll
            for (int k = 0; k < 6; ++k) v += Rq[p][k] * (R)a.ext_D[gpi * 36 + k * 6 + q];
            RD[p][q] = v;
          }
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            R v = R(0);
#pragma unroll
            for (int k = 0; k < 6; ++k) v += RD[p][k] * Rq[q][k];
            Dh[p][q] = v;
          }
      } else if (!plastic) {
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
          for (int q = 0; q < 6; ++q) Dh[p][q] = (p == q ? R(2) * mu : R(0)) + (p < 3 && q < 3 ? lam : R(0));
      } else {
        // implicit function theorem on Eq. local_cpp (App. D) in the Hill eigenbasis:
        // Xi^-1 = E^-1 + dgamma (H - N (x) N) / phi, D = Xi - (Xi N)(Xi N)^T / (N Xi N + 2/3 H')
        const R iphy = Num<R>::div(R(1), phy);
        const R cph = (R)rm.dgamma * iphy;
        R nv[6], iDd[6], pv[6];
        R npn = R(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const R hi = (R)m.h[i];
          nv[i] = (i == 0) ? R(0) : hi * Teig[i] * iphy;
          const R ei = (i == 0) ? (R)m.kap3 : R(2) * mu;
          iDd[i] = Num<R>::div(R(1), Num<R>::div(R(1), ei) + cph * hi);
          pv[i] = nv[i] * iDd[i];
          npn += nv[i] * pv[i];
        }
        const R kap = Num<R>::div(cph, R(1) - cph * npn);
        const R qf = R(1) + kap * npn;
        R qv[6];
        R nqn = R(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) { qv[i] = pv[i] * qf; nqn += nv[i] * qv[i]; }
        const R beta = nqn + (R(2) / R(3)) * (R)rm.dsy;
        // W = Rq QH ; Dh = W diag(1/Dd) W^T + kap (W p)(W p)^T - (W q)(W q)^T / beta
        R W[6][6];
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            R s = R(0);
#pragma unroll
            for (int i = 0; i < 6; ++i) s += Rq[p][i] * m.QH[i * 6 + j];
            W[p][j] = s;
          }
        R Wp[6], Wq[6];
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          R s1 = R(0), s2 = R(0);
#pragma unroll
          for (int j = 0; j < 6; ++j) { s1 += W[p][j] * pv[j]; s2 += W[p][j] * qv[j]; }
          Wp[p] = s1;
          Wq[p] = s2;
        }
        const R ib = Num<R>::div(R(1), beta);
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
          for (int q = p; q < 6; ++q) {
            R s = R(0);
#pragma unroll
            for (int j = 0; j < 6; ++j) s += W[p][j] * W[q][j] * iDd[j];
            s += kap * Wp[p] * Wp[q] - ib * Wq[p] * Wq[q];
            Dh[p][q] = Dh[q][p] = s;
          }
      }
      // material tangent in the eigenbasis: Chat = 4 diag(f1) Dh diag(f1) + 4 D^2eps[That, .]
      R f1M[6];
#pragma unroll
      for (int p = 0; p < 6; ++p) f1M[p] = f1[pI(p)][pJ(p)];
      // second divided differences on the sorted eigenvalues (10 distinct values)
      R f2[3][3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
#pragma unroll
          for (int k = j; k < 3; ++k) {
            R v = dd2<R>(ev[i], ev[j], ev[k], f1[k][j], f1[j][i]);
            f2[i][j][k] = f2[i][k][j] = f2[j][i][k] = f2[j][k][i] = f2[k][i][j] = f2[k][j][i] = v;
          }
      R Ct[6][6];   // tensor-component matrix of Chat (no Mandel factors)
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int aa = pI(p), bb = pJ(p);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const int cc = pI(q), dd = pJ(q);
          // G(Y)_ab = 4 sum_k f2(a,k,b) (That_ak Y_kb + Y_ak That_kb) for the Mandel unit Y_q
          R gsum = R(0);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            R ykb = ((k == cc && bb == dd) || (k == dd && bb == cc)) ? R(1) : R(0);
            R yak = ((aa == cc && k == dd) || (aa == dd && k == cc)) ? R(1) : R(0);
            if (cc != dd) { ykb *= R(kISq2); yak *= R(kISq2); }
            gsum += f2[aa][k][bb] * (That[aa][k] * ykb + yak * That[k][bb]);
          }
          R cm = R(4) * f1M[p] * Dh[p][q] * f1M[q] + R(4) * gsum * (aa == bb ? R(1) : R(kSq2));
          Ct[p][q] = cm * (aa == bb ? R(1) : R(kISq2)) * (cc == dd ? R(1) : R(kISq2));
        }
      }
      // A_iJkL = delta_ik Shat_JL + sum_IK Ft_iI Chat_IJKL Ft_kK, scaled by w det J0
      R Xt[3][3][6];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J)
#pragma unroll
          for (int q = 0; q < 6; ++q)
            Xt[i][J][q] = Ft[i][0] * Ct[pidx(0, J)][q] + Ft[i][1] * Ct[pidx(1, J)][q] + Ft[i][2] * Ct[pidx(2, J)][q];
      R av[48];
#pragma unroll
      for (int P = 0; P < 9; ++P)
#pragma unroll
        for (int Qi = P; Qi < 9; ++Qi) {
          const int i = P / 3, J = P % 3, k = Qi / 3, L = Qi % 3;
          R s = Xt[i][J][pidx(0, L)] * Ft[k][0] + Xt[i][J][pidx(1, L)] * Ft[k][1] + Xt[i][J][pidx(2, L)] * Ft[k][2];
          if (i == k) s += Sh[J][L];
          av[asym(P, Qi)] = wd * s;
        }
      av[45] = av[46] = av[47] = R(0);
      if constexpr (FBAR) {
        // K^e = sum_q [ g_a . (s A) . g_b + (M g_a) (x) v_b ] with M = w det J0 A : Fbar (the
        // stored gradients are rotated, so Fbar enters as Fbar Q = Ft)
        R mv[12];
#pragma unroll
        for (int P = 0; P < 9; ++P) {
          R m = R(0);
#pragma unroll
          for (int Qi = 0; Qi < 9; ++Qi) m += av[asym(P, Qi)] * Ft[Qi / 3][Qi % 3];
          mv[P] = m;
        }
        mv[9] = mv[10] = mv[11] = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) V4<R>::st(gp + kOffM + 4 * k, mv[4 * k], mv[4 * k + 1], mv[4 * k + 2], mv[4 * k + 3]);
#pragma unroll
        for (int k = 0; k < 45; ++k) av[k] *= fb_s;
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) V4<R>::st(gp + 4 * k, av[4 * k], av[4 * k + 1], av[4 * k + 2], av[4 * k + 3]);
    }
    }   // MAT != 1
  }

  // ---- status counters (one atomic per warp and counter)
  {
    const unsigned full = 0xffffffffu;
    unsigned bd = __ballot_sync(full, flag_detj), bl = __ballot_sync(full, flag_local);
    unsigned bp = __ballot_sync(full, flag_plastic);
    int mx = local_iters;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(full, mx, o));
    if (lane == 0) {
      if (bd) atomicAdd(&a.status->detj, __popc(bd));
      if (bl) atomicAdd(&a.status->local_fail, __popc(bl));
      if (bp) atomicAdd(&a.status->plastic, __popc(bp));
      if (mx > 0) atomicMax(&a.status->max_local_iters, mx);
    }
  }
  // an element's Gauss-point records are written and read by its own 8 threads, all in one
  // warp: a warp barrier suffices, and warps move on independently
  __syncwarp();
  if constexpr (MAT == 1) return;   // the strain pass assembles nothing
  // launched as a dependent of the previous launch: its writes to K and R must be complete
  // and visible before this launch adds to the same blocks (a no-op for the first launch)
  asm volatile("griddepcontrol.wait;\n" ::: "memory");

  // ---- S7/S8 phase 2: thread (element le, node row a = g)
  if constexpr (TANGENT) {
    // the element matrix: contraction, then the warp's four elements are staged row-major in
    // shared memory and written out with consecutive lanes on consecutive entries (a block's 9
    // values are contiguous in K), so that a warp store touches a few 32-byte sectors instead
    // of 32 scattered ones
    phase2_staged<R, FBAR>(a, sGp, le, g, e, lane, valid, node, blockIdx.x, ccount, pol);
    return;
  }
  if (!valid) return;
  const R* G = sGp + (size_t)le * kElStride;
  R Ra[3] = {R(0), R(0), R(0)};
  const int arow = g;
  {
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      const R* Aq = G + q * kGpStride;
      const R* gt = Aq + kOffG;
      const R ga0 = gt[arow * 3], ga1 = gt[arow * 3 + 1], ga2 = gt[arow * 3 + 2];
      R P[12];
#pragma unroll
      for (int k = 0; k < 3; ++k) V4<R>::ld(Aq + kOffP + 4 * k, P + 4 * k);
#pragma unroll
      for (int i = 0; i < 3; ++i) Ra[i] += P[i * 3] * ga0 + P[i * 3 + 1] * ga1 + P[i * 3 + 2] * ga2;
    }
  }
  {
    // node of row a = g is the node this thread gathered in phase 1
    const bool store = Stream<int32_t>::ld(a.slot + (int64_t)e * 64 + arow * 9, pol) < 0;   // diagonal block (a, a)
    double* Rg = a.R + 3 * (int64_t)node;
    if (!(isfinite(Ra[0]) && isfinite(Ra[1]) && isfinite(Ra[2])))
      atomicAdd(&a.status->nonfinite, 1);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double v = (double)Ra[i];
      if (store) Rg[i] = v - (a.f_ext ? a.load * a.f_ext[3 * (int64_t)node + i] : 0.0);
      else atomicAdd(Rg + i, v);
    }
  }
}

// ----------------------------------------------------------------------------------------
// Material set-up (one thread per material): Lame constants, the Hill tensor in Mandel
// notation from (F, G, H, L, M, N) — phi^2 = (2/3)[F (T22-T33)^2 + G (T33-T11)^2 +
// H (T11-T22)^2 + 2L T23^2 + 2M T13^2 + 2N T12^2] in the material frame (App. A.1 written in
// the Hill constants) — rotated by Theta (X -> Theta^T X Theta), and its eigen-decomposition
// by cyclic Jacobi in FP64.  The hydrostatic direction is pinned as eigenvector 0.
__global__ void material_setup_kernel(const double* theta, const double* Theta, int64_t n_mat, MatRec* out,
                                      MatRecF* outf, int* bad) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_mat) return;
  const double* th = theta + id * 11;
  const double E = th[0], nu = th[1];
  const double Fh = th[2], Gh = th[3], Hh = th[4], Lh = th[5], Mh = th[6], Nh = th[7];
  MatRec r;
  r.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  r.mu = E / (2.0 * (1.0 + nu));
  r.kap3 = 3.0 * r.lam + 2.0 * r.mu;
  r.hard[0] = th[8];
  r.hard[1] = th[9];
  r.hard[2] = th[10];
  r.pad = 0.0;
  double Hl[6][6] = {};
  const double c = 2.0 / 3.0;
  Hl[0][0] = c * (Gh + Hh); Hl[1][1] = c * (Fh + Hh); Hl[2][2] = c * (Fh + Gh);
  Hl[0][1] = Hl[1][0] = -c * Hh;
  Hl[1][2] = Hl[2][1] = -c * Fh;
  Hl[0][2] = Hl[2][0] = -c * Gh;
  Hl[3][3] = c * Nh; Hl[4][4] = c * Lh; Hl[5][5] = c * Mh;
  double Hg[6][6];
  if (Theta != nullptr) {
    double Th[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Th[i][j] = Theta[id * 9 + i * 3 + j];
    double Rt[6][6];
    mandel_rotation<double>(Th, Rt);   // local Mandel = Rt * global Mandel
    double tmp[6][6];
    for (int p = 0; p < 6; ++p)
      for (int q = 0; q < 6; ++q) {
        double s = 0.0;
        for (int k = 0; k < 6; ++k) s += Hl[p][k] * Rt[k][q];
        tmp[p][q] = s;
      }
    for (int p = 0; p < 6; ++p)
      for (int q = 0; q < 6; ++q) {
        double s = 0.0;
        for (int k = 0; k < 6; ++k) s += Rt[k][p] * tmp[k][q];
        Hg[p][q] = s;
      }
  } else {
    for (int p = 0; p < 6; ++p)
      for (int q = 0; q < 6; ++q) Hg[p][q] = Hl[p][q];
  }
  // shift the hydrostatic eigenvalue 0 to -1 so that it is isolated: A = Hg - v0 v0^T
  const double v0 = 0.57735026918962576451;
  double A[6][6], V[6][6];
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q) {
      A[p][q] = Hg[p][q] - ((p < 3 && q < 3) ? v0 * v0 : 0.0);
      V[p][q] = (p == q) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < 6; ++p) {
      dia += A[p][p] * A[p][p];
      for (int q = p + 1; q < 6; ++q) off += A[p][q] * A[p][q];
    }
    if (off <= 1e-32 * dia) break;
    for (int p = 0; p < 5; ++p)
      for (int q = p + 1; q < 6; ++q) {
        double apq = A[p][q];
        if (apq == 0.0) continue;
        double thv = (A[q][q] - A[p][p]) / (2.0 * apq);
        double t = (fabs(thv) > 1e15) ? 0.5 / thv : (thv >= 0 ? 1.0 : -1.0) / (fabs(thv) + sqrt(thv * thv + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        A[p][p] -= t * apq;
        A[q][q] += t * apq;
        A[p][q] = A[q][p] = 0.0;
        for (int k = 0; k < 6; ++k) {
          if (k == p || k == q) continue;
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = A[p][k] = cs * akp - sn * akq;
          A[k][q] = A[q][k] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 6; ++k) {
          double vp = V[k][p], vq = V[k][q];
          V[k][p] = cs * vp - sn * vq;
          V[k][q] = sn * vp + cs * vq;
        }
      }
  }
  int i0 = 0;
  for (int j = 1; j < 6; ++j)
    if (fabs(A[j][j] + 1.0) < fabs(A[i0][i0] + 1.0)) i0 = j;
  // order: hydrostatic first, then the others in their Jacobi order
  int ord[6];
  ord[0] = i0;
  for (int j = 0, k = 1; j < 6; ++j)
    if (j != i0) ord[k++] = j;
  double hmin = 1e300;
  for (int k = 0; k < 6; ++k) {
    int j = ord[k];
    double hv = (k == 0) ? 0.0 : A[j][j];
    r.h[k] = hv;
    if (k > 0 && hv < hmin) hmin = hv;
    for (int i = 0; i < 6; ++i) r.QH[i * 6 + k] = V[i][j];
  }
  // exact hydrostatic vector, other columns re-orthogonalised against it
  for (int i = 0; i < 6; ++i) r.QH[i * 6 + 0] = (i < 3) ? v0 : 0.0;
  for (int k = 1; k < 6; ++k) {
    double d = v0 * (r.QH[0 * 6 + k] + r.QH[1 * 6 + k] + r.QH[2 * 6 + k]);
    double nn = 0.0;
    for (int i = 0; i < 6; ++i) {
      r.QH[i * 6 + k] -= d * ((i < 3) ? v0 : 0.0);
      nn += r.QH[i * 6 + k] * r.QH[i * 6 + k];
    }
    double inv = 1.0 / sqrt(nn);
    for (int i = 0; i < 6; ++i) r.QH[i * 6 + k] *= inv;
  }
  r.hmin = hmin;
  if (!(hmin > 0.0) || !(r.mu > 0.0) || !(r.kap3 > 0.0) || !isfinite(hmin)) atomicAdd(bad, 1);
  out[id] = r;
  if (outf != nullptr) {
    MatRecF f;
    for (int k = 0; k < 6; ++k) f.h64[k] = r.h[k];
    f.mu64 = r.mu;
    for (int k = 0; k < 3; ++k) f.hard64[k] = r.hard[k];
    f.lam = (float)r.lam; f.mu = (float)r.mu; f.kap3 = (float)r.kap3;
    for (int k = 0; k < 6; ++k) f.h[k] = (float)r.h[k];
    f.hmin = (float)r.hmin;
    for (int k = 0; k < 36; ++k) f.QH[k] = (float)r.QH[k];
    for (int k = 0; k < 3; ++k) f.hard[k] = (float)r.hard[k];
    f.pad = 0.0f;
    outf[id] = f;
  }
}

// sigma_y(alpha) cache recomputed in FP64 from alpha (history component 6).
template <typename R>
__global__ void sigma_cache_kernel(void* hist, const MatRec* mat, int per_element, int type, int64_t n_gp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_gp) return;
  const MatRec& m = mat[per_element ? (i >> 3) : 0];
  double sy, dsy;
  sigy64(type, Hard3{m.hard[0], m.hard[1], m.hard[2]}, (double)Hist<R>::comp(hist, 6, n_gp)[i], sy, dsy);
  Hist<R>::cache(hist, n_gp)[i] = sy;
}

template <typename R>
__global__ void hist_import_kernel(const double* user, void* hist, int64_t n_gp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 7 * n_gp) return;
  Hist<R>::comp(hist, 0, n_gp)[i] = (R)user[i];
}

template <typename R>
__global__ void hist_export_kernel(const void* hist, double* user, int64_t n_gp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 7 * n_gp) return;
  user[i] = (double)Hist<R>::comp(const_cast<void*>(hist), 0, n_gp)[i];
}

}  // namespace

void launch_material_setup(const double* theta, const double* Theta, int64_t n_mat, MatRec* out,
                                MatRecF* outf, int* bad, cudaStream_t s) {
  int threads = 64;
  int blocks = (int)((n_mat + threads - 1) / threads);
  material_setup_kernel<<<blocks, threads, 0, s>>>(theta, Theta, n_mat, out, outf, bad);
}

void launch_sigma_cache(void* hist, bool fp64, const MatRec* mat, int mat_per_element, int hardening, int64_t n_gp,
                        cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((n_gp + threads - 1) / threads);
  if (fp64) sigma_cache_kernel<double><<<blocks, threads, 0, s>>>(hist, mat, mat_per_element, hardening, n_gp);
  else sigma_cache_kernel<float><<<blocks, threads, 0, s>>>(hist, mat, mat_per_element, hardening, n_gp);
}

void launch_hist_import(const double* user, void* hist, bool fp64, int64_t n_gp, cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((7 * n_gp + threads - 1) / threads);
  if (fp64) hist_import_kernel<double><<<blocks, threads, 0, s>>>(user, hist, n_gp);
  else hist_import_kernel<float><<<blocks, threads, 0, s>>>(user, hist, n_gp);
}

void launch_hist_export(const void* hist, double* user, bool fp64, int64_t n_gp, cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((7 * n_gp + threads - 1) / threads);
  if (fp64) hist_export_kernel<double><<<blocks, threads, 0, s>>>(hist, user, n_gp);
  else hist_export_kernel<float><<<blocks, threads, 0, s>>>(hist, user, n_gp);
}

template <typename R, bool TANGENT, bool UNIF, bool FBAR, int MAT = 0>
static void launch_typed(const SweepArgs& a, const std::vector<int64_t>& off, cudaStream_t s) {
  using MR = typename MatOf<R>::T;
  const size_t smem = sizeof(R) * (size_t)kElemsPerCta * Lay<FBAR>::kElStride;
  // the dynamic shared-memory limit is a per-device function attribute: set it on every call
  // (a host-side call, no synchronisation) so that each device the handle runs on has it
  cudaFuncSetAttribute(gp_sweep_kernel<R, TANGENT, UNIF, FBAR, MAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  MR rec;
  if (UNIF) memcpy(&rec, a.mat_host, sizeof(MR));   // host copy of the single record
  else memset(&rec, 0, sizeof(MR));
  // launches after the first are programmatic dependents of the previous launch: their
  // Gauss-point updates (phase 1) overlap the previous launch's last CTAs, and their assembly
  // (phase 2) waits for that launch to complete (griddepcontrol.wait).  The first launch is
  // an ordinary one: it reads what the kernels before the sweep wrote (u).
  bool first = true;
  for (size_t c = 0; c + 1 < off.size(); ++c) {
    int64_t cnt = off[c + 1] - off[c];
    if (cnt <= 0) continue;
    unsigned blocks = (unsigned)((cnt + kElemsPerCta - 1) / kElemsPerCta);
    if (first) {
      gp_sweep_kernel<R, TANGENT, UNIF, FBAR, MAT><<<blocks, kThreads, smem, s>>>(a, rec, off[c], cnt);
      first = false;
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, gp_sweep_kernel<R, TANGENT, UNIF, FBAR, MAT>, a, rec, off[c], cnt);
  }
}

template <typename R, bool FBAR>
static int64_t resident_ctas() {
  const size_t smem = sizeof(R) * (size_t)kElemsPerCta * Lay<FBAR>::kElStride;
  auto* k = gp_sweep_kernel<R, true, true, FBAR, 0>;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess)
    return -1;
  return (int64_t)per_sm * sms;
}

int64_t sweep_resident_ctas(bool fp64, bool fbar) {
  if (fp64) return fbar ? resident_ctas<double, true>() : resident_ctas<double, false>();
  return fbar ? resident_ctas<float, true>() : resident_ctas<float, false>();
}

int64_t sweep_elems_per_cta() { return kElemsPerCta; }

template <typename R, bool FBAR>
static void launch_mode(const SweepArgs& a, int mode, const std::vector<int64_t>& off, cudaStream_t s) {
  const bool u = a.mat_host != nullptr;
  if (mode == HFE_SWEEP_TANGENT) u ? launch_typed<R, true, true, FBAR>(a, off, s) : launch_typed<R, true, false, FBAR>(a, off, s);
  else u ? launch_typed<R, false, true, FBAR>(a, off, s) : launch_typed<R, false, false, FBAR>(a, off, s);
}

void launch_gp_sweep_ext(const SweepArgs& a, bool fp64, int pass, int mode, const std::vector<int64_t>& launch_off,
                         cudaStream_t s) {
  if (fp64) {
    if (pass == 1) launch_typed<double, false, true, false, 1>(a, launch_off, s);
    else if (mode == HFE_SWEEP_TANGENT) launch_typed<double, true, true, false, 2>(a, launch_off, s);
    else launch_typed<double, false, true, false, 2>(a, launch_off, s);
  } else {
    if (pass == 1) launch_typed<float, false, true, false, 1>(a, launch_off, s);
    else if (mode == HFE_SWEEP_TANGENT) launch_typed<float, true, true, false, 2>(a, launch_off, s);
    else launch_typed<float, false, true, false, 2>(a, launch_off, s);
  }
}

void launch_gp_sweep(const SweepArgs& a, bool fp64, int mode, const std::vector<int64_t>& launch_off,
                     cudaStream_t s) {
  if (fp64) a.fbar ? launch_mode<double, true>(a, mode, launch_off, s) : launch_mode<double, false>(a, mode, launch_off, s);
  else a.fbar ? launch_mode<float, true>(a, mode, launch_off, s) : launch_mode<float, false>(a, mode, launch_off, s);
}

}  // namespace hfe
