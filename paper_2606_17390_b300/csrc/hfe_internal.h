// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hfe.h"

namespace hfe {

// Per-material record (FP64).  The Hill tensor is held in Mandel notation
// (t = (T11, T22, T33, sqrt2 T12, sqrt2 T23, sqrt2 T13)) through its eigen-decomposition
// H_M = QH diag(h) QH^T; column 0 of QH is the hydrostatic direction (1,1,1,0,0,0)/sqrt3
// with h[0] = 0 (the Hill tensor is pressure-insensitive), so the isotropic elasticity is
// diagonal in the same basis with eigenvalues kap3 = 3 lambda + 2 mu (column 0) and 2 mu.
struct MatRec {
  double lam, mu, kap3;
  double h[6];
  double hmin;        // smallest deviatoric eigenvalue of H_M
  double QH[36];      // QH[i*6 + j]: component i of eigenvector j
  double hard[3];     // hardening parameters (h1, h2, h3)
  double pad;
};

// Mixed-precision record: FP32 copies for the FP32 arithmetic, plus the FP64 values the
// FP64 steps of the return mapping need.
struct MatRecF {
  double h64[6];
  double mu64;
  double hard64[3];
  float lam, mu, kap3;
  float h[6];
  float hmin;
  float QH[36];
  float hard[3];
  float pad;
};

// Device status counters written by the kernels (read back by the host after each call).
struct DevStatus {
  int local_fail;      // return mappings that hit the iteration bound
  int nonfinite;       // non-finite values met
  int detj;            // det(dX/dxi) <= 0 or det F <= 0 or stretch <= 0
  int max_local_iters;
  int plastic;         // plastic Gauss points in the sweep
  int krylov_breakdown;
  int pad[2];
};

// History storage.  FP64 path: double [8][n_gp] = eps_p (6), alpha, sigma_y(alpha).
// Mixed path: float [7][n_gp] = eps_p (6), alpha, followed by double [n_gp] sigma_y(alpha)
// at byte offset 28 n_gp (the FP64 yield-stress cache of the FP64 return-mapping steps).
inline size_t hist_bytes(int64_t n_gp, bool fp64) { return fp64 ? 64 * (size_t)n_gp : 36 * (size_t)n_gp; }

struct SweepArgs {
  const double* X;         // [n_nodes*3]
  const float* dX32;       // [n_el*21] X_a - X_0 of nodes 1..7 (mixed path)
  const int32_t* conn;     // [n_el*8]
  const double* u;         // [n_dof]
  const void* hist;        // layout above
  void* hist_trial;
  const void* mat;         // MatRec* or MatRecF* (device)
  const void* mat_host;    // host copy of the record when one material serves every element, else nullptr
  int mat_per_element;
  int hardening;
  const int32_t* elems;    // element ids in launch order (conflict-free ranges)
  const int32_t* slot;     // [n_el*64] block index | store flag (bit 31)
  void* K;                 // [n_blocks*9] float or double
  double* R;               // [n_dof]
  const double* f_ext;     // [n_dof] or nullptr
  double load;
  double* sigma;           // [n_gp*6] Cauchy stress output or nullptr
  DevStatus* status;
  int64_t n_gp;
  int local_maxit;
  double local_tol;
  int fbar;                // F-bar element (Eq. Fbar)
  // external material model (FP64, uniform material, standard element): the strain pass
  // writes ext_eps; the assembly pass reads ext_T, ext_D and ext_plastic
  double* ext_eps;         // [n_gp*6] Mandel log strain
  const double* ext_T;     // [n_gp*6] Mandel stress
  const double* ext_D;     // [n_gp*36] Mandel dT/deps, row-major
  const uint8_t* ext_plastic;   // [n_gp]
};

void launch_material_setup(const double* theta, const double* Theta, int64_t n_mat, MatRec* out,
                           MatRecF* outf, int* bad, cudaStream_t s);
// mode: HFE_SWEEP_RESIDUAL / HFE_SWEEP_TANGENT; fp64 selects the plain FP64 kernel.
// CTAs of the tangent sweep kernel resident on the current device at once (occupancy x SMs;
// <= 0 on a failed query), and the elements one CTA takes
int64_t sweep_resident_ctas(bool fp64, bool fbar);
int64_t sweep_elems_per_cta();
void launch_gp_sweep(const SweepArgs& a, bool fp64, int mode, const std::vector<int64_t>& launch_off,
                     cudaStream_t s);
// The Barlat Yld2004-18p material of a handle (barlat.cu): parameters and local controls,
// and the strain-driven update of every Gauss point between the two external sweep passes.
struct BarlatModel;
BarlatModel* barlat_model_new(const hfe_barlat_material* mat, const hfe_cpp_options* opt, hfe_status* st);
void barlat_model_free(BarlatModel* m);
// hist / hist_trial in the handle's layout (fp64: double [8][n_gp]; mixed: float [7][n_gp] and
// the FP64 sigma_y cache); work: [n_gp*15] doubles, iters: [n_gp] int32, st: [n_gp] int8
void launch_barlat_gp(const BarlatModel* m, bool fp64_hist, const double* eps_M, const void* hist,
                      void* hist_trial, int64_t n_gp, double* T_M, double* D_M, uint8_t* plastic, int tangent,
                      DevStatus* status, double* work, int32_t* iters, int8_t* st, cudaStream_t s);
// External material model (FP64 or mixed sweep): pass 1 = strain pass (ext_eps out), pass 2 =
// assembly with ext_T / ext_D / ext_plastic (mode HFE_SWEEP_RESIDUAL or HFE_SWEEP_TANGENT).
void launch_gp_sweep_ext(const SweepArgs& a, bool fp64, int pass, int mode, const std::vector<int64_t>& launch_off,
                         cudaStream_t s);
void launch_sigma_cache(void* hist, bool fp64, const MatRec* mat, int mat_per_element, int hardening,
                        int64_t n_gp, cudaStream_t s);
// user layout double [7][n_gp] <-> internal layout (the cache is not touched)
void launch_hist_import(const double* user, void* hist, bool fp64, int64_t n_gp, cudaStream_t s);
void launch_hist_export(const void* hist, double* user, bool fp64, int64_t n_gp, cudaStream_t s);

}  // namespace hfe
