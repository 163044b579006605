// Library handle and host helpers shared by the translation units (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hfe_internal.h"
#include "pattern.h"
#include "solver.h"

namespace hfe {
struct AdjointWork;
struct StepHook;
}  // namespace hfe

using hfe::DevStatus;
using hfe::MatRec;
using hfe::MatRecF;
using hfe::Pattern;
using hfe::PcgScalars;

namespace hfe {
// One linear system: block-CSR values in the pattern of the handle and the Krylov workspace
// (precision R = double if fp64 else float), with its CUDA graph of CG iterations.
struct LinSys {
  void* K = nullptr;
  void *vx = nullptr, *vr = nullptr, *vz = nullptr, *vp = nullptr, *vq = nullptr, *vminv = nullptr;
  void* vp2 = nullptr;   // second search direction (persistent CG)
  void *vrh = nullptr, *vy = nullptr, *vt = nullptr;   // BiCGSTAB work vectors
  void* vxt = nullptr;   // truncated-CG direction kept while BiCGSTAB runs
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  bool fp64 = true;
};
}  // namespace hfe

struct hfe_handle {
  hfe_options opt;
  int fp64 = 1;
  cudaStream_t user = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
  int64_t n_nodes = 0, n_el = 0, n_dof = 0, n_gp = 0, n_fixed = 0, n_mat = 1;
  int hardening = 0;
  Pattern P;
  // Barlat Yld2004-18p material (hfe_set_barlat; FP64 handles): the model and the per-Gauss-
  // point exchange buffers of its sweep (Mandel strain, stress, tangent, plastic flag)
  hfe::BarlatModel* barlat = nullptr;
  double *ext_eps = nullptr, *ext_T = nullptr, *ext_D = nullptr, *ext_work = nullptr;
  uint8_t* ext_pl = nullptr;
  int32_t* ext_it = nullptr;
  int8_t* ext_st = nullptr;
  // device buffers
  double* X = nullptr;
  int32_t* conn = nullptr;
  double* u = nullptr;
  void* hist = nullptr;         // internal history layout (hist_bytes)
  void* hist_trial = nullptr;
  float* dX32 = nullptr;        // mixed path: per-element coordinate differences
  double* hist_io = nullptr;    // FP64 [7][n_gp] staging for state transfer (lazy)
  int64_t* rowptr = nullptr;
  int32_t* cols = nullptr;
  int32_t* chunk32 = nullptr;   // row chunks of the streamed CG SpMV, FP32 / FP64 values
  int32_t* chunk64 = nullptr;
  int64_t n_chunk32 = 0, n_chunk64 = 0;
  int64_t* diag_slot = nullptr;
  int32_t* slot = nullptr;
  int32_t* elems = nullptr;
  void* K = nullptr;
  double* R = nullptr;
  double* f_ext = nullptr;
  int64_t* fixed_dof = nullptr;
  double* fixed_val = nullptr;
  uint8_t* freem = nullptr;
  double* theta = nullptr;
  double* Theta = nullptr;
  MatRec* mat64 = nullptr;
  MatRecF* matf = nullptr;
  MatRec h_mat64;               // host copies of the record when n_mat == 1
  MatRecF h_matf;
  DevStatus* status = nullptr;
  PcgScalars* sc = nullptr;
  double* part = nullptr;
  int* bad = nullptr;
  void* vx = nullptr; void* vr = nullptr; void* vz = nullptr; void* vp = nullptr; void* vq = nullptr;
  void* vminv = nullptr;
  double* tmp64 = nullptr;     // n_dof doubles
  double* b64 = nullptr;       // n_dof doubles (predictor right-hand side)
  double t_state = 0.0;        // load factor of the stored state
  double pcg_rtol_now = 0.0;   // CG tolerance of the current Newton solve (0: opt.pcg_rtol)
  bool allow_truncated = false;  // Newton solves may stop at negative curvature
  bool allow_indefinite = false; // Newton and adjoint solves: indefinite K -> BiCGSTAB
  bool pcg_truncated = false;
  int64_t n_bicgstab = 0;        // Newton corrections solved by the BiCGSTAB fallback
  // K and R in the handle are those of the last Newton iteration of the step that produced
  // the stored state (the next step's predictor reuses them); cleared by anything that
  // changes the state, the material or K
  bool pred_valid = false;
  double* u_start = nullptr;     // start-of-step displacement, restored when a step fails
  double* sigma = nullptr;     // n_gp * 6, allocated on demand
  // warm start: the displacement each pass converged to at its requested load factors
  // (warm_t[k], slot k of warm_u, warm_cap slots of n_dof doubles), kept across passes
  // extrapolated predictor: the last converged (sub)step solutions, newest first (extrap_n
  // valid of 3 slots of n_dof doubles, allocated when options.predictor >= 2)
  double* extrap_u[3] = {nullptr, nullptr, nullptr};
  double extrap_t[3] = {0.0, 0.0, 0.0};
  int extrap_n = 0;
  int warm_mode = 0;
  double* warm_u = nullptr;
  int warm_cap = 0;
  std::vector<double> warm_t;
  // pinned host mirrors of the device scalars
  PcgScalars* h_sc = nullptr;
  DevStatus* h_status = nullptr;
  int* h_bad = nullptr;
  hfe::LinSys ls;              // the handle's own system (K and vectors above)
  hfe::LinSys ls_fb64;         // F-bar on the mixed path: FP64 copy of K and FP64 Krylov vectors
  size_t device_bytes = 0;
  std::string err;
  std::vector<void*> allocs;
  hfe::AdjointWork* adj = nullptr;
};

// The handle's block-CSR pattern with the row chunks of the streamed CG SpMV.
inline hfe::Csr csr_of(const hfe_handle* h) {
  hfe::Csr K{h->rowptr, h->cols, h->n_nodes, h->P.n_blocks};
  K.chunk32 = h->chunk32;
  K.n_chunk32 = h->n_chunk32;
  K.chunk64 = h->chunk64;
  K.n_chunk64 = h->n_chunk64;
  return K;
}


namespace hfe {

#define HFE_TRY(expr)              \
  do {                             \
    hfe_status _st = (expr);       \
    if (_st != HFE_OK) return _st; \
  } while (0)

// Called by the Newton driver around each commit (used by the adjoint's forward pass).
struct StepHook {
  virtual ~StepHook() {}
  // t_new: load factor of the (sub)step being committed; marker: index of the requested
  // load factor it reaches, -1 for an intermediate substep of adaptive stepping
  virtual hfe_status before_commit(hfe_handle* h, double t_new) = 0;
  virtual hfe_status after_commit(hfe_handle* h, double t_new, int marker) = 0;
};

// order the internal stream after the caller's stream, and the caller's after ours on exit
struct StreamScope {
  hfe_handle* h;
  explicit StreamScope(hfe_handle* hh) : h(hh) {
    cudaEventRecord(h->ev_in, h->user);
    cudaStreamWaitEvent(h->s, h->ev_in, 0);
  }
  ~StreamScope() {
    cudaEventRecord(h->ev_out, h->s);
    cudaStreamWaitEvent(h->user, h->ev_out, 0);
  }
};

hfe_status fail(hfe_handle* h, hfe_status st, const std::string& msg);
hfe_status cuda_check(hfe_handle* h, cudaError_t e, const char* what);
template <typename T>
hfe_status dalloc(hfe_handle* h, T** p, size_t count);
bool is_device_ptr(const void* p);
hfe_status copy_in(hfe_handle* h, void* dst, const void* src, size_t bytes);
hfe_status copy_out(hfe_handle* h, void* dst, const void* src, size_t bytes);
hfe_status read_status(hfe_handle* h);
hfe_status import_history(hfe_handle* h, const double* user, void* dst);
hfe_status export_history(hfe_handle* h, const void* src, double* user);
hfe_status sweep(hfe_handle* h, const double* u_dev, double load, int mode, double* Rdst, double* sigma_dev);
// sweep with explicit K values, history buffers and precision (FP64 systems of the adjoint)
hfe_status sweep_ex(hfe_handle* h, const double* u_dev, double load, int mode, double* Rdst, double* sigma_dev,
                    void* K, const void* hist, void* hist_trial, bool fp64);
hfe_status solve_sys(hfe_handle* h, LinSys& ls, const double* b, double bscale, int64_t* iters);
hfe_status check_sweep_status(hfe_handle* h);
hfe_status solve_any(hfe_handle* h, const double* b, double bscale, int64_t* iters);
float elapsed(cudaEvent_t a, cudaEvent_t b);
hfe_status newton_steps(hfe_handle* h, int n_steps, const double* t, double* u_out, double* sigma_out,
                        double* hist_out, hfe_stats* st, StepHook* hook);

// adjoint.cu
hfe_status adjoint_run(hfe_handle* h, int n_steps, const double* t, const double* u_target, double w,
                       double* J_out, double* grad_out, hfe_stats* stats);
void adjoint_free(AdjointWork* w);

}  // namespace hfe
