// C ABI of the library (include/hfe.h): handle set-up, state transfer, the Gauss-point
// sweep, the Krylov solve and the load-step Newton driver (paper Eq. Stiffness_mat and the
// load-step loop of Algorithm adjoint_ad's forward pass).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "stepping.h"

using namespace hfe;

namespace hfe {

hfe_status fail(hfe_handle* h, hfe_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

hfe_status cuda_check(hfe_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HFE_OK;
  return fail(h, HFE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
hfe_status dalloc(hfe_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, HFE_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  h->allocs.push_back(q);
  h->device_bytes += count * sizeof(T);
  *p = reinterpret_cast<T*>(q);
  return HFE_OK;
}

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// copy `bytes` from a host or device source into device memory on the handle's stream
hfe_status copy_in(hfe_handle* h, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return HFE_OK;
  cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  return cuda_check(h, cudaMemcpyAsync(dst, src, bytes, k, h->s), "copy in");
}

// copy device memory out to a host or device destination; host copies complete on return
hfe_status copy_out(hfe_handle* h, void* dst, const void* src, size_t bytes) {
  if (bytes == 0 || dst == nullptr) return HFE_OK;
  bool dev = is_device_ptr(dst);
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s),
                     "copy out"));
  if (!dev) HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "sync"));
  return HFE_OK;
}

hfe_status upload_material(hfe_handle* h, const hfe_material* m) {
  if (m == nullptr || m->theta == nullptr) return fail(h, HFE_EINVAL, "material: theta is NULL");
  if (!(m->n_mat == 1 || m->n_mat == h->n_el)) return fail(h, HFE_EINVAL, "material: n_mat must be 1 or n_el");
  if (m->hardening != HFE_HARDENING_SWIFT && m->hardening != HFE_HARDENING_VOCE)
    return fail(h, HFE_EINVAL, "material: unknown hardening law");
  if (h->mat64 != nullptr && m->n_mat != h->n_mat) return fail(h, HFE_EINVAL, "material: n_mat changed");
  if (h->mat64 != nullptr && m->hardening != h->hardening) return fail(h, HFE_EINVAL, "material: hardening changed");
  h->n_mat = m->n_mat;
  h->hardening = m->hardening;
  if (h->mat64 == nullptr) {
    HFE_TRY(dalloc(h, &h->theta, (size_t)h->n_mat * 11));
    HFE_TRY(dalloc(h, &h->mat64, (size_t)h->n_mat));
    HFE_TRY(dalloc(h, &h->matf, (size_t)h->n_mat));
  }
  HFE_TRY(copy_in(h, h->theta, m->theta, sizeof(double) * h->n_mat * 11));
  if (m->Theta != nullptr) {
    if (h->Theta == nullptr) HFE_TRY(dalloc(h, &h->Theta, (size_t)h->n_mat * 9));
    HFE_TRY(copy_in(h, h->Theta, m->Theta, sizeof(double) * h->n_mat * 9));
  } else if (h->Theta != nullptr) {
    h->Theta = nullptr;   // buffer stays in allocs; identity axes from now on
  }
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->s), "memset"));
  launch_material_setup(h->theta, h->Theta, h->n_mat, h->mat64, h->matf, h->bad, h->s);
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->h_bad, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->s), "copy"));
  if (h->n_mat == 1) {
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(&h->h_mat64, h->mat64, sizeof(MatRec), cudaMemcpyDeviceToHost, h->s), "copy"));
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(&h->h_matf, h->matf, sizeof(MatRecF), cudaMemcpyDeviceToHost, h->s), "copy"));
  }
  HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "material set-up"));
  if (*h->h_bad != 0) return fail(h, HFE_EINVAL, "material: " + std::to_string(*h->h_bad) +
                                                     " record(s) with non-positive Hill eigenvalue or elastic modulus");
  return HFE_OK;
}

hfe_status read_status(hfe_handle* h) {
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->h_status, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->s),
                     "status"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->h_sc, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, h->s), "scalars"));
  HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "kernels"));
  return cuda_check(h, cudaGetLastError(), "kernel launch");
}

hfe_status ensure_hist_io(hfe_handle* h) {
  if (h->hist_io == nullptr) HFE_TRY(dalloc(h, &h->hist_io, 7 * (size_t)h->n_gp));
  return HFE_OK;
}

// user history (FP64 [7][n_gp], host or device) into an internal history buffer
hfe_status import_history(hfe_handle* h, const double* user, void* dst) {
  const double* src = user;
  if (!is_device_ptr(user)) {
    HFE_TRY(ensure_hist_io(h));
    HFE_TRY(copy_in(h, h->hist_io, user, sizeof(double) * 7 * h->n_gp));
    src = h->hist_io;
  }
  launch_hist_import(src, dst, h->fp64 != 0, h->n_gp, h->s);
  return HFE_OK;
}

// internal history buffer out to FP64 [7][n_gp] (host or device)
hfe_status export_history(hfe_handle* h, const void* src, double* user) {
  if (is_device_ptr(user)) {
    launch_hist_export(src, user, h->fp64 != 0, h->n_gp, h->s);
    return HFE_OK;
  }
  HFE_TRY(ensure_hist_io(h));
  launch_hist_export(src, h->hist_io, h->fp64 != 0, h->n_gp, h->s);
  return copy_out(h, user, h->hist_io, sizeof(double) * 7 * h->n_gp);
}

// one sweep on the internal stream; u may be any device pointer; R into Rdst (device)
hfe_status sweep_ex(hfe_handle* h, const double* u_dev, double load, int mode, double* Rdst, double* sigma_dev,
                    void* K, const void* hist, void* hist_trial, bool fp64) {
  SweepArgs a;
  a.X = h->X;
  a.dX32 = h->dX32;
  a.conn = h->conn;
  a.u = u_dev;
  a.hist = hist;
  a.hist_trial = hist_trial;
  a.mat = fp64 ? (const void*)h->mat64 : (const void*)h->matf;
  a.mat_host = h->n_mat == 1 ? (fp64 ? (const void*)&h->h_mat64 : (const void*)&h->h_matf) : nullptr;
  a.mat_per_element = h->n_mat > 1 ? 1 : 0;
  a.hardening = h->hardening;
  a.elems = h->elems;
  a.slot = h->slot;
  a.K = K;
  a.R = Rdst;
  a.f_ext = h->f_ext;
  a.load = load;
  a.sigma = sigma_dev;
  a.status = h->status;
  a.n_gp = h->n_gp;
  a.local_maxit = h->opt.local_maxit;
  a.local_tol = h->opt.local_tol;
  a.fbar = h->opt.fbar;
  a.ext_eps = h->ext_eps;
  a.ext_T = h->ext_T;
  a.ext_D = h->ext_D;
  a.ext_plastic = h->ext_pl;
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->status, 0, sizeof(DevStatus), h->s), "memset"));
  if (h->barlat != nullptr) {   // Barlat: strain pass, the Gauss-point update, assembly pass
    launch_gp_sweep_ext(a, fp64, 1, mode, h->P.launch_off, h->s);
    launch_barlat_gp(h->barlat, fp64, h->ext_eps, hist, hist_trial, h->n_gp, h->ext_T, h->ext_D, h->ext_pl,
                     mode == HFE_SWEEP_TANGENT ? 1 : 0, h->status, h->ext_work, h->ext_it, h->ext_st, h->s);
    launch_gp_sweep_ext(a, fp64, 2, mode, h->P.launch_off, h->s);
    return HFE_OK;
  }
  launch_gp_sweep(a, fp64, mode, h->P.launch_off, h->s);
  return HFE_OK;
}

hfe_status sweep(hfe_handle* h, const double* u_dev, double load, int mode, double* Rdst, double* sigma_dev) {
  return sweep_ex(h, u_dev, load, mode, Rdst, sigma_dev, h->K, h->hist, h->hist_trial, h->fp64 != 0);
}

hfe_status check_sweep_status(hfe_handle* h) {
  const DevStatus& st = *h->h_status;
  if (st.detj > 0)
    return fail(h, HFE_EDETJ, std::to_string(st.detj) + " Gauss point(s) with det J <= 0 or not a number");
  if (st.nonfinite > 0) return fail(h, HFE_ENONFINITE, "non-finite internal force");
  if (st.local_fail > 0)
    return fail(h, HFE_ELOCAL, std::to_string(st.local_fail) + " local return mapping(s) hit local_maxit");
  return HFE_OK;
}

template <typename R>
PcgVecs<R> vecs(LinSys& ls) {
  PcgVecs<R> v;
  v.x = (R*)ls.vx; v.r = (R*)ls.vr; v.z = (R*)ls.vz; v.p = (R*)ls.vp; v.q = (R*)ls.vq; v.minv = (R*)ls.vminv;
  v.p2 = (R*)ls.vp2;
  v.rh = (R*)ls.vrh; v.y = (R*)ls.vy; v.t = (R*)ls.vt;
  return v;
}

template <typename R>
hfe_status build_pcg_graph(hfe_handle* h, LinSys& ls, int len) {
  if (ls.graph != nullptr && ls.graph_len == len) return HFE_OK;
  if (ls.graph != nullptr) {
    cudaGraphExecDestroy(ls.graph);
    ls.graph = nullptr;
  }
  Csr K = csr_of(h);
  PcgVecs<R> v = vecs<R>(ls);
  const int block3 = h->opt.precond == HFE_PRECOND_BLOCK3;
  cudaGraph_t g;
  HFE_TRY(cuda_check(h, cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal), "capture"));
  for (int i = 0; i < len; ++i) pcg_iteration<R>(K, (const R*)ls.K, h->freem, v, block3, h->sc, h->part, h->s);
  HFE_TRY(cuda_check(h, cudaStreamEndCapture(h->s, &g), "end capture"));
  cudaError_t e = cudaGraphInstantiate(&ls.graph, g, 0);
  cudaGraphDestroy(g);
  HFE_TRY(cuda_check(h, e, "graph instantiate"));
  ls.graph_len = len;
  return HFE_OK;
}

// A Newton correction whose CG met negative curvature (p.Kp <= 0: the tangent is
// indefinite at this iterate): solve the same system with preconditioned BiCGSTAB, which
// needs no definiteness, as a direct solver would; if that fails too, the truncated CG
// direction (Steihaug) is kept when there is one.  x in v.x either way.
template <typename R>
hfe_status indefinite_fallback(hfe_handle* h, LinSys& ls, const Csr& K, PcgVecs<R>& v, int block3, const double* b,
                               double bscale) {
  const int cg_iters = h->h_sc->iters;
  const bool have_truncated = h->allow_truncated && cg_iters > 0 && std::isfinite(h->h_sc->rr);
  const size_t bytes = (ls.fp64 ? sizeof(double) : sizeof(float)) * h->n_dof;
  if (have_truncated) HFE_TRY(cuda_check(h, cudaMemcpyAsync(ls.vxt, v.x, bytes, cudaMemcpyDeviceToDevice, h->s), "copy"));
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->sc, 0, sizeof(PcgScalars), h->s), "memset"));
  const double rt = h->pcg_rtol_now > 0.0 ? h->pcg_rtol_now : h->opt.pcg_rtol;
  HFE_TRY(cuda_check(h, bicgstab_persistent<R>(K, (const R*)ls.K, h->freem, v, block3, b, bscale, rt * rt,
                                               h->opt.pcg_maxit, h->sc, h->part, partial_slots(),
                                               (uint64_t)h->opt.barrier_spin_limit, h->s),
                     "BiCGSTAB launch"));
  HFE_TRY(read_status(h));
  h->n_bicgstab++;
  h->h_sc->iters += cg_iters;
  if (h->h_sc->gs.timeout) return fail(h, HFE_EBARRIER, "BiCGSTAB: a grid barrier wait ran out");
  if (h->h_sc->done) return HFE_OK;
  if (have_truncated && h->allow_truncated) {
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(v.x, ls.vxt, bytes, cudaMemcpyDeviceToDevice, h->s), "copy"));
    h->pcg_truncated = true;
    return HFE_OK;
  }
  return fail(h, HFE_EPCG, "indefinite matrix: CG broke down and BiCGSTAB did not converge");
}

// The solve as one cooperative launch (preconditioner set up and scalars zeroed by the
// caller); the same outcomes as the chunked form below.
template <typename R>
hfe_status pcg_solve_persistent(hfe_handle* h, LinSys& ls, Csr K, PcgVecs<R>& v, int block3, const double* b,
                                double bscale, int64_t* iters_out) {
  const double rt = h->pcg_rtol_now > 0.0 ? h->pcg_rtol_now : h->opt.pcg_rtol;
  if (h->opt.pcg_persistent == 2) {   // direct loads of K: no row chunks
    K.chunk32 = K.chunk64 = nullptr;
    K.n_chunk32 = K.n_chunk64 = 0;
  }
  HFE_TRY(cuda_check(h, pcg_persistent<R>(K, (const R*)ls.K, h->freem, v, block3, b, bscale, rt * rt,
                                          h->opt.pcg_maxit, h->sc, h->part, partial_slots(),
                                          (uint64_t)h->opt.barrier_spin_limit, h->s),
                     "persistent CG launch"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->h_bad, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->s), "copy"));
  HFE_TRY(read_status(h));
  const PcgScalars& sc = *h->h_sc;
  if (iters_out) *iters_out = sc.iters;
  if (sc.gs.timeout) return fail(h, HFE_EBARRIER, "persistent CG: a grid barrier wait ran out");
  // a Newton correction may run on a tangent that is indefinite at some nodes (the surrogate
  // blocks keep the preconditioner SPD and truncated CG stops at negative curvature); a plain
  // solve of a matrix that is not SPD is refused
  if (*h->h_bad != 0 && !h->allow_indefinite)
    return fail(h, HFE_EPCG, "preconditioner: " + std::to_string(*h->h_bad) + " diagonal blocks not positive definite");
  if (!std::isfinite(sc.rr0)) return fail(h, HFE_ENONFINITE, "non-finite right-hand side");
  if (sc.done) return HFE_OK;
  if (sc.breakdown) {
    // negative curvature (p.Ap <= 0) in a Newton correction: BiCGSTAB, else the truncated
    // CG direction
    if (h->allow_indefinite) return indefinite_fallback<R>(h, ls, K, v, block3, b, bscale);
    return fail(h, HFE_EPCG, "CG breakdown (p.Ap <= 0 or non-finite)");
  }
  return fail(h, HFE_EPCG, "CG did not converge: |r|/|b| = " + std::to_string(std::sqrt(sc.rr / sc.rr0)));
}

// Solve Kt x = bscale * b with PCG (b device FP64 [n_dof]); x left in h->vx (precision R).
template <typename R>
hfe_status pcg_solve(hfe_handle* h, LinSys& ls, const double* b, double bscale, int64_t* iters_out) {
  Csr K = csr_of(h);
  PcgVecs<R> v = vecs<R>(ls);
  const int block3 = h->opt.precond == HFE_PRECOND_BLOCK3;
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->s), "memset"));
  precond_setup<R>(K, (const R*)ls.K, h->diag_slot, h->freem, v.minv, block3, h->bad, h->s);
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->sc, 0, sizeof(PcgScalars), h->s), "memset"));
  if (h->opt.pcg_persistent) return pcg_solve_persistent<R>(h, ls, K, v, block3, b, bscale, iters_out);
  {
    const double rt = h->pcg_rtol_now > 0.0 ? h->pcg_rtol_now : h->opt.pcg_rtol;
    const double rt2 = rt * rt;
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(&h->sc->target, &rt2, sizeof(double), cudaMemcpyHostToDevice, h->s),
                       "copy"));
    HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "sync"));   // rt2 lives on this stack frame
  }
  pcg_init<R>(b, bscale, h->freem, v, block3, h->n_nodes, h->sc, h->part, h->s);
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->h_bad, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->s), "copy"));
  HFE_TRY(read_status(h));
  // a Newton correction may run on a tangent that is indefinite at some nodes (the surrogate
  // blocks keep the preconditioner SPD and truncated CG stops at negative curvature); a plain
  // solve of a matrix that is not SPD is refused
  if (*h->h_bad != 0 && !h->allow_indefinite)
    return fail(h, HFE_EPCG, "preconditioner: " + std::to_string(*h->h_bad) + " diagonal blocks not positive definite");
  const double rr0 = h->h_sc->rr0;
  if (!std::isfinite(rr0)) return fail(h, HFE_ENONFINITE, "non-finite right-hand side");
  int64_t it = 0;
  if (rr0 > 0.0) {
    const double rtc = h->pcg_rtol_now > 0.0 ? h->pcg_rtol_now : h->opt.pcg_rtol;
    const double target = rtc * rtc * rr0;
    const int m = std::max(1, h->opt.pcg_check_every);
    HFE_TRY(build_pcg_graph<R>(h, ls, m));
    bool done = false;
    while (it < h->opt.pcg_maxit) {
      HFE_TRY(cuda_check(h, cudaGraphLaunch(ls.graph, h->s), "graph launch"));
      it += m;
      HFE_TRY(read_status(h));
      if (h->h_sc->done || h->h_sc->rr <= target) { done = true; break; }
      if (h->h_sc->breakdown) {
        // negative curvature (p.Ap <= 0): the kernels froze x at the last iterate; in a
        // Newton correction BiCGSTAB takes over, else the truncated CG direction is kept
        if (h->allow_indefinite) {
          HFE_TRY((indefinite_fallback<R>(h, ls, K, v, block3, b, bscale)));
          if (iters_out) *iters_out = h->h_sc->iters;
          return HFE_OK;
        }
        return fail(h, HFE_EPCG, "CG breakdown (p.Ap <= 0 or non-finite)");
      }
    }
    if (!done) {
      if (iters_out) *iters_out = it;
      return fail(h, HFE_EPCG, "CG did not converge: |r|/|b| = " + std::to_string(std::sqrt(h->h_sc->rr / rr0)));
    }
  } else {
    HFE_TRY(cuda_check(h, cudaMemsetAsync(v.x, 0, sizeof(R) * h->n_dof, h->s), "memset"));
  }
  if (iters_out) *iters_out = it;
  return HFE_OK;
}

// Non-symmetric K (F-bar element): preconditioned BiCGSTAB in one cooperative launch.
template <typename R>
hfe_status bicg_solve(hfe_handle* h, LinSys& ls, const double* b, double bscale, int64_t* iters_out) {
  Csr K = csr_of(h);
  PcgVecs<R> v = vecs<R>(ls);
  const int block3 = h->opt.precond == HFE_PRECOND_BLOCK3;
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->s), "memset"));
  precond_setup<R>(K, (const R*)ls.K, h->diag_slot, h->freem, v.minv, block3, h->bad, h->s);
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->sc, 0, sizeof(PcgScalars), h->s), "memset"));
  const double rt = h->pcg_rtol_now > 0.0 ? h->pcg_rtol_now : h->opt.pcg_rtol;
  HFE_TRY(cuda_check(h, bicgstab_persistent<R>(K, (const R*)ls.K, h->freem, v, block3, b, bscale, rt * rt,
                                               h->opt.pcg_maxit, h->sc, h->part, partial_slots(),
                                               (uint64_t)h->opt.barrier_spin_limit, h->s),
                     "BiCGSTAB launch"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->h_bad, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->s), "copy"));
  HFE_TRY(read_status(h));
  const PcgScalars& sc = *h->h_sc;
  if (iters_out) *iters_out = sc.iters;
  if (sc.gs.timeout) return fail(h, HFE_EBARRIER, "BiCGSTAB: a grid barrier wait ran out");
  if (!std::isfinite(sc.rr0)) return fail(h, HFE_ENONFINITE, "non-finite right-hand side");
  if (sc.done) return HFE_OK;
  if (sc.breakdown)
    return fail(h, HFE_EPCG, "BiCGSTAB breakdown (" + std::string(sc.breakdown == 1 ? "rh.v = 0" : sc.breakdown == 3 ? "|t| = 0" :
                                                                   sc.breakdown == 5 ? "too many restarts" : "non-finite") +
                                 ") after " + std::to_string(sc.iters) + " iterations, |r|/|b| = " +
                                 std::to_string(std::sqrt(sc.rr / sc.rr0)));
  return fail(h, HFE_EPCG, "BiCGSTAB did not converge: |r|/|b| = " + std::to_string(std::sqrt(sc.rr / sc.rr0)));
}

hfe_status solve_sys(hfe_handle* h, LinSys& ls, const double* b, double bscale, int64_t* iters) {
  if (!h->opt.fbar)
    return ls.fp64 ? pcg_solve<double>(h, ls, b, bscale, iters) : pcg_solve<float>(h, ls, b, bscale, iters);
  if (ls.fp64) return bicg_solve<double>(h, ls, b, bscale, iters);
  // mixed path: BiCGSTAB diverges in FP32 on ill-conditioned meshes (its recurrences are not
  // monotone), so the FP32 tangent is widened to FP64 and solved there; x back in FP32
  LinSys& l64 = h->ls_fb64;
  if (l64.K == nullptr) {
    unsigned char* p = nullptr;
    HFE_TRY(dalloc(h, &p, sizeof(double) * (9 * h->P.n_blocks + kKPad))); l64.K = p;
    for (void** v : {&l64.vx, &l64.vr, &l64.vz, &l64.vp, &l64.vq, &l64.vp2, &l64.vrh, &l64.vy, &l64.vt, &l64.vxt}) {
      HFE_TRY(dalloc(h, &p, sizeof(double) * h->n_dof));
      *v = p;
    }
    HFE_TRY(dalloc(h, &p, sizeof(double) * 9 * h->n_nodes)); l64.vminv = p;
    l64.fp64 = true;
  }
  to_double((const float*)ls.K, (double*)l64.K, 9 * h->P.n_blocks, h->s);
  HFE_TRY(bicg_solve<double>(h, l64, b, bscale, iters));
  to_float((const double*)l64.vx, (float*)ls.vx, h->n_dof, h->s);
  return HFE_OK;
}

hfe_status solve_any(hfe_handle* h, const double* b, double bscale, int64_t* iters) {
  return solve_sys(h, h->ls, b, bscale, iters);
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace hfe

extern "C" {

void hfe_default_options(hfe_options* o, int precision) {
  std::memset(o, 0, sizeof(*o));
  o->precision = precision;
  // mixed: 1e-7 keeps the displacement within ~5e-7 of the exact solution on the 100^3 cube
  // (1e-6 left 2e-5 - 6e-5 there, above the 1e-5 target)
  o->newton_rtol = precision == HFE_PRECISION_FP64 ? 1e-10 : 1e-7;
  o->newton_atol = 1.0;
  o->newton_maxit = 25;
  o->newton_stag_tol = 1e-4;
  o->pcg_rtol = precision == HFE_PRECISION_FP64 ? 1e-12 : 1e-6;
  o->pcg_maxit = 20000;
  o->pcg_check_every = 16;
  o->precond = HFE_PRECOND_BLOCK3;
  o->local_maxit = 50;
  o->local_tol = 1e-14;
  o->ckpt_every = 1;
  o->predictor = 2;
  o->ew_forcing = 0;
  o->pcg_persistent = 1;
  o->adaptive = 1;
  o->cutback = 0.5;
  o->max_cutbacks = 8;
  o->fbar = 0;
  o->barrier_spin_limit = (int64_t)1 << 25;
  o->assembly_l2_bytes = -1;
}

hfe_status hfe_create(const hfe_mesh* mesh, const hfe_bc* bc, const hfe_material* mat, const hfe_options* opt,
                      void* stream, hfe_handle** out) {
  if (out == nullptr) return HFE_EINVAL;
  *out = nullptr;
  if (mesh == nullptr || mesh->X == nullptr || mesh->conn == nullptr || mesh->n_nodes <= 0 || mesh->n_el <= 0)
    return HFE_EINVAL;
  hfe_handle* h = new (std::nothrow) hfe_handle();
  if (h == nullptr) return HFE_ENOMEM;
  *out = h;
  if (opt) h->opt = *opt;
  else hfe_default_options(&h->opt, HFE_PRECISION_FP64);
  if (h->opt.precision != HFE_PRECISION_FP64 && h->opt.precision != HFE_PRECISION_MIXED)
    return fail(h, HFE_EINVAL, "options: unknown precision");
  if (h->opt.adaptive && !(h->opt.cutback > 0.0 && h->opt.cutback < 1.0))
    return fail(h, HFE_EINVAL, "options: cutback must lie in (0, 1)");
  if (h->opt.max_cutbacks < 0) return fail(h, HFE_EINVAL, "options: max_cutbacks must be >= 0");
  if (h->opt.predictor < 0 || h->opt.predictor > 3) return fail(h, HFE_EINVAL, "options: predictor must be 0 to 3");
  if (h->opt.barrier_spin_limit < 0) return fail(h, HFE_EINVAL, "options: barrier_spin_limit must be >= 0");
  if (h->opt.assembly_l2_bytes < -1) return fail(h, HFE_EINVAL, "options: assembly_l2_bytes must be >= -1");
  h->fp64 = h->opt.precision == HFE_PRECISION_FP64;
  h->user = reinterpret_cast<cudaStream_t>(stream);
  HFE_TRY(cuda_check(h, cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking), "stream"));
  HFE_TRY(cuda_check(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming), "event"));
  HFE_TRY(cuda_check(h, cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming), "event"));
  HFE_TRY(cuda_check(h, cudaEventCreate(&h->t0), "event"));
  HFE_TRY(cuda_check(h, cudaEventCreate(&h->t1), "event"));
  h->n_nodes = mesh->n_nodes;
  h->n_el = mesh->n_el;
  h->n_dof = 3 * h->n_nodes;
  h->n_gp = 8 * h->n_el;
  // host copies of the mesh (pageable or device input)
  std::vector<int32_t> conn_h(h->n_el * 8);
  if (is_device_ptr(mesh->conn)) {
    if (cudaMemcpy(conn_h.data(), mesh->conn, conn_h.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(h, HFE_ECUDA, "copy conn");
  } else {
    std::memcpy(conn_h.data(), mesh->conn, conn_h.size() * 4);
  }
  std::string perr;
  // launch order: slabs of K rows (blocks of 9 values of the handle's precision) of
  // assembly_l2_bytes, or (-1) of 0.4-0.8 of this device's L2 as the planner picks, the rest
  // of L2 left to the streamed per-point data
  hfe::SlabPlan plan;
  {
    const int64_t bb = 9 * (h->fp64 ? 8 : 4);
    int64_t lo = 0, hi = 0;
    if (h->opt.assembly_l2_bytes == -1) {
      int dev = 0, l2 = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        return fail(h, HFE_ECUDA, "L2 size query");
      lo = (int64_t)l2 * 2 / 5;
      hi = (int64_t)l2 * 4 / 5;
    } else {
      lo = hi = h->opt.assembly_l2_bytes;
    }
    if (hi > 0) {
      plan.min_blocks = std::max<int64_t>(1, lo / bb);
      plan.max_blocks = std::max<int64_t>(1, hi / bb);
      plan.resident_ctas = sweep_resident_ctas(h->fp64 != 0, h->opt.fbar != 0);
      plan.el_per_cta = sweep_elems_per_cta();
      if (plan.resident_ctas <= 0) return fail(h, HFE_ECUDA, "sweep occupancy query");
    }
  }
  if (!build_pattern(h->n_nodes, h->n_el, conn_h.data(), plan, h->P, perr))
    return fail(h, HFE_EINVAL, "mesh: " + perr);
  StreamScope scope(h);
  // device allocations
  const bool f64 = h->fp64 != 0;
  const size_t rsz = f64 ? 8 : 4;
  HFE_TRY(dalloc(h, &h->X, h->n_dof));
  HFE_TRY(dalloc(h, &h->conn, h->n_el * 8));
  HFE_TRY(dalloc(h, &h->u, h->n_dof));
  {
    unsigned char* b = nullptr;
    HFE_TRY(dalloc(h, &b, hist_bytes(h->n_gp, f64))); h->hist = b;
    HFE_TRY(dalloc(h, &b, hist_bytes(h->n_gp, f64))); h->hist_trial = b;
  }
  if (!f64) {   // coordinate differences X_a - X_0 (a = 1..7) per element, rounded once to FP32
    std::vector<double> Xh(h->n_dof);
    if (is_device_ptr(mesh->X)) cudaMemcpy(Xh.data(), mesh->X, 8 * h->n_dof, cudaMemcpyDeviceToHost);
    else std::memcpy(Xh.data(), mesh->X, 8 * h->n_dof);
    std::vector<float> dx(21 * (size_t)h->n_el);
    for (int64_t e = 0; e < h->n_el; ++e) {
      const int64_t n0 = conn_h[e * 8];
      for (int a = 1; a < 8; ++a) {
        const int64_t na = conn_h[e * 8 + a];
        for (int c = 0; c < 3; ++c) dx[e * 21 + (a - 1) * 3 + c] = (float)(Xh[3 * na + c] - Xh[3 * n0 + c]);
      }
    }
    HFE_TRY(dalloc(h, &h->dX32, dx.size()));
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->dX32, dx.data(), 4 * dx.size(), cudaMemcpyHostToDevice, h->s), "copy"));
    HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "sync"));
  }
  HFE_TRY(dalloc(h, &h->rowptr, h->n_nodes + 1));
  HFE_TRY(dalloc(h, &h->cols, h->P.n_blocks + kKPad));
  HFE_TRY(dalloc(h, &h->diag_slot, h->n_nodes));
  HFE_TRY(dalloc(h, &h->slot, h->n_el * 64));
  HFE_TRY(dalloc(h, &h->elems, h->n_el));
  {
    unsigned char* k = nullptr;
    HFE_TRY(dalloc(h, &k, rsz * (9 * h->P.n_blocks + kKPad)));
    h->K = k;
  }
  HFE_TRY(dalloc(h, &h->R, h->n_dof));
  HFE_TRY(dalloc(h, &h->freem, h->n_dof));
  HFE_TRY(dalloc(h, &h->status, 1));
  HFE_TRY(dalloc(h, &h->sc, 1));
  HFE_TRY(dalloc(h, &h->part, partial_slots()));
  HFE_TRY(dalloc(h, &h->bad, 1));
  HFE_TRY(dalloc(h, &h->tmp64, h->n_dof));
  HFE_TRY(dalloc(h, &h->b64, h->n_dof));
  HFE_TRY(dalloc(h, &h->u_start, h->n_dof));
  {
    unsigned char* b = nullptr;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->vx = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->vr = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->vz = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->vp = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->vq = b;
    HFE_TRY(dalloc(h, &b, rsz * 9 * h->n_nodes)); h->vminv = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->ls.vp2 = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->ls.vrh = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->ls.vy = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->ls.vt = b;
    HFE_TRY(dalloc(h, &b, rsz * h->n_dof)); h->ls.vxt = b;
  }
  h->ls.K = h->K;
  h->ls.vx = h->vx; h->ls.vr = h->vr; h->ls.vz = h->vz; h->ls.vp = h->vp; h->ls.vq = h->vq; h->ls.vminv = h->vminv;
  h->ls.fp64 = f64;
  if (cudaMallocHost(&h->h_sc, sizeof(PcgScalars)) != cudaSuccess ||
      cudaMallocHost(&h->h_status, sizeof(DevStatus)) != cudaSuccess || cudaMallocHost(&h->h_bad, sizeof(int)) != cudaSuccess)
    return fail(h, HFE_ENOMEM, "pinned host allocation failed");
  HFE_TRY(copy_in(h, h->X, mesh->X, sizeof(double) * h->n_dof));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->conn, conn_h.data(), conn_h.size() * 4, cudaMemcpyHostToDevice, h->s), "copy"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->rowptr, h->P.rowptr.data(), 8 * (h->n_nodes + 1), cudaMemcpyHostToDevice, h->s),
                     "copy"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->cols, h->P.cols.data(), 4 * h->P.n_blocks, cudaMemcpyHostToDevice, h->s), "copy"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->diag_slot, h->P.diag_slot.data(), 8 * h->n_nodes, cudaMemcpyHostToDevice, h->s),
                     "copy"));
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->slot, h->P.slot.data(), 4 * h->P.slot.size(), cudaMemcpyHostToDevice, h->s),
                     "copy"));
  {
    // row chunks of the streamed SpMV of the one-launch CG (FP32 and FP64 block values)
    std::vector<int32_t> c32, c64;
    stream_chunks(h->P.rowptr.data(), h->n_nodes, stream_rows<float>(), stream_max_blocks<float>(), c32);
    stream_chunks(h->P.rowptr.data(), h->n_nodes, stream_rows<double>(), stream_max_blocks<double>(), c64);
    if (!c32.empty()) {
      HFE_TRY(dalloc(h, &h->chunk32, c32.size()));
      HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->chunk32, c32.data(), 4 * c32.size(), cudaMemcpyHostToDevice, h->s),
                         "copy"));
      h->n_chunk32 = (int64_t)c32.size() - 1;
    }
    if (!c64.empty()) {
      HFE_TRY(dalloc(h, &h->chunk64, c64.size()));
      HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->chunk64, c64.data(), 4 * c64.size(), cudaMemcpyHostToDevice, h->s),
                         "copy"));
      h->n_chunk64 = (int64_t)c64.size() - 1;
    }
    HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "sync"));   // c32, c64 live on this frame
  }
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->elems, h->P.elems.data(), 4 * h->n_el, cudaMemcpyHostToDevice, h->s), "copy"));
  // boundary data
  std::vector<uint8_t> freem(h->n_dof, 1);
  std::vector<int64_t> fdof;
  std::vector<double> fval;
  if (bc != nullptr && bc->n_fixed > 0) {
    if (bc->dof == nullptr || bc->value == nullptr) return fail(h, HFE_EINVAL, "bc: dof/value NULL");
    fdof.resize(bc->n_fixed);
    fval.resize(bc->n_fixed);
    if (is_device_ptr(bc->dof)) {
      cudaMemcpy(fdof.data(), bc->dof, 8 * bc->n_fixed, cudaMemcpyDeviceToHost);
      cudaMemcpy(fval.data(), bc->value, 8 * bc->n_fixed, cudaMemcpyDeviceToHost);
    } else {
      std::memcpy(fdof.data(), bc->dof, 8 * bc->n_fixed);
      std::memcpy(fval.data(), bc->value, 8 * bc->n_fixed);
    }
    for (int64_t i = 0; i < bc->n_fixed; ++i) {
      if (fdof[i] < 0 || fdof[i] >= h->n_dof) return fail(h, HFE_EINVAL, "bc: dof out of range");
      if (!freem[fdof[i]]) return fail(h, HFE_EINVAL, "bc: duplicate dof");
      freem[fdof[i]] = 0;
    }
  }
  h->n_fixed = (int64_t)fdof.size();
  HFE_TRY(dalloc(h, &h->fixed_dof, h->n_fixed));
  HFE_TRY(dalloc(h, &h->fixed_val, h->n_fixed));
  if (h->n_fixed) {
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->fixed_dof, fdof.data(), 8 * h->n_fixed, cudaMemcpyHostToDevice, h->s), "copy"));
    HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->fixed_val, fval.data(), 8 * h->n_fixed, cudaMemcpyHostToDevice, h->s), "copy"));
  }
  HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->freem, freem.data(), h->n_dof, cudaMemcpyHostToDevice, h->s), "copy"));
  if (bc != nullptr && bc->f_ext != nullptr) {
    HFE_TRY(dalloc(h, &h->f_ext, h->n_dof));
    HFE_TRY(copy_in(h, h->f_ext, bc->f_ext, sizeof(double) * h->n_dof));
  }
  HFE_TRY(upload_material(h, mat));
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->u, 0, sizeof(double) * h->n_dof, h->s), "memset"));
  HFE_TRY(cuda_check(h, cudaMemsetAsync(h->hist, 0, hist_bytes(h->n_gp, f64), h->s), "memset"));
  launch_sigma_cache(h->hist, f64, h->mat64, h->n_mat > 1, h->hardening, h->n_gp, h->s);
  HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "create"));
  return cuda_check(h, cudaGetLastError(), "create kernels");
}

void hfe_destroy(hfe_handle* h) {
  if (h == nullptr) return;
  if (h->s) cudaStreamSynchronize(h->s);
  adjoint_free(h->adj);
  hfe::barlat_model_free(h->barlat);
  if (h->ls.graph) cudaGraphExecDestroy(h->ls.graph);
  for (void* p : h->allocs) cudaFree(p);
  if (h->sigma) cudaFree(h->sigma);
  if (h->warm_u) cudaFree(h->warm_u);
  for (double* p : h->extrap_u)
    if (p) cudaFree(p);
  if (h->h_sc) cudaFreeHost(h->h_sc);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->h_bad) cudaFreeHost(h->h_bad);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->t0) cudaEventDestroy(h->t0);
  if (h->t1) cudaEventDestroy(h->t1);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
}

const char* hfe_last_error(const hfe_handle* h) { return h ? h->err.c_str() : "null handle"; }

hfe_status hfe_set_barlat(hfe_handle* h, const hfe_barlat_material* mat, const hfe_cpp_options* opt) {
  if (h == nullptr) return HFE_EINVAL;
  if (mat == nullptr) {   // back to the Hill-48 material of the handle
    hfe::barlat_model_free(h->barlat);
    h->barlat = nullptr;
    h->pred_valid = false;
    h->extrap_n = 0;
    return HFE_OK;
  }
  if (h->n_mat != 1) return fail(h, HFE_EINVAL, "Barlat material: the handle's material must be uniform");
  if (h->opt.fbar) return fail(h, HFE_EINVAL, "Barlat material: the standard element only");
  hfe_status st = HFE_OK;
  hfe::BarlatModel* m = hfe::barlat_model_new(mat, opt, &st);
  if (m == nullptr) return fail(h, st, "Barlat material: invalid parameters or options");
  if (h->ext_eps == nullptr) {
    const size_t ng = (size_t)h->n_gp;
    hfe_status a = dalloc(h, &h->ext_eps, 6 * ng);
    if (a == HFE_OK) a = dalloc(h, &h->ext_T, 6 * ng);
    if (a == HFE_OK) a = dalloc(h, &h->ext_D, 36 * ng);
    if (a == HFE_OK) a = dalloc(h, &h->ext_pl, ng);
    if (a == HFE_OK) a = dalloc(h, &h->ext_work, 15 * ng);
    if (a == HFE_OK) a = dalloc(h, &h->ext_it, ng);
    if (a == HFE_OK) a = dalloc(h, &h->ext_st, ng);
    if (a != HFE_OK) {
      hfe::barlat_model_free(m);
      return a;
    }
  }
  hfe::barlat_model_free(h->barlat);
  h->barlat = m;
  h->pred_valid = false;
  h->extrap_n = 0;
  return HFE_OK;
}

hfe_status hfe_get_info(const hfe_handle* h, hfe_info* info) {
  if (h == nullptr || info == nullptr) return HFE_EINVAL;
  info->n_nodes = h->n_nodes;
  info->n_el = h->n_el;
  info->n_dof = h->n_dof;
  info->n_gp = h->n_gp;
  info->n_blocks = h->P.n_blocks;
  info->n_fixed = h->n_fixed;
  info->n_colors = h->P.n_colors;
  info->n_slabs = h->P.n_slabs;
  info->n_launches = (int64_t)h->P.launch_off.size() - 1;
  info->precision = h->opt.precision;
  info->device_bytes = (int64_t)h->device_bytes;
  return HFE_OK;
}

hfe_status hfe_set_material(hfe_handle* h, const hfe_material* mat) {
  if (h == nullptr) return HFE_EINVAL;
  h->pred_valid = false;
  h->extrap_n = 0;
  StreamScope scope(h);
  HFE_TRY(upload_material(h, mat));
  launch_sigma_cache(h->hist, h->fp64 != 0, h->mat64, h->n_mat > 1, h->hardening, h->n_gp, h->s);
  return cuda_check(h, cudaStreamSynchronize(h->s), "set material");
}

hfe_status hfe_set_state(hfe_handle* h, const double* u, const double* hist) {
  if (h == nullptr) return HFE_EINVAL;
  h->pred_valid = false;
  h->extrap_n = 0;
  StreamScope scope(h);
  if (u) HFE_TRY(copy_in(h, h->u, u, sizeof(double) * h->n_dof));
  else HFE_TRY(cuda_check(h, cudaMemsetAsync(h->u, 0, sizeof(double) * h->n_dof, h->s), "memset"));
  if (hist) HFE_TRY(import_history(h, hist, h->hist));
  else HFE_TRY(cuda_check(h, cudaMemsetAsync(h->hist, 0, hist_bytes(h->n_gp, h->fp64 != 0), h->s), "memset"));
  launch_sigma_cache(h->hist, h->fp64 != 0, h->mat64, h->n_mat > 1, h->hardening, h->n_gp, h->s);
  h->t_state = 0.0;
  return cuda_check(h, cudaStreamSynchronize(h->s), "set state");
}

hfe_status hfe_set_load(hfe_handle* h, double t) {
  if (h == nullptr || !std::isfinite(t)) return HFE_EINVAL;
  h->pred_valid = false;
  h->extrap_n = 0;
  h->t_state = t;
  return HFE_OK;
}

hfe_status hfe_get_load(const hfe_handle* h, double* t) {
  if (h == nullptr || t == nullptr) return HFE_EINVAL;
  *t = h->t_state;
  return HFE_OK;
}

hfe_status hfe_get_state(hfe_handle* h, double* u, double* hist) {
  if (h == nullptr) return HFE_EINVAL;
  StreamScope scope(h);
  HFE_TRY(copy_out(h, u, h->u, sizeof(double) * h->n_dof));
  if (hist) HFE_TRY(export_history(h, h->hist, hist));
  return cuda_check(h, cudaStreamSynchronize(h->s), "get state");
}

hfe_status hfe_gp_sweep(hfe_handle* h, const double* u, double load, int mode, double* R_out, double* rnorm_out,
                        double* hist_trial_out, hfe_stats* stats) {
  if (h == nullptr || u == nullptr) return HFE_EINVAL;
  if (mode != HFE_SWEEP_RESIDUAL && mode != HFE_SWEEP_TANGENT) return fail(h, HFE_EINVAL, "sweep: unknown mode");
  h->pred_valid = false;   // R (and K) no longer those of the last converged Newton iteration
  auto w0 = std::chrono::steady_clock::now();
  StreamScope scope(h);
  const double* ud = u;
  if (!is_device_ptr(u)) {
    HFE_TRY(copy_in(h, h->tmp64, u, sizeof(double) * h->n_dof));
    ud = h->tmp64;
  }
  double* Rd = (R_out != nullptr && is_device_ptr(R_out)) ? R_out : h->R;
  cudaEventRecord(h->t0, h->s);
  HFE_TRY(sweep(h, ud, load, mode, Rd, nullptr));
  cudaEventRecord(h->t1, h->s);
  if (rnorm_out != nullptr) {
    const bool dev = is_device_ptr(rnorm_out);
    free_norm(Rd, h->freem, h->n_dof, h->sc, h->part, h->s, dev ? rnorm_out : h->b64);
    if (!dev) HFE_TRY(copy_out(h, rnorm_out, h->b64, sizeof(double)));
  }
  if (R_out != nullptr && Rd != R_out) HFE_TRY(copy_out(h, R_out, Rd, sizeof(double) * h->n_dof));
  if (hist_trial_out) HFE_TRY(export_history(h, h->hist_trial, hist_trial_out));
  if (stats != nullptr) {
    HFE_TRY(read_status(h));
    std::memset(stats, 0, sizeof(*stats));
    stats->sweeps = 1;
    stats->plastic_gps = h->h_status->plastic;
    stats->local_fail = h->h_status->local_fail;
    stats->max_local_iters = h->h_status->max_local_iters;
    stats->sweep_ms = elapsed(h->t0, h->t1);
    stats->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
    return check_sweep_status(h);
  }
  return cuda_check(h, cudaGetLastError(), "sweep launch");
}

hfe_status hfe_get_bsr(hfe_handle* h, int64_t* rowptr, int32_t* cols, double* vals) {
  if (h == nullptr) return HFE_EINVAL;
  if (rowptr) std::memcpy(rowptr, h->P.rowptr.data(), 8 * (h->n_nodes + 1));
  if (cols) std::memcpy(cols, h->P.cols.data(), 4 * h->P.n_blocks);
  if (vals) {
    StreamScope scope(h);
    const size_t n = 9 * (size_t)h->P.n_blocks;
    if (h->fp64) {
      HFE_TRY(cuda_check(h, cudaMemcpyAsync(vals, h->K, 8 * n, cudaMemcpyDeviceToHost, h->s), "copy"));
    } else {
      std::vector<float> tmp(n);
      HFE_TRY(cuda_check(h, cudaMemcpyAsync(tmp.data(), h->K, 4 * n, cudaMemcpyDeviceToHost, h->s), "copy"));
      HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "sync"));
      for (size_t i = 0; i < n; ++i) vals[i] = tmp[i];
    }
    HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "sync"));
  }
  return HFE_OK;
}

hfe_status hfe_spmv(hfe_handle* h, const double* x, double* y) {
  if (h == nullptr || x == nullptr || y == nullptr) return HFE_EINVAL;
  StreamScope scope(h);
  HFE_TRY(copy_in(h, h->tmp64, x, sizeof(double) * h->n_dof));
  Csr K = csr_of(h);
  if (h->fp64) {
    spmv<double>(K, (const double*)h->K, h->freem, h->tmp64, (double*)h->vq, nullptr, nullptr, h->s);
    HFE_TRY(copy_out(h, y, h->vq, sizeof(double) * h->n_dof));
  } else {
    to_float(h->tmp64, (float*)h->vp, h->n_dof, h->s);
    spmv<float>(K, (const float*)h->K, h->freem, (const float*)h->vp, (float*)h->vq, nullptr, nullptr, h->s);
    to_double((const float*)h->vq, h->tmp64, h->n_dof, h->s);
    HFE_TRY(copy_out(h, y, h->tmp64, sizeof(double) * h->n_dof));
  }
  return cuda_check(h, cudaStreamSynchronize(h->s), "spmv");
}

hfe_status hfe_solve(hfe_handle* h, const double* b, double* x, hfe_stats* stats) {
  if (h == nullptr || b == nullptr || x == nullptr) return HFE_EINVAL;
  StreamScope scope(h);
  HFE_TRY(copy_in(h, h->tmp64, b, sizeof(double) * h->n_dof));
  int64_t it = 0;
  cudaEventRecord(h->t0, h->s);
  hfe_status st = solve_any(h, h->tmp64, 1.0, &it);
  cudaEventRecord(h->t1, h->s);
  if (st != HFE_OK) return st;
  if (h->fp64) HFE_TRY(copy_out(h, x, h->vx, sizeof(double) * h->n_dof));
  else {
    to_double((const float*)h->vx, h->tmp64, h->n_dof, h->s);
    HFE_TRY(copy_out(h, x, h->tmp64, sizeof(double) * h->n_dof));
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    cudaStreamSynchronize(h->s);
    stats->pcg_iters = h->h_sc->iters;
    stats->solve_ms = elapsed(h->t0, h->t1);
  }
  return cuda_check(h, cudaStreamSynchronize(h->s), "solve");
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Extrapolated predictor (Sec. 2.2, automatic time stepping): u = sum_k w_k u_k on the free
// dofs, w_k the Lagrange weights in the load factor of the stored (sub)step solutions.
namespace {
constexpr int kExtrapBlock = 256;

__global__ void __launch_bounds__(kExtrapBlock) extrapolate_kernel(double* __restrict__ u, const double* __restrict__ u0,
                                                                   const double* __restrict__ u1,
                                                                   const double* __restrict__ u2, double w0, double w1,
                                                                   double w2, const uint8_t* __restrict__ freem,
                                                                   int64_t n_dof) {
  const int64_t d = (int64_t)blockIdx.x * kExtrapBlock + threadIdx.x;
  if (d >= n_dof || !freem[d]) return;
  double v = w0 * u0[d] + w1 * u1[d];
  if (u2 != nullptr) v += w2 * u2[d];
  u[d] = v;
}

// stores (t, u) as the newest solution of the extrapolation history
hfe_status extrap_push(hfe_handle* h, double t) {
  double* oldest = h->extrap_u[2];
  h->extrap_u[2] = h->extrap_u[1];
  h->extrap_u[1] = h->extrap_u[0];
  h->extrap_u[0] = oldest;
  h->extrap_t[2] = h->extrap_t[1];
  h->extrap_t[1] = h->extrap_t[0];
  h->extrap_t[0] = t;
  h->extrap_n = std::min(h->extrap_n + 1, 3);
  return cuda_check(h, cudaMemcpyAsync(h->extrap_u[0], h->u, sizeof(double) * h->n_dof, cudaMemcpyDeviceToDevice, h->s),
                    "copy");
}

// the number of stored solutions the extrapolation to t_new uses (1 = none: u_{n-1} stays)
// and their Lagrange weights
int extrap_weights(const hfe_handle* h, double t_new, double w[3]) {
  return extrapolation_weights(h->extrap_t, h->extrap_n, h->opt.predictor == 2 ? 2 : 3, t_new, w);
}
}  // namespace

// ---------------------------------------------------------------------------------------
// Warm-start record: room for n_steps displacements, the slots already recorded kept.
namespace {
hfe_status warm_reserve(hfe_handle* h, int n_steps) {
  if (n_steps > h->warm_cap) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * (size_t)n_steps * h->n_dof) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, HFE_ENOMEM, "warm-start record");
    }
    double* nu = static_cast<double*>(p);
    if (h->warm_u != nullptr) {
      cudaError_t e = cudaMemcpyAsync(nu, h->warm_u, sizeof(double) * (size_t)h->warm_cap * h->n_dof,
                                      cudaMemcpyDeviceToDevice, h->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
      if (e != cudaSuccess) {
        cudaFree(nu);
        return cuda_check(h, e, "warm-start record");
      }
      cudaFree(h->warm_u);
    }
    h->device_bytes += sizeof(double) * (size_t)(n_steps - h->warm_cap) * h->n_dof;
    h->warm_u = nu;
    h->warm_cap = n_steps;
  }
  if ((int)h->warm_t.size() < n_steps) h->warm_t.resize(n_steps, std::numeric_limits<double>::quiet_NaN());
  return HFE_OK;
}
}  // namespace

extern "C" hfe_status hfe_set_warm_start(hfe_handle* h, int mode) {
  if (h == nullptr || mode < HFE_WARM_OFF || mode > HFE_WARM_USE) return HFE_EINVAL;
  if (mode == HFE_WARM_OFF && h->warm_u != nullptr) {
    StreamScope scope(h);
    cudaStreamSynchronize(h->s);
    cudaFree(h->warm_u);
    h->device_bytes -= sizeof(double) * (size_t)h->warm_cap * h->n_dof;
    h->warm_u = nullptr;
    h->warm_cap = 0;
    h->warm_t.clear();
  }
  h->warm_mode = mode;
  return HFE_OK;
}

extern "C" hfe_status hfe_set_barrier_spin_limit(hfe_handle* h, int64_t limit) {
  if (h == nullptr || limit < 0) return HFE_EINVAL;
  h->opt.barrier_spin_limit = limit;
  return HFE_OK;
}

// ---------------------------------------------------------------------------------------
// Newton driver (shared with the adjoint's forward pass).
hfe_status hfe::newton_steps(hfe_handle* h, int n_steps, const double* t, double* u_out_dev_or_host,
                            double* sigma_out, double* hist_out, hfe_stats* st, StepHook* hook) {
  auto w0 = std::chrono::steady_clock::now();
  hfe_stats loc;
  std::memset(&loc, 0, sizeof(loc));
  const bool u_out_dev = is_device_ptr(u_out_dev_or_host);
  const int64_t bicg0 = h->n_bicgstab;
  // one load (sub)step from the stored state to t_new: predictor, Newton, commit; marker =
  // index of the requested load factor it reaches, or -1 for an intermediate substep
  // guess: the warm-start record slot of this requested step, or nullptr for a cold start
  auto one_step = [&](const double t_new, const int marker, const double* guess) -> hfe_status {
      double ref = -1.0, prev = 0.0, prev_solve = -1.0, eta_prev = 1e-3;
      double step_scale = 0.0;   // fraction of the last correction (in ls.vx) currently applied
      const double t_prev = h->t_state;
      // the newest stored solution must be the stored state; anything else is a history of
      // another pass (a state reset that did not clear it) and is dropped
      if (h->extrap_n > 0 && h->extrap_t[0] != t_prev) h->extrap_n = 0;
      if (h->opt.predictor >= 2 && h->extrap_n == 0) HFE_TRY(extrap_push(h, t_prev));
      double wex[3];
      const int kex = (h->opt.predictor >= 2 && guess == nullptr) ? extrap_weights(h, t_new, wex) : 1;
      // the tangent predictor's solve; it also starts an extrapolating run until two solutions
      // are stored (a step from u_{n-1} with the new Dirichlet values alone can land on another
      // equilibrium branch of the perforated plate)
      const bool solve_pred = guess == nullptr && (h->opt.predictor == 1 || (h->opt.predictor >= 2 && kex == 1));
      // the predictor solve is loose; a warm start or an extrapolation makes none
      bool last_tight = !solve_pred || !h->opt.ew_forcing;
      bool force_tight = false;
      int backtracks = 0;
      HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->u_start, h->u, sizeof(double) * h->n_dof, cudaMemcpyDeviceToDevice, h->s),
                         "copy"));
      if (h->opt.predictor >= 1) {
        // tangent predictor on the converged start-of-step state u_{n-1}:
        // K du = -(R(u_{n-1}) + K du_D - dt f_ext) on the free dofs, du_D = Dirichlet increment,
        // with K and R of the previous step's last Newton iteration (its consistent tangent at
        // u_{n-1}); without them (first step, or after the state was set) the sweep at
        // (u_{n-1}, h_{n-1}).  The norm of its right-hand side is the Newton reference of the
        // step whatever starts it (this solve, an extrapolation or a warm start).
        if (!h->pred_valid) {
          cudaEventRecord(h->t0, h->s);
          HFE_TRY(sweep(h, h->u, t_prev, HFE_SWEEP_TANGENT, h->R, nullptr));
          cudaEventRecord(h->t1, h->s);
          HFE_TRY(read_status(h));
          loc.sweeps++;
          loc.sweep_ms += elapsed(h->t0, h->t1);
          HFE_TRY(check_sweep_status(h));
        }
        h->pred_valid = false;
        HFE_TRY(cuda_check(h, cudaMemsetAsync(h->tmp64, 0, sizeof(double) * h->n_dof, h->s), "memset"));
        set_dirichlet(h->tmp64, h->fixed_dof, h->fixed_val, t_new - t_prev, h->n_fixed, h->s);
        Csr K = csr_of(h);
        if (h->fp64) {
          spmv_rows<double>(K, (const double*)h->K, h->freem, h->tmp64, (double*)h->vq, h->s);
          predictor_rhs<double>(h->R, (const double*)h->vq, h->f_ext, t_new - t_prev, h->freem, h->b64, h->n_dof, h->s);
        } else {
          to_float(h->tmp64, (float*)h->vp, h->n_dof, h->s);
          spmv_rows<float>(K, (const float*)h->K, h->freem, (const float*)h->vp, (float*)h->vq, h->s);
          predictor_rhs<float>(h->R, (const float*)h->vq, h->f_ext, t_new - t_prev, h->freem, h->b64, h->n_dof, h->s);
        }
        free_norm(h->b64, h->freem, h->n_dof, h->sc, h->part, h->s, nullptr);
        HFE_TRY(read_status(h));
        ref = std::max(std::sqrt(h->h_sc->norm2), h->opt.newton_atol);
        set_dirichlet(h->u, h->fixed_dof, h->fixed_val, t_new, h->n_fixed, h->s);
        if (kex > 1) {
          const unsigned blocks = (unsigned)((h->n_dof + kExtrapBlock - 1) / kExtrapBlock);
          extrapolate_kernel<<<blocks, kExtrapBlock, 0, h->s>>>(h->u, h->extrap_u[0], h->extrap_u[1],
                                                              kex == 3 ? h->extrap_u[2] : nullptr, wex[0], wex[1],
                                                              wex[2], h->freem, h->n_dof);
          HFE_TRY(cuda_check(h, cudaGetLastError(), "extrapolate"));
        } else if (h->h_sc->norm2 > 0.0 && solve_pred) {
          cudaEventRecord(h->t0, h->s);
          if (h->opt.ew_forcing) h->pcg_rtol_now = std::max(h->opt.pcg_rtol, 1e-3);   // predictor: rough solve
          h->allow_truncated = true;
          h->allow_indefinite = true;
          hfe_status pst = solve_any(h, h->b64, 1.0, nullptr);
          h->allow_truncated = false;
          h->allow_indefinite = false;
          h->pcg_rtol_now = 0.0;
          HFE_TRY(pst);
          cudaEventRecord(h->t1, h->s);
          cudaEventSynchronize(h->t1);
          loc.solve_ms += elapsed(h->t0, h->t1);
          loc.pcg_iters += h->h_sc->iters;
          if (h->fp64) add_update<double>(h->u, (const double*)h->vx, h->freem, h->n_dof, h->s);
          else add_update<float>(h->u, (const float*)h->vx, h->freem, h->n_dof, h->s);
          step_scale = 1.0;
        }
      } else {
        set_dirichlet(h->u, h->fixed_dof, h->fixed_val, t_new, h->n_fixed, h->s);
        if (guess != nullptr) {
          // the reference of a step from u_{n-1}: the residual there with the new Dirichlet values
          cudaEventRecord(h->t0, h->s);
          HFE_TRY(sweep(h, h->u, t_new, HFE_SWEEP_RESIDUAL, h->R, nullptr));
          cudaEventRecord(h->t1, h->s);
          free_norm(h->R, h->freem, h->n_dof, h->sc, h->part, h->s, nullptr);
          HFE_TRY(read_status(h));
          loc.sweeps++;
          loc.sweep_ms += elapsed(h->t0, h->t1);
          HFE_TRY(check_sweep_status(h));
          if (h->h_sc->nonfinite > 0) return fail(h, HFE_ENONFINITE, "non-finite residual");
          ref = std::max(std::sqrt(h->h_sc->norm2), h->opt.newton_atol);
        }
      }
      if (guess != nullptr) {
        // warm start: the previous pass's converged displacement at this load factor
        HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->u, guess, sizeof(double) * h->n_dof, cudaMemcpyDeviceToDevice, h->s),
                           "copy"));
        set_dirichlet(h->u, h->fixed_dof, h->fixed_val, t_new, h->n_fixed, h->s);
        step_scale = 0.0;
      }
      int stall = 0;
      bool conv = false;
      for (int it = 0; it <= h->opt.newton_maxit; ++it) {
        cudaEventRecord(h->t0, h->s);
        HFE_TRY(sweep(h, h->u, t_new, HFE_SWEEP_TANGENT, h->R, nullptr));
        cudaEventRecord(h->t1, h->s);
        free_norm(h->R, h->freem, h->n_dof, h->sc, h->part, h->s, nullptr);
        HFE_TRY(read_status(h));
        loc.sweeps++;
        loc.sweep_ms += elapsed(h->t0, h->t1);
        if ((h->h_status->detj > 0 || h->h_status->nonfinite > 0 || h->h_sc->nonfinite > 0) && step_scale > 0.0 &&
            backtracks < 6) {
          // the last correction inverted an element or produced non-finite values: halve it
          const double c = -0.5 * step_scale;
          if (h->fp64) add_update<double>(h->u, (const double*)h->vx, h->freem, h->n_dof, h->s, c);
          else add_update<float>(h->u, (const float*)h->vx, h->freem, h->n_dof, h->s, c);
          step_scale *= 0.5;
          ++backtracks;
          --it;
          continue;
        }
        HFE_TRY(check_sweep_status(h));
        loc.plastic_gps = h->h_status->plastic;
        loc.max_local_iters = std::max<int32_t>(loc.max_local_iters, (int32_t)h->h_status->max_local_iters);
        if (h->h_sc->nonfinite > 0) return fail(h, HFE_ENONFINITE, "non-finite residual");
        const double nrm = std::sqrt(h->h_sc->norm2);
        loc.last_residual = nrm;
        if (ref < 0.0) ref = std::max(nrm, h->opt.newton_atol);
        if (nrm <= h->opt.newton_rtol * ref) {
          // accept only after a correction solved to pcg_rtol: with an ill-conditioned K a small
          // residual after a loose solve can still hide a large error in the soft modes
          if (last_tight || !h->opt.ew_forcing) { conv = true; break; }
          force_tight = true;
        }
        const bool slow = it >= 1 && nrm > 0.5 * prev;
        if (!h->fp64 && it >= 2) {   // mixed: accept a stagnated residual below newton_stag_tol
          // (only after solves at the tightest tolerance, so an inexact solve cannot stall it)
          stall = (slow && last_tight) ? stall + 1 : 0;
          if (stall >= 2 && nrm <= h->opt.newton_stag_tol * ref) { conv = true; break; }
        }
        prev = nrm;
        if (it == h->opt.newton_maxit) break;
        int64_t pit = 0;
        cudaEventRecord(h->t0, h->s);
        // inexact Newton: Eisenstat-Walker forcing (choice 2, gamma = 0.9, alpha = 2) with their
        // safeguard, bounded below by pcg_rtol; the converged solution does not depend on it
        if (h->opt.ew_forcing) {
          double eta = 1e-3;
          if (prev_solve > 0.0) {
            const double ratio = nrm / prev_solve;
            eta = 0.9 * ratio * ratio;
            const double safe = 0.9 * eta_prev * eta_prev;
            if (safe > 0.1) eta = std::max(eta, safe);
          }
          eta = std::min(eta, 0.5);
          if (slow || force_tight) eta = h->opt.pcg_rtol;   // slow progress or final correction: solve tightly
          eta = std::max(eta, h->opt.pcg_rtol);
          h->pcg_rtol_now = eta;
          eta_prev = eta;
        }
        prev_solve = nrm;
        last_tight = !h->opt.ew_forcing || h->pcg_rtol_now <= h->opt.pcg_rtol * 1.0000001;
        h->allow_truncated = true;
        h->allow_indefinite = true;
        h->pcg_truncated = false;
        hfe_status sst = solve_any(h, h->R, -1.0, &pit);
        h->allow_truncated = false;
        h->allow_indefinite = false;
        h->pcg_rtol_now = 0.0;
        HFE_TRY(sst);
        if (h->pcg_truncated) last_tight = false;
        cudaEventRecord(h->t1, h->s);
        cudaEventSynchronize(h->t1);
        loc.solve_ms += elapsed(h->t0, h->t1);
        loc.pcg_iters += h->h_sc->iters;
        (void)pit;
        if (h->fp64) add_update<double>(h->u, (const double*)h->vx, h->freem, h->n_dof, h->s);
        else add_update<float>(h->u, (const float*)h->vx, h->freem, h->n_dof, h->s);
        step_scale = 1.0;
        backtracks = 0;
        loc.newton_iters++;
      }
      if (!conv)
        return fail(h, HFE_ENEWTON, "Newton did not converge at t = " + std::to_string(t_new) + ", |R| = " +
                                        std::to_string(loc.last_residual));
      if (hook) HFE_TRY(hook->before_commit(h, t_new));
      if (sigma_out != nullptr && marker == n_steps - 1) {
        if (h->sigma == nullptr) {
          if (cudaMalloc(&h->sigma, sizeof(double) * 6 * h->n_gp) != cudaSuccess) return fail(h, HFE_ENOMEM, "sigma");
        }
        HFE_TRY(sweep(h, h->u, t_new, HFE_SWEEP_RESIDUAL, h->R, h->sigma));
        HFE_TRY(read_status(h));
        HFE_TRY(copy_out(h, sigma_out, h->sigma, sizeof(double) * 6 * h->n_gp));
      }
      std::swap(h->hist, h->hist_trial);   // commit h_n = H(u_n, h_{n-1})
      if (!h->fp64) launch_sigma_cache(h->hist, false, h->mat64, h->n_mat > 1, h->hardening, h->n_gp, h->s);
      if (h->warm_mode != HFE_WARM_OFF && marker >= 0) {
        HFE_TRY(cuda_check(h, cudaMemcpyAsync(h->warm_u + (size_t)marker * h->n_dof, h->u, sizeof(double) * h->n_dof,
                                              cudaMemcpyDeviceToDevice, h->s), "copy"));
        h->warm_t[marker] = t_new;
      }
      if (u_out_dev_or_host != nullptr && marker >= 0) {
        double* dst = u_out_dev_or_host + (size_t)marker * h->n_dof;
        if (u_out_dev) HFE_TRY(cuda_check(h, cudaMemcpyAsync(dst, h->u, 8 * h->n_dof, cudaMemcpyDeviceToDevice, h->s), "copy"));
        else HFE_TRY(copy_out(h, dst, h->u, sizeof(double) * h->n_dof));
      }
      h->t_state = t_new;
      h->pred_valid = true;
      if (h->opt.predictor >= 2) HFE_TRY(extrap_push(h, t_new));
      if (hook) HFE_TRY(hook->after_commit(h, t_new, marker));
      return HFE_OK;
  };
  // a failed attempt leaves the stored state at the last converged step
  auto attempt = [&](const double t_new, const int marker, const double* guess) -> hfe_status {
    const hfe_status s = one_step(t_new, marker, guess);
    if (s != HFE_OK) {
      h->pred_valid = false;
      h->allow_truncated = h->allow_indefinite = false;
      h->pcg_rtol_now = 0.0;
      cudaMemcpyAsync(h->u, h->u_start, sizeof(double) * h->n_dof, cudaMemcpyDeviceToDevice, h->s);
      cudaStreamSynchronize(h->s);
    }
    return s;
  };
  // Adaptive load stepping (Sec. 2.2 Implementation Aspects): each requested load factor is
  // first reached in one step; a step whose Newton fails (no convergence, an inverted
  // element, non-finite values, a failed solve or local return mapping) is rejected and
  // retried with the increment times `cutback`, down to the interval times
  // cutback^max_cutbacks; after two accepted substeps in a row the increment grows back by
  // 1/cutback, clipped so that the requested load factors are hit exactly.  A reduced
  // increment carries over to the next interval.
  // Increments are handled as magnitudes along the direction of each interval, so loading
  // and unloading intervals are stepped alike.
  //
  // Warm start: the record is sized for this pass first; a requested step whose record slot
  // holds the same load factor starts from it and spans its whole interval.
  if (h->warm_mode != HFE_WARM_OFF) HFE_TRY(warm_reserve(h, n_steps));
  if (h->opt.predictor >= 2 && h->extrap_u[0] == nullptr) {
    for (double*& p : h->extrap_u) {
      void* q = nullptr;
      if (cudaMalloc(&q, sizeof(double) * h->n_dof) != cudaSuccess) {
        cudaGetLastError();
        for (double*& r : h->extrap_u) {
          if (r) cudaFree(r);
          r = nullptr;
        }
        return fail(h, HFE_ENOMEM, "extrapolation history");
      }
      p = static_cast<double*>(q);
    }
    h->device_bytes += 3 * sizeof(double) * (size_t)h->n_dof;
    h->extrap_n = 0;
  }
  double inc_carry = 0.0;
  for (int n = 0; n < n_steps; ++n) {
    int cuts = 0, ok_run = 0;
    const double span = t[n] - h->t_state;
    const double dirn = span < 0.0 ? -1.0 : 1.0;
    double inc_try = std::fabs(span);
    const double inc_min = inc_try * std::pow(h->opt.cutback, (double)h->opt.max_cutbacks);
    const double* guess = nullptr;
    if (h->warm_mode == HFE_WARM_USE && n < (int)h->warm_t.size() &&
        std::fabs(h->warm_t[n] - t[n]) <= 1e-12 * std::max(1.0, std::fabs(t[n])))
      guess = h->warm_u + (size_t)n * h->n_dof;
    if (guess == nullptr && inc_carry > 0.0 && inc_carry < inc_try) inc_try = inc_carry;
    if (guess != nullptr) loc.warm_steps++;
    for (;;) {
      const double remaining = std::fabs(t[n] - h->t_state);
      const double inc = std::min(inc_try, remaining);
      const bool hits = inc >= remaining * (1.0 - 1e-12);
      const double t_new = hits ? t[n] : h->t_state + dirn * inc;
      const double* g = hits ? guess : nullptr;
      const hfe_status s = attempt(t_new, hits ? n : -1, g);
      const bool recoverable = s == HFE_ENEWTON || s == HFE_EDETJ || s == HFE_ENONFINITE || s == HFE_EPCG ||
                               s == HFE_ELOCAL;
      if (s != HFE_OK && g != nullptr && recoverable) {
        // a failed warm attempt is retried cold over the same increment
        guess = nullptr;
        loc.warm_retries++;
        continue;
      }
      if (s == HFE_OK) {
        loc.substeps++;
        if (hits) break;
        if (++ok_run >= 2) {
          inc_try = inc / h->opt.cutback;
          ok_run = 0;
        } else {
          inc_try = inc;
        }
        continue;
      }
      if (!h->opt.adaptive || !recoverable || inc * h->opt.cutback < inc_min * (1.0 - 1e-9)) {
        loc.bicgstab_solves = h->n_bicgstab - bicg0;
        if (st) *st = loc;
        return s;
      }
      ++cuts;
      loc.cutbacks++;
      ok_run = 0;
      inc_try = inc * h->opt.cutback;
    }
    inc_carry = cuts > 0 ? inc_try : 0.0;
    loc.steps_done = n + 1;
  }
  if (hist_out) HFE_TRY(export_history(h, h->hist, hist_out));
  HFE_TRY(cuda_check(h, cudaStreamSynchronize(h->s), "forward"));
  loc.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  loc.bicgstab_solves = h->n_bicgstab - bicg0;
  if (st) *st = loc;
  return HFE_OK;
}

extern "C" hfe_status hfe_forward(hfe_handle* h, int n_steps, const double* t, double* u_out, double* sigma_out,
                                  double* hist_out, hfe_stats* stats) {
  if (h == nullptr || t == nullptr || n_steps <= 0) return HFE_EINVAL;
  StreamScope scope(h);
  std::vector<double> th(n_steps);
  std::memcpy(th.data(), t, sizeof(double) * n_steps);
  return newton_steps(h, n_steps, th.data(), u_out, sigma_out, hist_out, stats, nullptr);
}

extern "C" hfe_status hfe_adjoint(hfe_handle* h, int n_steps, const double* t, const double* u_target, double w,
                                  double* J_out, double* grad_out, hfe_stats* stats) {
  if (h == nullptr || t == nullptr || n_steps <= 0 || u_target == nullptr) return HFE_EINVAL;
  StreamScope scope(h);
  return adjoint_run(h, n_steps, t, u_target, w, J_out, grad_out, stats);
}
