"""Thin Python binding of the C ABI in include/hfe.h (argument marshalling only).

Every computation runs in ``libhfe.so`` (hand-written CUDA for sm_103a).  There is no CPU
fallback: if the library is missing or no CUDA device is present the calls raise.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they must be contiguous
and of the documented dtype (float64 for reals, int32 for ``conn``, int64 for dofs).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["HfeError", "Solver", "lib", "LIB_PATH", "STATUS", "material_arrays"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhfe.so")

STATUS = {0: "HFE_OK", -1: "HFE_EINVAL", -2: "HFE_ENOMEM", -3: "HFE_ECUDA", -4: "HFE_EDETJ",
          1: "HFE_ENEWTON", 2: "HFE_ELOCAL", 3: "HFE_EPCG", 4: "HFE_ENONFINITE", 5: "HFE_EBARRIER"}
PRECISION = {"fp64": 0, "mixed": 1}
HARDENING = {"swift": 0, "voce": 1}
SWEEP_RESIDUAL, SWEEP_TANGENT = 0, 1


class HfeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_el", C.c_int64), ("X", C.c_void_p), ("conn", C.c_void_p)]


class _BC(C.Structure):
    _fields_ = [("n_fixed", C.c_int64), ("dof", C.c_void_p), ("value", C.c_void_p), ("f_ext", C.c_void_p)]


class _Material(C.Structure):
    _fields_ = [("hardening", C.c_int), ("n_mat", C.c_int64), ("theta", C.c_void_p), ("Theta", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("newton_rtol", C.c_double), ("newton_atol", C.c_double),
                ("newton_maxit", C.c_int), ("newton_stag_tol", C.c_double), ("pcg_rtol", C.c_double),
                ("pcg_maxit", C.c_int), ("pcg_check_every", C.c_int), ("precond", C.c_int),
                ("local_maxit", C.c_int), ("local_tol", C.c_double), ("ckpt_every", C.c_int),
                ("predictor", C.c_int), ("ew_forcing", C.c_int), ("pcg_persistent", C.c_int),
                ("adaptive", C.c_int), ("cutback", C.c_double), ("max_cutbacks", C.c_int), ("fbar", C.c_int),
                ("barrier_spin_limit", C.c_int64), ("assembly_l2_bytes", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int64), ("pcg_iters", C.c_int64), ("sweeps", C.c_int64),
                ("plastic_gps", C.c_int64), ("local_fail", C.c_int64), ("max_local_iters", C.c_int32),
                ("steps_done", C.c_int32), ("last_residual", C.c_double), ("sweep_ms", C.c_double),
                ("solve_ms", C.c_double), ("total_ms", C.c_double), ("bicgstab_solves", C.c_int64),
                ("substeps", C.c_int64), ("cutbacks", C.c_int64), ("warm_steps", C.c_int64),
                ("warm_retries", C.c_int64), ("refine_pcg_iters", C.c_int64), ("reverse_pcg_iters", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_el", C.c_int64), ("n_dof", C.c_int64), ("n_gp", C.c_int64),
                ("n_blocks", C.c_int64), ("n_fixed", C.c_int64), ("n_colors", C.c_int32),
                ("precision", C.c_int32), ("device_bytes", C.c_int64), ("n_slabs", C.c_int64),
                ("n_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def lib():
    """Load libhfe.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2606_17390_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    L.hfe_default_options.argtypes = [C.POINTER(Options), i32]
    L.hfe_default_options.restype = None
    L.hfe_create.argtypes = [C.POINTER(_Mesh), C.POINTER(_BC), C.POINTER(_Material), C.POINTER(Options), vp,
                             C.POINTER(vp)]
    L.hfe_destroy.argtypes = [vp]
    L.hfe_destroy.restype = None
    L.hfe_last_error.argtypes = [vp]
    L.hfe_last_error.restype = C.c_char_p
    L.hfe_get_info.argtypes = [vp, C.POINTER(Info)]
    L.hfe_set_material.argtypes = [vp, C.POINTER(_Material)]
    L.hfe_set_state.argtypes = [vp, vp, vp]
    L.hfe_set_load.argtypes = [vp, dbl]
    L.hfe_get_load.argtypes = [vp, C.POINTER(dbl)]
    L.hfe_get_state.argtypes = [vp, vp, vp]
    L.hfe_gp_sweep.argtypes = [vp, vp, dbl, i32, vp, vp, vp, C.POINTER(Stats)]
    L.hfe_get_bsr.argtypes = [vp, vp, vp, vp]
    L.hfe_spmv.argtypes = [vp, vp, vp]
    L.hfe_solve.argtypes = [vp, vp, vp, C.POINTER(Stats)]
    L.hfe_forward.argtypes = [vp, i32, vp, vp, vp, vp, C.POINTER(Stats)]
    L.hfe_adjoint.argtypes = [vp, i32, vp, vp, dbl, vp, vp, C.POINTER(Stats)]
    L.hfe_set_barrier_spin_limit.argtypes = [vp, C.c_int64]
    for name in ("hfe_create", "hfe_get_info", "hfe_set_material", "hfe_set_state", "hfe_get_state",
                 "hfe_set_load", "hfe_get_load",
                 "hfe_gp_sweep", "hfe_get_bsr", "hfe_spmv", "hfe_solve", "hfe_forward", "hfe_adjoint",
                 "hfe_set_barrier_spin_limit"):
        getattr(L, name).restype = i32
    _LIB = L
    return L


def _ptr(x, dtype=None):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {x.dtype}")
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(type(x))


def material_arrays(theta, Theta=None):
    th = np.ascontiguousarray(np.atleast_2d(np.asarray(theta, dtype=np.float64)))
    Th = None
    if Theta is not None:
        Th = np.asarray(Theta, dtype=np.float64)
        if Th.ndim == 2:
            Th = Th[None]
        if Th.shape[0] == 1 and th.shape[0] > 1:
            Th = np.repeat(Th, th.shape[0], axis=0)
        Th = np.ascontiguousarray(Th.reshape(-1, 9))
        if np.allclose(Th, np.eye(3).ravel()[None]):
            Th = None
    return th, Th


class Solver:
    """One handle of the library: mesh, Dirichlet data, material and workspaces on the GPU."""

    def __init__(self, X, conn, fixed_dof, fixed_val, theta, hardening, Theta=None, precision="fp64",
                 f_ext=None, stream=None, **options):
        L = lib()
        self._keep = []
        X = np.ascontiguousarray(X, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        dof = np.ascontiguousarray(fixed_dof, dtype=np.int64)
        val = np.ascontiguousarray(fixed_val, dtype=np.float64)
        th, Th = material_arrays(theta, Theta)
        self.Theta_axes = Theta
        self.n_nodes, self.n_el = X.shape[0], conn.shape[0]
        self.n_dof, self.n_gp = 3 * self.n_nodes, 8 * self.n_el
        self.hardening = hardening
        self.n_mat = th.shape[0]
        mesh = _Mesh(self.n_nodes, self.n_el, _ptr(X), _ptr(conn))
        fe = None if f_ext is None else np.ascontiguousarray(f_ext, dtype=np.float64)
        bc = _BC(dof.size, _ptr(dof), _ptr(val), _ptr(fe))
        mat = _Material(HARDENING[hardening], th.shape[0], _ptr(th), _ptr(Th))
        opt = Options()
        L.hfe_default_options(C.byref(opt), PRECISION[precision])
        for k, v in options.items():
            if not hasattr(opt, k):
                raise KeyError(k)
            setattr(opt, k, v)
        self.options = opt
        self.precision = precision
        h = C.c_void_p()
        st = L.hfe_create(C.byref(mesh), C.byref(bc), C.byref(mat), C.byref(opt), stream, C.byref(h))
        self._h = h
        if st != 0:
            msg = L.hfe_last_error(h).decode() if h.value else "hfe_create failed"
            self.close()
            raise HfeError(st, msg)

    # -- helpers
    def _check(self, st):
        if st != 0:
            raise HfeError(st, lib().hfe_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hfe_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self):
        inf = Info()
        self._check(lib().hfe_get_info(self._h, C.byref(inf)))
        return inf.as_dict()

    # -- state and material
    def set_material(self, theta, Theta=None):
        th, Th = material_arrays(theta, Theta)
        mat = _Material(HARDENING[self.hardening], th.shape[0], _ptr(th), _ptr(Th))
        self._check(lib().hfe_set_material(self._h, C.byref(mat)))

    def set_state(self, u=None, hist=None):
        self._check(lib().hfe_set_state(self._h, _ptr(u), _ptr(hist)))

    def set_load(self, t):
        """Load factor of the stored state (hfe_set_state resets it to 0)."""
        self._check(lib().hfe_set_load(self._h, float(t)))

    def get_load(self):
        t = C.c_double()
        self._check(lib().hfe_get_load(self._h, C.byref(t)))
        return t.value

    def get_state(self):
        u = np.empty(self.n_dof)
        hist = np.empty((7, self.n_gp))
        self._check(lib().hfe_get_state(self._h, _ptr(u), _ptr(hist)))
        return u, hist

    # -- hot path
    def sweep(self, u, load=1.0, tangent=True, R_out=None, hist_out=None, stats=True, rnorm_out=None):
        """One Gauss-point sweep; returns (R, hist_trial, stats).  Host arrays are allocated
        unless the caller passes its own (host or device) output buffers; rnorm_out (a
        1-element buffer) receives the FP64 norm of R over the free dofs."""
        R = np.empty(self.n_dof) if R_out is None else R_out
        H = hist_out
        s = Stats() if stats else None
        st = lib().hfe_gp_sweep(self._h, _ptr(u), float(load), SWEEP_TANGENT if tangent else SWEEP_RESIDUAL,
                                _ptr(R), _ptr(rnorm_out), _ptr(H), C.byref(s) if s is not None else None)
        self._check(st)
        return R, H, (s.as_dict() if s is not None else None)

    def get_bsr(self, values=True):
        inf = self.info()
        rowptr = np.empty(self.n_nodes + 1, dtype=np.int64)
        cols = np.empty(inf["n_blocks"], dtype=np.int32)
        vals = np.empty(9 * inf["n_blocks"]) if values else None
        self._check(lib().hfe_get_bsr(self._h, _ptr(rowptr), _ptr(cols), _ptr(vals)))
        return rowptr, cols, (vals.reshape(-1, 3, 3) if values else None)

    def spmv(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64) if isinstance(x, np.ndarray) else x
        y = np.empty(self.n_dof) if isinstance(x, np.ndarray) else x.new_empty(self.n_dof)
        self._check(lib().hfe_spmv(self._h, _ptr(x), _ptr(y)))
        return y

    def set_barlat(self, mat, **options):
        """Give this handle (FP64 or mixed) the Barlat material `mat` (inputs.BarlatMaterial-like)
        through hfe_set_barlat, with the local controls of cpp_options; mat None returns it to
        Hill-48."""
        f = lib().hfe_set_barlat
        f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        f.restype = C.c_int
        if mat is None:
            self._check(f(self._h, None, None))
            return
        m = barlat_material(mat)
        o = cpp_options(**options)
        self._check(f(self._h, C.byref(m), C.byref(o)))

    WARM_MODES = {"off": 0, "record": 1, "use": 2}

    def set_warm_start(self, mode):
        """hfe_set_warm_start: "off" (cold steps, record freed), "record" (record each pass's
        displacement at its requested load factors) or "use" (record, and start each requested
        step's Newton iteration from the recorded displacement at the same load factor)."""
        f = lib().hfe_set_warm_start
        f.argtypes = [C.c_void_p, C.c_int]
        f.restype = C.c_int
        self._check(f(self._h, self.WARM_MODES[mode] if isinstance(mode, str) else int(mode)))

    def set_barrier_spin_limit(self, limit):
        """hfe_set_barrier_spin_limit: the bound (polls) of every grid-barrier wait in the
        one-launch Krylov solves of the calls that follow."""
        self._check(lib().hfe_set_barrier_spin_limit(self._h, int(limit)))
        self.options.barrier_spin_limit = int(limit)

    def solve(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64) if isinstance(b, np.ndarray) else b
        x = np.empty(self.n_dof) if isinstance(b, np.ndarray) else b.new_empty(self.n_dof)
        s = Stats()
        self._check(lib().hfe_solve(self._h, _ptr(b), _ptr(x), C.byref(s)))
        return x, s.as_dict()

    def forward(self, t, u_out=None, sigma_out=None, hist_out=None, want_u=True):
        t = np.ascontiguousarray(t, dtype=np.float64)
        if u_out is None and want_u:
            u_out = np.empty((t.size, self.n_dof))
        s = Stats()
        self._check(lib().hfe_forward(self._h, int(t.size), _ptr(t), _ptr(u_out), _ptr(sigma_out),
                                      _ptr(hist_out), C.byref(s)))
        return u_out, s.as_dict()

    def adjoint(self, t, u_target, w=1.0, grad_out=None):
        """Misfit J = w sum_n ||u^n - u_target^n||^2 of a forward run from the zero state and its
        gradient dJ/dtheta by the discrete adjoint; returns (J, grad [n_mat, 11], stats)."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        if isinstance(u_target, np.ndarray):
            u_target = np.ascontiguousarray(u_target, dtype=np.float64)
        if grad_out is None:
            grad_out = np.empty((self.n_mat, 11))
        J = C.c_double()
        s = Stats()
        self._check(lib().hfe_adjoint(self._h, int(t.size), _ptr(t), _ptr(u_target), float(w), C.byref(J),
                                      _ptr(grad_out), C.byref(s)))
        return J.value, grad_out, s.as_dict()


def from_inputs(mesh, bc, mat, precision="fp64", theta=None, **options):
    """Solver for the dataclasses of paper_2606_17390_b300.inputs."""
    th = mat.theta_vector() if theta is None else theta
    return Solver(mesh.X, mesh.conn, bc.dof, bc.value, th, mat.hardening, mat.Theta, precision=precision,
                  **options)


FREE_NORM_STATIC_MAX_DOF = 4194304   # HFE_FREE_NORM_STATIC_MAX_DOF of include/hfe.h


def free_norm_static(r, free_mask, norm_out, stream=None):
    """||r_free||_2 into norm_out[0] through hfe_free_norm_static, which needs no handle and
    allocates no device memory (its reduction scratch is a static device array of the library).
    r: float64 CUDA tensor [n], free_mask: uint8 CUDA tensor [n] (0 = Dirichlet dof),
    norm_out: float64 CUDA tensor [>= 1], all on the current device; stream: a cudaStream_t
    handle (int) or None for the legacy default stream.  Asynchronous on that stream.  Calls
    that overlap on one device race on the shared scratch."""
    L = lib()
    f = L.hfe_free_norm_static
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    n = int(r.numel()) if hasattr(r, "numel") else int(np.asarray(r).size)
    st = f(_ptr(r), _ptr(free_mask), n, _ptr(norm_out), stream)
    if st != 0:
        if n > FREE_NORM_STATIC_MAX_DOF:
            msg = f"n = {n} exceeds the static scratch limit of {FREE_NORM_STATIC_MAX_DOF} dofs"
        elif st == -1:
            msg = "invalid argument (r, free_mask and norm_out must be device memory of the current device)"
        else:
            msg = "CUDA error in set-up or launch"
        raise HfeError(st, "hfe_free_norm_static: " + msg)


# ---------------------------------------------------------------- Barlat material points
CPP_STATUS = {0: "converged", 1: "elastic", 2: "maxit", 3: "singular", 4: "nonfinite"}
BARLAT_MAX_M = 32   # HFE_BARLAT_MAX_M of include/hfe.h


class BarlatMaterialC(C.Structure):
    _fields_ = [("c1", C.c_double * 9), ("c2", C.c_double * 9), ("m", C.c_int), ("E", C.c_double),
                ("nu", C.c_double), ("hardening", C.c_int), ("h", C.c_double * 3), ("Theta", C.c_double * 9),
                ("orthotropic", C.c_int), ("d", C.c_double * 9)]


class CppOptions(C.Structure):
    _fields_ = [("kmax", C.c_int), ("line_search", C.c_int), ("jmax", C.c_int), ("beta", C.c_double),
                ("eta", C.c_double), ("tol", C.c_double), ("precision", C.c_int)]


def barlat_material(mat) -> BarlatMaterialC:
    """hfe_barlat_material from an object with c1, c2, m, E, nu, hardening ('swift'|'voce'),
    h, Theta (None = identity) and optionally d (nine orthotropic stiffness coefficients in the
    material frame; None = isotropic E, nu), e.g. inputs.BarlatMaterial."""
    s = BarlatMaterialC()
    s.c1[:] = [float(v) for v in mat.c1]
    s.c2[:] = [float(v) for v in mat.c2]
    s.m = int(mat.m)
    s.E, s.nu = float(mat.E), float(mat.nu)
    s.hardening = HARDENING[mat.hardening]
    s.h[:] = [float(v) for v in mat.h]
    Th = np.eye(3) if getattr(mat, "Theta", None) is None else np.asarray(mat.Theta, dtype=np.float64)
    s.Theta[:] = [float(v) for v in Th.reshape(9)]
    d = getattr(mat, "d", None)
    s.orthotropic = 0 if d is None else 1
    s.d[:] = [0.0] * 9 if d is None else [float(v) for v in d]
    return s


def _check(st, name):
    if st != 0:
        raise HfeError(st, name + (": invalid argument (material, options, sizes, or pointers not on the "
                                   "current device)" if st == -1 else ": CUDA error"))


def barlat_phi(mat, T, with_N=False, stream=None):
    """phi (and N = dphi/dT if with_N) for stresses T, a float64 CUDA tensor [n, 6], through
    hfe_barlat_phi.  Returns phi [n] (and N [n, 6]) as CUDA tensors, queued on `stream`
    (a cudaStream_t handle or None for the legacy default stream)."""
    import torch
    L = lib()
    f = L.hfe_barlat_phi
    f.argtypes = [C.POINTER(BarlatMaterialC), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    n = int(T.shape[0])
    phi = torch.empty(n, dtype=torch.float64, device=T.device)
    N = torch.empty((n, 6), dtype=torch.float64, device=T.device) if with_N else None
    m = barlat_material(mat)
    _check(f(C.byref(m), _ptr(T), n, _ptr(phi), _ptr(N), stream), "hfe_barlat_phi")
    return (phi, N) if with_N else phi


def cpp_options(line_search=True, kmax=40, jmax=10, beta=1e-4, eta=0.1, tol=1e-13, precision="fp64") -> CppOptions:
    return CppOptions(int(kmax), int(bool(line_search)), int(jmax), float(beta), float(eta), float(tol),
                      PRECISION[precision])


def barlat_return_map(mat, T_trial, alpha_n, tangent=False, stream=None, out=None, **options):
    """Elastic predictor / plastic corrector for n trial stresses T_trial (float64 CUDA [n, 6])
    with alpha_n (float64 CUDA [n]) through hfe_barlat_return_map; options as cpp_options.
    Returns a dict of CUDA tensors T [n, 6], alpha [n], dgamma [n], iters (int32) [n],
    status (int8) [n] and, if tangent, tangent [n, 6, 6] = dT/dT_trial.  `out`, a dict of
    such tensors, is written in place instead of allocating."""
    import torch
    L = lib()
    f = L.hfe_barlat_return_map
    f.argtypes = [C.POINTER(BarlatMaterialC), C.POINTER(CppOptions), C.c_void_p, C.c_void_p, C.c_int64,
                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    n = int(T_trial.shape[0])
    dev = T_trial.device
    if out is None:
        out = dict(T=torch.empty((n, 6), dtype=torch.float64, device=dev),
                   alpha=torch.empty(n, dtype=torch.float64, device=dev),
                   dgamma=torch.empty(n, dtype=torch.float64, device=dev),
                   iters=torch.empty(n, dtype=torch.int32, device=dev),
                   status=torch.empty(n, dtype=torch.int8, device=dev))
        if tangent:
            out["tangent"] = torch.empty((n, 6, 6), dtype=torch.float64, device=dev)
    m = barlat_material(mat)
    o = cpp_options(**options)
    st = f(C.byref(m), C.byref(o), _ptr(T_trial), _ptr(alpha_n), n, _ptr(out["T"]), _ptr(out["alpha"]),
           _ptr(out["dgamma"]), _ptr(out["iters"]), _ptr(out["status"]), _ptr(out.get("tangent")), stream)
    _check(st, "hfe_barlat_return_map")
    return out
