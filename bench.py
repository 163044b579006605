"""Benchmark of the Gauss-point sweep on the 100^3 hex8 cube (3,090,903 dofs, 8,000,000 Gauss
points; Hill-48 with Swift hardening, clamped-platen compression).

One step = one pass of the per-Newton-iteration element sweep through the C ABI
(hfe_gp_sweep, tangent mode): gather, kinematics, log strain, Hill-48 return mapping,
consistent tangent, post-processing, element contraction, conflict-free scatter into the
block-CSR matrix, and the FP64 residual norm over the free dofs.  The state is the
deterministic mid-step compression state of paper_2606_17390_b300.inputs.compression_state
(every Gauss point plastic).  Inputs (history 512 MB, K 982 MB) exceed the 126 MB L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the CPU baseline runs the oracle single-threaded (set before numpy loads its BLAS)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

from paper_2606_17390_b300 import inputs  # noqa: E402

METRIC = "Gauss-point updates/s (FP32-mixed vs FP64) at 3M DOF; adjoint/forward time ratio"
UNIT = "GP/s"
LOAD = 0.5
# FP32 flops per Gauss point of the tangent sweep counted from the formulation (kinematics
# 0.6k, eigen-decomposition 0.5k, return mapping and recovery 0.7k, post-processor and
# rotated gradients 0.4k, algorithmic tangent in the eigenbasis of C 1.7k, dP/dF 1.0k,
# element contraction with the symmetric K^e 3.4k).
ALG_FLOPS_PER_GP = 8.3e3
# algorithmic DRAM bytes per element of a mixed tangent sweep (one node per element on a
# large structured mesh): conn 32, nodal X (FP32) 12 and u (FP64) 24, history in 8 Gauss
# points x (7 FP32 values + the FP64 sigma_y cache) = 288, history out 8 x 7 FP32 = 224 (the
# trial cache is not written: it is recomputed from alpha when a step is committed), R 24,
# K 27 blocks x 36 B = 972
ALG_BYTES_PER_EL = 32 + 12 + 24 + 288 + 224 + 24 + 972


def _peaks():
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(x, dist, device):
    """The largest x over the ranks of the process group (x itself on one process): the job's
    time is its slowest rank's.  Any backend (NCCL on GPUs, gloo on the host)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: the units all ranks processed over the (max-over-ranks) time."""
    return world * units_per_rank / seconds


def measured_fp32_tflops(dev, stream, n=8192, reps=10):
    """FP32 throughput of a plain library GEMM on this GPU: cuBLAS SGEMM (C = A B, n^3, TF32
    off, so every product is an FP32 FMA on the CUDA cores), best of reps after 3 warm-ups,
    CUDA events on the launching stream: 2 n^3 / t.  The denominator of the sweep kernel's
    ALU roofline, measured the way the driver measures the bf16 peak."""
    import torch
    mm = torch.backends.cuda.matmul
    old = (getattr(mm, "fp32_precision", None), mm.allow_tf32)
    if old[0] is not None:
        mm.fp32_precision = "ieee"
    mm.allow_tf32 = False
    try:
        with torch.cuda.stream(stream):
            g = torch.Generator(device=dev).manual_seed(0)
            a = torch.randn(n, n, device=dev, generator=g)
            b = torch.randn(n, n, device=dev, generator=g)
            c = torch.empty(n, n, device=dev)
            for _ in range(3):
                torch.matmul(a, b, out=c)
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                torch.matmul(a, b, out=c)
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            del a, b, c
    finally:
        if old[0] is not None:
            mm.fp32_precision = old[0]
        mm.allow_tf32 = old[1]
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def workload(n):
    mesh, bc, mat, _ = inputs.config2_problem(n=n)
    u, hist = inputs.compression_state(mesh, LOAD)
    return mesh, bc, mat, u, hist


def cpu_oracle_rate(mesh, mat, u, hist, target_s=12.0, seed=0):
    """The FP64 oracle (as it stands) on a bounded sample of the same workload: the tangent
    sweep of a seeded random sample of elements plus the assembly of their contributions,
    single-threaded.  Returns (GP/s, description, cores, seconds)."""
    from oracle import element, solver
    hist_el = np.ascontiguousarray(hist.T.reshape(mesh.n_el, 8, 7))
    rng = np.random.default_rng(seed)
    prob = solver.Problem(X=mesh.X, conn=mesh.conn.astype(np.int64), fixed_dof=np.zeros(0, np.int64),
                          fixed_val=np.zeros(0), theta=mat.theta_vector(), hardening=mat.hardening)

    def run(k):
        els = np.sort(rng.choice(mesh.n_el, size=k, replace=False))
        sub = solver.Problem(X=mesh.X, conn=prob.conn[els], fixed_dof=prob.fixed_dof, fixed_val=prob.fixed_val,
                             theta=prob.theta, hardening=prob.hardening)
        t0 = time.perf_counter()
        es = element.element_sweep(mesh.X, sub.conn, u, hist_el[els], sub.theta, sub.hardening)
        solver.assemble_R(sub, es["Re"])
        solver.assemble_K(sub, es["Ke"])
        return time.perf_counter() - t0

    t_probe = run(64)
    k = int(min(mesh.n_el, max(64, 64 * target_s / max(t_probe, 1e-3))))
    dt = run(k)
    return 8 * k / dt, f"oracle tangent sweep + assembly of {k} random elements ({8 * k} Gauss points) of the same state", 1, dt


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def _oracle_worker_init():
    from oracle import element, solver  # noqa: F401  (imported once per worker)


def _oracle_chunk(job):
    """One worker's share of the all-cores CPU baseline: the oracle's tangent sweep and the
    assembly of a chunk of elements in local node numbering; returns its seconds."""
    from oracle import element, solver
    X, conn, u, hist_el, theta, hardening = job
    sub = solver.Problem(X=X, conn=conn, fixed_dof=np.zeros(0, np.int64), fixed_val=np.zeros(0), theta=theta,
                         hardening=hardening)
    t0 = time.perf_counter()
    es = element.element_sweep(X, conn, u, hist_el, theta, hardening)
    solver.assemble_R(sub, es["Re"])
    solver.assemble_K(sub, es["Ke"])
    return time.perf_counter() - t0


def _local_chunk(mesh, u, hist_el, els, theta, hardening):
    nodes, inv = np.unique(mesh.conn[els].ravel(), return_inverse=True)
    return (np.ascontiguousarray(mesh.X[nodes]), inv.reshape(-1, 8).astype(np.int64),
            np.ascontiguousarray(u.reshape(-1, 3)[nodes].ravel()), np.ascontiguousarray(hist_el[els]), theta, hardening)


def cpu_oracle_rate_all_cores(mesh, mat, u, hist, per_worker_s=6.0, seed=0, cores=None):
    """The same oracle sample work spread over the host cores this process may run on: a pool
    of spawned worker processes (one BLAS thread each), each sweeping and assembling an equal
    chunk of seeded random elements sized for about per_worker_s seconds.  The rate is the
    Gauss points of all chunks over the wall time of the timed map (workers already started
    and their imports done).  Returns (GP/s, description, cores, seconds)."""
    import multiprocessing
    if cores is None:   # the permitted cores, at most 64 (the host is shared with other jobs)
        avail = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        cores = max(1, min(64, avail))
    theta, hardening = mat.theta_vector(), mat.hardening
    hist_el = np.ascontiguousarray(hist.T.reshape(mesh.n_el, 8, 7))
    rng = np.random.default_rng(seed)
    probe = np.sort(rng.choice(mesh.n_el, size=min(64, mesh.n_el), replace=False))
    t_probe = _oracle_chunk(_local_chunk(mesh, u, hist_el, probe, theta, hardening))
    k = int(max(8, len(probe) * per_worker_s / max(t_probe, 1e-3)))
    k = min(k, mesh.n_el // cores)
    els = rng.choice(mesh.n_el, size=k * cores, replace=False).reshape(cores, k)
    jobs = [_local_chunk(mesh, u, hist_el, np.sort(e), theta, hardening) for e in els]
    warm = [_local_chunk(mesh, u, hist_el, probe[:2], theta, hardening)] * cores
    # bounded waits: a pool whose workers fail to start keeps replacing them instead of failing
    with multiprocessing.get_context("spawn").Pool(cores, initializer=_oracle_worker_init) as pool:
        pool.map_async(_oracle_chunk, warm, chunksize=1).get(timeout=300)
        t0 = time.perf_counter()
        pool.map_async(_oracle_chunk, jobs, chunksize=1).get(timeout=max(300.0, 20.0 * per_worker_s))
        wall = time.perf_counter() - t0
    desc = (f"oracle tangent sweep + assembly of {k * cores} random elements ({8 * k * cores} Gauss points) of "
            f"the same state, {cores} spawned worker processes with {k} elements each")
    return 8 * k * cores / wall, desc, cores, wall


def _von_mises6(sig):
    """von Mises stress of Cauchy stresses given as 6 components (11, 22, 33, 12, 23, 13)."""
    s11, s22, s33, s12, s23, s13 = (sig[:, k] for k in range(6))
    return np.sqrt(0.5 * ((s11 - s22) ** 2 + (s22 - s33) ** 2 + (s33 - s11) ** 2) + 3.0 * (s12 ** 2 + s23 ** 2 + s13 ** 2))


def config1_forward_section(stream):
    """Config 1's forward (perforated 200 x 100 x 4 plate, Voce, 20 load steps) in FP64 and in
    FP32-mixed on the same inputs, one requested step per hfe_forward call (the handle carries
    its state, its extrapolation history and any reduced increment from call to call), with the
    displacement and the Cauchy stress of every step copied out: wall time and Newton / CG
    counts of each precision, and per step the mixed result's error against the FP64 one,
    max|du| / max|u| and max|dvm| / max vm.  A run that fails reports its error instead of
    ending the benchmark."""
    from paper_2606_17390_b300 import hfe
    m1, bc1, mat1, t1 = inputs.config1_problem()
    out = {"workload": f"config 1: perforated plate 200x100x4 ({m1.n_el} elements, {m1.n_dof} dofs), Voce, "
                       f"{len(t1)} steps; one hfe_forward call per step, u and sigma copied out each step"}
    res = {}
    for prec in ("fp64", "mixed"):
        try:
            us, vms = [], []
            tot = {"newton_iters": 0, "pcg_iters": 0, "substeps": 0, "cutbacks": 0}
            sig = np.empty((8 * m1.n_el, 6))
            with hfe.from_inputs(m1, bc1, mat1, precision=prec, stream=stream.cuda_stream) as s1:
                t0 = time.perf_counter()
                for t in t1:
                    u, st = s1.forward(np.array([t]), sigma_out=sig)
                    us.append(u[0].copy())
                    vms.append(_von_mises6(sig))
                    for k in tot:
                        tot[k] += st[k]
                wall = time.perf_counter() - t0
            res[prec] = (us, vms)
            out[prec] = {"wall_s": wall, **tot}
        except Exception as e:
            out[prec] = {"error": f"{type(e).__name__}: {e}"[:200]}
    if "fp64" in res and "mixed" in res:
        (u64, vm64), (umx, vmmx) = res["fp64"], res["mixed"]
        du = [float(np.abs(a - b).max() / np.abs(b).max()) for a, b in zip(umx, u64)]
        dvm = [float(np.abs(a - b).max() / b.max()) for a, b in zip(vmmx, vm64)]
        out["fp64_over_mixed"] = out["fp64"]["wall_s"] / out["mixed"]["wall_s"]
        out["mixed_vs_fp64"] = {"u_rel_per_step": du, "vm_rel_per_step": dvm, "u_rel_max": max(du),
                                "vm_rel_max": max(dvm), "tolerance": {"u": 1e-5, "vm": 1e-4},
                                "within_tolerance": bool(max(du) <= 1e-5 and max(dvm) <= 1e-4)}
    return out


def config3_fd_section(stream, h=1e-6):
    """Config 3's gradient check at full size (200 x 100 x 4 plate, Swift, 20 steps, the nine
    uniform parameters at the seeded +-20 % point, target = FP64 forward at the true
    parameters + N(0, (1e-3 max|u|)^2)): the adjoint gradient (FP64 handle, and the default
    mixed handle with the FP64 refinement) against central differences of J with a relative
    step h per parameter, each J from an FP64 forward solve (Newton 1e-12) that starts every
    load step from the pass at the evaluation point (warm start).  Compared as
    theta_i dJ/dtheta_i."""
    from paper_2606_17390_b300 import hfe
    m3, bc3, mat3, t3 = inputs.config3_problem()
    th_true = mat3.theta_vector()
    th = inputs.perturbed_theta(th_true)
    idx = np.arange(2, 11)
    fp64 = dict(newton_rtol=1e-12, pcg_rtol=1e-13)
    t0 = time.perf_counter()
    with hfe.from_inputs(m3, bc3, mat3, precision="fp64", theta=th_true, stream=stream.cuda_stream, **fp64) as s:
        u_true, _ = s.forward(t3)
    u_gt = u_true + inputs.noise(u_true.shape, 1e-3 * np.abs(u_true).max())
    out = {"workload": f"config 3: perforated plate 200x100x4 ({m3.n_el} elements, {m3.n_dof} dofs), Swift, "
                       f"{len(t3)} steps, 9 parameters (F, G, H, L, M, N, K, eps0, n)", "relative_step": h}
    grads = {}
    for prec, opts in (("fp64", fp64), ("mixed", {})):
        with hfe.from_inputs(m3, bc3, mat3, precision=prec, theta=th, stream=stream.cuda_stream, **opts) as s:
            J, g, _ = s.adjoint(t3, u_gt)
        grads[prec] = th[idx] * g[0][idx]
        out[f"J_{prec}"] = J
    d_fd = np.empty(idx.size)
    with hfe.from_inputs(m3, bc3, mat3, precision="fp64", theta=th, stream=stream.cuda_stream, **fp64) as s:
        s.set_warm_start("record")
        s.forward(t3, want_u=False)
        s.set_warm_start("use")
        for k, i in enumerate(idx):
            Jpm = []
            for sgn in (1.0, -1.0):
                tp = th.copy()
                tp[i] *= 1.0 + sgn * h
                s.set_material(tp, mat3.Theta)
                s.set_state(None, None)
                u, _ = s.forward(t3)
                Jpm.append(float(np.sum((u - u_gt) ** 2)))
            d_fd[k] = (Jpm[0] - Jpm[1]) / (2.0 * h)
        s.set_warm_start("off")
    names = ["F", "G", "H", "L", "M", "N", "K", "eps0", "n"]
    out["theta_dJ_dtheta_fd"] = dict(zip(names, d_fd.tolist()))
    for prec, d in grads.items():
        out[f"theta_dJ_dtheta_{prec}"] = dict(zip(names, d.tolist()))
        out[f"{prec}_vs_fd_rel_norm"] = float(np.linalg.norm(d - d_fd) / np.linalg.norm(d_fd))
        out[f"{prec}_vs_fd_rel_per_parameter"] = dict(zip(names, (np.abs(d - d_fd) / np.abs(d_fd)).tolist()))
    out["mixed_vs_fp64_rel_norm"] = float(np.linalg.norm(grads["mixed"] - grads["fp64"]) / np.linalg.norm(grads["fp64"]))
    out["wall_s"] = time.perf_counter() - t0
    return out


def directional_fd_check(mesh, bc, mat, ts, theta, grad, u_gt, stream, h=1e-6, seed=41):
    """The adjoint gradient along a seeded direction against central differences of J: v with
    entries U(-1, 1) on the nine identified parameters, theta(s) = theta * (1 + s v), and
    dJ/ds = sum_i grad_i theta_i v_i against (J(h) - J(-h)) / 2h, each J from an FP64 forward
    (Newton 1e-12) that starts every load step from a recorded pass at theta (warm start)."""
    from paper_2606_17390_b300 import hfe
    idx = np.arange(2, 11)
    v = np.zeros_like(theta)
    v[idx] = np.random.default_rng(seed).uniform(-1.0, 1.0, idx.size)
    d_adj = float(np.sum(grad * theta * v))
    t0 = time.perf_counter()
    Js = []
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=theta, stream=stream.cuda_stream,
                         newton_rtol=1e-12, pcg_rtol=1e-13) as s:
        s.set_warm_start("record")
        s.forward(ts, want_u=False)
        s.set_warm_start("use")
        for sgn in (1.0, -1.0):
            s.set_material(theta * (1.0 + sgn * h * v), mat.Theta)
            s.set_state(None, None)
            u, _ = s.forward(ts)
            Js.append(float(np.sum((u - u_gt) ** 2)))
        s.set_warm_start("off")
    d_fd = (Js[0] - Js[1]) / (2.0 * h)
    return {"direction": f"theta_i (1 + s v_i), v_i ~ U(-1, 1) on the 9 parameters (seed {seed})",
            "relative_step": h, "dJ_ds_adjoint": d_adj, "dJ_ds_central_difference": d_fd,
            "relative_error": abs(d_adj - d_fd) / abs(d_fd), "seconds": time.perf_counter() - t0,
            "forward": "FP64, Newton 1e-12, warm-started from a pass at the evaluation point"}


def inverse_section(nx, stream, maxfun=90):
    """The inverse loop on config 3 (Sec. 3.3 normalisation rho in [-1, 1], L-BFGS-B with the
    paper's stopping criteria, warm start under the 10 % rule): nine parameters from the seeded
    +-20 % start, bounds theta_true x [0.5, 1.5], noisy target from the mixed forward at the true
    parameters; w scales J at the start to 1e3 (so that the relative stopping tests act).
    Reports the recovered parameters against the true ones, iterations, evaluations and the
    time per evaluation (one gradient call each)."""
    from paper_2606_17390_b300 import hfe, inverse
    m3, bc3, mat3, t3 = inputs.config3_problem(nx, nx // 2, 4 if nx >= 200 else 2)
    th_true = mat3.theta_vector()
    th0 = inputs.perturbed_theta(th_true)
    idx = np.arange(2, 11)
    tmin, tref = 0.5 * th_true[idx], th_true[idx]
    with hfe.from_inputs(m3, bc3, mat3, precision="mixed", theta=th_true, stream=stream.cuda_stream) as s:
        u_true, _ = s.forward(t3)
    u_gt = u_true + inputs.noise(u_true.shape, 1e-3 * np.abs(u_true).max())
    with hfe.from_inputs(m3, bc3, mat3, precision="mixed", theta=th0, stream=stream.cuda_stream) as s:
        J0, _, _ = s.adjoint(t3, u_gt)
        w = 1e3 / J0
        res = inverse.identify(s, t3, u_gt, th0, idx, tmin, tref, w=w, criteria=dict(maxfun=maxfun),
                               warm_start=True)
    names = ["F", "G", "H", "L", "M", "N", "K", "eps0", "n"]
    rel = (res.theta[idx] - th_true[idx]) / th_true[idx]
    rel0 = (th0[idx] - th_true[idx]) / th_true[idx]
    return {"workload": f"config 3: perforated plate {nx}x{nx // 2} ({m3.n_el} elements, {m3.n_dof} dofs), "
                        f"{len(t3)} steps, 9 parameters, mixed forward with FP64 refinement, warm start",
            "w": w, "J_start": float(res.history[0][0]), "J_end": res.J, "iterations": res.iterations,
            "evaluations": res.evaluations, "warm_passes": res.warm_passes, "success": res.success,
            "message": res.message, "seconds": res.seconds, "seconds_per_evaluation": res.seconds / max(1, res.evaluations),
            "theta_true": dict(zip(names, th_true[idx].tolist())),
            "theta_start": dict(zip(names, th0[idx].tolist())),
            "theta_recovered": dict(zip(names, res.theta[idx].tolist())),
            "relative_error_start": dict(zip(names, rel0.tolist())),
            "relative_error_recovered": dict(zip(names, rel.tolist()))}


def barlat_map_section(reps, stream, dev, with_cpu):
    """Device time of hfe_barlat_return_map on the App. B robustness map and on a 64-times
    larger batch (CUDA events on the launching stream, after 3 warm-up launches), outcome
    counts, and the oracle's rate on a bounded sample of the same map."""
    import torch
    from paper_2606_17390_b300 import hfe
    mat = inputs.barlat_verification_material()
    n = 16000
    angle, scale = inputs.pi_plane_sample(n)
    with torch.cuda.stream(stream):
        d = torch.from_numpy(inputs.principal_plane_directions(angle)).to(dev)
        phi = hfe.barlat_phi(mat, d, stream=stream.cuda_stream)
        Tt = (torch.from_numpy(scale).to(dev)[:, None] / phi[:, None]) * d
        a0 = torch.zeros(n, dtype=torch.float64, device=dev)
        big_T, big_a = Tt.repeat(64, 1).contiguous(), a0.repeat(64).contiguous()

    def run(T, a, reps_, **kw):
        with torch.cuda.stream(stream):
            out = hfe.barlat_return_map(mat, T, a, stream=stream.cuda_stream, **kw)
            for _ in range(3):
                hfe.barlat_return_map(mat, T, a, stream=stream.cuda_stream, out=out, **kw)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps_):
                hfe.barlat_return_map(mat, T, a, stream=stream.cuda_stream, out=out, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps_
        st = out["status"].cpu().numpy()
        it = out["iters"].cpu().numpy()
        conv = st == 0
        return {"ms": ms, "points_per_s": T.shape[0] / (ms * 1e-3), "converged": int(conv.sum()),
                "at_kmax": int((st == 2).sum()), "other": int((~conv & (st != 2)).sum()),
                "mean_iters_converged": float(it[conv].mean()) if conv.any() else None,
                "launches": 2 if kw.get("precision") == "mixed" else 1}

    sec = {"workload": "line-search robustness map: 16,000 seeded pi-plane trial states between the yield surface "
                       "and 30 times it; Yld2004-18p verification parameters (m = 8, E = 1000, nu = 0.3, "
                       "sigma0 = 1, perfect plasticity); k_max 40, beta 1e-4, eta 0.1, tol 1e-13; inputs are "
                       "0.8 MB (compute-bound, L2 irrelevant)"}
    for prec in ("mixed", "fp64"):
        for ls in (True, False):
            sec[f"{prec}_{'line_search' if ls else 'newton'}"] = run(Tt, a0, reps, precision=prec, line_search=ls)
        sec[f"{prec}_line_search_1M"] = run(big_T, big_a, max(2, reps // 10), precision=prec, line_search=True)
    if with_cpu:
        from oracle import barlat as BA
        model = BA.Barlat(mat.c1, mat.c2, mat.m)
        dd = inputs.principal_plane_directions(angle)
        To = (scale / model.phi_poly(dd))[:, None] * dd
        t0 = time.perf_counter()
        _, _, conv_o = BA.cpp(model, mat.E, mat.nu, mat.hardening, mat.h, To, np.zeros(n), kmax=40)
        dt = time.perf_counter() - t0
        sec["cpu_baseline"] = {"points_per_s": n / dt, "cores": 1, "kind": "oracle", "seconds": dt,
                               "converged": int(conv_o.sum()),
                               "sample": "the oracle's closest-point projection with the line search on the whole "
                                         "16,000-point map (FP64 numpy, vectorised over the points, 1 thread)"}
        k = n
        sec["mixed_over_oracle"] = sec["mixed_line_search"]["points_per_s"] / (k / dt)
        sec["fp64_over_oracle"] = sec["fp64_line_search"]["points_per_s"] / (k / dt)
    return sec


def barlat_fe_section(n, stream, dev, reps=5):
    """Device time per FP64 tangent sweep of an n^3 cube at the compression state, with the
    paper's Yld2004-18p coefficients (rotated 30 degrees about z, config 0's elasticity and
    Swift hardening; the local projection with the FP32 iteration and FP64 finish, or all
    FP64), and with the Hill-48 material of the same configuration."""
    import torch
    from paper_2606_17390_b300 import hfe
    mesh, bc, mat, _ = inputs.config2_problem(n=n)
    u, hist = inputs.compression_state(mesh, LOAD)
    bm = inputs.barlat_verification_material()
    th = mat.theta_vector()
    bm.E, bm.nu, bm.hardening, bm.h = th[0], th[1], "swift", (th[8], th[9], th[10])
    a = np.deg2rad(30.0)
    bm.Theta = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    out = {"workload": f"hex8 cube {n}^3 ({mesh.n_el} elements, {8 * mesh.n_el} Gauss points), clamped-platen "
                       "compression mid-step state, tangent sweep (FP64 and mixed handles); Yld2004-18p (m = 8) "
                       "vs Hill-48"}
    cases = {"barlat_mixed_projection": ("fp64", "mixed"), "barlat_fp64_projection": ("fp64", "fp64"),
             "hill": ("fp64", None), "barlat_mixed_handle": ("mixed", "mixed"), "hill_mixed_handle": ("mixed", None)}
    for name, (handle, projection) in cases.items():
        with torch.cuda.stream(stream):
            s = hfe.from_inputs(mesh, bc, mat, precision=handle, stream=stream.cuda_stream)
            if projection is not None:
                s.set_barlat(bm, precision=projection)
            s.set_state(u, hist)
            u_d = torch.from_numpy(u).to(dev)
            R_d = torch.empty(mesh.n_dof, dtype=torch.float64, device=dev)
            _, _, st = s.sweep(u_d, LOAD, tangent=True, R_out=R_d, stats=True)
            for _ in range(2):
                s.sweep(u_d, LOAD, tangent=True, R_out=R_d, stats=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                s.sweep(u_d, LOAD, tangent=True, R_out=R_d, stats=False)
            e1.record(stream)
            torch.cuda.synchronize()
            s.close()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_sweep": ms, "gp_per_s": 8 * mesh.n_el / (ms * 1e-3), "plastic_gps": st["plastic_gps"]}
    out["barlat_over_hill"] = out["barlat_mixed_projection"]["ms_per_sweep"] / out["hill"]["ms_per_sweep"]
    out["barlat_over_hill_mixed_handle"] = (out["barlat_mixed_handle"]["ms_per_sweep"] /
                                            out["hill_mixed_handle"]["ms_per_sweep"])
    return out


def reference_arm(args, rank):
    """The oracle timed as it stands: each step is a bounded sample (a seeded random set of
    elements of the same state, about ref_step_s seconds of CPU work); ms_per_step is the
    measured time of one such sample, value the Gauss points of the samples over their time."""
    if rank != 0:
        return
    mesh, bc, mat, u, hist = workload(args.n)
    gps, times = [], []
    for i in range(args.warmup + args.steps):
        r, desc, cores, dt = cpu_oracle_rate(mesh, mat, u, hist, target_s=args.ref_step_s, seed=i)
        if i >= args.warmup:
            gps.append(r * dt)
            times.append(dt)
    value = float(np.sum(gps) / np.sum(times))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "step": "one bounded sample of the workload (see cpu_baseline.sample), timed as measured",
            "full_workload_ms_extrapolated": 1e3 * 8 * mesh.n_el / value,
            "extrapolated": "full_workload_ms_extrapolated scales the measured rate to all "
                            f"{8 * mesh.n_el} Gauss points; it was not run",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"hex8 cube {args.n}^3, {mesh.n_dof} dofs, {8 * mesh.n_el} Gauss points, "
                                   "Hill-48 + Swift, clamped compression, mid-step state; CPU oracle on a sample",
                       "n_el": mesh.n_el, "n_dof": mesh.n_dof, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", "--cube-n", dest="n", type=int, default=100,
                    help="cube edge in elements (100 = 3.09M dofs); --cube-n is the same option under "
                         "torch.distributed.run, whose own options make --n ambiguous")
    ap.add_argument("--fp64-steps", type=int, default=5, help="steps of the FP64 comparison (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pcg-iters", type=int, default=200, help="PCG iterations timed for context (0 = skip)")
    ap.add_argument("--adjoint-nx", type=int, default=200, help="plate resolution of the adjoint ratio run (0 = skip)")
    ap.add_argument("--adjoint-steps", type=int, default=20)
    ap.add_argument("--warm-delta", type=float, default=0.01,
                    help="relative parameter change of the warm-start forward comparison (0 = skip)")
    ap.add_argument("--fbar-steps", type=int, default=20, help="timed F-bar tangent sweeps (0 = skip)")
    ap.add_argument("--adjoint-config", type=int, default=3, choices=(3, 4),
                    help="3: nine uniform parameters on the 200x100x4 plate; 4: per-element fields (use --adjoint-nx 400)")
    ap.add_argument("--forward-n", type=int, default=100, help="cube size of the end-to-end forward run (0 = skip)")
    ap.add_argument("--forward-steps", type=int, default=10)
    ap.add_argument("--assembly-l2-mb", type=float, default=-1.0,
                    help="K bytes (MB) of a slab of the sweep's launch order (-1: the library default, "
                         "3/4 of L2; 0: colour order)")
    ap.add_argument("--no-gradient-check", dest="gradient_check", action="store_false",
                    help="skip the directional central-difference check of the config-3 gradient")
    ap.add_argument("--config3-fd", action="store_true",
                    help="config 3's full-size gradient against FP64 central differences (18 forward solves)")
    ap.add_argument("--inverse-nx", type=int, default=0,
                    help="plate resolution of the config-3 inverse loop (0 = skip; 200 = config 3)")
    ap.add_argument("--inverse-maxfun", type=int, default=90)
    ap.add_argument("--no-config1-forward", dest="config1_forward", action="store_false",
                    help="skip config 1's full-size forward in FP64 and FP32-mixed (per-step errors)")
    ap.add_argument("--forward-predictors", default="2",
                    help="comma-separated options.predictor values of the forward run (first one reported); "
                         "0 restarts each step from the previous displacement, which inverts the elements "
                         "next to a platen at this size and is left to cutbacks (very slow)")
    ap.add_argument("--ref-step-s", type=float, default=6.0, help="CPU seconds per reference-arm step")
    ap.add_argument("--barlat-reps", type=int, default=20,
                    help="timed launches of the Barlat line-search map (0 = skip)")
    ap.add_argument("--barlat-fe-n", type=int, default=40,
                    help="cube edge of the FP64 Barlat tangent sweep timed against Hill-48 (0 = skip)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch
    from paper_2606_17390_b300 import hfe
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    mesh, bc, mat, u, hist = workload(args.n)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    def make(precision, **opts):
        if args.assembly_l2_mb >= 0:
            opts.setdefault("assembly_l2_bytes", int(args.assembly_l2_mb * 2 ** 20))
        s = hfe.from_inputs(mesh, bc, mat, precision=precision, stream=stream.cuda_stream, **opts)
        s.set_state(u, hist)
        return s

    solver = make(args.precision)
    info = solver.info()
    hist_mb = (64 if args.precision == "fp64" else 36) * 8 * mesh.n_el / 1e6
    k_mb = (72 if args.precision == "fp64" else 36) * info["n_blocks"] / 1e6
    u_d = torch.from_numpy(u).to(dev)
    R_d = torch.empty(mesh.n_dof, dtype=torch.float64, device=dev)
    rn_d = torch.empty(1, dtype=torch.float64, device=dev)

    def step(s):
        s.sweep(u_d, LOAD, tangent=True, R_out=R_d, rnorm_out=rn_d, stats=False)

    # correctness / status of the workload before timing
    _, _, st0 = solver.sweep(u_d, LOAD, tangent=True, R_out=R_d, rnorm_out=rn_d, stats=True)
    for _ in range(args.warmup):
        step(solver)
    torch.cuda.synchronize()

    def timed(s, k):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            step(s)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        if dist is not None:
            dist.barrier()
        return ms

    with ClockSampler(local) as clk:
        ms_total = timed(solver, args.steps)
    ms_step = ms_total / args.steps
    value = whole_job_rate(world, 8 * mesh.n_el, ms_step * 1e-3)

    # the same sweep without the tangent and assembly (residual and history only), for context
    def step_res(s):
        s.sweep(u_d, LOAD, tangent=False, R_out=R_d, rnorm_out=rn_d, stats=False)
    step_res(solver)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_res = max(3, args.steps // 4)
    e0.record(stream)
    for _ in range(k_res):
        step_res(solver)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_res = e0.elapsed_time(e1) / k_res

    # per-launch device time of the dominant kernel (gp_sweep, one launch per colour),
    # CUDA events on the library's launching stream (hfe_stats.sweep_ms)
    sweep_ms = []
    for _ in range(5):
        _, _, st = solver.sweep(u_d, LOAD, tangent=True, R_out=R_d, rnorm_out=rn_d, stats=True)
        sweep_ms.append(st["sweep_ms"])
    sweep_ms_avg = float(np.mean(sweep_ms))
    launch_ms = sweep_ms_avg / info["n_launches"]
    el_per_launch = mesh.n_el / info["n_launches"]
    flops_launch = ALG_FLOPS_PER_GP * 8 * el_per_launch
    peak_derived = 148 * 128 * 2 * 2.032e9 / 1e12      # FP32 FMA lanes x 2 flop x max SM clock
    peak_fp32 = measured_fp32_tflops(dev, stream)
    roofline = {"bound": "alu", "achieved": flops_launch / (launch_ms * 1e-3) / 1e12, "peak": peak_fp32,
                "unit": "TFLOP/s", "frac": None, "traffic": None,
                "kernel": "gp_sweep_kernel<float,true>", "launch_ms": launch_ms,
                "alg_flops_per_launch": flops_launch, "alg_bytes_per_launch": ALG_BYTES_PER_EL * el_per_launch,
                "hbm_frac_of_measured": None,
                "peak_source": "measured in this run: cuBLAS FP32 SGEMM 8192^3, TF32 off, best of 10",
                "peak_derived": peak_derived, "frac_of_derived": None,
                "derived_source": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz"}
    roofline["frac"] = roofline["achieved"] / peak_fp32
    roofline["frac_of_derived"] = roofline["achieved"] / peak_derived
    peaks, src = _peaks()
    roofline["hbm_frac_of_measured"] = ALG_BYTES_PER_EL * el_per_launch / (launch_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
    traffic_file = os.path.join(HERE, "profiles", "gp_sweep_traffic.json")
    if os.path.exists(traffic_file):
        with open(traffic_file) as f:
            tr = json.load(f)
        if (tr.get("precision") == args.precision and tr.get("n") == args.n
                and tr.get("n_launches") == info["n_launches"]):
            roofline["traffic"] = tr.get("dram_bytes_per_launch")

    # end to end through the C ABI with host buffers (pinned): u in, R and |R_free| out
    u_h = torch.from_numpy(u).pin_memory()
    R_h = torch.empty(mesh.n_dof, dtype=torch.float64).pin_memory()
    rn_h = torch.empty(1, dtype=torch.float64).pin_memory()
    k_e2e = max(3, args.steps // 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        solver.sweep(u_h, LOAD, tangent=True, R_out=R_h, rnorm_out=rn_h, stats=False)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / k_e2e, dist, dev)
    e2e = {"value": whole_job_rate(world, 8 * mesh.n_el, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 8 * mesh.n_dof,
           "d2h_bytes_per_step": 8 * mesh.n_dof + 8, "ms_per_step": 1e3 * e2e_s}

    # the linear solve of the Newton step on the same mesh: block-Jacobi PCG with the BSR SpMV
    # (elastic tangent at u = 0, fixed iteration count), for context
    pcg = None
    if args.pcg_iters > 0:
        s_pcg = hfe.from_inputs(mesh, bc, mat, precision=args.precision, stream=stream.cuda_stream,
                                pcg_maxit=args.pcg_iters, pcg_rtol=1e-30, pcg_check_every=args.pcg_iters)
        s_pcg.sweep(np.zeros(mesh.n_dof), 0.0, tangent=True)
        free = np.ones(mesh.n_dof)
        free[bc.dof] = 0.0
        b = torch.from_numpy(free).to(dev)
        try:
            s_pcg.solve(b)
        except hfe.HfeError:
            pass                       # the iteration cap is the point: time per iteration
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            s_pcg.solve(b)
        except hfe.HfeError:
            pass
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        n_blocks = info["n_blocks"]
        bytes_spmv = n_blocks * (9 * (4 if args.precision == "mixed" else 8) + 4)
        pcg = {"iters": args.pcg_iters, "ms_per_iter": ms / args.pcg_iters,
               "spmv_alg_bytes": bytes_spmv}
        s_pcg.close()

    # FP64 form of the same sweep (the comparison the metric names)
    fp64 = None
    if args.fp64_steps > 0 and args.precision == "mixed":
        solver.close()
        s64 = make("fp64")
        step(s64)
        ms64 = timed(s64, args.fp64_steps) / args.fp64_steps
        fp64 = {"value": world * 8 * mesh.n_el / (ms64 * 1e-3), "ms_per_step": ms64, "steps": args.fp64_steps,
                "mixed_speedup": ms64 / ms_step}
        s64.close()
    else:
        solver.close()

    # the F-bar element's tangent sweep on the same state (option fbar, non-symmetric K), for context
    fbar = None
    if args.fbar_steps > 0:
        sfb = make(args.precision, fbar=1)
        step(sfb)
        msfb = timed(sfb, args.fbar_steps) / args.fbar_steps
        fbar = {"value": world * 8 * mesh.n_el / (msfb * 1e-3), "ms_per_step": msfb, "steps": args.fbar_steps,
                "over_standard": msfb / ms_step}
        sfb.close()

    # adjoint/forward time ratio (second part of the metric) on the config-3 problem: perforated
    # plate, Swift parameters perturbed by +-20 %, noisy synthetic target; the gradient call runs
    # its own forward pass (mixed, each step ending with an FP64 Newton iteration) and the FP64
    # reverse sweep
    adjoint = None
    if args.adjoint_nx > 0:
        nx = args.adjoint_nx
        if args.adjoint_config == 4:
            # per-element F, G, H, sigma0 fields (config 4); the gradient is taken at the
            # spatially uniform mean parameters, the start of an inverse run
            m3, bc3, mat3, th_true, t3 = inputs.config4_problem(nx, nx // 2, 4 if nx >= 200 else 2,
                                                                args.adjoint_steps)
            th_eval = np.tile(mat3.theta_vector(), (m3.n_el, 1))
            what = "per-element F, G, H, sigma0 (4 x n_el parameters), Voce"
        else:
            m3, bc3, mat3, t3 = inputs.config3_problem(nx, nx // 2, 4 if nx >= 200 else 2, args.adjoint_steps)
            th_true = mat3.theta_vector()
            th_eval = inputs.perturbed_theta(th_true)
            what = "9 Swift/Hill parameters"
        with hfe.from_inputs(m3, bc3, mat3, precision="mixed", theta=th_true, stream=stream.cuda_stream) as s3:
            u_true, _ = s3.forward(t3)
        u_gt = u_true + inputs.noise(u_true.shape, 1e-3 * np.abs(u_true).max())
        warm = None
        with hfe.from_inputs(m3, bc3, mat3, precision="mixed", theta=th_eval, stream=stream.cuda_stream) as s3:
            s3.set_state(None, None)
            if args.warm_delta > 0:
                s3.set_warm_start("record")   # this pass is the record of the warm-start run below
            t0 = time.perf_counter()
            _, fst = s3.forward(t3, want_u=False)
            t_fwd = time.perf_counter() - t0
            t0 = time.perf_counter()
            J3, g3, ast = s3.adjoint(t3, u_gt)
            t_adj = time.perf_counter() - t0
            gcheck = None
            if args.adjoint_config == 3 and args.gradient_check:
                try:
                    gcheck = directional_fd_check(m3, bc3, mat3, t3, th_eval, g3[0], u_gt, stream)
                except Exception as e:   # reported in the line instead of ending the benchmark
                    gcheck = {"error": f"{type(e).__name__}: {e}"[:200]}
            if args.warm_delta > 0:
                # warm start (Sec. 3.6): the next evaluation of an inverse loop, parameters moved
                # by up to warm_delta (relative, seeded), forward from the record vs cold
                rng = np.random.default_rng(31)
                th_next = th_eval * (1 + args.warm_delta * rng.uniform(-1, 1, th_eval.shape))
                s3.set_material(th_next, s3.Theta_axes)
                s3.set_warm_start("use")
                s3.set_state(None, None)
                t0 = time.perf_counter()
                _, wst = s3.forward(t3, want_u=False)
                t_warm = time.perf_counter() - t0
                s3.set_warm_start("off")
                s3.set_state(None, None)
                t0 = time.perf_counter()
                _, cst = s3.forward(t3, want_u=False)
                t_cold = time.perf_counter() - t0
                warm = {"parameter_change": f"every parameter x (1 + {args.warm_delta} U(-1, 1)), seed 31",
                        "cold_forward_s": t_cold, "warm_forward_s": t_warm, "speedup": t_cold / t_warm,
                        "cold_newton_iters": cst["newton_iters"], "warm_newton_iters": wst["newton_iters"],
                        "cold_pcg_iters": cst["pcg_iters"], "warm_pcg_iters": wst["pcg_iters"],
                        "warm_steps": wst["warm_steps"], "warm_retries": wst["warm_retries"],
                        "cold_substeps": cst["substeps"], "warm_substeps": wst["substeps"]}
        adjoint = {"workload": f"config {args.adjoint_config}: perforated plate {nx}x{nx // 2} ({m3.n_el} elements, "
                               f"{m3.n_dof} dofs), {args.adjoint_steps} steps, {what}",
                   "forward_s": t_fwd, "gradient_call_s": t_adj, "reverse_s": ast["solve_ms"] * 1e-3,
                   "gradient_forward_pass_s": ast["sweep_ms"] * 1e-3,
                   "gradient_pcg_iters": {"forward_newton": ast["pcg_iters"] - ast["refine_pcg_iters"]
                                          - ast["reverse_pcg_iters"], "fp64_refinement": ast["refine_pcg_iters"],
                                          "reverse": ast["reverse_pcg_iters"]},
                   "gradient_over_forward": t_adj / t_fwd, "reverse_over_forward": ast["solve_ms"] * 1e-3 / t_fwd,
                   "forward_newton_iters": fst["newton_iters"], "forward_pcg_iters": fst["pcg_iters"],
                   "forward_substeps": fst["substeps"], "gradient_substeps": ast["substeps"],
                   "warm_start": warm, "gradient_check": gcheck}

    # end-to-end forward solve of the 100^3 clamped-platen compression (10 load steps, mixed):
    # Newton, PCG and substep counts, and the in-solve Gauss-point update rate
    forward = None
    if args.forward_n > 0:
        m2, bc2, mat2, t2 = inputs.config2_problem(args.forward_n, args.forward_steps)
        names = {0: "previous", 1: "tangent", 2: "linear_extrapolation", 3: "quadratic_extrapolation"}
        runs = {}
        for pm in [int(x) for x in args.forward_predictors.split(",")]:
            with hfe.from_inputs(m2, bc2, mat2, precision=args.precision, stream=stream.cuda_stream,
                                 predictor=pm) as s2:
                t0 = time.perf_counter()
                _, st2 = s2.forward(t2, want_u=False)
                wall = time.perf_counter() - t0
            print(f"forward {args.forward_n}^3, predictor {pm}: {wall:.1f} s, {st2['newton_iters']} Newton, "
                  f"{st2['pcg_iters']} PCG, {st2['substeps']} substeps", file=sys.stderr, flush=True)
            runs[names[pm]] = {"wall_s": wall, "newton_iters": st2["newton_iters"], "pcg_iters": st2["pcg_iters"],
                               "substeps": st2["substeps"], "cutbacks": st2["cutbacks"], "sweeps": st2["sweeps"],
                               "sweep_s": st2["sweep_ms"] * 1e-3, "solve_s": st2["solve_ms"] * 1e-3,
                               "in_solve_gp_per_s": st2["sweeps"] * 8 * m2.n_el / (st2["sweep_ms"] * 1e-3)}
        first = next(iter(runs.values()))
        forward = {"workload": f"hex8 cube {args.forward_n}^3 ({m2.n_dof} dofs), 10 % compression between clamped "
                               f"platens, {args.forward_steps} load steps, {args.precision}", **first}
        if len(runs) > 1:
            forward["predictors"] = runs

    # Barlat Yld2004-18p material points: the line-search robustness map (16,000 pi-plane trial
    # states between the yield surface and 30 times it, the verification parameters, perfect
    # plasticity, k_max 40), with and without the line search, FP64 and mixed, plus a
    # 1,024,000-point batch (the map 64 times) for throughput; the oracle on a bounded sample
    barlat = None
    if args.barlat_reps > 0:
        barlat = barlat_map_section(args.barlat_reps, stream, dev, rank == 0 and not args.no_cpu_baseline)

    # the Barlat model in the hex8 path (FP64): tangent sweeps of an n^3 cube at the
    # compression state (strain pass, Gauss-point update, assembly pass) against the FP64
    # Hill-48 sweep of the same state
    barlat_fe = None
    if args.barlat_fe_n > 0:
        barlat_fe = barlat_fe_section(args.barlat_fe_n, stream, dev)

    config1 = config1_forward_section(stream) if args.config1_forward else None
    config3_fd = inverse_run = None
    if args.config3_fd:
        try:
            config3_fd = config3_fd_section(stream)
        except Exception as e:   # reported in the line instead of ending the benchmark
            config3_fd = {"error": f"{type(e).__name__}: {e}"[:200]}
    if args.inverse_nx > 0:
        try:
            inverse_run = inverse_section(args.inverse_nx, stream, args.inverse_maxfun)
        except Exception as e:
            inverse_run = {"error": f"{type(e).__name__}: {e}"[:200]}

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu_baseline:
        r, desc, cores, dt = cpu_oracle_rate(mesh, mat, u, hist)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc, "seconds": dt,
               "cpu_model": cpu_model()}
        try:
            r, desc, cores, dt = cpu_oracle_rate_all_cores(mesh, mat, u, hist)
            cpu_all = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc, "seconds": dt,
                       "cpu_model": cpu_model()}
        except Exception as e:  # the single-thread baseline above stands on its own
            cpu_all = {"unavailable": f"{type(e).__name__}: {e}"[:200]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": f"hex8 cube {args.n}^3 ({mesh.n_dof} dofs, {8 * mesh.n_el} Gauss points), "
                                       "Hill-48 + Swift, clamped-platen compression, mid-step state, tangent sweep "
                                       "+ assembly + residual norm",
                           "n_el": mesh.n_el, "n_dof": mesh.n_dof, "n_blocks": info["n_blocks"],
                           "precision": args.precision,
                           "l2": f"inputs larger than L2 (history {hist_mb:.0f} MB, K {k_mb:.0f} MB)",
                           "launch_order": f"{info['n_slabs']} slabs of K rows x {info['n_colors']} colours = "
                                           f"{info['n_launches']} launches per sweep",
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "fp64": fp64,
                "residual_sweep": {"ms_per_step": ms_res, "value": world * 8 * mesh.n_el / (ms_res * 1e-3)},
                "pcg": pcg, "adjoint": adjoint, "forward": forward, "config1_forward": config1, "config3_gradient_fd": config3_fd,
                "inverse": inverse_run, "fbar_sweep": fbar,
                "barlat_map": barlat, "barlat_fe_sweep": barlat_fe,
                "gpu_launches": (info["n_launches"] + 1) * args.steps,
                "clocks": clk.summary(), "peaks_source": src,
                "plastic_gps": st0["plastic_gps"], "max_local_iters": st0["max_local_iters"]}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
