"""Host logic of bench.py on several processes (CPU, gloo): the job's time is the max over
the ranks and the whole-job rate counts every rank's units; under torch.distributed.run the
reference arm runs and prints on rank 0 only.  The GPU path itself runs replicas only: every
rank's sweep is independent, there is no collective on the data path."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")   # ranks take 10 and 15 ms
        out[rank] = (ms, bench.whole_job_rate(world, 1000, ms * 1e-3))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, rate = out[0]
    assert ms == 15.0                                  # the slowest rank
    assert rate == pytest.approx(2 * 1000 / 0.015)     # all ranks' units over the job time


def test_reference_arm_prints_on_rank_zero_only():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-step-s", "0.2",
           "--cube-n", "4"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0


def test_all_cores_cpu_baseline_spawned_pool():
    """The all-cores CPU baseline: a spawned pool of 2 workers sweeps equal chunks of random
    elements of the bench state (local node numbering) with the oracle, and one worker's
    chunk gives the same element results as the oracle on the global mesh."""
    import bench
    from oracle import element
    mesh, _, mat, u, hist = bench.workload(6)
    r, desc, cores, dt = bench.cpu_oracle_rate_all_cores(mesh, mat, u, hist, per_worker_s=0.2, cores=2)
    assert cores == 2 and r > 0 and dt > 0 and "2 spawned worker processes" in desc
    hist_el = np.ascontiguousarray(hist.T.reshape(mesh.n_el, 8, 7))
    els = np.array([3, 17, 40, 101])
    X, conn, uu, h, th, hard = bench._local_chunk(mesh, u, hist_el, els, mat.theta_vector(), mat.hardening)
    loc = element.element_sweep(X, conn, uu, h, th, hard)
    glo = element.element_sweep(mesh.X, mesh.conn[els].astype(np.int64), u, hist_el[els], th, hard)
    assert np.array_equal(loc["Re"], glo["Re"]) and np.array_equal(loc["Ke"], glo["Ke"])
