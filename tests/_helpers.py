"""Shared helpers of the GPU parity tests (state construction and format conversions)."""
import numpy as np
import scipy.sparse as sp

from paper_2606_17390_b300 import inputs


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def bsr_to_csr(rowptr, cols, vals, n_nodes):
    return sp.bsr_matrix((vals, cols, rowptr), shape=(3 * n_nodes, 3 * n_nodes)).tocsr()


def hist_oracle_to_soa(h):
    """(n_el, 8, 7) -> [7][n_gp]"""
    return np.ascontiguousarray(h.reshape(-1, 7).T)


def hist_soa_to_oracle(h, n_el):
    return np.ascontiguousarray(h.T.reshape(n_el, 8, 7))


def mixed_state(mesh, seed, strain=0.0015, noise=1.2, eps_scale=0.0008, alpha_max=0.02):
    """A displacement (affine strain + nodal noise of `noise` x element size x strain) and a
    random history giving a mix of elastic and plastic Gauss points."""
    rng = np.random.default_rng(seed)
    G = strain * rng.uniform(-1, 1, (3, 3))
    h = np.ptp(mesh.X[:, 0]) / max(1, round(np.ptp(mesh.X[:, 0]) / np.abs(np.diff(np.unique(mesh.X[:, 0]))).max()))
    u = (mesh.X @ G.T + noise * strain * h * rng.uniform(-1, 1, mesh.X.shape)).ravel()
    ep, al = inputs.random_history(mesh.n_el * 8, seed + 1, eps_scale, alpha_max)
    hist = np.concatenate([ep, al[:, None]], axis=1).reshape(mesh.n_el, 8, 7)
    return u, hist


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
