"""hfe_free_norm_static — the FP64 free-dof residual norm whose reduction scratch is a static
device array of the library (no allocation) — against the norm that hfe_gp_sweep returns for
the same residual, called twice in a row; plus its size limit, empty input and rejected
pointers.  Collected last so that it also runs after every other GPU test."""
import os
import re

import numpy as np
import pytest

from paper_2606_17390_b300 import hfe, inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hfe.h")
LOAD = 0.5
TOL = 1e-12   # the two sides sum the same FP64 squares in different orders


def test_limit_matches_header():
    m = re.search(r"#define\s+HFE_FREE_NORM_STATIC_MAX_DOF\s+(\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == hfe.FREE_NORM_STATIC_MAX_DOF


def _free_mask(torch, n_dof, fixed):
    mask = torch.ones(n_dof, dtype=torch.uint8, device="cuda")
    mask[torch.from_numpy(np.asarray(fixed, dtype=np.int64)).cuda()] = 0
    return mask


@pytest.mark.gpu
@pytest.mark.parametrize("n", [5, 40])
def test_matches_sweep_norm_on_two_calls(n):
    """Config-2 compression state on an n^3 cube (5^3: 648 dofs, one CTA with a ragged tail;
    40^3: 206,763 dofs, 51 CTAs) — the residual and its free-dof norm from hfe_gp_sweep, then
    the static-scratch norm of the same residual twice."""
    import torch
    mesh, bc, mat, _ = inputs.config2_problem(n, 10)
    u, hist = inputs.compression_state(mesh, LOAD)
    R = torch.empty(mesh.n_dof, dtype=torch.float64, device="cuda")
    rn = torch.empty(1, dtype=torch.float64, device="cuda")
    with hfe.from_inputs(mesh, bc, mat, precision="mixed") as s:
        s.set_state(None, np.ascontiguousarray(hist))
        s.sweep(torch.from_numpy(u).cuda(), LOAD, tangent=False, R_out=R, rnorm_out=rn, stats=True)
    torch.cuda.synchronize()
    mask = _free_mask(torch, mesh.n_dof, bc.dof)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    hfe.free_norm_static(R, mask, out[0:1], stream=stream)
    hfe.free_norm_static(R, mask, out[1:2], stream=stream)
    torch.cuda.synchronize()
    ref = rn.item()
    first, second = out.tolist()
    assert ref > 0.0
    assert abs(first - ref) <= TOL * ref, (first, ref)
    assert abs(second - ref) <= TOL * ref, (second, ref)
    assert first == second   # fixed summation order


@pytest.mark.gpu
def test_maximum_size_empty_and_rejections():
    import torch
    nmax = hfe.FREE_NORM_STATIC_MAX_DOF
    g = torch.Generator(device="cuda").manual_seed(11)
    r = torch.randn(nmax + 1, dtype=torch.float64, device="cuda", generator=g)
    mask = (torch.rand(nmax + 1, device="cuda", generator=g) < 0.9).to(torch.uint8)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    # the largest accepted size (1,024 CTAs) against a plain FP64 sum of the same squares
    hfe.free_norm_static(r[:nmax], mask[:nmax], out)
    torch.cuda.synchronize()
    rh, mh = r[:nmax].cpu().numpy(), mask[:nmax].cpu().numpy()
    ref = float(np.sqrt(np.sum(rh[mh != 0] ** 2)))
    assert abs(out.item() - ref) <= TOL * ref
    # one dof beyond the limit: rejected before anything is launched (the buffers are valid)
    out.fill_(-1.0)
    with pytest.raises(hfe.HfeError, match="exceeds the static scratch limit") as e:
        hfe.free_norm_static(r, mask, out)
    assert e.value.status == -1
    torch.cuda.synchronize()
    assert out.item() == -1.0
    # host memory is rejected
    with pytest.raises(hfe.HfeError) as e:
        hfe.free_norm_static(r[:16].cpu(), mask[:16].cpu(), out)
    assert e.value.status == -1
    # empty input: +0.0
    hfe.free_norm_static(r[:0], mask[:0], out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
