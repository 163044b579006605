"""Barlat Yld2004-18p material points on the GPU (hfe_barlat_phi, hfe_barlat_return_map)
against the oracle: phi and N on random stresses for several parameter sets and frames; the
closest-point projection with and without the App. B line search on a sample of the pi-plane
robustness map (converged stresses, iteration counts, outcomes); the implicit-differentiation
tangent; Swift hardening with shear components in a rotated frame; the full 16,000-point map
at the benchmark's launch configuration on sampled points; the elastic branch, empty input,
non-finite input and rejected arguments.

Each side builds its own trial stresses from the same seeded (angle, scale) sample: the
scaling to the yield surface uses that side's phi."""
import numpy as np
import pytest

from oracle import barlat as BA
from paper_2606_17390_b300 import hfe, inputs

pytestmark = pytest.mark.gpu

ONES = (1.0,) * 9


def _models():
    rng = np.random.default_rng(5)
    mat = inputs.barlat_verification_material()
    out = [mat]
    m2 = inputs.barlat_verification_material()
    m2.Theta = inputs.random_rotation(1)
    out.append(m2)
    for m in (2, 4, 6, 12):
        out.append(inputs.BarlatMaterial(c1=tuple(rng.uniform(-0.2, 1.6, 9)), c2=tuple(rng.uniform(-0.2, 1.6, 9)),
                                         m=m, E=1000.0, nu=0.3, Theta=inputs.random_rotation(m)))
    out.append(inputs.BarlatMaterial(c1=ONES, c2=ONES, m=8, E=1000.0, nu=0.3))
    return out


def _oracle_model(mat):
    return BA.Barlat(mat.c1, mat.c2, mat.m, mat.Theta)


def _cuda(a, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda() if dtype is None else \
        torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.parametrize("k", range(7))
def test_phi_and_flow_against_oracle(k):
    mat = _models()[k]
    T = inputs.random_stresses(1000, seed=60 + k, scale=3.0)
    phi_d, N_d = hfe.barlat_phi(mat, _cuda(T), with_N=True)
    N_o, phi_o = _oracle_model(mat).flow(T)
    assert np.abs(phi_d.cpu().numpy() - phi_o).max() <= 1e-12 * phi_o.max()
    assert np.abs(N_d.cpu().numpy() - N_o).max() <= 1e-11 * np.abs(N_o).max()


def _gpu_trials(mat, angle, scale, alpn):
    """GPU side of the recipe (perfect plasticity, so sigma_y(alpha_n) = sigma0):
    T_tr = scale * sigma0 * d / phi_gpu(d)."""
    import torch
    assert mat.hardening == "voce" and mat.h[1] == 0.0
    d = _cuda(inputs.principal_plane_directions(angle))
    phi = hfe.barlat_phi(mat, d)
    return (torch.from_numpy(scale * mat.h[0]).cuda()[:, None] / phi[:, None]) * d


def _oracle_trials(model, mat, angle, scale, alpn):
    d = inputs.principal_plane_directions(angle)
    return (scale * BA.sigma_y(mat.hardening, mat.h, alpn) / model.phi_poly(d))[:, None] * d


def _compare_map(mat, n, line_search, seed, kmax=40, precision="fp64"):
    angle, scale = inputs.pi_plane_sample(n, seed=seed)
    alpn = np.zeros(n)
    model = _oracle_model(mat)
    Tt_o = _oracle_trials(model, mat, angle, scale, alpn)
    y, it_o, conv_o = BA.cpp(model, mat.E, mat.nu, mat.hardening, mat.h, Tt_o, alpn,
                             line_search=line_search, kmax=kmax)
    Tt_d = _gpu_trials(mat, angle, scale, alpn)
    assert np.abs(Tt_d.cpu().numpy() - Tt_o).max() <= 1e-13 * np.abs(Tt_o).max()
    out = hfe.barlat_return_map(mat, Tt_d, _cuda(alpn), line_search=line_search, kmax=kmax, precision=precision)
    st = out["status"].cpu().numpy()
    it_d = out["iters"].cpu().numpy()
    T_d = out["T"].cpu().numpy()
    return dict(y=y, it_o=it_o, conv_o=conv_o, st=st, it_d=it_d, T_d=T_d, dg_d=out["dgamma"].cpu().numpy(),
                al_d=out["alpha"].cpu().numpy(), Tt=Tt_o)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_line_search_map_sample_against_oracle(precision):
    """2,000 points of the map with the line search: the points converge on both sides to the
    same stress.  FP64: iteration counts agree (rounding may move a count by one at a Goldstein
    or tolerance tie).  Mixed: the FP32 iterates differ from the FP64 ones by rounding and the
    FP64 polish adds an iteration or two, so counts agree within a few."""
    mat = inputs.barlat_verification_material()
    r = _compare_map(mat, 2000, True, seed=101, precision=precision)
    conv_d = r["st"] == hfe_status("converged")
    assert (r["st"] != hfe_status("elastic")).all()
    assert np.isin(r["st"], [hfe_status("converged"), hfe_status("maxit")]).all()
    both = conv_d & r["conv_o"]
    assert (conv_d == r["conv_o"]).mean() >= 0.99
    # a disagreement is only allowed near the iteration cap
    dis = np.nonzero(conv_d != r["conv_o"])[0]
    assert (np.maximum(r["it_o"][dis], r["it_d"][dis]) >= 35).all()
    scale = np.abs(r["Tt"]).max(axis=1)
    err = np.abs(r["T_d"][both] - r["y"][both, :6]).max(axis=1) / scale[both]
    assert err.max() <= 1e-11, err.max()
    assert np.abs(r["dg_d"][both] - r["y"][both, 7]).max() <= 1e-11 * np.abs(r["y"][both, 7]).max()
    assert np.abs(r["al_d"][both] - r["y"][both, 6]).max() <= 1e-11 * np.abs(r["y"][both, 6]).max()
    dit = r["it_d"][both] - r["it_o"][both]
    if precision == "fp64":
        assert (dit == 0).mean() >= 0.99, (dit == 0).mean()
        assert np.abs(dit).max() <= 2
    else:
        assert (np.abs(dit) <= 2).mean() >= 0.98, (np.abs(dit) <= 2).mean()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plain_newton_map_sample_against_oracle(precision):
    """Standard Newton on the same kind of sample: points that converge on both sides agree;
    the number left unconverged is close (the failing trajectories oscillate, so rounding may
    move individual points)."""
    mat = inputs.barlat_verification_material()
    r = _compare_map(mat, 1000, False, seed=102, precision=precision)
    conv_d = r["st"] == hfe_status("converged")
    both = conv_d & r["conv_o"]
    assert both.sum() >= 200
    scale = np.abs(r["Tt"]).max(axis=1)
    err = np.abs(r["T_d"][both] - r["y"][both, :6]).max(axis=1) / scale[both]
    assert err.max() <= 1e-11
    fail_o, fail_d = (~r["conv_o"]).sum(), (~conv_d).sum()
    assert fail_o >= 300 and abs(int(fail_o) - int(fail_d)) <= 0.05 * 1000
    assert (r["st"][~conv_d] != hfe_status("elastic")).all()


def hfe_status(name):
    return {v: k for k, v in hfe.CPP_STATUS.items()}[name]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_rotated_swift_with_shear_and_tangent(k, precision):
    """Swift hardening, a rotated material frame, trial stresses with shear components and
    alpha_n > 0: stress, alpha, dgamma and dT/dT_tr against the oracle."""
    mat = _models()[k]
    mat.hardening, mat.h, mat.E, mat.nu = "swift", (500.0, 0.01, 0.2), 70000.0, 0.33
    n = 64
    rng = np.random.default_rng(70 + k)
    alpn = rng.uniform(0.0, 0.05, n)
    model = _oracle_model(mat)
    T = inputs.random_stresses(n, seed=71 + k, scale=1.0)
    sy = BA.sigma_y("swift", mat.h, alpn)
    Ttr = T * (sy * rng.uniform(1.05, 4.0, n) / model.phi_poly(T))[:, None]
    y, it_o, conv_o = BA.cpp(model, mat.E, mat.nu, "swift", mat.h, Ttr, alpn, kmax=60)
    assert conv_o.all()
    D_o = BA.cpp_tangent(model, mat.E, mat.nu, "swift", mat.h, y, Ttr, alpn)
    out = hfe.barlat_return_map(mat, _cuda(Ttr), _cuda(alpn), tangent=True, kmax=60, precision=precision)
    assert (out["status"].cpu().numpy() == hfe_status("converged")).all()
    sc = np.abs(Ttr).max()
    assert np.abs(out["T"].cpu().numpy() - y[:, :6]).max() <= 1e-11 * sc
    assert np.abs(out["alpha"].cpu().numpy() - y[:, 6]).max() <= 1e-12 * max(1.0, np.abs(y[:, 6]).max())
    assert np.abs(out["dgamma"].cpu().numpy() - y[:, 7]).max() <= 1e-11 * np.abs(y[:, 7]).max()
    D_d = out["tangent"].cpu().numpy()
    assert np.abs(D_d - D_o).max() <= 1e-8 * np.abs(D_o).max()
    assert np.abs(out["iters"].cpu().numpy() - it_o).max() <= (1 if precision == "fp64" else 3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_map_launch_configuration_sampled(precision):
    """The full 16,000-point map in one launch, as the benchmark runs it: 400 sampled points
    against the oracle, every point converged with the line search, and the standard-Newton
    launch leaves thousands unconverged."""
    mat = inputs.barlat_verification_material()
    angle, scale = inputs.pi_plane_sample(16000)
    alpn = np.zeros(16000)
    Tt_d = _gpu_trials(mat, angle, scale, alpn)
    out = hfe.barlat_return_map(mat, Tt_d, _cuda(alpn), line_search=True, kmax=40, precision=precision)
    st = out["status"].cpu().numpy()
    # the slow points of the map need up to about 52 iterations: with kmax = 40 a few hundredths
    # of a percent stay at the cap, and none of them fails in any other way
    assert np.isin(st, [hfe_status("converged"), hfe_status("maxit")]).all()
    assert (st == hfe_status("maxit")).sum() <= 200
    idx = np.random.default_rng(9).choice(16000, 400, replace=False)
    model = _oracle_model(mat)
    Tt_o = _oracle_trials(model, mat, angle[idx], scale[idx], alpn[idx])
    y, it_o, conv_o = BA.cpp(model, mat.E, mat.nu, mat.hardening, mat.h, Tt_o, alpn[idx], kmax=40)
    both = conv_o & (st[idx] == hfe_status("converged"))
    assert both.mean() >= 0.98
    T_d = out["T"].cpu().numpy()[idx]
    assert np.abs(T_d[both] - y[both, :6]).max() <= 1e-11 * np.abs(Tt_o).max()
    out_nw = hfe.barlat_return_map(mat, Tt_d, _cuda(alpn), line_search=False, kmax=40, precision=precision)
    n_fail = int((out_nw["status"].cpu().numpy() != hfe_status("converged")).sum())
    assert 8000 <= n_fail <= 11000, n_fail


def test_elastic_empty_nonfinite_and_rejections():
    import torch
    mat = inputs.barlat_verification_material()
    angle, _ = inputs.pi_plane_sample(8, seed=3)
    d = _cuda(inputs.principal_plane_directions(angle))
    phi = hfe.barlat_phi(mat, d)
    Tin = (0.9 / phi)[:, None] * d                                  # inside the yield surface
    Tin[:, :3] += 5.0                                               # plus a pressure
    a0 = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = hfe.barlat_return_map(mat, Tin, a0, tangent=True)
    assert (out["status"].cpu().numpy() == hfe_status("elastic")).all()
    out_m = hfe.barlat_return_map(mat, Tin, a0, precision="mixed")
    assert (out_m["status"].cpu().numpy() == hfe_status("elastic")).all()
    # on the yield surface to within the FP32 band: decided in FP64 on the mixed path
    Ton = (1.0 / phi)[:, None] * d
    Ton[:4] *= 1.0 + 1e-9
    Ton[4:] *= 1.0 - 1e-9
    st_on = hfe.barlat_return_map(mat, Ton, a0, precision="mixed")["status"].cpu().numpy()
    st_64 = hfe.barlat_return_map(mat, Ton, a0)["status"].cpu().numpy()
    assert (st_on[4:] == hfe_status("elastic")).all() and (st_on[:4] == hfe_status("converged")).all()
    assert (st_64 == st_on).all()
    assert torch.equal(out["T"], Tin)
    assert (out["iters"].cpu().numpy() == 0).all()
    assert torch.equal(out["tangent"].cpu(), torch.eye(6, dtype=torch.float64).expand(8, 6, 6))
    # a pure pressure: phi = 0 up to the rounding of the deviatoric projection; elastic
    P = torch.zeros((2, 6), dtype=torch.float64, device="cuda")
    P[0, :3] = 3.0
    phi_p = hfe.barlat_phi(mat, P).cpu().numpy()
    assert phi_p[0] <= 1e-14 * 3.0 and phi_p[1] == 0.0
    out_p = hfe.barlat_return_map(mat, P, torch.zeros(2, dtype=torch.float64, device="cuda"))
    assert (out_p["status"].cpu().numpy() == hfe_status("elastic")).all()
    # empty input
    e = torch.empty((0, 6), dtype=torch.float64, device="cuda")
    r = hfe.barlat_return_map(mat, e, torch.empty(0, dtype=torch.float64, device="cuda"))
    assert r["T"].shape == (0, 6)
    # a non-finite trial stress is reported per point
    bad = Tin.clone()
    bad[2, 0] = float("nan")
    bad[3, 1] = float("inf")
    out = hfe.barlat_return_map(mat, bad * 10.0, a0)
    st = out["status"].cpu().numpy()
    assert st[2] == hfe_status("nonfinite") and st[3] == hfe_status("nonfinite")
    assert (st[[0, 1, 4, 5, 6, 7]] == hfe_status("converged")).all()
    assert np.isnan(hfe.barlat_phi(mat, bad).cpu().numpy()[2:4]).all()
    # rejected arguments
    for bad_m in (7, 0, 34):
        mm = inputs.barlat_verification_material()
        mm.m = bad_m
        with pytest.raises(hfe.HfeError) as ex:
            hfe.barlat_phi(mm, d)
        assert ex.value.status == -1
    mm = inputs.barlat_verification_material()
    mm.Theta = 2.0 * np.eye(3)
    with pytest.raises(hfe.HfeError):
        hfe.barlat_return_map(mm, Tin, a0)
    with pytest.raises(hfe.HfeError):
        hfe.barlat_return_map(mat, Tin.cpu(), a0.cpu())
    with pytest.raises(hfe.HfeError):
        hfe.barlat_return_map(mat, Tin, a0, eta=1.5)
    # the mixed path reports non-finite inputs the same way
    st_m = hfe.barlat_return_map(mat, bad * 10.0, a0, precision="mixed")["status"].cpu().numpy()
    assert st_m[2] == hfe_status("nonfinite") and st_m[3] == hfe_status("nonfinite")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_orthotropic_elasticity_and_voce_against_oracle(precision):
    """An orthotropic, rotated E (nine coefficients in the material frame) with Voce hardening
    (Q > 0, alpha_n > 0) in a rotated Barlat frame: stress, alpha, dgamma and the tangent
    against the oracle; the isotropic coefficients through the orthotropic table give the
    (E, nu) result."""
    mat = inputs.barlat_verification_material()
    mat.Theta = inputs.random_rotation(101)
    mat.h = (1.0, 0.6, 15.0)
    mat.d = (2.0e3, 1.4e3, 1.1e3, 0.5e3, 0.45e3, 0.4e3, 0.35e3, 0.3e3, 0.25e3)
    Eg = BA.orthotropic_tensor(mat.d, mat.Theta)   # the elasticity frame is the material frame
    model = _oracle_model(mat)
    n = 96
    rng = np.random.default_rng(103)
    alpn = rng.uniform(0.0, 0.05, n)
    T = inputs.random_stresses(n, seed=104, scale=1.0)
    sy = BA.sigma_y("voce", mat.h, alpn)
    Ttr = T * (sy * rng.uniform(1.05, 6.0, n) / model.phi_poly(T))[:, None]
    y, it_o, conv_o = BA.cpp(model, Eg, None, "voce", mat.h, Ttr, alpn, kmax=60)
    assert conv_o.all()
    D_o = BA.cpp_tangent(model, Eg, None, "voce", mat.h, y, Ttr, alpn)
    out = hfe.barlat_return_map(mat, _cuda(Ttr), _cuda(alpn), tangent=True, kmax=60, precision=precision)
    assert (out["status"].cpu().numpy() == hfe_status("converged")).all()
    sc = np.abs(Ttr).max()
    assert np.abs(out["T"].cpu().numpy() - y[:, :6]).max() <= 1e-11 * sc
    assert np.abs(out["alpha"].cpu().numpy() - y[:, 6]).max() <= 1e-12
    assert np.abs(out["dgamma"].cpu().numpy() - y[:, 7]).max() <= 1e-11 * np.abs(y[:, 7]).max()
    assert np.abs(out["tangent"].cpu().numpy() - D_o).max() <= 1e-8 * np.abs(D_o).max()
    # isotropic coefficients through the orthotropic table = the (E, nu) path
    lam, mu = BA.lame(mat.E, mat.nu)
    iso = inputs.barlat_verification_material()
    iso.Theta, iso.h = mat.Theta, mat.h
    iso_d = inputs.barlat_verification_material()
    iso_d.Theta, iso_d.h = mat.Theta, mat.h
    iso_d.d = (lam + 2 * mu,) * 3 + (lam,) * 3 + (mu,) * 3
    a = hfe.barlat_return_map(iso, _cuda(Ttr), _cuda(alpn), precision=precision)
    b = hfe.barlat_return_map(iso_d, _cuda(Ttr), _cuda(alpn), precision=precision)
    assert np.abs(a["T"].cpu().numpy() - b["T"].cpu().numpy()).max() <= 1e-12 * sc
    # a non-positive stiffness coefficient is rejected
    bad = inputs.barlat_verification_material()
    bad.d = (0.0,) + mat.d[1:]
    with pytest.raises(hfe.HfeError):
        hfe.barlat_return_map(bad, _cuda(Ttr), _cuda(alpn))
