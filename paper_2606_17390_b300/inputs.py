"""Seeded synthetic inputs shared by the CUDA path, the oracle-based tests and the bench.

This module holds no arithmetic of the method: it only builds meshes, boundary-condition
lists, parameter sets, load-factor sequences and random states.  Every generator is
deterministic in its ``seed``.

Conventions (used by both sides):
* hex8 node order is the C3D8/VTK order: bottom face 0-1-2-3 counter-clockwise seen
  from +z, top face 4-7 above them;
* degrees of freedom are node-major: dof = 3*node + component;
* a Dirichlet entry (dof, value) prescribes u[dof] = t * value at load factor t.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Mesh", "Dirichlet", "Material", "box_mesh", "grf_plate_mesh", "roller_uniaxial_bcs",
    "clamp_displace_bcs", "config0_problem", "config1_problem", "config2_problem",
    "config2h_problem", "config1_material", "config0_material", "load_factors",
    "random_deformation_gradients", "random_history", "distorted_box_mesh",
    "hill_from_r_values", "compression_state", "config3_problem", "perturbed_theta", "noise",
]


@dataclasses.dataclass
class Mesh:
    X: np.ndarray      # float64 [n_nodes, 3], mm
    conn: np.ndarray   # int32 [n_el, 8], C3D8 order

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_el(self) -> int:
        return int(self.conn.shape[0])

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes


@dataclasses.dataclass
class Dirichlet:
    dof: np.ndarray    # int64 [n_fixed], sorted, unique
    value: np.ndarray  # float64 [n_fixed], prescribed value at load factor t = 1


@dataclasses.dataclass
class Material:
    """Isotropic elasticity (E, nu), Hill-48 (F, G, H, L, M, N) in the material frame,
    hardening law 'swift' (h = K, eps0, n) or 'voce' (h = sigma0, Q, b), and the material
    axes Theta (3x3, columns = material axes in global coordinates)."""
    E: float
    nu: float
    F: float
    G: float
    H: float
    L: float
    M: float
    N: float
    hardening: str
    h1: float
    h2: float
    h3: float
    Theta: np.ndarray = dataclasses.field(default_factory=lambda: np.eye(3))

    def theta_vector(self) -> np.ndarray:
        """Parameters in the order E, nu, F, G, H, L, M, N, h1, h2, h3."""
        return np.array([self.E, self.nu, self.F, self.G, self.H, self.L, self.M, self.N,
                         self.h1, self.h2, self.h3], dtype=np.float64)

    def with_theta(self, th) -> "Material":
        th = np.asarray(th, dtype=np.float64)
        return dataclasses.replace(self, E=th[0], nu=th[1], F=th[2], G=th[3], H=th[4],
                                   L=th[5], M=th[6], N=th[7], h1=th[8], h2=th[9], h3=th[10])


THETA_NAMES = ["E", "nu", "F", "G", "H", "L", "M", "N", "h1", "h2", "h3"]


def box_mesh(nx: int, ny: int, nz: int, Lx: float = 1.0, Ly: float = 1.0,
             Lz: float = 1.0) -> Mesh:
    """Structured nx*ny*nz hex8 grid on [0,Lx]x[0,Ly]x[0,Lz]; node id = i + (nx+1)(j + (ny+1)k),
    element id = i + nx(j + ny k)."""
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    zs = np.linspace(0.0, Lz, nz + 1)
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    X = np.stack([Xg.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i = i.transpose(2, 1, 0).ravel()
    j = j.transpose(2, 1, 0).ravel()
    k = k.transpose(2, 1, 0).ravel()

    def nid(a, b, c):
        return a + (nx + 1) * (b + (ny + 1) * c)

    conn = np.stack([nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k), nid(i, j + 1, k),
                     nid(i, j, k + 1), nid(i + 1, j, k + 1), nid(i + 1, j + 1, k + 1),
                     nid(i, j + 1, k + 1)], axis=1).astype(np.int32)
    return Mesh(X=X, conn=conn)


def distorted_box_mesh(n: int, seed: int, amp: float = 0.2, L: float = 1.0) -> Mesh:
    """n^3 box whose interior nodes are moved by up to amp*h in each direction (boundary
    nodes stay on their faces, only moved tangentially)."""
    m = box_mesh(n, n, n, L, L, L)
    rng = np.random.default_rng(seed)
    h = L / n
    d = rng.uniform(-amp * h, amp * h, size=m.X.shape)
    on_lo = np.isclose(m.X, 0.0)
    on_hi = np.isclose(m.X, L)
    d[on_lo | on_hi] = 0.0
    return Mesh(X=m.X + d, conn=m.conn)


def _gaussian_smooth_2d(w: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(w, sigma=sigma, mode="reflect")


def _smooth_grf(nx: int, ny: int, seed: int, corr: float, upsample: int) -> np.ndarray:
    """(ny, nx) Gaussian random field: white noise (seed) on the (nx/upsample)*(ny/upsample)
    base grid, repeated `upsample` times per axis, Gaussian filter of std
    corr*upsample/sqrt(2) elements (covariance exp(-r^2/(2 corr^2)) on the base grid)."""
    rng = np.random.default_rng(seed)
    bx, by = nx // upsample, ny // upsample
    w = rng.standard_normal((by, bx))
    if upsample > 1:
        w = np.repeat(np.repeat(w, upsample, axis=0), upsample, axis=1)
    return _gaussian_smooth_2d(w, corr * upsample / math.sqrt(2.0))


def _largest_component(keep2d: np.ndarray) -> np.ndarray:
    """Largest 4-connected component of the kept columns (face connectivity in 3-D since
    every column spans the full thickness)."""
    from scipy.ndimage import label
    lab, nlab = label(keep2d)
    if nlab > 1:
        sizes = np.bincount(lab.ravel())
        sizes[0] = 0
        keep2d = lab == int(np.argmax(sizes))
    return keep2d


def _column_mesh(keep2d: np.ndarray, nz: int, Lx: float, Ly: float, Lz: float):
    """Hex mesh of the kept through-thickness columns of an (ny, nx) grid; returns the mesh
    and the column index j*nx + i of every element."""
    ny, nx = keep2d.shape
    full = box_mesh(nx, ny, nz, Lx, Ly, Lz)
    col_keep = keep2d.ravel()                      # index j*nx + i
    el_col = np.arange(full.n_el) % (nx * ny)
    sel = col_keep[el_col]
    conn = full.conn[sel]
    used = np.unique(conn)
    remap = -np.ones(full.n_nodes, dtype=np.int64)
    remap[used] = np.arange(used.size)
    return Mesh(X=full.X[used].copy(), conn=remap[conn].astype(np.int32)), el_col[sel]


def grf_plate_mesh(nx: int = 200, ny: int = 100, nz: int = 4, Lx: float = 100.0,
                   Ly: float = 50.0, Lz: float = 2.0, seed: int = 1, corr: float = 8.0,
                   percentile: float = 70.0, grip_cols: int = 4, upsample: int = 1) -> Mesh:
    """Perforated plate: a 2-D Gaussian random field on the nx*ny element columns
    (white noise, seed `seed`, on the (nx/upsample)*(ny/upsample) base grid, repeated
    `upsample` times per axis, then a Gaussian filter of std corr*upsample/sqrt(2) elements,
    i.e. covariance exp(-r^2/(2 corr^2)) on the base grid) removes every through-thickness
    column whose value exceeds its `percentile`; `grip_cols` columns at each x end stay
    solid; the largest face-connected component is kept and orphan nodes are dropped."""
    g = _smooth_grf(nx, ny, seed, corr, upsample)
    keep2d = g <= np.percentile(g, percentile)
    keep2d[:, :grip_cols * upsample] = True
    keep2d[:, nx - grip_cols * upsample:] = True
    return _column_mesh(_largest_component(keep2d), nz, Lx, Ly, Lz)[0]


def _face_nodes(mesh: Mesh, axis: int, where: str) -> np.ndarray:
    c = mesh.X[:, axis]
    v = c.min() if where == "min" else c.max()
    return np.nonzero(np.isclose(c, v, rtol=0.0, atol=1e-9 * max(1.0, abs(v))))[0]


def _make_dirichlet(pairs: dict) -> Dirichlet:
    dof = np.array(sorted(pairs), dtype=np.int64)
    val = np.array([pairs[d] for d in dof], dtype=np.float64)
    return Dirichlet(dof=dof, value=val)


def roller_uniaxial_bcs(mesh: Mesh, disp: float, axis: int = 0) -> Dirichlet:
    """Symmetry rollers on the three minimum faces (u_k = 0 on x_k = min) and a normal
    displacement `disp` on the maximum face along `axis`: homogeneous uniaxial stress."""
    pairs = {}
    for k in range(3):
        for n in _face_nodes(mesh, k, "min"):
            pairs[3 * int(n) + k] = 0.0
    for n in _face_nodes(mesh, axis, "max"):
        pairs[3 * int(n) + axis] = float(disp)
    return _make_dirichlet(pairs)


def clamp_displace_bcs(mesh: Mesh, disp) -> Dirichlet:
    """x = min face clamped (u = 0); x = max face displaced by the 3-vector `disp`."""
    pairs = {}
    for n in _face_nodes(mesh, 0, "min"):
        for k in range(3):
            pairs[3 * int(n) + k] = 0.0
    for n in _face_nodes(mesh, 0, "max"):
        for k in range(3):
            pairs[3 * int(n) + k] = float(disp[k])
    return _make_dirichlet(pairs)


def load_factors(n_steps: int) -> np.ndarray:
    return np.arange(1, n_steps + 1, dtype=np.float64) / n_steps


def config0_material() -> Material:
    """Hill-48 (F,G,H,L,M,N) = (0.25,0.30,0.70,1.5,1.5,1.5), E = 70 GPa, nu = 0.33,
    Swift K = 500 MPa, eps0 = 0.01, n = 0.2 (units mm, N, MPa)."""
    return Material(E=70000.0, nu=0.33, F=0.25, G=0.30, H=0.70, L=1.5, M=1.5, N=1.5,
                    hardening="swift", h1=500.0, h2=0.01, h3=0.2)


def config1_material() -> Material:
    """Hill-48 as config0_material, Voce sigma0 = 150 MPa, Q = 120 MPa, b = 12."""
    return Material(E=70000.0, nu=0.33, F=0.25, G=0.30, H=0.70, L=1.5, M=1.5, N=1.5,
                    hardening="voce", h1=150.0, h2=120.0, h3=12.0)


def config0_problem(n: int = 4, n_steps: int = 10):
    """Unit cube n^3, roller symmetry BCs, u_x(x=1) = 0.05 t: uniaxial tension to 5 %."""
    mesh = box_mesh(n, n, n)
    return mesh, roller_uniaxial_bcs(mesh, 0.05, axis=0), config0_material(), load_factors(n_steps)


def config1_problem(nx: int = 200, ny: int = 100, nz: int = 4, n_steps: int = 20, seed: int = 1):
    """Perforated 100 x 50 x 2 mm plate, clamped at x = 0, u_x = 2 mm at x = 100 (u_y = u_z = 0),
    Hill-48 with Voce hardening; `nx, ny, nz` can be reduced for small cases (the GRF
    correlation length scales with nx/200)."""
    corr = 8.0 * nx / 200.0
    mesh = grf_plate_mesh(nx, ny, nz, 100.0, 50.0, 2.0, seed=seed, corr=corr,
                          grip_cols=max(1, (4 * nx) // 200))
    return mesh, clamp_displace_bcs(mesh, (2.0, 0.0, 0.0)), config1_material(), load_factors(n_steps)


def config4_problem(nx: int = 400, ny: int = 200, nz: int = 4, n_steps: int = 20):
    """Config 1's 100 x 50 x 2 mm domain at 0.25 mm (400 x 200 x 4): the holes of the same
    random field at twice the resolution (seed 1 white noise on the 200 x 100 base grid,
    upsampled 2x, Gaussian filter of std 16/sqrt(2) fine columns, 70th percentile, 2 mm grips
    at both ends), config-1 loading and Voce material, and per-element Hill F, G, H and
    sigma0 = mean * (1 + 0.15 g_k / max|g_k|) with g_k smooth random fields of the same
    construction (seeds 5, 6, 7, 8).  Other (nx, ny), e.g. a 40 x 20 x 2 re-mesh, sample the
    400 x 200 hole mask and fields at their element-column centres.  Returns (mesh, bc,
    material with the mean values, theta [n_el, 11], t)."""
    NX, NY, up = 400, 200, 2
    keep_f = (lambda g: g <= np.percentile(g, 70.0))(_smooth_grf(NX, NY, 1, 8.0, up))
    keep_f[:, :4 * up] = True
    keep_f[:, NX - 4 * up:] = True
    fields = [_smooth_grf(NX, NY, sd, 8.0, up) for sd in (5, 6, 7, 8)]
    fields = [1.0 + 0.15 * g / np.abs(g).max() for g in fields]
    fi = np.minimum(((np.arange(nx) + 0.5) * NX / nx).astype(np.int64), NX - 1)
    fj = np.minimum(((np.arange(ny) + 0.5) * NY / ny).astype(np.int64), NY - 1)
    keep = keep_f[np.ix_(fj, fi)]
    mesh, col = _column_mesh(_largest_component(keep), nz, 100.0, 50.0, 2.0)
    mat = config1_material()
    theta = np.tile(mat.theta_vector(), (mesh.n_el, 1))
    cj, ci = fj[col // nx], fi[col % nx]
    for k, idx in enumerate((2, 3, 4, 8)):      # F, G, H, sigma0
        theta[:, idx] *= fields[k][cj, ci]
    return mesh, clamp_displace_bcs(mesh, (2.0, 0.0, 0.0)), mat, theta, load_factors(n_steps)


def config2_problem(n: int = 100, n_steps: int = 10):
    """Unit cube n^3, x = 0 clamped, x = 1 face u = (-0.1 t, 0, 0): 10 % compression between
    clamped platens (heterogeneous elastic/plastic mix), config-0 material."""
    mesh = box_mesh(n, n, n)
    return mesh, clamp_displace_bcs(mesh, (-0.1, 0.0, 0.0)), config0_material(), load_factors(n_steps)


def config2h_problem(n: int = 100, n_steps: int = 10):
    """Homogeneous variant of config2_problem: roller symmetry BCs, u_x(x=1) = -0.1 t."""
    mesh = box_mesh(n, n, n)
    return mesh, roller_uniaxial_bcs(mesh, -0.1, axis=0), config0_material(), load_factors(n_steps)


def compression_state(mesh: Mesh, t: float, strain: float = 0.1, bulge: float = 0.3,
                      alpha_lag: float = 0.85, H: float = 0.70, G: float = 0.30):
    """A seeded-free, deterministic mid-step state of the clamped-platen compression of the
    unit cube (config 2) at load factor t: displacement u_x = -strain t X, lateral bulge
    u_y = bulge strain t (Y - 1/2) 4X(1-X), u_z likewise (zero on both clamped faces, so the
    Dirichlet data hold exactly), and a history that lags behind it: alpha = alpha_lag *
    strain * t * (1 + 4X(1-X)) / 2 with eps_p = alpha * diag(-1, H, G) (the traceless
    compression flow direction of a Hill material with G + H = 1).  Returns u [n_dof] and
    the history [7][n_gp] at the Gauss points' elements' centres."""
    X = mesh.X
    s = 4.0 * X[:, 0] * (1.0 - X[:, 0])
    u = np.stack([-strain * t * X[:, 0], bulge * strain * t * (X[:, 1] - 0.5) * s,
                  bulge * strain * t * (X[:, 2] - 0.5) * s], axis=1).ravel()
    xc = X[mesh.conn].mean(axis=1)
    sc = 4.0 * xc[:, 0] * (1.0 - xc[:, 0])
    alpha_el = alpha_lag * strain * t * 0.5 * (1.0 + sc)
    alpha = np.repeat(alpha_el, 8)
    hist = np.zeros((7, alpha.size))
    hist[0] = -alpha
    hist[1] = H * alpha
    hist[2] = G * alpha
    hist[6] = alpha
    return u, hist


def config3_problem(nx: int = 200, ny: int = 100, nz: int = 4, n_steps: int = 20):
    """Config-1 mesh and loading with the nine uniform parameters of the gradient check
    (F, G, H, L, M, N, K, eps0, n): Swift hardening with the config-0 values as the 'true'
    set.  Returns (mesh, bc, material_true, t)."""
    mesh, bc, _, ts = config1_problem(nx, ny, nz, n_steps)
    return mesh, bc, config0_material(), ts


def perturbed_theta(theta_true, seed: int = 4, rel: float = 0.2, indices=(2, 3, 4, 5, 6, 7, 8, 9, 10)):
    """theta_true * (1 + rel * U(-1, 1)) on the given parameter indices (seeded)."""
    rng = np.random.default_rng(seed)
    th = np.array(theta_true, dtype=np.float64)
    idx = np.asarray(indices)
    th[..., idx] = th[..., idx] * (1.0 + rel * rng.uniform(-1.0, 1.0, size=th[..., idx].shape))
    return th


def noise(shape, scale: float, seed: int = 3) -> np.ndarray:
    """Gaussian noise N(0, scale^2) of the given shape (seeded), added to target fields."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def hill_from_r_values(r11, r22, r33, r12, r23, r13):
    """(F, G, H, L, M, N) from the normalised yield ratios: the inverse of
    r11 = 1/sqrt(G+H), r22 = 1/sqrt(F+H), r33 = 1/sqrt(F+G), r12 = sqrt(3/(2N)),
    r23 = sqrt(3/(2L)), r13 = sqrt(3/(2M)).  Pure parameter bookkeeping."""
    a, b, c = 1.0 / r11 ** 2, 1.0 / r22 ** 2, 1.0 / r33 ** 2   # G+H, F+H, F+G
    F = 0.5 * (b + c - a)
    G = 0.5 * (a + c - b)
    H = 0.5 * (a + b - c)
    return F, G, H, 1.5 / r23 ** 2, 1.5 / r13 ** 2, 1.5 / r12 ** 2


def random_deformation_gradients(n: int, seed: int, scale: float = 0.05) -> np.ndarray:
    """n deformation gradients I + scale * U(-1,1)^{3x3}; det > 0 for scale < 0.3."""
    rng = np.random.default_rng(seed)
    return np.eye(3)[None] + scale * rng.uniform(-1.0, 1.0, size=(n, 3, 3))


def random_history(n: int, seed: int, eps_scale: float = 0.02, alpha_max: float = 0.05):
    """Random traceless plastic log strains (n, 6; order 11,22,33,12,23,13) and alpha (n,)."""
    rng = np.random.default_rng(seed)
    ep = eps_scale * rng.uniform(-1.0, 1.0, size=(n, 6))
    ep[:, :3] -= ep[:, :3].mean(axis=1, keepdims=True)
    alpha = alpha_max * rng.uniform(0.0, 1.0, size=n)
    return ep, alpha


# ------------------------------------------------------------------ Barlat material points
@dataclasses.dataclass
class BarlatMaterial:
    """Yld2004-18p parameters: c1 = (c'12, c'13, c'21, c'23, c'31, c'32, c'44, c'55, c'66),
    c2 the same for c'', even exponent m, isotropic E and nu (or nine orthotropic stiffness
    coefficients d in the material frame), hardening law and parameters ((sigma0, Q, b) for
    Voce, (K, eps0, n) for Swift), material frame Theta (columns = axes)."""
    c1: tuple
    c2: tuple
    m: int
    E: float
    nu: float
    hardening: str = "voce"
    h: tuple = (1.0, 0.0, 0.0)
    Theta: np.ndarray = None
    d: tuple = None   # orthotropic stiffness (E1111, E2222, E3333, E1122, E1133, E2233, E1212, E2323, E1313)


def barlat_verification_material() -> BarlatMaterial:
    """The Yld2004-18p verification parameters of the paper's table (m = 8, E = 1000,
    nu = 0.3, sigma0 = 1, perfect plasticity = Voce with Q = 0)."""
    return BarlatMaterial(
        c1=(-0.069888, 0.936408, 0.079143, 1.003060, 0.524741, 1.363180, 1.023770, 1.069060, 0.954322),
        c2=(0.981171, 0.476741, 0.575316, 0.866827, 1.145010, -0.079294, 1.051660, 1.147100, 1.404620),
        m=8, E=1000.0, nu=0.3, hardening="voce", h=(1.0, 0.0, 0.0))


def principal_plane_directions(angle) -> np.ndarray:
    """Unit deviatoric directions of the principal-stress (pi) plane as stress components
    (..., 6) of a diagonal stress: sqrt(2/3) (cos a, cos(a - 2 pi/3), cos(a + 2 pi/3))."""
    a = np.asarray(angle, dtype=np.float64)
    d = np.zeros(a.shape + (6,))
    s = math.sqrt(2.0 / 3.0)
    d[..., 0] = s * np.cos(a)
    d[..., 1] = s * np.cos(a - 2.0 * math.pi / 3.0)
    d[..., 2] = s * np.cos(a + 2.0 * math.pi / 3.0)
    return d


def pi_plane_sample(n: int = 16000, seed: int = 17390, scale_max: float = 30.0):
    """The line-search robustness map's trial states: n points of the pi plane between the
    yield surface and the same surface scaled by scale_max, as (angle (n,), scale (n,)) drawn
    uniformly from [0, 2 pi) x (1, scale_max].  The trial stress of a point is
    scale * sigma_y(alpha_n) * d(angle) / phi(d(angle)), d = principal_plane_directions: the
    scaling to the yield surface is the method's arithmetic and is done by each side."""
    rng = np.random.default_rng(seed)
    angle = rng.uniform(0.0, 2.0 * math.pi, size=n)
    scale = scale_max - (scale_max - 1.0) * rng.uniform(0.0, 1.0, size=n)   # (1, scale_max]
    return angle, scale


def random_stresses(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Random stress components (n, 6), uniform in [-scale, scale]."""
    rng = np.random.default_rng(seed)
    return scale * rng.uniform(-1.0, 1.0, size=(n, 6))


def random_rotation(seed: int) -> np.ndarray:
    """A random proper rotation (3, 3) (QR of a Gaussian matrix, signs fixed)."""
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q
