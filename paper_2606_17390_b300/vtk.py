"""Legacy-VTK (ASCII, unstructured grid) output of a hex8 result for visual post-processing:
the reference or deformed node coordinates, node fields (the displacement u) and element
fields (e.g. the Gauss-point average of the von Mises stress or of the equivalent plastic
strain alpha).  Host-side file writing only; the node order of the library's hex8 elements is
VTK_HEXAHEDRON's (cell type 12), so the connectivity is written as it is.
"""
from __future__ import annotations

import numpy as np

__all__ = ["VTK_HEXAHEDRON", "von_mises", "gauss_point_average", "write_vtk"]

VTK_HEXAHEDRON = 12


def von_mises(sigma6):
    """sqrt(3/2 s:s) of stresses given as 6 components (11, 22, 33, 12, 23, 13), [..., 6]."""
    s = np.asarray(sigma6, dtype=np.float64)
    p = (s[..., 0] + s[..., 1] + s[..., 2]) / 3.0
    d0, d1, d2 = s[..., 0] - p, s[..., 1] - p, s[..., 2] - p
    ss = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * (s[..., 3] ** 2 + s[..., 4] ** 2 + s[..., 5] ** 2)
    return np.sqrt(1.5 * ss)


def gauss_point_average(values, n_el):
    """Element averages of a per-Gauss-point quantity stored element-major ([n_el * 8, ...],
    the order of hfe_forward's sigma_out) or as history components ([n_el * 8])."""
    v = np.asarray(values, dtype=np.float64)
    return v.reshape(n_el, 8, *v.shape[1:]).mean(axis=1)


def _block(f, name, a):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        f.write(f"SCALARS {name} double 1\nLOOKUP_TABLE default\n")
        np.savetxt(f, a[:, None], fmt="%.17g")
    elif a.ndim == 2 and a.shape[1] == 3:
        f.write(f"VECTORS {name} double\n")
        np.savetxt(f, a, fmt="%.17g")
    else:
        raise ValueError(f"{name}: scalars [n] or 3-vectors [n, 3] only, got shape {a.shape}")


def write_vtk(path, X, conn, u=None, deformed=False, point_data=None, cell_data=None, title="hfe result"):
    """Write the mesh (X [n_nodes, 3], conn [n_el, 8]) with u [n_nodes * 3 or n_nodes, 3] as the
    node vector "u" (and as the coordinate offset when deformed), further node fields
    point_data {name: [n_nodes] or [n_nodes, 3]} and element fields cell_data {name: [n_el] or
    [n_el, 3]}."""
    X = np.asarray(X, dtype=np.float64)
    conn = np.asarray(conn, dtype=np.int64)
    n_nodes, n_el = X.shape[0], conn.shape[0]
    if conn.ndim != 2 or conn.shape[1] != 8 or conn.min() < 0 or conn.max() >= n_nodes:
        raise ValueError("conn must be [n_el, 8] with node ids in [0, n_nodes)")
    pd = dict(point_data or {})
    if u is not None:
        U = np.asarray(u, dtype=np.float64).reshape(n_nodes, 3)
        pd = {"u": U, **pd}
        if deformed:
            X = X + U
    for name, a in pd.items():
        if np.asarray(a).shape[0] != n_nodes:
            raise ValueError(f"point field {name}: {n_nodes} rows expected")
    cd = dict(cell_data or {})
    for name, a in cd.items():
        if np.asarray(a).shape[0] != n_el:
            raise ValueError(f"cell field {name}: {n_el} rows expected")
    with open(path, "w") as f:
        f.write(f"# vtk DataFile Version 3.0\n{title.splitlines()[0][:255]}\nASCII\nDATASET UNSTRUCTURED_GRID\n")
        f.write(f"POINTS {n_nodes} double\n")
        np.savetxt(f, X, fmt="%.17g")
        f.write(f"CELLS {n_el} {9 * n_el}\n")
        np.savetxt(f, np.hstack([np.full((n_el, 1), 8, np.int64), conn]), fmt="%d")
        f.write(f"CELL_TYPES {n_el}\n")
        np.savetxt(f, np.full((n_el, 1), VTK_HEXAHEDRON, np.int64), fmt="%d")
        if pd:
            f.write(f"POINT_DATA {n_nodes}\n")
            for name, a in pd.items():
                _block(f, name, a)
        if cd:
            f.write(f"CELL_DATA {n_el}\n")
            for name, a in cd.items():
                _block(f, name, a)
