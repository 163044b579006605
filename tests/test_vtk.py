"""Legacy-VTK output (paper_2606_17390_b300/vtk.py): the file parses back to the same mesh,
node and element fields (round trip at full precision, hexahedron cell type 12, deformed
coordinates X + u), von Mises from 6 stress components equals the oracle's tensor
definition, element averages follow the element-major Gauss-point order, and inconsistent
shapes are refused."""
import numpy as np
import pytest

from oracle import material
from paper_2606_17390_b300 import inputs, vtk


def _parse(path):
    tok = open(path).read().split("\n")
    assert tok[0].startswith("# vtk DataFile") and tok[2] == "ASCII" and tok[3] == "DATASET UNSTRUCTURED_GRID"
    words = " ".join(tok[4:]).split()
    out, i, section = {"point": {}, "cell": {}}, 0, None
    while i < len(words):
        w = words[i]
        if w == "POINTS":
            n = int(words[i + 1]); i += 3
            out["X"] = np.array(words[i:i + 3 * n], float).reshape(n, 3); i += 3 * n
        elif w == "CELLS":
            n, m = int(words[i + 1]), int(words[i + 2]); i += 3
            out["cells"] = np.array(words[i:i + m], int).reshape(n, 9); i += m
        elif w == "CELL_TYPES":
            n = int(words[i + 1]); i += 2
            out["types"] = np.array(words[i:i + n], int); i += n
        elif w in ("POINT_DATA", "CELL_DATA"):
            section, count = ("point" if w == "POINT_DATA" else "cell"), int(words[i + 1]); i += 2
        elif w == "SCALARS":
            name = words[i + 1]; i += 6
            out[section][name] = np.array(words[i:i + count], float); i += count
        elif w == "VECTORS":
            name = words[i + 1]; i += 3
            out[section][name] = np.array(words[i:i + 3 * count], float).reshape(count, 3); i += 3 * count
        else:
            raise AssertionError(w)
    return out


def test_round_trip_and_deformed_coordinates(tmp_path):
    mesh = inputs.distorted_box_mesh(3, seed=2, amp=0.2)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(mesh.n_dof) * 1e-3
    sig = rng.standard_normal((8 * mesh.n_el, 6)) * 100.0
    vm = vtk.gauss_point_average(vtk.von_mises(sig), mesh.n_el)
    alpha = rng.uniform(0, 0.1, 8 * mesh.n_el)
    p = tmp_path / "r.vtk"
    vtk.write_vtk(p, mesh.X, mesh.conn, u=u, deformed=True,
                  cell_data={"von_mises": vm, "alpha": vtk.gauss_point_average(alpha, mesh.n_el)})
    r = _parse(p)
    assert np.array_equal(r["X"], mesh.X + u.reshape(-1, 3))
    assert np.array_equal(r["cells"][:, 0], np.full(mesh.n_el, 8)) and np.array_equal(r["cells"][:, 1:], mesh.conn)
    assert np.all(r["types"] == vtk.VTK_HEXAHEDRON)
    assert np.array_equal(r["point"]["u"], u.reshape(-1, 3))
    assert np.array_equal(r["cell"]["von_mises"], vm)
    assert np.allclose(r["cell"]["alpha"], alpha.reshape(mesh.n_el, 8).mean(axis=1), rtol=0, atol=1e-15)


def test_von_mises_matches_the_tensor_definition():
    s6 = np.random.default_rng(3).standard_normal((50, 6))
    assert np.allclose(vtk.von_mises(s6), material.von_mises(material.sym(s6)), rtol=1e-14, atol=0)
    uniax = np.zeros(6)
    uniax[0] = 250.0
    assert vtk.von_mises(uniax) == pytest.approx(250.0, rel=1e-15)


def test_shapes_refused(tmp_path):
    mesh = inputs.box_mesh(2, 2, 1)
    with pytest.raises(ValueError):
        vtk.write_vtk(tmp_path / "a.vtk", mesh.X, mesh.conn[:, :7])
    with pytest.raises(ValueError):
        vtk.write_vtk(tmp_path / "b.vtk", mesh.X, mesh.conn, cell_data={"x": np.zeros(mesh.n_el + 1)})
    bad = mesh.conn.copy()
    bad[0, 0] = mesh.n_nodes
    with pytest.raises(ValueError):
        vtk.write_vtk(tmp_path / "c.vtk", mesh.X, bad)
