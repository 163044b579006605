"""The host-side assembly set-up (csrc/pattern.cpp, compiled here by the host C++ compiler
without CUDA) against an independent numpy construction: the block-CSR pattern (one 3x3
block per pair of nodes sharing an element, sorted columns, the diagonal slot), the element
colouring (no two elements of a colour share a node; 8 colours on a structured hex mesh),
the element-to-block slot map, and the first-writer flags (exactly one per block, on its
first touch in launch order); malformed meshes are refused with a message."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2606_17390_b300 import inputs

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_17390_b300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <string>
#include <vector>
#include "pattern.h"
template <typename T> static void put(FILE* f, const std::vector<T>& v) {
  long long n = (long long)v.size();
  fwrite(&n, 8, 1, f);
  fwrite(v.data(), sizeof(T), v.size(), f);
}
int main(int argc, char** argv) {
  FILE* in = fopen(argv[1], "rb");
  long long nn, ne;
  if (fread(&nn, 8, 1, in) != 1 || fread(&ne, 8, 1, in) != 1) return 3;
  std::vector<int32_t> conn(ne * 8);
  if (fread(conn.data(), 4, conn.size(), in) != conn.size()) return 3;
  fclose(in);
  hfe::Pattern P;
  std::string err;
  if (!hfe::build_pattern(nn, ne, conn.data(), P, err)) {
    fprintf(stderr, "%s\n", err.c_str());
    return 2;
  }
  FILE* out = fopen(argv[2], "wb");
  put(out, P.rowptr); put(out, P.cols); put(out, P.diag_slot); put(out, P.slot);
  put(out, P.elems); put(out, P.color_off);
  fclose(out);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("pattern")
    (d / "driver.cpp").write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(d / "driver.cpp"),
                    os.path.join(CSRC, "pattern.cpp"), "-o", str(exe)], check=True)
    return exe, d


def _run(driver, n_nodes, conn):
    exe, d = driver
    inp, out = d / "conn.bin", d / "pattern.bin"
    with open(inp, "wb") as f:
        np.array([n_nodes, conn.shape[0]], dtype=np.int64).tofile(f)
        np.ascontiguousarray(conn, dtype=np.int32).tofile(f)
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True)
    if r.returncode != 0:
        return None, r.stderr.strip()
    buf = open(out, "rb").read()
    parts, off = [], 0
    for dt in (np.int64, np.int32, np.int64, np.int32, np.int32, np.int64):
        n = int(np.frombuffer(buf, np.int64, 1, off)[0])
        off += 8
        parts.append(np.frombuffer(buf, dt, n, off).copy())
        off += n * np.dtype(dt).itemsize
    return dict(zip(("rowptr", "cols", "diag_slot", "slot", "elems", "color_off"), parts)), ""


def _check(P, n_nodes, conn):
    n_el = conn.shape[0]
    # pattern: every node pair sharing an element, rows sorted
    pairs = np.unique(np.stack([np.repeat(conn, 8, axis=1).ravel(), np.tile(conn, (1, 8)).ravel()], 1), axis=0)
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(pairs[:, 0], minlength=n_nodes))])
    assert np.array_equal(P["rowptr"], rowptr)
    assert np.array_equal(P["cols"], pairs[:, 1])
    rows = np.repeat(np.arange(n_nodes), np.diff(rowptr))
    assert np.array_equal(rows[P["diag_slot"]], np.arange(n_nodes))
    assert np.array_equal(P["cols"][P["diag_slot"]], np.arange(n_nodes))
    # slot map: block (conn[e][a], conn[e][b]) with bit 31 the first-writer flag
    raw = P["slot"].view(np.uint32)
    first = (raw >> 31).astype(bool)
    slot = (raw & 0x7FFFFFFF).astype(np.int64).reshape(n_el, 8, 8)
    assert np.array_equal(rows[slot], np.broadcast_to(conn[:, :, None], slot.shape))
    assert np.array_equal(P["cols"][slot], np.broadcast_to(conn[:, None, :], slot.shape))
    # colouring: a permutation grouped by colour, no shared node inside a colour
    elems, off = P["elems"], P["color_off"]
    assert np.array_equal(np.sort(elems), np.arange(n_el)) and off[0] == 0 and off[-1] == n_el
    for c in range(len(off) - 1):
        nodes = conn[elems[off[c]:off[c + 1]]].ravel()
        assert np.unique(nodes).size == nodes.size, c
    # first writers: one per block, at its first touch in launch order
    order = (elems[:, None] * 64 + np.arange(64)[None, :]).ravel()
    s_launch = slot.reshape(-1)[order]
    _, first_idx = np.unique(s_launch, return_index=True)
    expect = np.zeros(order.size, bool)
    expect[first_idx] = True
    assert np.array_equal(first.reshape(-1)[order], expect)
    assert first.sum() == P["cols"].size
    return len(off) - 1


def test_structured_box_eight_colours(driver):
    mesh = inputs.box_mesh(5, 4, 3)
    P, err = _run(driver, mesh.n_nodes, mesh.conn)
    assert P is not None, err
    assert _check(P, mesh.n_nodes, mesh.conn) == 8


@pytest.mark.parametrize("case", ["distorted", "plate", "shuffled"])
def test_unstructured_meshes(driver, case):
    if case == "distorted":
        mesh = inputs.distorted_box_mesh(4, seed=3, amp=0.2)
        conn = mesh.conn
    elif case == "plate":
        mesh, _, _, _ = inputs.config1_problem(nx=24, ny=12, nz=2, n_steps=2)
        conn = mesh.conn
    else:
        mesh = inputs.box_mesh(4, 4, 2)
        conn = mesh.conn[np.random.default_rng(5).permutation(mesh.n_el)]
    P, err = _run(driver, mesh.n_nodes, conn)
    assert P is not None, err
    assert _check(P, mesh.n_nodes, np.asarray(conn, dtype=np.int64)) >= 8


def test_malformed_meshes_refused(driver):
    mesh = inputs.box_mesh(2, 2, 2)
    bad = mesh.conn.copy()
    bad[3, 5] = mesh.n_nodes
    assert _run(driver, mesh.n_nodes, bad) == (None, "conn[29] out of range")
    bad = mesh.conn.copy()
    bad[1, 2] = bad[1, 0]
    P, err = _run(driver, mesh.n_nodes, bad)
    assert P is None and "repeats a node" in err
    P, err = _run(driver, mesh.n_nodes + 1, mesh.conn)
    assert P is None and err == f"node {mesh.n_nodes} belongs to no element"
