"""The host-side assembly set-up (csrc/pattern.cpp, compiled here by the host C++ compiler
without CUDA) against an independent numpy construction: the block-CSR pattern (one 3x3
block per pair of nodes sharing an element, sorted columns, the diagonal slot), the element
colouring (no two elements of a colour share a node; 8 colours on a structured hex mesh),
the launch order (one colour of one slab of K rows per launch, slabs in row order), the
element-to-block slot map, and the first-writer flags (exactly one per block, on its first
touch in launch order); malformed meshes are refused with a message.  Also the cut of the
rows into the chunks that the streamed CG copies into shared memory (stream_chunks)."""
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
  long long nn, ne, plan[4];
  if (fread(&nn, 8, 1, in) != 1 || fread(&ne, 8, 1, in) != 1 || fread(plan, 8, 4, in) != 4) return 3;
  std::vector<int32_t> conn(ne * 8);
  if (fread(conn.data(), 4, conn.size(), in) != conn.size()) return 3;
  fclose(in);
  hfe::Pattern P;
  std::string err;
  hfe::SlabPlan sp;
  sp.min_blocks = plan[0]; sp.max_blocks = plan[1]; sp.resident_ctas = plan[2]; sp.el_per_cta = plan[3];
  if (!hfe::build_pattern(nn, ne, conn.data(), sp, P, err)) {
    fprintf(stderr, "%s\n", err.c_str());
    return 2;
  }
  FILE* out = fopen(argv[2], "wb");
  put(out, P.rowptr); put(out, P.cols); put(out, P.diag_slot); put(out, P.slot);
  put(out, P.elems); put(out, P.launch_off);
  std::vector<long long> ns{(long long)P.n_slabs, (long long)P.slab_blocks};
  put(out, ns);
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


def _run(driver, n_nodes, conn, slab_blocks=0, plan=None):
    """plan = (min_blocks, max_blocks, resident_ctas, el_per_cta); slab_blocks > 0 fixes the size."""
    exe, d = driver
    inp, out = d / "conn.bin", d / "pattern.bin"
    if plan is None:
        plan = (slab_blocks, slab_blocks, 1, 16)
    with open(inp, "wb") as f:
        np.array([n_nodes, conn.shape[0], *plan], dtype=np.int64).tofile(f)
        np.ascontiguousarray(conn, dtype=np.int32).tofile(f)
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True)
    if r.returncode != 0:
        return None, r.stderr.strip()
    buf = open(out, "rb").read()
    parts, off = [], 0
    for dt in (np.int64, np.int32, np.int64, np.int32, np.int32, np.int64, np.int64):
        n = int(np.frombuffer(buf, np.int64, 1, off)[0])
        off += 8
        parts.append(np.frombuffer(buf, dt, n, off).copy())
        off += n * np.dtype(dt).itemsize
    return dict(zip(("rowptr", "cols", "diag_slot", "slot", "elems", "launch_off", "n_slabs"), parts)), ""


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
    # launch ranges: a permutation cut into ranges, no shared node inside a range
    elems, off = P["elems"], P["launch_off"]
    assert np.array_equal(np.sort(elems), np.arange(n_el)) and off[0] == 0 and off[-1] == n_el
    assert np.all(np.diff(off) > 0)
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


def _colours(conn):
    """Greedy colouring in element order: an element takes the smallest colour that no earlier
    element sharing a node has."""
    n_el = conn.shape[0]
    colour = np.full(n_el, -1)
    by_node = {}
    for e in range(n_el):
        used = {colour[o] for n in conn[e] for o in by_node.get(int(n), [])}
        c = 0
        while c in used:
            c += 1
        colour[e] = c
        for n in conn[e]:
            by_node.setdefault(int(n), []).append(e)
    return colour


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


@pytest.mark.parametrize("slab_blocks", [60, 250, 10 ** 9])
def test_slab_launch_order(driver, slab_blocks):
    """Launches ordered by slab (slab_blocks consecutive K blocks, an element in the slab of
    the first block of its lowest node's row), then by colour; one (slab, colour) per launch."""
    mesh = inputs.box_mesh(6, 5, 4)
    conn = np.asarray(mesh.conn, dtype=np.int64)
    P, err = _run(driver, mesh.n_nodes, mesh.conn, slab_blocks)
    assert P is not None, err
    n_launch = _check(P, mesh.n_nodes, conn)
    colour = _colours(conn)
    slab = P["rowptr"][conn.min(axis=1)] // slab_blocks
    assert int(P["n_slabs"][0]) == slab.max() + 1
    assert int(P["n_slabs"][1]) == (0 if slab_blocks == 0 else slab_blocks)
    elems, off = P["elems"], P["launch_off"]
    key = slab[elems] * 64 + colour[elems]
    assert np.all(np.diff(key) >= 0)                     # slabs in order, colours within a slab
    for c in range(n_launch):                            # one (slab, colour) per launch, all of it
        k = np.unique(key[off[c]:off[c + 1]])
        assert k.size == 1 and np.count_nonzero(key == k[0]) == off[c + 1] - off[c]
    assert n_launch == np.unique(slab * 64 + colour).size
    if slab_blocks == 10 ** 9:
        assert n_launch == 8 and int(P["n_slabs"][0]) == 1
    else:
        assert int(P["n_slabs"][0]) > 1
    # within a launch the elements keep their id order
    for c in range(n_launch):
        assert np.all(np.diff(elems[off[c]:off[c + 1]]) > 0)


def _waves(conn, rowptr, colour, sb, resident, epc):
    first = rowptr[conn.min(axis=1)]
    _, cnt = np.unique((first // sb) * 64 + colour, return_counts=True)
    return int(np.sum(-(-(-(-cnt // epc)) // resident)))


def test_slab_size_planner(driver):
    """With a size range, the planner takes, among the 32 sizes min + (max - min) k / 31, one
    with the fewest waves of resident CTAs (sum over launches of ceil(CTAs / resident)), the
    largest such size; the launch order is then the fixed-size order of that size."""
    mesh = inputs.box_mesh(9, 8, 7)
    conn = np.asarray(mesh.conn, dtype=np.int64)
    colour = _colours(conn)
    lo, hi, res, epc = 300, 1200, 3, 4
    P, err = _run(driver, mesh.n_nodes, mesh.conn, plan=(lo, hi, res, epc))
    assert P is not None, err
    sizes = [lo + (hi - lo) * k // 31 for k in range(32)]
    waves = {sb: _waves(conn, P["rowptr"], colour, sb, res, epc) for sb in sizes}
    best = min(waves.values())
    chosen = int(P["n_slabs"][1])
    assert chosen == max(sb for sb in sizes if waves[sb] == best)
    assert len(set(waves.values())) > 1                     # the choice is not a trivial one
    F, _ = _run(driver, mesh.n_nodes, mesh.conn, chosen)
    for key in ("elems", "launch_off", "slot"):
        assert np.array_equal(P[key], F[key]), key
    _check(P, mesh.n_nodes, conn)


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


CHUNK_DRIVER = r"""
#include <cstdio>
#include <string>
#include <vector>
#include "pattern.h"
int main(int argc, char** argv) {
  FILE* in = fopen(argv[1], "rb");
  long long nn, par[2];
  if (fread(&nn, 8, 1, in) != 1 || fread(par, 8, 2, in) != 2) return 3;
  std::vector<int64_t> rowptr(nn + 1);
  if (fread(rowptr.data(), 8, rowptr.size(), in) != rowptr.size()) return 3;
  fclose(in);
  std::vector<int32_t> out;
  hfe::stream_chunks(rowptr.data(), nn, (int)par[0], (int)par[1], out);
  FILE* o = fopen(argv[2], "wb");
  long long n = (long long)out.size();
  fwrite(&n, 8, 1, o);
  fwrite(out.data(), 4, out.size(), o);
  fclose(o);
  return 0;
}
"""


@pytest.fixture(scope="module")
def chunk_driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("chunks")
    (d / "driver.cpp").write_text(CHUNK_DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(d / "driver.cpp"),
                    os.path.join(CSRC, "pattern.cpp"), "-o", str(exe)], check=True)
    return exe, d


def _chunks(chunk_driver, rowptr, max_rows, max_blocks):
    exe, d = chunk_driver
    inp, out = d / "rowptr.bin", d / "chunks.bin"
    with open(inp, "wb") as f:
        np.array([len(rowptr) - 1, max_rows, max_blocks], dtype=np.int64).tofile(f)
        np.asarray(rowptr, dtype=np.int64).tofile(f)
    subprocess.run([str(exe), str(inp), str(out)], check=True)
    buf = open(out, "rb").read()
    n = int(np.frombuffer(buf, np.int64, 1, 0)[0])
    return np.frombuffer(buf, np.int32, n, 8).copy()


@pytest.mark.parametrize("max_rows,max_blocks", [(32, 764), (32, 100), (7, 60), (1, 27)])
def test_stream_chunks_cover_rows_within_limits(chunk_driver, max_rows, max_blocks):
    """The rows of the streamed CG cut into chunks: consecutive, covering every row once, each
    within max_rows rows and max_blocks blocks, and greedy (one more row would break a limit)."""
    mesh, _, _, _ = inputs.config1_problem(nx=24, ny=12, nz=2, n_steps=2)
    conn = np.asarray(mesh.conn, dtype=np.int64)
    pairs = np.unique(np.stack([np.repeat(conn, 8, axis=1).ravel(), np.tile(conn, (1, 8)).ravel()], 1), axis=0)
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(pairs[:, 0], minlength=mesh.n_nodes))])
    c = _chunks(chunk_driver, rowptr, max_rows, max_blocks)
    assert c[0] == 0 and c[-1] == mesh.n_nodes and np.all(np.diff(c) > 0)
    rows = np.diff(c)
    blocks = rowptr[c[1:]] - rowptr[c[:-1]]
    assert rows.max() <= max_rows and blocks.max() <= max_blocks
    for k in range(len(c) - 2):   # every chunk but the last stops because the next row breaks a limit
        nxt_rows, nxt_blocks = rows[k] + 1, rowptr[c[k + 1] + 1] - rowptr[c[k]]
        assert nxt_rows > max_rows or nxt_blocks > max_blocks


def test_stream_chunks_empty_when_a_row_is_too_long(chunk_driver):
    rowptr = np.array([0, 5, 40, 45])
    assert _chunks(chunk_driver, rowptr, 32, 30).size == 0
    assert np.array_equal(_chunks(chunk_driver, rowptr, 32, 45), [0, 3])
    assert np.array_equal(_chunks(chunk_driver, rowptr, 2, 45), [0, 2, 3])
