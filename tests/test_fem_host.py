"""The library's host-side FEM data for the coupled loop's solves (fem_host.h), on the CPU.

The builder is plain C++; the test compiles it with g++ into a small harness, runs it on
synthetic grids and checks its CSR matrices against the oracle's matrix-free Galerkin
operators (the same products for random vectors), its element contributions against the
values they sum to, and its boundary data against closed forms of the channel geometry.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1006_0532_gb300 import synth
from helpers import base_params

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1006_0532_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("femh") / "harness")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "fem_host_harness.cpp")], check=True)
    return exe


def element_frame(g):
    """Vertices with x taken as the image nearest to vertex A, and twice the signed area."""
    x = g.node_xy[g.tri, 0].copy()
    if g.period_x > 0:
        for k in (1, 2):
            x[:, k] -= g.period_x * np.round((x[:, k] - x[:, 0]) / g.period_x)
    y = g.node_xy[g.tri, 1].copy()
    a2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    return x, y, a2


def run(harness, g, tmp_path):
    x, y, a2 = element_frame(g)
    d = str(tmp_path)
    g.tri.astype(np.int32).tofile(os.path.join(d, "tri"))
    g.edge_tag.astype(np.int8).tofile(os.path.join(d, "tag"))
    x.tofile(os.path.join(d, "vx"))
    y.tofile(os.path.join(d, "vy"))
    a2.tofile(os.path.join(d, "area2"))
    rc = subprocess.run([harness, d, str(g.nn), str(g.tri.shape[0])]).returncode
    if rc:
        return rc, None
    rd = lambda n, t: np.fromfile(os.path.join(d, n), t)
    m = {n: rd(n, np.int32) for n in ("row", "col", "dpos", "cptr", "clist", "boff", "bnb")}
    m.update({n: rd(n, np.float64) for n in ("mval", "kval", "kdiag", "mlump", "nrm", "blen", "scal")})
    m["cls"] = rd("cls", np.int8)
    return 0, m


def csr_apply(m, val, v):
    row, col = m["row"], m["col"]
    out = np.zeros(row.size - 1)
    for n in range(row.size - 1):
        out[n] = val[row[n]:row[n + 1]] @ v[col[row[n]:row[n + 1]]]
    return out


def grids():
    ch = synth.workload("channel_2k")["grid"]
    fs = synth.Grid(node_xy=ch.node_xy, tri=ch.tri, edge_tag=np.where(ch.edge_tag == 1, 2, ch.edge_tag).astype(np.int8),
                    period_x=ch.period_x)
    return [("channel", ch), ("freeslip", fs), ("canyon", synth.canyon_workload("canyon_2k")["grid"])]


@pytest.mark.parametrize("name,g", grids())
def test_csr_matrices_equal_the_oracles_operators(harness, tmp_path, name, g):
    """M x and K x from the CSR arrays equal the oracle's element-by-element products for
    random x (periodic seam included); the diagonal positions point at the diagonal; every
    entry's contributions are its (element, a, b) pairs with the right nodes."""
    rc, m = run(harness, g, tmp_path)
    assert rc == 0
    o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = rng.normal(size=g.nn)
        for which, key in ((0, "mval"), (1, "kval")):
            want = o.fem_apply(which, v)
            got = csr_apply(m, m[key], v)
            assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    row, col = m["row"], m["col"]
    assert np.array_equal(col[m["dpos"]], np.arange(g.nn))
    assert np.array_equal(m["kdiag"], m["kval"][m["dpos"]])
    for k in range(0, col.size, 7):
        r = np.searchsorted(row, k, side="right") - 1
        for code in m["clist"][m["cptr"][k]:m["cptr"][k + 1]]:
            e, a, b = code // 9, (code % 9) // 3, code % 3
            assert g.tri[e, a] == r and g.tri[e, b] == col[k]
    assert m["cptr"][-1] == 9 * g.tri.shape[0]


def test_channel_boundary_data_closed_forms(harness, tmp_path):
    """Walls at y = 0 and 1 of the periodic channel (length 2): outward normals (0, -1) and
    (0, 1), every wall node of class 1 and no other node classed; the wall edges at the
    nodes add up to twice the total wall length; the shapefunction integrals add up to the
    area 2; C_xi = 2.3.  The same grid with free-slip rows: class 2 there, C_xi = 1."""
    g = synth.workload("channel_2k")["grid"]
    rc, m = run(harness, g, tmp_path)
    assert rc == 0
    y = g.node_xy[:, 1]
    bottom, top = y == 0.0, y == 1.0
    assert np.array_equal(m["cls"], np.where(bottom | top, 1, 0).astype(np.int8))
    nrm = m["nrm"].reshape(-1, 2)
    assert np.allclose(nrm[bottom], [0.0, -1.0], atol=1e-15) and np.allclose(nrm[top], [0.0, 1.0], atol=1e-15)
    assert np.abs(nrm[~(bottom | top)]).max() == 0.0
    assert abs(m["blen"].sum() - 2 * 2 * 2.0) < 1e-12
    assert abs(m["mlump"].sum() - 2.0) < 1e-12 and abs(m["scal"][0] - 2.0) < 1e-12
    assert m["scal"][1] == 2.3
    fs = synth.Grid(node_xy=g.node_xy, tri=g.tri, edge_tag=np.where(g.edge_tag == 1, 2, g.edge_tag).astype(np.int8),
                    period_x=g.period_x)
    rc, m2 = run(harness, fs, tmp_path)
    assert rc == 0
    assert np.array_equal(m2["cls"], np.where(bottom | top, 2, 0).astype(np.int8))
    assert m2["boff"][-1] == 0 and m2["scal"][1] == 1.0


def test_a_node_of_no_element_is_refused(harness, tmp_path):
    """A grid with a node that no element uses has no equation for it: the builder refuses."""
    g = synth.workload("channel_2k")["grid"]
    extra = synth.Grid(node_xy=np.vstack([g.node_xy, [[0.5, 0.5]]]), tri=g.tri, edge_tag=g.edge_tag,
                       period_x=g.period_x)
    rc, _ = run(harness, extra, tmp_path)
    assert rc == 4
