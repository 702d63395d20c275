"""The coupled loop's kernel arithmetic (eulerian_ops.h), run on the CPU against the oracle.

Every kernel of the coupled loop maps its threads onto one inline function per node, entry or
element.  The test compiles those functions with g++ into a harness that applies them over
a whole grid in the kernels' order.  It compares the results with the oracle: Eq. 12's
right-hand side and length scale, Eq. 59's wall values, the assembled matrix M + L_e^2 K,
Eq. 33's source and Eq. 61's flux, the Galerkin load, and both solves driven through the
library's per-node conjugate-gradient functions.  What this leaves to the GPU tests is the
launch structure and the two-stage sums around these functions.
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
    exe = str(tmp_path_factory.mktemp("eops") / "harness")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "eulerian_ops_harness.cpp")], check=True)
    return exe


def random_fields(g, seed):
    rng = np.random.default_rng(seed)
    F = synth.uniform_fields(g.nn)
    A = rng.normal(size=(g.nn, 3, 3))
    R = A @ A.transpose(0, 2, 1) * rng.uniform(0.05, 1.0, size=(g.nn, 1, 1))
    F[:, 23], F[:, 24], F[:, 25] = R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]
    F[:, 26], F[:, 27], F[:, 28] = R[:, 0, 1], R[:, 0, 2], R[:, 1, 2]
    F[:, 5:11] = rng.normal(size=(g.nn, 6))
    F[:, 11:14] = rng.normal(size=(g.nn, 3))
    F[:, 29] = rng.uniform(0.5, 3.0, size=g.nn)
    return F


def run(harness, g, F, params, ustar, P, dt, Cp, d):
    x = g.node_xy[g.tri, 0].copy()
    for k in (1, 2):
        x[:, k] -= g.period_x * np.round((x[:, k] - x[:, 0]) / g.period_x)
    y = g.node_xy[g.tri, 1].copy()
    a2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    files = dict(tri=g.tri.astype(np.int32), tag=g.edge_tag.astype(np.int8), vx=x, vy=y, area2=a2,
                 fields=np.ascontiguousarray(F, dtype=np.float64),
                 consts=np.array([params[k] for k in ("C1", "C2", "Cv", "gamma5", "CL", "Ceta", "CT", "nu")]
                                 + [dt, Cp, 1e-13, 0.0]),
                 ustar=np.ascontiguousarray(ustar, dtype=np.float64), P=np.ascontiguousarray(P, dtype=np.float64))
    for k, v in files.items():
        v.tofile(os.path.join(d, k))
    subprocess.run([harness, d, str(g.nn), str(g.tri.shape[0])], check=True)
    rd = lambda n, t: np.fromfile(os.path.join(d, n), t)
    out = {n: rd(n, np.float64) for n in ("rhs", "L", "x", "aval", "src", "flux", "b", "wp", "dP")}
    out["iters"] = rd("iters", np.int32)
    out.update(fixed=rd("fixed", np.uint8), bad=rd("bad", np.int32), row=rd("row", np.int32),
               col=rd("col", np.int32))
    return out


def csr_apply(row, col, val, v):
    return np.array([val[row[n]:row[n + 1]] @ v[col[row[n]:row[n + 1]]] for n in range(row.size - 1)])


def cases():
    ch = synth.workload("channel_2k")
    cy = synth.canyon_workload("canyon_2k")
    return [("channel", ch["grid"], ch["params"]), ("canyon", cy["grid"], cy["params"])]


@pytest.mark.parametrize("name,g,params", cases())
def test_kernel_arithmetic_matches_oracle(harness, tmp_path, name, g, params):
    F = random_fields(g, 3)
    p = base_params(**{k: params[k] for k in ("nu",)}, period_x=g.period_x)
    o = oracle.Oracle(g, p, F)
    rng = np.random.default_rng(5)
    ustar, P = rng.normal(size=(g.nn, 3)), rng.normal(size=g.nn)
    dt, Cp = 1e-4, 5e-5
    r = run(harness, g, F, p, ustar, P, dt, Cp, str(tmp_path))
    assert r["bad"].tolist() == [0, 0]
    # Eqs. 12-18
    ro, Lo = o.wp_rhs()
    rhs = r["rhs"].reshape(9, g.nn).T.reshape(g.nn, 3, 3)
    assert np.abs(rhs - ro).max() <= 1e-14 * np.abs(ro).max()
    assert np.abs(r["L"] - Lo).max() <= 1e-14 * np.abs(Lo).max()
    # Eq. 59 and the symmetry conditions: fixed components carry the oracle solution's values
    fixed = r["fixed"].reshape(9, g.nn).T.astype(bool)
    xs = r["x"].reshape(9, g.nn).T
    wp, _ = o.wp_solve(ro, Lo, tol=1e-12)
    wp = wp.reshape(g.nn, 9)
    assert fixed.any()
    assert np.abs(xs[fixed] - wp[fixed]).max() <= 1e-15 * max(np.abs(wp).max(), 1.0)
    # the assembled M + L_e^2 K against the oracle's element-wise operator
    for _ in range(2):
        v = rng.normal(size=g.nn)
        want = o.wp_apply(Lo, v)
        got = csr_apply(r["row"], r["col"], r["aval"], v)
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # Eq. 33's source and Eq. 61's increment flux
    so, fo = o.pressure_rhs(ustar, P, dt, Cp)
    assert np.abs(r["src"] - so).max() <= 1e-13 * np.abs(so).max()
    assert np.abs(r["flux"] - fo).max() <= 1e-13 * max(np.abs(fo).max(), 1.0)
    assert np.abs(fo).max() > 0.0
    # the Galerkin load: -M src plus the wall-edge integrals (zero away from no-slip nodes)
    edge = r["b"] + o.fem_apply(0, r["src"])
    wall = np.zeros(g.nn, bool)
    for kk in range(3):
        msk = g.edge_tag[:, kk] == 1
        wall[g.tri[msk, (kk + 1) % 3]] = True
        wall[g.tri[msk, (kk + 2) % 3]] = True
    assert np.abs(edge[~wall]).max() <= 1e-12 * np.abs(r["b"]).max()
    assert np.abs(edge[wall]).max() > 0.0


@pytest.mark.parametrize("name,g,params", cases())
def test_solves_through_the_kernel_functions_match_oracle(harness, tmp_path, name, g, params):
    """Both solves driven through pcg_node, pcg_scalars, pcg_direction and pcg_trivial
    (tolerance 1e-13, zero initial guess) reproduce the oracle's solutions and iteration
    counts: the same stopping rule, masks and zero-load rule."""
    F = random_fields(g, 4)
    p = base_params(**{k: params[k] for k in ("nu",)}, period_x=g.period_x)
    o = oracle.Oracle(g, p, F)
    rng = np.random.default_rng(6)
    ustar, P = rng.normal(size=(g.nn, 3)), rng.normal(size=g.nn)
    r = run(harness, g, F, p, ustar, P, 1e-4, 5e-5, str(tmp_path))
    ro, Lo = o.wp_rhs()
    wo, io = o.wp_solve(ro, Lo, tol=1e-13)
    wg = r["wp"].reshape(9, g.nn).T.reshape(g.nn, 3, 3)
    assert np.abs(wg - wo).max() <= 1e-10 * np.abs(wo).max()
    assert abs(int(r["iters"][0]) - io) <= 1
    so, fo = o.pressure_rhs(ustar, P, 1e-4, 5e-5)
    do, ip = o.pressure_solve(so, fo, tol=1e-13)
    assert np.abs(r["dP"] - do).max() <= 1e-9 * np.abs(do).max()
    assert abs(int(r["iters"][1]) - ip) <= 1
