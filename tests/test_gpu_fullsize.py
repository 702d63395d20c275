"""Parity at the benchmark's full size (50,000 triangles, 500 particles per element, 25.0M
particles), in the benchmark's launch configuration (autotuned): the oracle follows a sample
of elements from the same initialisation (same ids and draws) through the statistics and
one step; the GPU runs the whole workload."""
import numpy as np
import pytest

import oracle
from paper_1006_0532_gb300 import synth
from helpers import period_diff

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
from paper_1006_0532_gb300 import _binding as B  # noqa: E402

PPE = 500


def _sample_elements(g, n_wall=4, n_inner=12, seed=11):
    rng = np.random.default_rng(seed)
    wall = np.where((g.edge_tag != 0).any(axis=1))[0]
    inner = np.setdiff1d(np.arange(g.ne), wall)
    return np.sort(np.concatenate([rng.choice(wall, n_wall, replace=False),
                                   rng.choice(inner, n_inner, replace=False)]))


def _rel(a, b, scale):
    return np.abs(a - b) / np.maximum(np.abs(b), scale)


def _thin_cells(g):
    """Elements thinner than 2e-3 (the graded cells near the walls)."""
    xy = g.node_xy[g.tri]                                  # [ne, 3, 2]
    dx = xy[:, [1, 2, 0], 0] - xy[:, :, 0]
    dx = (dx + 0.5 * g.period_x) % g.period_x - 0.5 * g.period_x
    dy = xy[:, [1, 2, 0], 1] - xy[:, :, 1]
    area2 = np.abs(dx[:, 0] * dy[:, 2] - dy[:, 0] * dx[:, 2])
    height = area2 / np.sqrt(dx ** 2 + dy ** 2).max(axis=1)
    return height < 2e-3


def test_full_size_sampled_parity_f64():
    """FP64 form: the oracle follows the sampled elements from the same initialisation (same
    ids and draws) through the statistics and one step: states within 1e-12, element
    indices, pointers and bins exact, element moments within 1e-10."""
    w = synth.workload("channel_50k")
    g = w["grid"]
    P = dict(w["params"], minnpel=0)           # particle-number control is global: off
    F = w["fields"]
    c = B.Context(dict(P, precision=0, sort_every=8))
    c.set_grid(g)
    c.set_fields(F)
    c.init_particles(PPE)
    assert c.np_ == PPE * g.ne == 25_000_000
    elems = _sample_elements(g)
    o = oracle.Oracle(g, P, F)
    o.init_elements(PPE, elems)
    ids = o.pids().astype(np.int64)
    sg, so = c.get_particles(), o.get_particles()
    assert np.array_equal(sg["elem"][ids], so["elem"])
    _check_states(g, sg, so, ids, np.ones(ids.shape[0], bool), 1e-12)
    eg, cg = c.element_stats()
    eo, co = o.element_stats()
    assert np.array_equal(cg[elems], co[elems])
    sc = np.sqrt(np.mean(eo[elems] ** 2, axis=0)) + 1e-300
    assert _rel(eg[elems], eo[elems], sc).max() <= 1e-10
    assert np.array_equal(sg["cp"][ids], so["cp"])
    vg, gg = c.bins()
    vo, go = o.bins()
    assert np.array_equal(gg[elems], go[elems])
    assert _rel(vg[elems], vo[elems], 1.0).max() <= 1e-12
    c.autotune(w["dt"])
    c.step(w["dt"])
    o.step(w["dt"])
    sg, so = c.get_particles(), o.get_particles()
    diff = sg["elem"][ids] != so["elem"]
    for i in np.where(diff)[0]:          # a particle on a shared edge may sit in either element
        assert o.lam(int(sg["elem"][ids][i]), so["x"][i], so["y"][i]).min() > -1e-12
    assert diff.sum() == 0
    _check_states(g, sg, so, ids, ~diff, 1e-12)
    assert c.check() == 0


def _check_states(g, sg, so, ids, mask, tol, worst=None, cls=None):
    dx = np.abs(period_diff(sg["x"][ids][mask], so["x"][mask], g.period_x))
    sx = np.sqrt(np.mean(so["x"] ** 2))
    assert (dx / sx).max() <= tol, ("x", float((dx / sx).max()))
    for k in ("y", "u", "v", "w", "om", "psi"):
        r = _rel(sg[k][ids][mask], so[k][mask], np.sqrt(np.mean(so[k] ** 2)) or 1.0)
        if r.size:
            if worst is not None:
                for c in (False, True):
                    m = cls == c
                    if m.any():
                        worst[(k, c)] = max(worst.get((k, c), 0.0), float(r[m].max()))
            assert r.max() <= tol, (k, float(r.max()))


def test_full_size_sampled_parity_f32():
    """FP32 form at the benchmark's size, one step from identical inputs: the oracle runs in
    FP64 from the GPU's own FP32-form state (FP32 velocities, frequencies and scalars; the
    positions' FP32 hi + lo pairs, exact in FP64) and the fields rounded to FP32, for the
    particles of sampled elements (4 at the walls).  Statistics of that state: counts,
    pointers and effective bins exact, element moments and conditional means within 1e-6.
    After one step every state within 1e-5, the graded wall cells included; exempt and
    counted are particles whose element differs (they lie on a shared edge to rounding) and
    those whose wall decision differs (the uniform and Eq. 53's probability agree to FP32
    rounding: one side stops the particle, U = 0)."""
    w = synth.workload("channel_50k")
    g = w["grid"]
    P = dict(w["params"], minnpel=0)           # particle-number control is global: off
    F = w["fields"].astype(np.float32).astype(np.float64)
    c = B.Context(dict(P, precision=1, sort_every=8))
    c.set_grid(g)
    c.set_fields(F)
    c.init_particles(PPE)
    assert c.np_ == PPE * g.ne == 25_000_000
    elems = _sample_elements(g)
    sg = c.get_particles()
    ids = np.where(np.isin(sg["elem"], elems))[0]
    thin = _thin_cells(g)
    o = oracle.Oracle(g, P, F)
    o.set_particles({k: sg[k][ids] for k in ("x", "y", "u", "v", "w", "om", "psi", "elem")}, 0, pid=ids)
    so = o.get_particles()
    assert np.array_equal(sg["elem"][ids], so["elem"])
    # statistics of identical values: exact pointers and bins, moments to FP32 accumulation
    assert np.array_equal(sg["cp"][ids], so["cp"])
    eg, cg = c.element_stats()
    eo, co = o.element_stats()
    assert np.array_equal(cg[elems], co[elems])
    sc = np.sqrt(np.mean(eo[elems] ** 2, axis=0)) + 1e-300
    assert _rel(eg[elems], eo[elems], sc).max() <= 1e-6
    vg, gg = c.bins()
    vo, go = o.bins()
    assert np.array_equal(gg[elems], go[elems])
    assert _rel(vg[elems], vo[elems], 1.0).max() <= 1e-6
    # one step in the benchmark's launch configuration
    c.autotune(w["dt"])
    c.step(w["dt"])
    o.step(w["dt"])
    sg, so = c.get_particles(), o.get_particles()
    diff = sg["elem"][ids] != so["elem"]
    for i in np.where(diff)[0]:          # a particle on a shared edge may sit in either element
        assert o.lam(int(sg["elem"][ids][i]), so["x"][i], so["y"][i]).min() > -1e-6
    stop_g = (sg["u"][ids] == 0) & (sg["v"][ids] == 0) & (sg["w"][ids] == 0)
    stop_o = (so["u"] == 0) & (so["v"] == 0) & (so["w"] == 0)
    wall_diff = stop_g != stop_o
    exempt = diff | wall_diff
    assert diff.sum() <= 5 and wall_diff.sum() <= 10, (int(diff.sum()), int(wall_diff.sum()))
    worst = {}
    _check_states(g, sg, so, ids, ~exempt, 1e-5, worst, thin[so["elem"][~exempt]])
    assert thin[so["elem"]].sum() > 1000          # the sample covers the graded wall cells
    assert c.check() == 0
    print("largest relative state errors (quantity, thin cell):", worst,
          "exempt:", int(diff.sum()), int(wall_diff.sum()))


def test_canyon_full_size_sampled_parity_f64():
    """The street canyon at full size (about 200,000 triangles graded to y+ = 1 at the floor,
    the cavity walls and corners; 100 particles per element, about 20M), FP64 form: the
    oracle follows sampled elements (8 at walls, the free-slip top or corners) from the same
    initialisation through the statistics and one step: states within 1e-12, element
    indices and conditioning pointers exact."""
    w = synth.canyon_workload("canyon_200k")
    g = w["grid"]
    P = dict(w["params"], minnpel=0)           # particle-number control is global: off
    c = B.Context(dict(P, precision=0, sort_every=8))
    c.set_grid(g)
    c.set_fields(w["fields"])
    c.init_particles(w["ppe"])
    elems = _sample_elements(g, n_wall=8, n_inner=8, seed=12)
    o = oracle.Oracle(g, P, w["fields"])
    o.init_elements(w["ppe"], elems)
    ids = o.pids().astype(np.int64)
    sg, so = c.get_particles(), o.get_particles()
    assert np.array_equal(sg["elem"][ids], so["elem"])
    assert np.abs(period_diff(sg["x"][ids], so["x"], g.period_x)).max() <= 1e-12 * g.period_x
    for k in ("y", "u", "v", "w", "om", "psi"):
        r = _rel(sg[k][ids], so[k], np.sqrt(np.mean(so[k] ** 2)) or 1.0).max()
        assert r <= 1e-12, (k, float(r))
    assert np.array_equal(sg["cp"][ids], so["cp"])
    eg, cg = c.element_stats()
    eo, co = o.element_stats()
    assert np.array_equal(cg[elems], co[elems])
    sc = np.sqrt(np.mean(eo[elems] ** 2, axis=0)) + 1e-300
    assert _rel(eg[elems], eo[elems], sc).max() <= 1e-10
    c.autotune(w["dt"])
    c.step(w["dt"])
    o.step(w["dt"])
    sg, so = c.get_particles(), o.get_particles()
    diff = sg["elem"][ids] != so["elem"]
    for i in np.where(diff)[0]:          # a particle on a shared edge may sit in either element
        assert o.lam(int(sg["elem"][ids][i]), so["x"][i], so["y"][i]).min() > -1e-12
    assert diff.sum() <= 2
    m = ~diff
    assert np.abs(period_diff(sg["x"][ids][m], so["x"][m], g.period_x)).max() <= 1e-12 * g.period_x
    for k in ("y", "u", "v", "w", "om", "psi"):
        r = _rel(sg[k][ids][m], so[k][m], np.sqrt(np.mean(so[k] ** 2)) or 1.0).max()
        assert r <= 1e-12, (k, float(r))
    d = o.diag()
    assert d["wall_hits"] > 0 or d["freeslip_hits"] > 0
    assert c.check() == 0
