"""GPU parity of the coupled loop's CUDA path (Eqs. 12-18, 33, 59, 61; Table 1).

Each test compares the CUDA path with the oracle on the same inputs in FP64; the solves use
the same stopping rule on both sides, so their results differ by the solver tolerance times
the conditioning, not by rounding alone.
"""
import numpy as np
import pytest

import oracle
from paper_1006_0532_gb300 import synth
from helpers import STATE_KEYS, base_params, period_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0532_gb300 import _binding as B  # noqa: E402


def gpu_ctx(grid, params, fields, precision=0):
    p = dict(params)
    p.setdefault("period_x", grid.period_x)
    p.update(precision=precision, sort_every=4)
    c = B.Context(p)
    c.set_grid(grid)
    c.set_fields(fields)
    return c


def both(grid, params, fields, precision=0):
    return oracle.Oracle(grid, params, fields), gpu_ctx(grid, params, fields, precision)


def rel(a, b):
    """Largest difference relative to the largest magnitude of the reference."""
    s = float(np.abs(b).max())
    return float(np.abs(a - b).max()) / (s if s > 0 else 1.0)


def random_fields(g, seed):
    """The channel fields with a random realisable <u_i u_j> and random mean gradients."""
    rng = np.random.default_rng(seed)
    F = synth.workload("channel_2k")["fields"].copy()
    A = rng.normal(size=(g.nn, 3, 3))
    R = A @ A.transpose(0, 2, 1) * rng.uniform(0.05, 1.0, size=(g.nn, 1, 1))
    F[:, 23], F[:, 24], F[:, 25] = R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]
    F[:, 26], F[:, 27], F[:, 28] = R[:, 0, 1], R[:, 0, 2], R[:, 1, 2]
    F[:, 5:11] = rng.normal(size=(g.nn, 6))
    F[:, 29] = rng.uniform(0.5, 3.0, size=g.nn)
    return F


def freeslip(g):
    tag = np.where(g.edge_tag == 1, 2, g.edge_tag).astype(np.int8)
    return synth.Grid(node_xy=g.node_xy, tri=g.tri, edge_tag=tag, period_x=g.period_x)


@pytest.fixture(scope="module")
def channel():
    w = synth.workload("channel_2k")
    return w, w["grid"]


def test_wp_rhs_matches_oracle(channel):
    """Eqs. 12-18 at every node: the kernel's contracted form of Eq. 13 against the oracle's
    term-by-term H_ijkl, and the length scale, within 1e-13."""
    w, g = channel
    F = random_fields(g, 1)
    o, c = both(g, w["params"], F)
    ro, Lo = o.wp_rhs()
    rg, Lg = c.wp_rhs()
    assert rel(rg, ro) < 1e-13
    assert rel(Lg, Lo) < 1e-13


@pytest.mark.parametrize("walls", [True, False])
def test_wp_solve_matches_oracle(channel, walls):
    """Eq. 12 by Galerkin FEM and Jacobi-PCG, with Eq. 59 at the walls or the symmetry
    conditions at free-slip rows: the same right-hand side and length scale, tolerance 1e-13
    on both sides, solutions within 1e-9 and iteration counts within two."""
    w, g = channel
    g = g if walls else freeslip(g)
    o, c = both(g, w["params"], w["fields"])
    rhs, L = o.wp_rhs()
    wo, io = o.wp_solve(rhs, L, tol=1e-13)
    wg, ig = c.wp_solve(rhs, L, tol=1e-13)
    assert rel(wg, wo) < 1e-9
    assert abs(ig - io) <= 2


def test_update_wp_matches_oracle(channel):
    """The coupled loop's update of slots 14-22 from their previous values; every other slot
    unchanged."""
    w, g = channel
    o, c = both(g, w["params"], w["fields"])
    o.update_wp(tol=1e-13)
    c.update_wp(tol=1e-13)
    fo, fg = o.fields(), c.fields()
    assert rel(fg[:, 14:23], fo[:, 14:23]) < 1e-9
    keep = [k for k in range(31) if not 14 <= k < 23]
    np.testing.assert_array_equal(fg[:, keep], w["fields"][:, keep])


def test_pressure_rhs_matches_oracle(channel):
    """Eq. 33's source (derivatives of Sect. 3.4) and Eq. 61's increment flux at the walls."""
    w, g = channel
    o, c = both(g, w["params"], w["fields"])
    rng = np.random.default_rng(3)
    ustar = rng.normal(size=(g.nn, 3))
    P = rng.normal(size=g.nn)
    so, fo = o.pressure_rhs(ustar, P, 1e-4, 5e-5)
    sg, fg = c.pressure_rhs(ustar, P, 1e-4, 5e-5)
    assert rel(sg, so) < 1e-12
    assert rel(fg, fo) < 1e-12
    assert np.abs(fo).max() > 0.0


def test_pressure_solve_matches_oracle(channel):
    """Eq. 33's singular Neumann-periodic system: the same load, zero-mean solutions within
    1e-8 of their largest value."""
    w, g = channel
    o, c = both(g, w["params"], w["fields"])
    rng = np.random.default_rng(4)
    src, flux = o.pressure_rhs(rng.normal(size=(g.nn, 3)), rng.normal(size=g.nn), 1e-4, 5e-5)
    do, io = o.pressure_solve(src, flux, tol=1e-13)
    dg, ig = c.pressure_solve(src, flux, tol=1e-13)
    assert rel(dg, do) < 1e-8
    assert abs(ig - io) <= 5


def test_solves_with_a_zero_load_return_zero(channel):
    w, g = channel
    c = gpu_ctx(freeslip(g), w["params"], w["fields"])
    rng = np.random.default_rng(5)
    wp, it = c.wp_solve(np.zeros((g.nn, 3, 3)), np.full(g.nn, 0.2), rng.normal(size=(g.nn, 3, 3)))
    assert it == 0 and np.abs(wp).max() == 0.0
    dP, it = c.pressure_solve(np.zeros(g.nn), np.zeros(g.nn), rng.normal(size=g.nn))
    assert it == 0 and np.abs(dP).max() == 0.0


def test_coupled_steps_match_oracle_f64(channel):
    """Two coupled steps (Table 1's order, C_p = dt/2) from the same particles and pressure:
    particle states within 1e-9, the pressure, its gradient slots and the elliptic-relaxation
    slots within 1e-7 of their largest values, nodal statistics within 1e-9."""
    w, g = channel
    o, c = both(g, w["params"], w["fields"])
    o.init_particles(25)
    c.init_particles(25)
    P0 = 0.2 * g.node_xy[:, 1] ** 2
    P = P0.copy()
    c.set_pressure(P0)
    dP = None
    for _ in range(2):
        dP, _, _ = o.coupled_step(w["dt"], P, dP, Cp=0.5 * w["dt"], tol=1e-13)
        c.coupled_step(w["dt"], Cp=0.5 * w["dt"], tol=1e-13)
    so, sg = o.get_particles(), c.get_particles()
    diff = sg["elem"] != so["elem"]
    assert diff.sum() <= 2
    for k in STATE_KEYS:
        a, b = sg[k][~diff], so[k][~diff]
        d = np.abs(period_diff(a, b, g.period_x)) if k == "x" else np.abs(a - b)
        assert float(d.max()) <= 1e-9 * max(float(np.abs(b).max()), 1e-300), k
    Pg, dPg = c.pressure()
    assert rel(Pg, P) < 1e-7 and rel(dPg, dP) < 1e-7
    fo, fg = o.fields(), c.fields()
    for sl in (slice(3, 5), slice(14, 23)):
        assert rel(fg[:, sl], fo[:, sl]) < 1e-7
    assert rel(c.nodal_stats(), o.nodal_stats()) < 1e-9
    assert c.check() == 0


def test_coupled_steps_fp32_stay_bounded(channel):
    """The FP32 form's coupled steps (FP64 solves) stay finite with a bounded increment."""
    w, g = channel
    c = gpu_ctx(g, w["params"], w["fields"], precision=1)
    c.init_particles(25)
    peaks = []
    for _ in range(4):
        c.coupled_step(w["dt"], Cp=0.5 * w["dt"], tol=1e-10)
        peaks.append(float(np.abs(c.pressure()[1]).max()))
    st = c.get_particles()
    for k in STATE_KEYS:
        assert np.isfinite(st[k]).all()
    assert max(peaks[1:]) < 2.0 * peaks[0]
    assert c.check() == 0


def test_canyon_solves_match_oracle():
    """The street canyon: walls with re-entrant and convex corners (bisector normals in Eq.
    59), a free-slip top and the periodic seam, for both solves."""
    w = synth.canyon_workload("canyon_2k")
    g = w["grid"]
    o, c = both(g, w["params"], w["fields"])
    rhs, L = o.wp_rhs()
    rg, Lg = c.wp_rhs()
    assert rel(rg, rhs) < 1e-13 and rel(Lg, L) < 1e-13
    wo, _ = o.wp_solve(rhs, L, tol=1e-13)
    wg, _ = c.wp_solve(rhs, L, tol=1e-13)
    assert rel(wg, wo) < 1e-9
    rng = np.random.default_rng(6)
    ustar, P = rng.normal(size=(g.nn, 3)), rng.normal(size=g.nn)
    so, fo = o.pressure_rhs(ustar, P, 1e-4, 5e-5)
    sg, fg = c.pressure_rhs(ustar, P, 1e-4, 5e-5)
    assert rel(sg, so) < 1e-12 and rel(fg, fo) < 1e-12
    do, _ = o.pressure_solve(so, fo, tol=1e-13)
    dg, _ = c.pressure_solve(so, fo, tol=1e-13)
    assert rel(dg, do) < 1e-8


def test_pressure_state_round_trip(channel):
    """pdfx_set_pressure stores P and clears the last increment; pdfx_get_pressure returns
    both bit for bit."""
    w, g = channel
    c = gpu_ctx(g, w["params"], w["fields"])
    P = np.random.default_rng(7).normal(size=g.nn)
    c.set_pressure(P)
    Pg, dPg = c.pressure()
    assert np.array_equal(Pg, P) and np.abs(dPg).max() == 0.0
