"""Pins of the oracle's elliptic-relaxation pieces (Eqs. 12-18, Eq. 59; no GPU).

The oracle builds H_ijkl of Eq. 13 term by term and contracts it; these tests check it
against contractions worked out by hand for special states, against invariants (the trace,
frame rotation) and against the limits of Eq. 16.  The FEM solve of Eq. 12 is checked
against exact solutions of the continuous problem (a periodic mode, the wall profile of
a channel with Eq. 59's wall value) with second-order convergence, and against the local
limit L = 0, where the Galerkin system returns the right-hand side itself.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1006_0532_gb300 import synth
from helpers import base_params

T4 = synth.TABLE4


def _freeslip_grid(nx, ny, jx=0.2, jy=0.1, seed=3):
    """A periodic channel grid whose two boundary rows are free-slip (no no-slip wall)."""
    g = synth.channel_grid(nx, ny, lx=1.0, jitter_x=jx, jitter_y=jy, seed=seed)
    tag = np.where(g.edge_tag == 1, 2, g.edge_tag).astype(np.int8)
    return synth.Grid(node_xy=g.node_xy, tri=g.tri, edge_tag=tag, period_x=g.period_x)


def _fields(nn, R, G, om):
    """Nodal fields with per-node <u_i u_j> R[nn][3][3], gradients G[nn][3][2], <omega>."""
    F = synth.uniform_fields(nn)
    F[:, 23] = R[:, 0, 0]
    F[:, 24] = R[:, 1, 1]
    F[:, 25] = R[:, 2, 2]
    F[:, 26] = R[:, 0, 1]
    F[:, 27] = R[:, 0, 2]
    F[:, 28] = R[:, 1, 2]
    F[:, 5:11] = np.asarray(G).reshape(nn, 6)
    F[:, 29] = om
    return F


def _random_state(nn, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(nn, 3, 3))
    R = A @ A.transpose(0, 2, 1) * rng.uniform(0.05, 1.0, size=(nn, 1, 1))
    G = rng.normal(size=(nn, 3, 2))
    om = rng.uniform(0.5, 3.0, size=nn)
    return R, G, om


def _rhs(grid, F, **kw):
    o = oracle.Oracle(grid, base_params(period_x=grid.period_x, **kw), F)
    return o.wp_rhs()


@pytest.fixture(scope="module")
def small_grid():
    return synth.channel_grid(6, 5, lx=1.0, seed=2)


# --------------------------------------------------------------------------------------
# The right-hand side of Eq. 12
# --------------------------------------------------------------------------------------

def test_rhs_without_mean_gradients_is_the_isotropic_term(small_grid):
    """With d<U_k>/dx_l = 0 only Eq. 12's first term is left: (1 - C1)/2 k <omega> on the
    diagonal and nothing off it, whatever the anisotropy of <u_i u_j>."""
    g = small_grid
    R, _, om = _random_state(g.nn, 1)
    rhs, _ = _rhs(g, _fields(g.nn, R, np.zeros((g.nn, 3, 2)), om))
    k = 0.5 * np.trace(R, axis1=1, axis2=2)
    want = 0.5 * (1 - T4["C1"]) * k * om
    np.testing.assert_allclose(np.diagonal(rhs, axis1=1, axis2=2), np.repeat(want[:, None], 3, 1),
                               rtol=1e-14, atol=0)
    off = rhs - np.einsum("nii->ni", rhs)[:, :, None] * np.eye(3)
    assert np.abs(off).max() == 0.0


def test_rhs_trace_identity(small_grid):
    """Contracting H_ijkl over i = j leaves C2 A_v delta_kl: the gamma5 terms of Eq. 13
    cancel in pairs (the two b terms because b is symmetric), so the trace of the
    right-hand side is 3 (1 - C1)/2 k <omega> + C2 A_v k div<U>, with A_v of Eq. 14 from
    LAPACK's determinant."""
    g = small_grid
    R, G, om = _random_state(g.nn, 2)
    rhs, _ = _rhs(g, _fields(g.nn, R, G, om))
    k = 0.5 * np.trace(R, axis1=1, axis2=2)
    av = np.minimum(1.0, T4["Cv"] * np.linalg.det(R) / (2 * k / 3) ** 3)
    div = G[:, 0, 0] + G[:, 1, 1]
    want = 1.5 * (1 - T4["C1"]) * k * om + T4["C2"] * av * k * div
    got = np.trace(rhs, axis1=1, axis2=2)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13 * np.abs(want).max())


def test_rhs_simple_shear_with_anisotropy(small_grid):
    """Principal-axes stresses R = diag(r1, r2, r3) in a simple shear d<U>/dy = S.  With
    b = diag(beta) of Eq. 15, the four terms of Eq. 13 contracted by hand give
        rhs_xy = k S (C2 A_v + gamma5/3 + gamma5 beta_1),
        rhs_yx = -k S (gamma5/3 + gamma5 beta_2),
    no other off-diagonal entry, and the isotropic diagonal, with A_v = min(1, C_v r1 r2 r3
    / (2k/3)^3)."""
    g = small_grid
    rng = np.random.default_rng(3)
    r = rng.uniform(0.1, 1.0, size=(g.nn, 3))
    R = np.zeros((g.nn, 3, 3))
    for i in range(3):
        R[:, i, i] = r[:, i]
    S = rng.uniform(-2.0, 2.0, size=g.nn)
    G = np.zeros((g.nn, 3, 2))
    G[:, 0, 1] = S
    om = rng.uniform(0.5, 2.0, size=g.nn)
    rhs, _ = _rhs(g, _fields(g.nn, R, G, om))
    tr = r.sum(1)
    k = 0.5 * tr
    beta = r / tr[:, None] - 1.0 / 3.0
    av = np.minimum(1.0, T4["Cv"] * r[:, 0] * r[:, 1] * r[:, 2] / (2 * k / 3) ** 3)
    g5, C2 = T4["gamma5"], T4["C2"]
    np.testing.assert_allclose(rhs[:, 0, 1], k * S * (C2 * av + g5 / 3 + g5 * beta[:, 0]), rtol=1e-13)
    np.testing.assert_allclose(rhs[:, 1, 0], -k * S * (g5 / 3 + g5 * beta[:, 1]), rtol=1e-13)
    for (i, j) in ((0, 2), (2, 0), (1, 2), (2, 1)):
        assert np.abs(rhs[:, i, j]).max() == 0.0
    iso = 0.5 * (1 - T4["C1"]) * k * om
    for i in range(3):
        np.testing.assert_allclose(rhs[:, i, i], iso, rtol=1e-13)


def test_rhs_isotropic_stress_and_two_component_limit(small_grid):
    """Isotropic <u_i u_j> = 2k/3 delta_ij gives b = 0 and det/(2k/3)^3 = 1, so A_v =
    min(1, C_v) = 1 and a pure strain G (symmetric) gives rhs = iso + C2 k G.  A
    two-component state (<w w> = 0, so det = 0 and A_v = 0) leaves a traceless mean-gradient
    part."""
    g = small_grid
    rng = np.random.default_rng(4)
    k = rng.uniform(0.1, 1.0, size=g.nn)
    om = rng.uniform(0.5, 2.0, size=g.nn)
    R = np.eye(3)[None] * (2 * k / 3)[:, None, None]
    a, b, s = rng.normal(size=(3, g.nn))
    G = np.zeros((g.nn, 3, 2))
    G[:, 0, 0], G[:, 1, 1], G[:, 0, 1], G[:, 1, 0] = a, b, s, s
    rhs, _ = _rhs(g, _fields(g.nn, R, G, om))
    iso = 0.5 * (1 - T4["C1"]) * k * om
    Gf = np.zeros((g.nn, 3, 3))
    Gf[:, :, :2] = G
    want = iso[:, None, None] * np.eye(3) + T4["C2"] * k[:, None, None] * Gf
    np.testing.assert_allclose(rhs, want, rtol=1e-13, atol=1e-15)
    R2 = np.zeros((g.nn, 3, 3))
    R2[:, 0, 0], R2[:, 1, 1] = rng.uniform(0.1, 1.0, size=(2, g.nn))
    R2[:, 0, 1] = R2[:, 1, 0] = 0.3 * np.sqrt(R2[:, 0, 0] * R2[:, 1, 1])
    rhs2, _ = _rhs(g, _fields(g.nn, R2, G, om))
    k2 = 0.5 * np.trace(R2, axis1=1, axis2=2)
    np.testing.assert_allclose(np.trace(rhs2, axis1=1, axis2=2), 1.5 * (1 - T4["C1"]) * k2 * om,
                               rtol=1e-13)


def test_rhs_rotates_with_the_frame(small_grid):
    """Eq. 12's right-hand side is a tensor function of <u_i u_j> and d<U_k>/dx_l: rotating
    both about z by Q rotates it to Q rhs Q^T (a slot mix-up, e.g. <uw> for <vw>, or a
    component treated out of its tensor position, breaks this)."""
    g = small_grid
    R, G, om = _random_state(g.nn, 5)
    Gf = np.zeros((g.nn, 3, 3))
    Gf[:, :, :2] = G
    rhs, _ = _rhs(g, _fields(g.nn, R, G, om))
    th = 0.7
    Q = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rq = Q @ R @ Q.T
    Gq = Q @ Gf @ Q.T
    assert np.abs(Gq[:, :, 2]).max() < 1e-15
    rhs_q, _ = _rhs(g, _fields(g.nn, Rq, Gq[:, :, :2], om))
    np.testing.assert_allclose(rhs_q, Q @ rhs @ Q.T, rtol=0, atol=1e-13 * np.abs(rhs).max())


def test_length_scale_limits():
    """Eq. 16 in its two limits, on a grid with no-slip walls (Eq. 17's C_xi = 1 + 1.3 for a
    unit normal) and on the same grid with free-slip boundaries (no wall: C_xi = 1).
    k = 0 with nu > 0: eps = nu C_T^2 <omega>^2 (Eq. 18) and L = C_L C_eta (nu^3/eps)^(1/4)
    = C_L C_eta (nu / (C_T <omega>))^(1/2) on both grids.  nu = 0: eps = k <omega> and
    L = C_L C_xi k^(1/2) / <omega>."""
    gw = synth.channel_grid(6, 5, lx=1.0, seed=2)
    gf = _freeslip_grid(6, 5, seed=2)
    rng = np.random.default_rng(6)
    om = rng.uniform(0.5, 3.0, size=gw.nn)
    zeroR = np.zeros((gw.nn, 3, 3))
    G0 = np.zeros((gw.nn, 3, 2))
    nu = 2e-3
    want = T4["CL"] * T4["Ceta"] * np.sqrt(nu / (T4["CT"] * om))
    for g in (gw, gf):
        _, L = _rhs(g, _fields(g.nn, zeroR, G0, om), nu=nu)
        np.testing.assert_allclose(L, want, rtol=1e-13)
    k = rng.uniform(0.1, 2.0, size=gw.nn)
    R = np.eye(3)[None] * (2 * k / 3)[:, None, None]
    for g, cxi in ((gw, 2.3), (gf, 1.0)):
        _, L = _rhs(g, _fields(g.nn, R, G0, om), nu=0.0)
        np.testing.assert_allclose(L, T4["CL"] * cxi * np.sqrt(k) / om, rtol=1e-13)


def test_rhs_rejects_zero_dissipation(small_grid):
    """A node with eps = 0 (k = 0 and nu = 0) has no length scale: the call fails."""
    g = small_grid
    F = _fields(g.nn, np.zeros((g.nn, 3, 3)), np.zeros((g.nn, 3, 2)), np.ones(g.nn))
    with pytest.raises(RuntimeError):
        _rhs(g, F, nu=0.0)


# --------------------------------------------------------------------------------------
# The FEM solve of Eq. 12
# --------------------------------------------------------------------------------------

def test_solve_local_limit_returns_the_rhs():
    """L = 0 leaves the consistent mass matrix on both sides (Galerkin projection of a
    linear right-hand side), so wp = rhs at every node; off-diagonal components meet their
    zero Dirichlet value at the free-slip rows, which the test's right-hand side also has."""
    g = _freeslip_grid(10, 9, seed=5)
    o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
    rng = np.random.default_rng(7)
    f = rng.normal(size=(g.nn, 3, 3))
    y = g.node_xy[:, 1]
    edge = (y == 0.0) | (y == 1.0)
    off = ~np.eye(3, dtype=bool)
    f[np.ix_(edge, *[np.arange(3)] * 2)] *= np.where(off, 0.0, 1.0)
    wp, it = o.wp_solve(f, np.zeros(g.nn))
    np.testing.assert_allclose(wp, f, rtol=0, atol=1e-11)
    assert it < 200


def test_solve_keeps_constants_under_natural_conditions():
    """With no Dirichlet node a constant is in the stiffness matrix's null space (its rows
    sum to zero), so a constant diagonal right-hand side is the solution for any L."""
    g = _freeslip_grid(10, 9, seed=5)
    o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
    f = np.zeros((g.nn, 3, 3))
    f[:, 0, 0], f[:, 1, 1], f[:, 2, 2] = 0.3, -1.2, 2.5
    L = np.random.default_rng(8).uniform(0.05, 0.4, size=g.nn)
    wp, _ = o.wp_solve(f, L)
    np.testing.assert_allclose(wp, f, rtol=0, atol=1e-12)


def test_solve_periodic_mode_converges_at_second_order():
    """wp - L^2 lap wp = c + a cos(2 pi x) on the periodic strip with zero normal derivative
    at the free-slip rows has the exact solution c + a cos(2 pi x) / (1 + (2 pi L)^2) for the
    diagonal components.  The nodal error of the linear-triangle Galerkin solution falls by
    about 4 per halving of h, across the periodic seam."""
    errs = []
    Lc, c, a = 0.2, 1.0, 0.5
    for n in (8, 16, 32):
        g = _freeslip_grid(n, n + 1, seed=3)
        o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
        x = g.node_xy[:, 0]
        f = np.zeros((g.nn, 3, 3))
        for i in range(3):
            f[:, i, i] = c + a * np.cos(2 * np.pi * x)
        wp, _ = o.wp_solve(f, np.full(g.nn, Lc))
        exact = c + a * np.cos(2 * np.pi * x) / (1 + (2 * np.pi * Lc) ** 2)
        errs.append(max(np.abs(wp[:, i, i] - exact).max() for i in range(3)))
        assert np.abs(wp[:, ~np.eye(3, dtype=bool)]).max() == 0.0
    assert errs[-1] < 1.5e-3
    assert errs[0] / errs[2] > 10.0


def test_solve_channel_wall_profile_with_eq59():
    """The channel of Sect. 4.1 with walls at y = 0 and 1: Eq. 59 with the outward normals
    (0, -1) and (0, 1) sets only wp_22 = -4.5 eps at the walls (the paper states this for
    its channel); the other components are 0 there.  For constant L and a constant
    right-hand side c the continuous solution is c + (w - c) cosh((y - 1/2)/L) / cosh(1/(2L))
    with w the wall value; the FEM solution converges to it at second order."""
    om, nu = 2.0, 1e-3
    uu = (0.2, 0.2, 0.2, 0.0, 0.0, 0.0)
    k = 0.3
    eps = om * (k + nu * T4["CT"] ** 2 * om)
    Lc, c = 0.15, 0.7
    errs = []
    for ny in (9, 17, 33):
        g = synth.channel_grid(ny - 1, ny, lx=1.0, jitter_x=0.2, jitter_y=0.1, seed=3)
        F = synth.uniform_fields(g.nn, uu=uu, omega=om)
        o = oracle.Oracle(g, base_params(period_x=g.period_x, nu=nu), F)
        f = np.zeros((g.nn, 3, 3))
        f[:, 0, 0] = f[:, 1, 1] = f[:, 2, 2] = c
        wp, _ = o.wp_solve(f, np.full(g.nn, Lc))
        y = g.node_xy[:, 1]
        wall = (y == 0.0) | (y == 1.0)
        want_wall = np.zeros((3, 3))
        want_wall[1, 1] = -4.5 * eps
        np.testing.assert_allclose(wp[wall], np.broadcast_to(want_wall, wp[wall].shape), rtol=1e-15)
        prof = lambda w: c + (w - c) * np.cosh((y - 0.5) / Lc) / math.cosh(0.5 / Lc)
        e = max(np.abs(wp[:, 1, 1] - prof(-4.5 * eps)).max(),
                np.abs(wp[:, 0, 0] - prof(0.0)).max(), np.abs(wp[:, 2, 2] - prof(0.0)).max())
        errs.append(e)
        assert np.abs(wp[:, ~np.eye(3, dtype=bool)]).max() == 0.0
    assert errs[2] < 0.012
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.5


def test_solve_wall_values_on_the_street_canyon():
    """Eq. 59 at every no-slip node of the street canyon (floor, cavity walls and its
    corners): wp = -4.5 eps n n^T with a unit n in the plane, so its trace is -4.5 eps, it
    is symmetric of rank one and has no z entries; straight floor nodes away from corners
    have n = (0, -1)."""
    w = synth.canyon_workload("canyon_2k")
    g = w["grid"]
    o = oracle.Oracle(g, w["params"], w["fields"])
    rhs, L = o.wp_rhs()
    wp, _ = o.wp_solve(rhs, L)
    F = w["fields"]
    nu, CT = w["params"]["nu"], T4["CT"]
    k = 0.5 * F[:, 23:26].sum(1)
    eps = F[:, 29] * (k + nu * CT ** 2 * F[:, 29])
    wallnode = np.zeros(g.nn, bool)
    for kk in range(3):
        m = g.edge_tag[:, kk] == 1
        wallnode[g.tri[m, (kk + 1) % 3]] = True
        wallnode[g.tri[m, (kk + 2) % 3]] = True
    assert wallnode.sum() > 20
    Wn = wp[wallnode]
    np.testing.assert_allclose(np.trace(Wn, axis1=1, axis2=2), -4.5 * eps[wallnode], rtol=1e-13)
    np.testing.assert_allclose(Wn, Wn.transpose(0, 2, 1), rtol=0, atol=1e-15 * np.abs(Wn).max())
    assert np.abs(Wn[:, 2, :]).max() == 0.0 and np.abs(Wn[:, :, 2]).max() == 0.0
    det2 = Wn[:, 0, 0] * Wn[:, 1, 1] - Wn[:, 0, 1] ** 2
    assert np.abs(det2).max() < 1e-12 * np.abs(Wn).max() ** 2
    assert (np.abs(Wn[:, 0, 1]) < 1e-14 * np.abs(Wn).max()).sum() > 10


def test_update_wp_writes_the_solution_into_the_fields():
    """The coupled-loop update solves from the fields' wp_ij (slots 14-22) and writes the
    solution back there, leaving every other slot as it was; a second update from that
    solution needs no iteration."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    o = oracle.Oracle(g, w["params"], w["fields"])
    before = o.fields()
    rhs, L = o.wp_rhs()
    want, _ = o.wp_solve(rhs, L, before[:, 14:23])
    it = o.update_wp()
    assert it > 0
    after = o.fields()
    np.testing.assert_array_equal(after[:, 14:23], want.reshape(g.nn, 9))
    keep = [s for s in range(32) if not 14 <= s < 23]
    np.testing.assert_array_equal(after[:, keep], before[:, keep])
    assert o.update_wp() == 0


def test_solve_free_slip_symmetry_conditions():
    """Sect. 4.1's symmetry conditions at a free-slip row: off-diagonal components are held
    at zero there and diagonal ones have zero normal derivative.  With a constant
    right-hand side c in every component and constant L on the free-slip strip, the
    diagonal solution is c everywhere and the off-diagonal one follows
    c (1 - cosh((y - 1/2)/L) / cosh(1/(2L))), to second order."""
    Lc, c = 0.2, 0.9
    errs = []
    for n in (8, 16, 32):
        g = _freeslip_grid(n, n + 1, seed=4)
        o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
        wp, _ = o.wp_solve(np.full((g.nn, 3, 3), c), np.full(g.nn, Lc))
        y = g.node_xy[:, 1]
        np.testing.assert_allclose(np.diagonal(wp, axis1=1, axis2=2), c, rtol=1e-12)
        prof = c * (1 - np.cosh((y - 0.5) / Lc) / math.cosh(0.5 / Lc))
        off = wp[:, ~np.eye(3, dtype=bool)]
        edge = (y == 0.0) | (y == 1.0)
        assert np.abs(off[edge]).max() == 0.0
        errs.append(np.abs(off - prof[:, None]).max())
    assert errs[2] < 4e-3 and errs[0] / errs[2] > 10.0


# --------------------------------------------------------------------------------------
# The pressure projection (Eq. 33 with Eq. 61) and the coupled step
# --------------------------------------------------------------------------------------

def _unwrapped(g):
    """Element vertex coordinates with x taken as the image nearest to vertex A."""
    x = g.node_xy[g.tri, 0].copy()
    for k in (1, 2):
        x[:, k] -= g.period_x * np.round((x[:, k] - x[:, 0]) / g.period_x)
    return x, g.node_xy[g.tri, 1]


def _areas(g):
    x, y = _unwrapped(g)
    return 0.5 * ((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))


def test_pressure_solve_periodic_mode_converges_at_second_order():
    """lap dP = -5 pi^2 cos(2 pi x) cos(pi y) on the periodic strip with zero normal
    derivative at the free-slip rows: the zero-mean solution is cos(2 pi x) cos(pi y), which
    the Galerkin solution approaches at second order; its integral is zero."""
    errs = []
    for n in (8, 16, 32):
        g = _freeslip_grid(n, n + 1, seed=3)
        o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
        x, y = g.node_xy.T
        exact = np.cos(2 * np.pi * x) * np.cos(np.pi * y)
        dP, _ = o.pressure_solve(-5 * np.pi ** 2 * exact, np.zeros(g.nn))
        errs.append(np.abs(dP - exact).max())
        assert abs(np.sum(_areas(g)[:, None] / 3 * dP[g.tri])) < 1e-13
    assert errs[2] < 0.01 and errs[0] / errs[2] > 10.0


def test_pressure_solve_wall_flux_converges_at_second_order():
    """lap dP = 1 in the walled channel with outward normal derivative 1 on the wall y = 1
    and 0 on y = 0 (compatible: the source integrates to the boundary flux) has the
    zero-mean solution y^2/2 - 1/6; the flux enters through the edge integrals of the weak
    form."""
    errs = []
    for n in (8, 16, 32):
        g = synth.channel_grid(n, n + 1, lx=1.0, seed=3)
        o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
        y = g.node_xy[:, 1]
        dP, _ = o.pressure_solve(np.ones(g.nn), np.where(y == 1.0, 1.0, 0.0))
        errs.append(np.abs(dP - (y * y / 2 - 1.0 / 6.0)).max())
    assert errs[2] < 3e-4 and errs[0] / errs[2] > 10.0


def test_pressure_rhs_linear_fields_closed_form():
    """Eq. 33's source and Eq. 61's increment flux for fields linear in y, for which every
    node-transferred derivative is exact: <U>* = (a y, b y, 0) has divergence b; P = c y has
    zero laplacian; with laplacian slots (lx, ly) and <uu>, <vv>, <uv> with y-slopes s1, s2,
    s3, the wall y = 0 (n = (0, -1)) gets -nu ly + s2 + c and the wall y = 1 (n = (0, 1))
    gets nu ly - s2 - c; other nodes get 0."""
    g = synth.channel_grid(10, 9, lx=1.0, seed=6)
    nu = 3e-3
    y = g.node_xy[:, 1]
    F = synth.uniform_fields(g.nn, lap=(0.4, -0.7, 0.0))
    s1, s2, s3 = 0.3, -0.5, 0.8
    F[:, 23] = 0.5 + s1 * y
    F[:, 24] = 0.6 + s2 * y
    F[:, 26] = 0.1 + s3 * y
    o = oracle.Oracle(g, base_params(period_x=g.period_x, nu=nu), F)
    a, b, c, dt, Cp = 1.3, 0.25, -2.0, 1e-3, 1e-3
    ustar = np.stack([a * y, b * y, np.zeros(g.nn)], 1)
    src, flux = o.pressure_rhs(ustar, c * y, dt, Cp)
    np.testing.assert_allclose(src, b / dt, rtol=1e-10)
    want = np.where(y == 0.0, -nu * (-0.7) + s2 + c, np.where(y == 1.0, nu * (-0.7) - s2 - c, 0.0))
    np.testing.assert_allclose(flux, want, rtol=1e-10, atol=1e-12)


def test_pressure_rhs_stabilisation_term():
    """Eq. 33's C_p term with P = y^2 on a lattice whose node transfers give the exact
    second derivative 2 two rows from the walls: src = (div <U>* - 2 C_p) / dt there."""
    from test_oracle_pins import _same_diagonal_lattice
    g = _same_diagonal_lattice(12, 9)
    o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
    y = g.node_xy[:, 1]
    dt, Cp = 2e-3, 0.05
    src, _ = o.pressure_rhs(np.stack([0 * y, 0.5 * y, 0 * y], 1), y * y, dt, Cp)
    deep = (y > 1.5 / 8) & (y < 1 - 1.5 / 8)
    np.testing.assert_allclose(src[deep], (0.5 - 2 * Cp) / dt, rtol=1e-10)


def _elem_grad(g, q):
    """Element gradients of a nodal field (shapefunction derivatives in the element frame)."""
    x, yv = _unwrapped(g)
    t = g.tri
    A2 = (x[:, 1] - x[:, 0]) * (yv[:, 2] - yv[:, 0]) - (x[:, 2] - x[:, 0]) * (yv[:, 1] - yv[:, 0])
    qv = q[t]
    gx = (qv[:, 0] * (yv[:, 1] - yv[:, 2]) + qv[:, 1] * (yv[:, 2] - yv[:, 0]) + qv[:, 2] * (yv[:, 0] - yv[:, 1])) / A2
    gy = (qv[:, 0] * (x[:, 2] - x[:, 1]) + qv[:, 1] * (x[:, 0] - x[:, 2]) + qv[:, 2] * (x[:, 1] - x[:, 0])) / A2
    return gx, gy


def test_coupled_step_against_the_particle_step():
    """The coupled step of Table 1 moves the particles exactly as the particle-path step does
    after the same elliptic-relaxation update (positions, frequency, scalar and element are
    untouched by the projection), and differs only by Eq. 31's correction: each particle's
    u, v drop by dt times its element's gradient of the pressure increment.  The increment
    has zero integral, P advances by it, the pressure-gradient slots hold its node-transferred
    gradient and the elliptic-relaxation slots the solution."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    dt = w["dt"]
    o1 = oracle.Oracle(g, w["params"], w["fields"])
    o2 = oracle.Oracle(g, w["params"], w["fields"])
    o1.init_particles(60)
    o2.init_particles(60)
    P0 = 0.2 * g.node_xy[:, 1] ** 2
    P = P0.copy()
    dP, wi, pi = o1.coupled_step(dt, P)
    assert wi > 0 and pi > 0
    o2.update_wp()
    o2.step(dt)
    s1, s2 = o1.get_particles(), o2.get_particles()
    for k in ("x", "y", "w", "om", "psi", "elem"):
        np.testing.assert_array_equal(s1[k], s2[k])
    gx, gy = _elem_grad(g, dP)
    e = s1["elem"]
    np.testing.assert_allclose(s1["u"], s2["u"] - dt * gx[e], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s1["v"], s2["v"] - dt * gy[e], rtol=0, atol=1e-13)
    assert np.abs(dt * gy).max() > 1e-6
    np.testing.assert_array_equal(P, P0 + dP)
    f1, f2 = o1.fields(), o2.fields()
    np.testing.assert_array_equal(f1[:, 14:23], f2[:, 14:23])
    np.testing.assert_allclose(f1[:, 3:5], o1.node_gradient(P), rtol=0, atol=1e-14)
    assert abs(np.sum(_areas(g)[:, None] / 3 * dP[g.tri])) < 1e-12 * np.abs(dP).max()


def test_coupled_step_statistics_shift_with_the_correction():
    """Eq. 31 shifts every particle of an element by the same vector, so the element means
    shift by it, while the central moments, the velocity ordering and with it the bins and
    their conditional scalar means stay as they were before the correction."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    dt = w["dt"]
    o1 = oracle.Oracle(g, w["params"], w["fields"])
    o2 = oracle.Oracle(g, w["params"], w["fields"])
    o1.init_particles(60)
    o2.init_particles(60)
    P = 0.2 * g.node_xy[:, 1] ** 2
    dP, _, _ = o1.coupled_step(dt, P)
    o2.update_wp()
    o2.step(dt)
    (m1, c1), (m2, c2) = o1.element_stats(), o2.element_stats()
    np.testing.assert_array_equal(c1, c2)
    gx, gy = _elem_grad(g, dP)
    has = c1 > 0
    np.testing.assert_allclose(m1[has, 1], m2[has, 1] - dt * gx[has], rtol=0, atol=1e-13)
    np.testing.assert_allclose(m1[has, 2], m2[has, 2] - dt * gy[has], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(m1[:, 3], m2[:, 3])
    scale = np.abs(m2[:, 4:10]).max()
    np.testing.assert_allclose(m1[:, 4:10], m2[:, 4:10], rtol=0, atol=1e-12 * scale)
    np.testing.assert_array_equal(m1[:, 10:], m2[:, 10:])
    (v1, g1), (v2, g2) = o1.bins(), o2.bins()
    np.testing.assert_array_equal(g1, g2)
    np.testing.assert_array_equal(v1, v2)
    np.testing.assert_array_equal(o1.get_particles()["cp"], o2.get_particles()["cp"])


def test_pressure_stabilisation_factor():
    """Eq. 33 with a divergence-free <U>* and no wall flux leaves lap dP = -(C_p / dt) lap P^n,
    so dP = -(C_p / dt) P^n for a zero-mean P^n: P^{n+1} = (1 - C_p / dt) P^n, which is
    stable only for C_p < 2 dt.  On a smooth mode the Galerkin solution of the two-pass
    laplacian's load approaches that factor as h falls (slower than second order on the
    coarse grids: the node-transferred second derivatives are one-sided at the boundary
    rows)."""
    errs = []
    dt, Cp = 1e-3, 4e-4
    for n in (8, 16, 32):
        g = _freeslip_grid(n, n + 1, seed=6)
        o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
        x, y = g.node_xy.T
        P = np.cos(2 * np.pi * x) * np.cos(np.pi * y)
        src, flux = o.pressure_rhs(np.zeros((g.nn, 3)), P, dt, Cp)
        assert np.abs(flux).max() == 0.0
        dP, _ = o.pressure_solve(src, flux)
        errs.append(np.abs(dP + (Cp / dt) * P).max() / (Cp / dt))
    assert errs[2] < 0.04 and errs[0] / errs[2] > 8.0


@pytest.mark.parametrize("name", ["channel_tiny", "canyon_2k"])
def test_coupled_steps_stay_bounded(name):
    """Six coupled steps (C_p = dt/2) on the channel (walls) and on the street canyon
    (walls, cavity corners, free-slip top): states stay finite, every particle stays in the
    domain and is found by the walk, the solves converge every step and the pressure
    increment does not grow from step to step."""
    w = synth.workload(name) if name == "channel_tiny" else synth.canyon_workload(name)
    g = w["grid"]
    o = oracle.Oracle(g, w["params"], w["fields"])
    o.init_particles(20 if name == "canyon_2k" else 60)
    o.derive_fields()
    P = np.zeros(g.nn)
    dP, peak = None, []
    for _ in range(6):
        dP, wi, pi = o.coupled_step(w["dt"], P, dP, Cp=0.5 * w["dt"], tol=1e-10)
        peak.append(np.abs(dP).max())
    st = o.get_particles()
    for k in ("x", "y", "u", "v", "w", "om", "psi"):
        assert np.isfinite(st[k]).all()
    d = o.diag()
    assert d["lost"] == 0 and d["walk_brute"] == 0
    assert max(peak[1:]) < 2.0 * peak[0]
    assert np.isfinite(P).all()


def test_solves_with_a_zero_load_return_zero_at_once():
    """A zero right-hand side with zero boundary values has the zero solution; both solves
    return it from any initial guess without iterating (a stopping rule relative to a zero
    load could never be met)."""
    g = _freeslip_grid(8, 9, seed=2)
    o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
    rng = np.random.default_rng(10)
    wp, it = o.wp_solve(np.zeros((g.nn, 3, 3)), np.full(g.nn, 0.2), rng.normal(size=(g.nn, 3, 3)))
    assert it == 0 and np.abs(wp).max() == 0.0
    dP, it = o.pressure_solve(np.zeros(g.nn), np.zeros(g.nn), rng.normal(size=g.nn))
    assert it == 0 and np.abs(dP).max() == 0.0
