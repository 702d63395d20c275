"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than its own formulas: published
known answers, closed forms of the stochastic recursions, invariants, textbook
distributions (scipy), brute force, or the paper's worked example.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1006_0532_gb300 import synth
from helpers import base_params, homogeneous_fields

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------
# Random numbers (Sect. 3.9)
# --------------------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_open_interval():
    assert oracle.lib().orc_uniform(0) == 0.5 / 2 ** 32
    assert oracle.lib().orc_uniform(0xffffffff) == (2 ** 32 - 0.5) / 2 ** 32
    assert 0.0 < oracle.lib().orc_uniform(0) and oracle.lib().orc_uniform(0xffffffff) < 1.0


def _gaussians(n, seed=11):
    out = []
    for pid in range(n // 6):
        xi, _ = oracle.step_gaussians(seed, 0, pid, 3)
        out.append(xi)
    return np.concatenate(out)


def test_box_muller_standard_normal():
    g = _gaussians(120000)
    n = g.size
    assert abs(g.mean()) < 5 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.skew(g)) < 5 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(g)) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(g, "norm").pvalue > 1e-3
    # the six per-particle Gaussians are mutually uncorrelated
    m = g.reshape(-1, 6)
    c = np.corrcoef(m.T)
    assert np.max(np.abs(c - np.eye(6))) < 5 / math.sqrt(m.shape[0])


def test_gamma_sampler_distribution():
    # Eq. 58 / Sect. 3.7: gamma with mean m and variance C4 m^2 is Gamma(1/C4, C4 m).
    C4, m = 0.25, 3.0
    n = 40000
    draws = np.array([oracle.gamma_draw(5, 0, pid, 9, 2, 1.0 / C4, C4 * m)[0] for pid in range(n)])
    assert abs(draws.mean() - m) < 5 * math.sqrt(C4 * m * m / n)
    assert abs(draws.var() / (C4 * m * m) - 1.0) < 0.05
    assert stats.kstest(draws, stats.gamma(a=1.0 / C4, scale=C4 * m).cdf).pvalue > 1e-3


# --------------------------------------------------------------------------------------
# Shapefunctions and tracking (Sect. 3.4, 3.6)
# --------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def w2k():
    return synth.workload("channel_2k")


@pytest.fixture(scope="module")
def orc2k(w2k):
    return oracle.Oracle(w2k["grid"], w2k["params"], w2k["fields"])


def _unwrapped_vertices(grid, e):
    tri = grid.tri[e]
    xy = grid.node_xy[tri].copy()
    L = grid.period_x
    for k in (1, 2):
        d = xy[k, 0] - xy[0, 0]
        if d > L / 2:
            xy[k, 0] -= L
        elif d < -L / 2:
            xy[k, 0] += L
    return xy


def test_area_coordinates_vertices_and_sum(orc2k, w2k):
    g = w2k["grid"]
    rng = np.random.default_rng(0)
    for e in rng.integers(0, g.ne, 200):
        xy = _unwrapped_vertices(g, e)
        for k in range(3):
            lam = orc2k.lam(e, xy[k, 0] % g.period_x, xy[k, 1])
            assert np.allclose(lam, np.eye(3)[k], atol=1e-12)
        r = rng.dirichlet([1, 1, 1])
        p = r @ xy
        lam = orc2k.lam(e, p[0] % g.period_x, p[1])
        assert abs(lam.sum() - 1.0) < 1e-14
        assert np.allclose(lam, r, atol=1e-11)


def test_linear_fields_interpolated_exactly(w2k):
    g = w2k["grid"]
    o = oracle.Oracle(g, w2k["params"])
    # a field linear in y (x is periodic, so use y and constants only)
    F = np.zeros((g.nn, 32))
    F[:, 0] = 3.0 * g.node_xy[:, 1] - 1.0
    F[:, 7] = 2.5
    o.set_fields(F)
    rng = np.random.default_rng(1)
    for e in rng.integers(0, g.ne, 100):
        xy = _unwrapped_vertices(g, e)
        p = rng.dirichlet([1, 1, 1]) @ xy
        q = o.interp(e, o.lam(e, p[0] % g.period_x, p[1]))
        assert abs(q[0] - (3.0 * p[1] - 1.0)) < 1e-12
        assert abs(q[7] - 2.5) < 1e-13


def test_neighbors_symmetric(orc2k, w2k):
    nb = orc2k.neighbors()
    g = w2k["grid"]
    for e in range(g.ne):
        for k in range(3):
            f = nb[e, k]
            if f < 0:
                assert g.edge_tag[e, k] != 0
            else:
                assert e in nb[f]
                shared = set(g.tri[e]) & set(g.tri[f])
                assert len(shared) == 2 and g.tri[e, k] not in shared


def test_walk_equals_brute_force(orc2k, w2k):
    """Sect. 3.6: the neighbour walk finds the element that brute force finds."""
    g = w2k["grid"]
    rng = np.random.default_rng(2)
    hops_seen = []
    for _ in range(3000):
        e0 = int(rng.integers(0, g.ne))
        xy = _unwrapped_vertices(g, e0)
        c = xy.mean(0)
        p = c + rng.normal(0, 0.05, 2)          # up to a few elements away, crosses the seam
        p[1] = np.clip(p[1], 1e-9, 1 - 1e-9)
        x = p[0] % g.period_x
        e, hops = orc2k.walk(e0, x, p[1])
        b = orc2k.brute(x, p[1])
        assert b >= 0 and e >= 0
        if e != b:
            # only a point on a shared edge may be claimed by either element
            assert orc2k.lam(e, x, p[1]).min() > -1e-12
            assert orc2k.lam(b, x, p[1]).min() > -1e-12
        hops_seen.append(hops)
    assert max(hops_seen) < 64


# --------------------------------------------------------------------------------------
# Stochastic updates: closed forms of the Euler-Maruyama recursions
# --------------------------------------------------------------------------------------

def _homog_oracle(grid, params, fields):
    o = oracle.Oracle(grid, params, fields)
    return o


def _middle(st, lo=0.2, hi=0.8):
    return (st["y"] > lo) & (st["y"] < hi)


@pytest.fixture(scope="module")
def grid_small():
    return synth.channel_grid(16, 9, seed=4)


def test_glm_ornstein_uhlenbeck_transient(grid_small):
    """Eq. 27 with constant coefficients: U' = (1 - a dt) U - dP dt + b sqrt(dt) xi.

    Mean: m_n = -(dP/a) (1 - r^n); variance: s_n = r^{2n} s_0 + b^2/(a(2 - a dt)) (1 - r^{2n}),
    r = 1 - a dt, a = (eps/2 - p)/k, b^2 = C0 eps.  (Ornstein-Uhlenbeck under Euler-Maruyama.)
    """
    k, Om, p_iso, C0, dt, n = 1.5e-4, 1.0, 0.0, 2.0, 0.05, 40
    nu = 0.0
    dPx = -0.01
    F, eps = homogeneous_fields(grid_small, k, Om, nu, p_iso=p_iso, dP=(dPx, 0.0))
    P = base_params(nu=nu, c0_mode=1, C0=C0, source_on=0, seed=21)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(400)
    for _ in range(n):
        o.step(dt)
    st = o.get_particles()
    m = _middle(st)
    a = (eps / 2 - p_iso) / k
    b2 = C0 * eps
    r = 1 - a * dt
    s0 = 2 * k / 3
    var_n = r ** (2 * n) * s0 + b2 / (a * (2 - a * dt)) * (1 - r ** (2 * n))
    mean_n = -(dPx / a) * (1 - r ** n)
    N = int(m.sum())
    assert N > 20000
    for key, mexp in (("u", mean_n), ("v", 0.0), ("w", 0.0)):
        vals = st[key][m]
        assert abs(vals.mean() - mexp) < 5 * math.sqrt(var_n / N)
        assert abs(vals.var() / var_n - 1) < 5 * math.sqrt(2.0 / N)


def test_glm_shared_wiener_increment(grid_small):
    """Eqs. 7 and 27 use the same dW: Cov(dU_x, dY) = 2 nu S dt, Var(dU_x) = 2 nu S^2 dt,
    E[dU_x] = (-dP_x + 2 nu lap U_x) dt, E[dY] = V dt (one step, G = 0, C0 = 0)."""
    k, Om, nu, dt, S = 1e-4, 1.0, 1e-3, 1e-2, 3.0
    lapx, dPx = 0.7, -0.2
    F, eps = homogeneous_fields(grid_small, k, Om, nu, grad=(0, S, 0, 0, 0, 0), lap=(lapx, 0, 0),
                                dP=(dPx, 0.0))
    P = base_params(nu=nu, c0_mode=1, C0=0.0, source_on=0, seed=22)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(300)
    s0 = o.get_particles()
    o.step(dt)
    s1 = o.get_particles()
    m = _middle(s0, 0.3, 0.7)
    dU = (s1["u"] - s0["u"])[m]
    dY = (s1["y"] - s0["y"] - s0["v"] * dt)[m]
    N = dU.size
    assert abs(dU.mean() - (-dPx + 2 * nu * lapx) * dt) < 5 * math.sqrt(2 * nu * S * S * dt / N)
    assert abs(dU.var() / (2 * nu * S * S * dt) - 1) < 5 * math.sqrt(2.0 / N)
    cov = np.mean((dU - dU.mean()) * (dY - dY.mean()))
    assert abs(cov / (2 * nu * S * dt) - 1) < 5 * math.sqrt(2.0 / N)
    assert abs(dY.var() / (2 * nu * dt) - 1) < 5 * math.sqrt(2.0 / N)
    # v and w get no mean-gradient noise here
    assert np.allclose(s1["v"][m], s0["v"][m], atol=1e-15)


def test_position_viscous_diffusion(grid_small):
    """Eq. 7 with U = 0: displacement has zero mean and variance 2 nu dt per component."""
    nu, dt = 2e-4, 1e-2
    F, _ = homogeneous_fields(grid_small, 1e-12, 1.0, nu)
    P = base_params(nu=nu, c0_mode=1, C0=0.0, source_on=0, seed=23)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(300)
    s0 = o.get_particles()
    s0["u"][:] = 0
    s0["v"][:] = 0
    s0["w"][:] = 0
    o.set_particles(s0, 0)
    o.step(dt)
    s1 = o.get_particles()
    m = _middle(s0, 0.3, 0.7)
    L = grid_small.period_x
    dx = ((s1["x"] - s0["x"] + L / 2) % L - L / 2)[m]
    dy = (s1["y"] - s0["y"])[m]
    N = dx.size
    sig2 = 2 * nu * dt
    for d in (dx, dy):
        assert abs(d.mean()) < 5 * math.sqrt(sig2 / N)
        assert abs(d.var() / sig2 - 1) < 5 * math.sqrt(2.0 / N)


def test_frequency_cir_stationary_gamma(grid_small):
    """Eq. 19 with S_omega = 0 and constant <omega> = Om is a CIR process whose stationary
    law is Gamma(1/C4, C4 Om); under Euler-Maruyama the stationary variance is
    C4 Om^2 * 2 / (2 - C3 Om dt) and the mean is exactly Om."""
    Om, dt, C3, C4 = 2.0, 1e-3, 5.0, 0.25
    F, _ = homogeneous_fields(grid_small, 1e-4, Om, 0.0)
    P = base_params(nu=0.0, c0_mode=1, C0=0.0, Cw1=0.0, Cw2=0.0, source_on=0, seed=24)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(80)
    s = o.get_particles()
    s["om"][:] = Om                      # start from a delta at the mean
    s["u"][:] = 0
    s["v"][:] = 0
    s["w"][:] = 0
    o.set_particles(s, 0)
    for _ in range(400):                 # C3 Om t = 4: relaxation e^-4 of the transient
        o.step(dt)
    w = o.get_particles()["om"]
    N = w.size
    var_em = C4 * Om * Om * 2 / (2 - C3 * Om * dt)
    trans = math.exp(-2 * C3 * Om * 400 * dt)
    assert abs(w.mean() - Om) < 5 * math.sqrt(var_em / N)
    assert abs(w.var() / var_em - 1) < 5 * math.sqrt(2.0 * 3 / N) + trans
    assert stats.kstest(w, stats.gamma(a=1 / C4, scale=C4 * Om).cdf).pvalue > 1e-4


def test_iecm_preserves_bin_means_and_decays_deviations(grid_small):
    """Eq. 24 with constant t_m: within each conditioning bin of the previous statistics
    the scalar mean is unchanged and every deviation from it shrinks by 1 - dt/t_m, with
    1/t_m = C_phi eps / (2k) = C_phi Om / 2 (IEM/IECM mixing rate; nu = 0)."""
    Om, dt, Cphi = 3.0, 1e-2, 2.0
    F, _ = homogeneous_fields(grid_small, 1e-6, Om, 0.0)
    P = base_params(nu=0.0, c0_mode=1, C0=0.0, tm_mode=1, Cphi=Cphi, source_on=0, seed=25,
                    bins=(3, 2, 2), min_per_bin=3)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(60)
    s0 = o.get_particles()
    rng = np.random.default_rng(3)
    s0["psi"] = rng.uniform(0, 1, s0["x"].size)
    o.set_particles(s0, 5)
    s0 = o.get_particles()
    o.step(dt)
    s1 = o.get_particles()
    key = s0["elem"].astype(np.int64) * 256 + s0["cp"]
    uniq, inv = np.unique(key, return_inverse=True)
    cnt = np.bincount(inv)
    mean0 = np.bincount(inv, s0["psi"]) / cnt
    mean1 = np.bincount(inv, s1["psi"]) / cnt
    assert np.allclose(mean1, mean0, rtol=0, atol=1e-14)
    ratio = 1 - dt * Cphi * Om / 2
    dev0 = s0["psi"] - mean0[inv]
    dev1 = s1["psi"] - mean0[inv]
    assert np.allclose(dev1, ratio * dev0, rtol=0, atol=1e-14)
    # element totals of psi are conserved (Sect. 3.3 statistics, no source, no walls on psi)
    e0 = np.bincount(s0["elem"], s0["psi"], minlength=grid_small.ne)
    e1 = np.bincount(s0["elem"], s1["psi"], minlength=grid_small.ne)
    assert np.allclose(e0, e1, atol=1e-12)


def test_eq11_c0_dissipates_energy_at_rate_eps(grid_small):
    """Eq. 11 (C0 from wp) makes the GLM consistent with dk/dt = -eps in homogeneous
    turbulence without production, for any wp: per step E[dk] = -eps dt + O(dt^2)."""
    k, Om, dt = 1.0, 1.0, 0.01
    F, eps = homogeneous_fields(grid_small, k, Om, 0.0)
    wp = np.array([[-0.6, 0.25, 0.0], [-0.1, -0.3, 0.05], [0.0, 0.15, -0.2]])   # anisotropic
    F[:, 14:23] = wp.reshape(9)
    P = base_params(nu=0.0, c0_mode=0, source_on=0, seed=27)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(800)
    s0 = o.get_particles()
    o.step(dt)
    s1 = o.get_particles()
    dk = 0.5 * ((s1["u"] ** 2 + s1["v"] ** 2 + s1["w"] ** 2) - (s0["u"] ** 2 + s0["v"] ** 2 + s0["w"] ** 2))
    sel = _middle(s0, 0.05, 0.95)
    dk = dk[sel]
    G = (wp - 0.5 * eps * np.eye(3)) / k
    Rs = np.cov(np.stack([s0[c][sel] for c in ("u", "v", "w")]))
    second = 0.5 * dt * dt * np.trace(G @ Rs @ G.T)
    # sample-covariance correction of the first-order term: tr(G (R_s - R)) dt
    first = dt * np.trace(G @ (Rs - (2 * k / 3) * np.eye(3)))
    assert abs(dk.mean() - (-eps * dt + first + second)) < 5 * dk.std() / math.sqrt(dk.size)
    assert abs(dk.mean() / (-eps * dt) - 1) < 0.1


def test_eq20_mean_frequency_source(grid_small):
    """Eq. 19 averaged with <omega> = Om: E[omega'] = Om (1 - S_omega Om dt), and Eq. 20 makes
    S_omega = C_w2 - C_w1 P / eps with production P = -<u v> dU/dy (the only shear here)."""
    Om, dt, S, uv = 2.0, 1e-3, 4.0, -0.1
    k = 1.0
    F, eps = homogeneous_fields(grid_small, k, Om, 0.0, grad=(0, S, 0, 0, 0, 0))
    F[:, 26] = uv
    C3, Cw1, Cw2 = 5.0, 0.5, 0.73
    P = base_params(nu=0.0, c0_mode=1, C0=0.0, source_on=0, seed=28, C3=C3, Cw1=Cw1, Cw2=Cw2)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(500)
    s0 = o.get_particles()
    s0["om"][:] = Om
    s0["u"][:] = s0["v"][:] = s0["w"][:] = 0.0
    o.set_particles(s0, 0)
    o.step(dt)
    w1 = o.get_particles()["om"]
    prod = -uv * S
    Sw = Cw2 - Cw1 * prod / eps
    sd = math.sqrt(2 * C3 * 0.25 * Om ** 3 * dt)
    assert abs(w1.mean() - Om * (1 - Sw * Om * dt)) < 5 * sd / math.sqrt(w1.size)
    assert abs(w1.std() / sd - 1) < 0.02


@pytest.mark.parametrize("case", ["no_mean_flow", "source_term"])
def test_eq25_micromixing_time_limits(grid_small, case):
    """Eq. 25 limits: with zero mean velocity the first argument is infinite, so
    t_m = max(k/eps, C_T sqrt(nu/eps)) = 1/Om for nu = 0; with C_t = 0 and a large k/eps
    it reduces to t_m = C_s (r0^2/eps)^(1/3).  Checked through the IECM decay ratio."""
    Om, dt = 3.0, 1e-3
    if case == "no_mean_flow":
        k, U, Cs, Ct, r0 = 1e-6, (0.0, 0.0, 0.0), 0.02, 0.7, 0.02
    else:
        k, U, Cs, Ct, r0 = 1e4, (1e-3, 0.0, 0.0), 0.5, 0.0, 0.05
    F, eps = homogeneous_fields(grid_small, k, Om, 0.0, U=U)
    P = base_params(nu=0.0, c0_mode=1, C0=0.0, tm_mode=0, Cs=Cs, Ct=Ct, src_r=r0, source_on=0,
                    seed=29, bins=(1, 1, 1), min_per_bin=1, C3=0.0, Cw1=0.0, Cw2=0.0)
    o = _homog_oracle(grid_small, P, F)
    o.init_particles(30)
    s0 = o.get_particles()
    rng = np.random.default_rng(5)
    s0["psi"] = rng.uniform(0, 1, s0["x"].size)
    s0["u"][:] = s0["v"][:] = s0["w"][:] = 0.0
    o.set_particles(s0, 0)
    s0 = o.get_particles()
    o.step(dt)
    s1 = o.get_particles()
    mean0 = np.bincount(s0["elem"], s0["psi"]) / np.bincount(s0["elem"])
    ratio = (s1["psi"] - mean0[s0["elem"]]) / (s0["psi"] - mean0[s0["elem"]])
    tm = 1.0 / Om if case == "no_mean_flow" else Cs * (r0 * r0 / eps) ** (1.0 / 3.0)
    assert np.allclose(ratio, 1 - dt / tm, rtol=1e-9)


# --------------------------------------------------------------------------------------
# Walls (Sect. 3.8)
# --------------------------------------------------------------------------------------

def test_wall_hit_probability_reflection_principle():
    """Eqs. 53-55: a particle at distance d from the wall with only viscous diffusion hits
    the wall during dt with probability P(d* < 0) + E[1{d* >= 0} f_w] = 2 Phi(-d/sigma),
    sigma^2 = 2 nu dt (reflection principle).  Hit particles get U = 0 (Eq. 56) and a
    gamma frequency with mean omega_w and variance C4 omega_w^2 (Eq. 58)."""
    g = synth.channel_grid(40, 6, seed=5)
    nu, dt, omw, C4 = 1e-3, 1e-3, 4.0, 0.25
    sig = math.sqrt(2 * nu * dt)
    F, _ = homogeneous_fields(g, 1e-12, 1.0, nu, omega_w=omw)
    # C3 = C_w1 = C_w2 = 0 freezes Eq. 19, so only the wall condition changes omega
    P = base_params(nu=nu, c0_mode=1, C0=0.0, C3=0.0, Cw1=0.0, Cw2=0.0, source_on=0, seed=26)
    o = oracle.Oracle(g, P, F)
    n = 30000
    rng = np.random.default_rng(4)
    for frac in (0.3, 1.0, 2.0):
        d = frac * sig
        x = rng.uniform(0, g.period_x, n)
        y = np.full(n, d)
        elem = np.array([o.brute(xi, d) for xi in x], dtype=np.int32)
        st = dict(x=x, y=y, u=np.zeros(n), v=np.zeros(n), w=np.zeros(n), om=np.ones(n),
                  psi=np.zeros(n), elem=elem)
        o.set_particles(st, 1)
        o.reset_diag()
        o.step(dt)
        dg = o.diag()
        s1 = o.get_particles()
        expected = 2 * stats.norm.cdf(-frac)
        frac_hit = dg["wall_hits"] / n
        assert abs(frac_hit - expected) < 5 * math.sqrt(expected * (1 - expected) / n)
        assert abs(dg["wall_hits_a"] / n - expected / 2) < 5 * math.sqrt(expected / 2 / n)
        assert s1["y"].min() >= 0.0
        hit = s1["om"] != 1.0                  # frequency was resampled by the wall condition
        assert hit.sum() == dg["wall_hits"]
        assert np.all(s1["u"][hit] == 0) and np.all(s1["v"][hit] == 0)
        if frac == 0.3:
            wv = s1["om"][hit]
            assert stats.kstest(wv, stats.gamma(a=1 / C4, scale=C4 * omw).cdf).pvalue > 1e-3


# --------------------------------------------------------------------------------------
# Binning (Sect. 3.5, Appendix A)
# --------------------------------------------------------------------------------------

def _bin_setup(counts, bins, mpb, seed=8):
    g = synth.channel_grid(8, 5, seed=6)
    F, _ = homogeneous_fields(g, 1e-4, 1.0, 0.0)
    P = base_params(nu=0.0, bins=bins, min_per_bin=mpb, source_on=0, seed=seed)
    o = oracle.Oracle(g, P, F)
    rng = np.random.default_rng(seed)
    xs, ys, es = [], [], []
    for e, c in enumerate(counts):
        xy = _unwrapped_vertices(g, e)
        for _ in range(c):
            p = rng.dirichlet([1, 1, 1]) @ xy
            xs.append(p[0] % g.period_x)
            ys.append(p[1])
            es.append(e)
    n = len(xs)
    st = dict(x=np.array(xs), y=np.array(ys), u=rng.normal(size=n), v=rng.normal(size=n),
              w=rng.normal(size=n), om=np.ones(n), psi=rng.uniform(size=n),
              elem=np.array(es, dtype=np.int32))
    # a few exact ties, as after no-slip wall hits
    st["u"][::7] = 0.0
    o.set_particles(st, 0)
    return g, o, st


def test_binning_worked_example():
    row = [l.split() for l in open(os.path.join(GOLDEN, "binning_worked_example.txt"))
           if l.strip() and not l.startswith("#")][0]
    N, b1, b2, b3, mpb, g1, g2, g3 = map(int, row)
    counts = [N] + [40] * 63
    g, o, st = _bin_setup(counts, (b1, b2, b3), mpb)
    v, gb = o.bins()
    assert tuple(gb[0]) == (g1, g2, g3)
    s = o.get_particles()
    idx = np.where(s["elem"] == 0)[0]
    order = sorted(idx, key=lambda p: (s["u"][p], p))
    # two groups of sizes 3 and 2 (Appendix A, i = 2 n / 5), the lower u in group 0
    assert [int(s["cp"][p]) for p in order] == [0, 0, 0, 1, 1]
    assert abs(v[0, 0] - s["psi"][order[:3]].mean()) < 1e-15
    assert abs(v[0, 1] - s["psi"][order[3:]].mean()) < 1e-15


def test_binning_uniform_counts_effective_bins():
    # 5x5x5 bins, at least 2 per bin: 150 -> 5*5*3 = 75, 300 -> 125, 1 -> 1, 9 -> 4*1*1
    counts = [150, 300, 1, 9, 0] + [20] * 59
    g, o, _ = _bin_setup(counts, (5, 5, 5), 2)
    _, gb = o.bins()
    assert tuple(gb[0]) == (5, 5, 3)
    assert tuple(gb[1]) == (5, 5, 5)
    assert tuple(gb[2]) == (1, 1, 1)
    assert tuple(gb[3]) == (4, 1, 1)
    assert tuple(gb[4]) == (1, 1, 1)


@pytest.mark.parametrize("bins,mpb", [((4, 4, 4), 2), ((3, 2, 5), 3), ((1, 4, 2), 2)])
def test_binning_characterisation(bins, mpb):
    """Sect. 3.5: bins are as equal in size as possible (App. A sizes), each holds at least
    min_per_bin particles, and bins are nested: level-1 groups are ordered by (u, id),
    inside them level-2 groups by (v, id), inside those the bins by (w, id).  The
    conditional mean of a bin is the mean scalar of its members."""
    rng = np.random.default_rng(9)
    counts = list(rng.integers(0, 130, 64))
    g, o, _ = _bin_setup(counts, bins, mpb)
    s = o.get_particles()
    v, gb = o.bins()
    for e in range(g.ne):
        idx = np.where(s["elem"] == e)[0]
        N = idx.size
        g1, g2, g3 = gb[e]
        G = g1 * g2 * g3
        assert G * mpb <= max(N, mpb)
        if N == 0:
            continue
        cp = s["cp"][idx].astype(int)
        sizes = np.bincount(cp, minlength=G)
        assert sizes.size == G
        expect = np.bincount((G * np.arange(N)) // N, minlength=G)
        assert np.array_equal(sizes, expect)
        if N >= mpb:
            assert sizes.min() >= mpb
        lvl1, lvl2 = cp // (g2 * g3), cp // g3
        for a, b in ((lvl1, None), (lvl2, lvl1), (cp, lvl2)):
            key = {id(lvl1): "u", id(lvl2): "v", id(cp): "w"}[id(a)]
            for grp in (np.unique(b) if b is not None else [None]):
                sel = np.ones(N, bool) if grp is None else (b == grp)
                sub_a = a[sel]
                vals = s[key][idx][sel]
                ids = idx[sel]
                for i in np.unique(sub_a)[:-1]:
                    lo = max(zip(vals[sub_a == i], ids[sub_a == i]))
                    hi = min(zip(vals[sub_a > i], ids[sub_a > i]))
                    assert lo < hi
        means = np.bincount(cp, s["psi"][idx], minlength=G) / sizes
        assert np.allclose(v[e, :G], means, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------------------
# Statistics (Sect. 3.3)
# --------------------------------------------------------------------------------------

def test_element_and_nodal_moments_definition():
    g, o, st = _bin_setup([50] * 30 + [0] * 2 + [1] + [50] * 31, (2, 2, 2), 2, seed=12)
    s = o.get_particles()
    em, cnt = o.element_stats()
    nm = o.nodal_stats()
    e = s["elem"]
    N = np.bincount(e, minlength=g.ne)
    assert np.array_equal(cnt, N)
    safe = np.maximum(N, 1)
    cols = {}
    for i, k in enumerate(("u", "v", "w")):
        cols[k] = np.bincount(e, s[k], minlength=g.ne) / safe
        assert np.allclose(em[:, 1 + i], cols[k], atol=1e-14)
    pairs = [("u", "u"), ("v", "v"), ("w", "w"), ("u", "v"), ("u", "w"), ("v", "w")]
    for j, (a, b) in enumerate(pairs):
        c = np.bincount(e, (s[a] - cols[a][e]) * (s[b] - cols[b][e]), minlength=g.ne) / safe
        assert np.allclose(em[:, 4 + j], c, atol=1e-14)
    mp = np.bincount(e, s["psi"], minlength=g.ne) / safe
    assert np.allclose(em[:, 11], mp, atol=1e-14)
    assert np.allclose(em[:, 12], np.bincount(e, (s["psi"] - mp[e]) ** 2, minlength=g.ne) / safe,
                       atol=1e-14)
    assert em[32, 4] == 0.0 and em[32, 0] == 1.0          # one particle: zero variance
    # nodes: plain mean over surrounding non-empty elements
    for n in range(g.nn):
        es = [k for k in range(g.ne) if n in g.tri[k] and N[k] > 0]
        if es:
            assert np.allclose(nm[n], em[es].mean(0), atol=1e-14)
        else:
            assert np.all(nm[n] == 0)


def test_moments_closed_form_two_values():
    g = synth.channel_grid(8, 5, seed=6)
    F, _ = homogeneous_fields(g, 1e-4, 1.0, 0.0)
    o = oracle.Oracle(g, base_params(nu=0.0, source_on=0), F)
    xy = _unwrapped_vertices(g, 3).mean(0)
    n = 4
    st = dict(x=np.full(n, xy[0] % g.period_x), y=np.full(n, xy[1]), u=np.array([1.0, -1.0, 1.0, -1.0]),
              v=np.array([2.0, 2.0, 0.0, 0.0]), w=np.zeros(n), om=np.array([1.0, 3.0, 1.0, 3.0]),
              psi=np.array([0.0, 1.0, 1.0, 0.0]), elem=np.full(n, 3, dtype=np.int32))
    o.set_particles(st, 0)
    em, _ = o.element_stats()
    # N, U, V, W, uu, vv, ww, uv, uw, vw, omega, phi, phi'^2
    assert np.allclose(em[3], [4, 0, 1, 0, 1, 1, 0, 0, 0, 0, 2, 0.5, 0.25], atol=1e-15)


# --------------------------------------------------------------------------------------
# Particle-number control (Sect. 3.7, Appendix B)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_redistribution_counts_properties(seed):
    rng = np.random.default_rng(seed)
    ne = 300
    counts = rng.integers(0, 60, ne).astype(np.int32)
    counts[rng.integers(0, ne, 20)] = rng.integers(100, 400, 20)
    minnpel = 25
    fin, moves = oracle.redistribution_counts(counts, minnpel)
    assert fin.sum() == counts.sum()
    deficit = np.maximum(minnpel - counts, 0)
    # feasible here: min reaches MINNPEL with exactly the deficit moved, one particle each
    assert fin.min() >= minnpel
    assert moves == deficit.sum()
    gain = fin - counts
    assert np.all(gain[counts >= minnpel] <= 0)          # only deficient elements receive
    assert np.all(fin[gain > 0] == minnpel)              # ...and only up to the threshold
    # donors are drained from the top: every donor ends at the same level or one above
    donors = gain < 0
    top = fin[donors]
    assert top.max() - top.min() <= 1
    assert np.all(counts[~donors & (gain == 0)] <= top.max())


def test_redistribution_infeasible_levels_out():
    counts = np.array([0, 0, 1, 10, 3], dtype=np.int32)
    fin, moves = oracle.redistribution_counts(counts, 100)
    assert fin.sum() == counts.sum()
    assert fin.max() - fin.min() <= 1
    fin2, moves2 = oracle.redistribution_counts(counts, 0)
    assert moves2 == 0 and np.array_equal(fin2, counts)


def test_redistribution_moves_particles():
    g = synth.channel_grid(8, 5, seed=6)
    F, _ = homogeneous_fields(g, 1e-4, 1.0, 0.0)
    counts = [40] * 64
    counts[5] = 0
    counts[9] = 2
    counts[20] = 140
    g, o, st = _bin_setup(counts, (2, 2, 2), 2, seed=13)
    o.set_params(base_params(nu=0.0, bins=(2, 2, 2), min_per_bin=2, source_on=0, seed=13,
                             minnpel=10, period_x=g.period_x))
    o.set_fields(F)
    s0 = o.get_particles()
    o.advance(1e-9)
    s_adv = o.get_particles()
    T = o.redistribute()
    s1 = o.get_particles()
    assert T == 18
    moved = np.where(s1["elem"] != s_adv["elem"])[0]
    assert moved.size == T
    # movers come from the donor (the fullest element), highest particle ids first
    donor_ids = np.where(s_adv["elem"] == 20)[0]
    assert set(moved) == set(np.sort(donor_ids)[-T:])
    for p in moved:
        r = s1["elem"][p]
        assert r in (5, 9)
        assert o.brute(s1["x"][p], s1["y"][p]) == r or o.lam(r, s1["x"][p], s1["y"][p]).min() > -1e-12
        src = r if counts[r] > 0 else None
        res = np.where(s_adv["elem"] == (src if src is not None else -1))[0]
        if src is not None:
            match = (s_adv["u"][res] == s1["u"][p]) & (s_adv["om"][res] == s1["om"][p])
            assert match.any()
    fin = np.bincount(s1["elem"], minlength=g.ne)
    assert fin[5] == 10 and fin[9] == 10


# --------------------------------------------------------------------------------------
# Whole step on the channel workload
# --------------------------------------------------------------------------------------

def test_step_tracking_and_domain(w2k):
    o = oracle.Oracle(w2k["grid"], w2k["params"], w2k["fields"])
    o.init_particles(20)
    s0 = o.get_particles()
    n0 = s0["x"].size
    for _ in range(3):
        o.step(w2k["dt"])
    s = o.get_particles()
    assert s["x"].size == n0
    assert s["y"].min() >= 0 and s["y"].max() <= 1
    assert s["x"].min() >= 0 and s["x"].max() < w2k["grid"].period_x
    rng = np.random.default_rng(5)
    for p in rng.integers(0, n0, 2000):
        e = s["elem"][p]
        assert o.lam(e, s["x"][p], s["y"][p]).min() >= -1e-12
    d = o.diag()
    assert d["lost"] == 0 and d["walk_brute"] == 0
    for k in ("u", "v", "w", "om", "psi"):
        assert np.all(np.isfinite(s[k]))


def test_init_particles_distribution(w2k):
    o = oracle.Oracle(w2k["grid"], w2k["params"], w2k["fields"])
    o.init_particles(30)
    s = o.get_particles()
    ne = w2k["grid"].ne
    assert np.array_equal(np.bincount(s["elem"], minlength=ne), np.full(ne, 30))
    for p in range(0, s["x"].size, 97):
        assert o.lam(s["elem"][p], s["x"][p], s["y"][p]).min() >= -1e-12
    # standardised velocity fluctuations about the local mean: N(0,1)
    z = []
    for p in range(0, s["x"].size, 3):
        e = s["elem"][p]
        q = o.interp(e, o.lam(e, s["x"][p], s["y"][p]))
        k = 0.5 * (q[23] + q[24] + q[25])
        z.append((s["u"][p] - q[0]) / math.sqrt(2 * k / 3))
        z.append(s["om"][p] / q[29])
    z = np.array(z)
    zu, zo = z[0::2], z[1::2]
    assert stats.kstest(zu, "norm").pvalue > 1e-3
    assert stats.kstest(zo, stats.gamma(a=4, scale=0.25).cdf).pvalue > 1e-3
    psi_in = (((s["x"] - 0.5) ** 2 + (s["y"] - 0.5) ** 2) <= 0.02 ** 2)
    assert np.array_equal(s["psi"] == 1.0, psi_in)


def test_element_subset_initialisation_matches_the_full_one():
    """orc_init_elements gives the listed elements' particles of a full initialisation (same
    ids, same draws), and a step of a subset given with its ids moves those particles as the
    full run does (the oracle following a sample of a run too large for it)."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    P = dict(w["params"], minnpel=0)
    full = oracle.Oracle(g, P, w["fields"])
    full.init_particles(30)
    sf = full.get_particles()
    elems = [3, 17, 40, 41, 63]
    sub = oracle.Oracle(g, P, w["fields"])
    sub.init_elements(30, elems)
    ss = sub.get_particles()
    ids = sub.pids()
    assert np.array_equal(ids, np.concatenate([np.arange(e * 30, e * 30 + 30) for e in elems]))
    for k in ("x", "y", "u", "v", "w", "om", "psi", "elem", "cp"):
        assert np.array_equal(ss[k], sf[k][ids]), k
    eo, _ = full.element_stats()
    es, _ = sub.element_stats()
    assert np.array_equal(es[elems], eo[elems])
    full.step(w["dt"])
    sub.step(w["dt"])
    sf, ss = full.get_particles(), sub.get_particles()
    for k in ("x", "y", "u", "v", "w", "om", "psi", "elem"):
        assert np.array_equal(ss[k], sf[k][ids]), k
    # the same subset given as a state with its ids
    sub2 = oracle.Oracle(g, P, w["fields"])
    st0 = oracle.Oracle(g, P, w["fields"])
    st0.init_elements(30, elems)
    sub2.set_particles(st0.get_particles(), 0, pid=st0.pids())
    sub2.step(w["dt"])
    assert np.array_equal(sub2.get_particles()["x"], ss["x"])


def _element_state(g, elems, n_per, rng, psi_fn):
    """Particles at random points of the given elements, Gaussian velocities, psi = psi_fn."""
    xs, ys, es = [], [], []
    for e in elems:
        xy = g.node_xy[g.tri[e]].copy()
        for k in (1, 2):
            d = xy[k, 0] - xy[0, 0]
            if g.period_x > 0 and abs(d) > g.period_x / 2:
                xy[k, 0] -= np.sign(d) * g.period_x
        lam = rng.dirichlet([2, 2, 2], size=n_per)
        p = lam @ xy
        xs.append(np.mod(p[:, 0], g.period_x) if g.period_x > 0 else p[:, 0])
        ys.append(p[:, 1])
        es.append(np.full(n_per, e, dtype=np.int32))
    n = n_per * len(elems)
    u, v, w = rng.normal(1.0, 0.3, n), rng.normal(0.0, 0.2, n), rng.normal(0.0, 0.25, n)
    return dict(x=np.concatenate(xs), y=np.concatenate(ys), u=u, v=v, w=w,
                om=np.full(n, 1.0), psi=psi_fn(u, v, w), elem=np.concatenate(es))


def test_fox_projection_orders_by_the_scalar_when_it_is_linear_in_velocity():
    """Eqs. 64-66: if phi' = c . u' exactly, alpha_a / s_a = c_a / s_phi, so the projected
    velocity is phi' / s_phi and the N_c conditional means are the means of the quantile
    groups of psi (sorted psi cut into N_c equal intervals)."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    rng = np.random.default_rng(41)
    elems = [5, 20, 33]
    st = _element_state(g, elems, 60, rng, lambda u, v, w_: 0.3 + 0.5 * u - 0.2 * v + 0.1 * w_)
    P = dict(w["params"], cond_mode=1, fox_bins=5, min_per_bin=2)
    o = oracle.Oracle(g, P, w["fields"])
    o.set_particles(st, 0)
    vc, gb = o.bins()
    for e in elems:
        psi = np.sort(st["psi"][st["elem"] == e])
        n = psi.shape[0]
        assert tuple(gb[e]) == (5, 1, 1)
        for i in range(5):
            lo, hi = -(-i * n // 5), -(-(i + 1) * n // 5)
            assert abs(vc[e, i] - psi[lo:hi].mean()) <= 1e-12
        assert np.all(np.diff(vc[e, :5]) > 0)


def test_fox_projection_degenerates_to_id_order_without_scalar_variance():
    """psi constant: s_phi = 0, alpha = 0, every particle has U_rho = 0 and the intervals
    follow particle ids; conditional means equal the constant."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    rng = np.random.default_rng(42)
    st = _element_state(g, [7], 40, rng, lambda u, v, w_: np.full(u.shape, 0.25))
    P = dict(w["params"], cond_mode=1, fox_bins=4, min_per_bin=2)
    o = oracle.Oracle(g, P, w["fields"])
    o.set_particles(st, 0)
    vc, gb = o.bins()
    assert tuple(gb[7]) == (4, 1, 1)
    assert np.all(vc[7, :4] == 0.25)
    cp = o.get_particles()["cp"]
    assert np.array_equal(cp, (4 * np.arange(40)) // 40)


# ----------------------------------------------------------------------------------------
# The simplified model of the particle-redistribution test (Sect. 3.7, Eqs. 46-52)
# ----------------------------------------------------------------------------------------

def _redist_run(ppe, alpha, steps, U0=(0.0, 0.0, 0.0), minnpel=0, seed=31):
    w = synth.redistribution_workload("redist_tiny", ppe=ppe)
    g = w["grid"]
    P = dict(w["params"], alpha=alpha, minnpel=minnpel, seed=seed)
    F = synth.uniform_fields(g.nn, U=U0, uu=(1.0, 1.0, 1.0, 0.0, 0.0, 0.0))
    o = oracle.Oracle(g, P, F)
    o.init_particles(ppe)
    return w, g, o


@pytest.mark.parametrize("alpha", [0.5, 0.0])
def test_simplified_model_mean_and_variance_closed_forms(alpha):
    """Eqs. 46-49 under Euler-Maruyama: the ensemble mean obeys Eq. 49,
    m_n = m_0 (1 - (1 - alpha) dt)^n (the interpolated nodal mean is the ensemble mean of a
    homogeneous field), and each component's fluctuation is the discrete OU process
    var_n = r^(2n) var_0 + 2 dt (1 - r^(2n)) / (1 - r^2), r = 1 - dt, whatever alpha is
    (alpha <U> is common to all particles; free-slip reflection only flips the sign of v)."""
    ppe, n = 400, 60
    w, g, o = _redist_run(ppe, alpha, n, U0=(1.0, 0.0, 0.5))
    dt = w["dt"]
    st0 = o.get_particles()
    m0 = np.array([st0[k].mean() for k in ("u", "w")])
    v0 = np.array([st0[k].var() for k in ("u", "v", "w")])
    for _ in range(n):
        o.step(dt)
    st = o.get_particles()
    N = st["u"].size
    assert o.diag()["freeslip_hits"] > 0
    m = np.array([st[k].mean() for k in ("u", "w")])
    decay = (1.0 - (1.0 - alpha) * dt) ** n
    # statistical error of a mean of N unit-variance samples, plus the noise the per-step
    # increments add (at most sqrt(1/N))
    assert np.all(np.abs(m - m0 * decay) < 6.0 * math.sqrt(2.0 / N)), (m, m0 * decay)
    r = 1.0 - dt
    var = np.array([st[k].var() for k in ("u", "v", "w")])
    var_n = r ** (2 * n) * v0 + 2.0 * dt * (1.0 - r ** (2 * n)) / (1.0 - r * r)
    assert np.all(np.abs(var / var_n - 1.0) < 6.0 * math.sqrt(2.0 / N)), (var, var_n)


def test_simplified_model_with_redistribution_keeps_counts_and_variance():
    """Sect. 3.7 with particle-number control on the stretched grid (MINNPEL = ppe / 10,
    Eq. 51): particles are moved, no element stays below MINNPEL, and the ensemble variance
    stays on the discrete OU steady approach toward 2 / (2 - dt) (the paper's analytic
    steady state <u_i u_j> = delta_ij up to the Euler-Maruyama factor) within the
    statistical error plus the perturbation the copied velocities bring."""
    ppe, n = 200, 80
    w, g, o = _redist_run(ppe, 0.5, n, minnpel=20)
    dt = w["dt"]
    v0 = np.array([o.get_particles()[k].var() for k in ("u", "v", "w")])
    for _ in range(n):
        o.step(dt)
        _, cnt = o.element_stats()
        assert cnt.min() >= 20
    assert o.diag()["moves"] > 0
    st = o.get_particles()
    N = st["u"].size
    r = 1.0 - dt
    var = np.array([st[k].var() for k in ("u", "v", "w")])
    var_n = r ** (2 * n) * v0 + 2.0 * dt * (1.0 - r ** (2 * n)) / (1.0 - r * r)
    assert np.all(np.abs(var / var_n - 1.0) < 8.0 * math.sqrt(2.0 / N)), (var, var_n)


def test_simplified_model_rejects_no_slip_walls():
    w = synth.workload("channel_tiny")
    o = oracle.Oracle(w["grid"], dict(w["params"], model=1), w["fields"])
    o.init_particles(5)
    with pytest.raises(Exception):
        o.step(1e-3)


# ----------------------------------------------------------------------------------------
# Scalar post-processing (Sect. 4.1.2, Eqs. 67-69)
# ----------------------------------------------------------------------------------------

def test_scalar_stats_iem_uniform_closed_forms():
    """With one conditioning bin (IEM: <phi|V> = <phi> = 1/2) and psi evenly spaced on
    [0, 1], Eq. 67 gives t_m <2 Gamma (grad phi)^2 | psi> = psi (1 - psi); on the empirical
    PDF at bin centres the integral is low by dpsi^2 / 8, so the result is psi (1 - psi) -
    dpsi^2 / 4 exactly.  Eq. 68 gives 1/2, the conditional diffusion 1/2 - psi, and the mean
    dissipation (Eq. 67 integrated over psi) is 2 <phi'^2>.  Moments are those of the
    discrete uniform distribution; an empty element gives zeros."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    nb, m = 20, 10
    N = nb * m
    st = _element_state(g, [9], N, np.random.default_rng(5), lambda u, v, w_: np.zeros(u.shape))
    st["psi"] = (np.arange(N) + 0.5) / N
    P = dict(w["params"], bins=(1, 1, 1), min_per_bin=1)
    o = oracle.Oracle(g, P, w["fields"])
    o.set_particles(st, 0)
    s = o.scalar_stats([9, 10], nb)
    dpsi = 1.0 / nb
    centre = (np.arange(nb) + 0.5) * dpsi
    assert np.array_equal(s["count"][0], np.full(nb, m))
    assert np.all(s["count"][1] == 0) and np.all(s["mom"][1] == 0) and np.all(s["cdiss"][1] == 0)
    np.testing.assert_allclose(s["phit"][0], 0.5, atol=1e-14)
    np.testing.assert_allclose(s["cdiff"][0], 0.5 - centre, atol=1e-14)
    np.testing.assert_allclose(s["cdiss"][0], centre * (1 - centre) - dpsi ** 2 / 4, atol=1e-13)
    mean, m2, m3, m4, lo, hi = s["mom"][0]
    assert abs(mean - 0.5) < 1e-15 and lo == st["psi"][0] and hi == st["psi"][-1]
    assert abs(m2 - (N * N - 1) / (12.0 * N * N)) < 1e-15
    assert abs(m3) < 1e-15
    assert abs(m4 - (N * N - 1) * (3.0 * N * N - 7) / (240.0 * N ** 4)) < 1e-15
    chi = float(np.sum(s["cdiss"][0] * s["count"][0])) / N
    assert abs(chi - 2.0 * m2) < dpsi ** 2


def test_scalar_stats_conditional_means_balance_on_a_real_state():
    """After IECM steps with a source (channel_tiny), the conditional means are bin means
    (Appendix A), so over an element sum_p (psi_p - <phi|V>_p) = 0: the Eq. 67 integral
    reaches zero at psi = 1 (sum over bins of count * conditional diffusion), and Eq. 68's
    phi~ weighted by the counts returns <phi>."""
    w = synth.workload("channel_tiny")
    o = oracle.Oracle(w["grid"], w["params"], w["fields"])
    o.init_particles(60)
    for _ in range(5):
        o.step(w["dt"])
    em, cnt = o.element_stats()
    elems = np.arange(w["grid"].ne)
    s = o.scalar_stats(elems, 50)
    N = s["count"].sum(axis=1)
    assert np.array_equal(N, cnt)
    bal = np.sum(s["cdiff"] * s["count"], axis=1)
    assert np.all(np.abs(bal) <= 1e-12 * np.maximum(N, 1))
    mean_from_phit = np.sum(s["phit"] * s["count"], axis=1) / np.maximum(N, 1)
    np.testing.assert_allclose(mean_from_phit[N > 0], em[N > 0, 11], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s["mom"][N > 0, 0], em[N > 0, 11], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s["mom"][N > 0, 1], em[N > 0, 12], rtol=1e-9, atol=1e-14)


def test_free_slip_reflection_beyond_the_start_element():
    """Sect. 4.2 with the walk's reflection: a particle starting in an element with no
    boundary line (second row of the stretched grid) that crosses the whole boundary row in
    one step ends at the mirror image of X + U dt across y = 0 (Eq. 46 moves it with U^n,
    without noise), in an element that contains it, counted once as a free-slip hit."""
    w = synth.redistribution_workload("redist_tiny")
    g = w["grid"]
    ys = np.sort(np.unique(np.round(g.node_xy[:, 1], 12)))
    row1 = ys[1]
    y_of = g.node_xy[g.tri, 1]                                     # [ne, 3]
    start = [e for e in range(g.ne) if y_of[e].min() > 0.5 * row1 and y_of[e].max() < 0.5]
    e0 = min(start, key=lambda e: y_of[e].min())                   # lowest such element
    lam = np.array([1.0, 1.0, 1.0]) / 3.0
    xy = g.node_xy[g.tri[e0]].copy()
    for k in (1, 2):
        d = xy[k, 0] - xy[0, 0]
        if abs(d) > g.period_x / 2:
            xy[k, 0] -= np.sign(d) * g.period_x
    x0, y0 = lam @ xy
    x0 %= g.period_x
    dt = w["dt"]
    target = -0.3 * row1                                          # below y = 0 before reflection
    st = dict(x=np.array([x0]), y=np.array([y0]), u=np.array([0.1]),
              v=np.array([(target - y0) / dt]), w=np.array([0.0]), om=np.array([1.0]),
              psi=np.array([0.0]), elem=np.array([e0], dtype=np.int32))
    P = dict(w["params"], minnpel=0)
    o = oracle.Oracle(g, P, w["fields"])
    o.set_particles(st, 0)
    o.step(dt)
    s = o.get_particles()
    assert abs(s["y"][0] - (-target)) <= 1e-14
    assert abs(((s["x"][0] - (x0 + 0.1 * dt)) + 0.5) % 1.0 - 0.5) <= 1e-14
    assert o.lam(int(s["elem"][0]), s["x"][0], s["y"][0]).min() >= -1e-12
    d = o.diag()
    assert d["freeslip_hits"] == 1 and d["lost"] == 0


# ----------------------------------------------------------------------------------------
# Corner walls of the street canyon (reading of Sect. 3.8 for corners)
# ----------------------------------------------------------------------------------------

def _one_particle_step(g, F, params, x, y, u, v, e=None):
    o = oracle.Oracle(g, params, F)
    if e is None:
        e = next(f for f in range(g.ne) if o.lam(f, x, y).min() >= 0.0)
    st = dict(x=np.array([x]), y=np.array([y]), u=np.array([u]), v=np.array([v]),
              w=np.array([0.0]), om=np.array([1.0]), psi=np.array([0.0]),
              elem=np.array([e], dtype=np.int32))
    o.set_particles(st, 0)
    return o


def test_concave_corner_reflects_across_both_walls():
    """Cavity floor y = 0 meets the cavity wall x = 1.5.  With nu = 0 Eq. 7 moves the
    particle by U dt alone; a particle driven across both wall lines is reflected across
    each (the second from the first's image), ending at the double mirror image; Eq. 56
    stops it and the hit counts once."""
    w = synth.canyon_workload("canyon_2k")
    g = w["grid"]
    P = dict(w["params"], nu=0.0, minnpel=0, source_on=0)
    h, dt = 0.004, 1e-3
    x0, y0 = 1.5 + 0.3 * h, 0.3 * h
    o = _one_particle_step(g, w["fields"], P, x0, y0, -0.8 * h / dt, -0.8 * h / dt)
    o.step(dt)
    s = o.get_particles()
    assert abs(s["x"][0] - (1.5 + 0.5 * h)) <= 1e-13 and abs(s["y"][0] - 0.5 * h) <= 1e-13
    assert s["u"][0] == 0.0 and s["v"][0] == 0.0 and s["w"][0] == 0.0
    assert o.lam(int(s["elem"][0]), s["x"][0], s["y"][0]).min() >= -1e-12
    d = o.diag()
    assert d["wall_hits"] == 1 and d["lost"] == 0


def test_convex_corner_applies_only_the_wall_in_front():
    """The channel floor y = 1 meets the cavity wall x = 1.5 at a convex corner.  A particle
    just left of the corner moving down crosses the floor line and is reflected across it
    alone: the cavity wall's line, oriented into the cavity, has the particle's element
    behind it and is not applied."""
    w = synth.canyon_workload("canyon_2k")
    g = w["grid"]
    P = dict(w["params"], nu=0.0, minnpel=0, source_on=0)
    h, dt = 0.004, 1e-3
    x0, y0 = 1.5 - 0.3 * h, 1.0 + 0.3 * h
    o = _one_particle_step(g, w["fields"], P, x0, y0, 0.0, -0.8 * h / dt)
    o.step(dt)
    s = o.get_particles()
    assert abs(s["x"][0] - x0) <= 1e-13 and abs(s["y"][0] - (1.0 + 0.5 * h)) <= 1e-13
    assert s["v"][0] == 0.0
    d = o.diag()
    assert d["wall_hits"] == 1 and d["lost"] == 0


def _in_canyon_domain(x, y, tol=1e-12):
    """The street-canyon domain: channel [0, 4] x [1, 2] over cavity [1.5, 2.5] x [0, 1]."""
    chan = (y >= 1.0 - tol) & (y <= 2.0 + tol)
    cav = (x >= 1.5 - tol) & (x <= 2.5 + tol) & (y >= -tol) & (y <= 1.0 + tol)
    return chan | cav


def test_walk_equals_brute_force_on_the_canyon():
    """Sect. 3.6 on the street canyon: from random elements to random points of the domain
    a few elements away (through the periodic seam and around the cavity's re-entrant
    corners), the walk with its fall-back finds the element brute force finds."""
    w = synth.canyon_workload("canyon_2k")
    g = w["grid"]
    o = oracle.Oracle(g, w["params"], w["fields"])
    rng = np.random.default_rng(8)
    n = 0
    while n < 3000:
        e0 = int(rng.integers(0, g.ne))
        xy = _unwrapped_vertices(g, e0)
        p = xy.mean(0) + rng.normal(0, 0.08, 2)
        x = p[0] % g.period_x
        if not _in_canyon_domain(np.array([x]), np.array([p[1]]), -1e-9)[0]:
            continue
        n += 1
        e, hops = o.walk(e0, x, p[1])
        b = o.brute(x, p[1])
        assert b >= 0 and e >= 0, (e0, x, p[1])
        if e != b:
            assert o.lam(e, x, p[1]).min() > -1e-12
            assert o.lam(b, x, p[1]).min() > -1e-12


def test_canyon_steps_keep_particles_in_the_domain():
    """P12 on the street canyon (walls, corners, free-slip top, particle-number control):
    after 10 steps every particle lies in the domain and in its element, none is lost, and
    the particle count is unchanged."""
    w = synth.canyon_workload("canyon_2k")
    P = dict(w["params"], minnpel=w["ppe"] - 2)
    o = oracle.Oracle(w["grid"], P, w["fields"])
    o.init_particles(w["ppe"])
    n0 = o.np_
    for _ in range(10):
        o.step(5e-4)
    s = o.get_particles()
    assert s["x"].size == n0
    assert np.all(_in_canyon_domain(s["x"], s["y"]))
    rng = np.random.default_rng(6)
    for p in rng.integers(0, n0, 3000):
        assert o.lam(int(s["elem"][p]), s["x"][p], s["y"][p]).min() >= -1e-12
    d = o.diag()
    assert d["lost"] == 0 and d["wall_hits"] > 0 and d["moves"] > 0
    for k in ("u", "v", "w", "om", "psi"):
        assert np.all(np.isfinite(s[k]))


def test_cfl_time_step_closed_form():
    """Eq. 26 on an unjittered lattice, where every triangle has area dx dy / 2 and so
    every A_n does: with all particles at U = (2, 0, 0), omega = psi = 0 the nodal mean
    vectors have norm 2 and dt = CFL sqrt(dx dy / 2) / 2; with psi = 1 the literal norm of
    Z = (V, omega, psi) is sqrt(5).  A step with dt <= 0 takes that dt."""
    nx, ny = 8, 6
    g = synth.channel_grid(nx, ny, lx=2.0, jitter_x=0.0, jitter_y=0.0, seed=1)
    dx, dy = 2.0 / nx, 1.0 / (ny - 1)
    F = synth.uniform_fields(g.nn, U=(2.0, 0.0, 0.0))
    P = base_params(period_x=g.period_x, source_on=0, cfl=0.7)
    st = _element_state(g, list(range(g.ne)), 6, np.random.default_rng(3),
                        lambda u, v, w_: np.zeros(u.shape))
    for k, val in (("u", 2.0), ("v", 0.0), ("w", 0.0), ("om", 0.0)):
        st[k] = np.full(st["u"].shape, val)
    for psi, norm in ((0.0, 2.0), (1.0, math.sqrt(5.0))):
        st["psi"] = np.full(st["u"].shape, psi)
        o = oracle.Oracle(g, P, F)
        o.set_particles(st, 0)
        expect = 0.7 * math.sqrt(0.5 * dx * dy) / norm
        assert abs(o.cfl_dt() / expect - 1.0) < 1e-14
        o.step(0.0)
        assert abs(o.last_dt / expect - 1.0) < 1e-14


# ----------------------------------------------------------------------------------------
# Eulerian derivatives from nodal values (Sect. 3.4, Eqs. 39-40)
# ----------------------------------------------------------------------------------------

def _same_diagonal_lattice(nx, ny, lx=2.0):
    """A periodic lattice on [0, lx] x [0, 1] with every quad split along the same diagonal
    (so every interior node's star has as many elements above as below), walls at y = 0, 1."""
    xs, ys = np.arange(nx) * (lx / nx), np.linspace(0.0, 1.0, ny)
    X, Y = np.meshgrid(xs, ys)
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    tri = []
    for j in range(ny - 1):
        for i in range(nx):
            a, b = j * nx + i, j * nx + (i + 1) % nx
            c, d = (j + 1) * nx + (i + 1) % nx, (j + 1) * nx + i
            tri += [[a, b, c], [a, c, d]]
    tri = np.array(tri, dtype=np.int32)
    y = xy[:, 1]
    tag = np.zeros(tri.shape, dtype=np.int8)
    for k in range(3):
        p, q = tri[:, (k + 1) % 3], tri[:, (k + 2) % 3]
        tag[:, k] = (((y[p] == 0) & (y[q] == 0)) | ((y[p] == 1) & (y[q] == 1))).astype(np.int8)
    return synth.Grid(node_xy=xy, tri=tri, edge_tag=tag, period_x=lx)


def test_node_gradient_linear_and_quadratic():
    """Eqs. 39-40 with the node transfer: a field linear in y has the exact gradient at every
    node of a jittered periodic grid (element gradients are exact, their means too); y^2 on
    a lattice whose interior nodes see as many elements above as below gets 2y at the
    interior nodes, and the second pass gets the exact second derivative 2 at nodes two rows
    or more from the boundaries."""
    g = synth.channel_grid(12, 9, jitter_x=0.2, jitter_y=0.1, seed=6)
    o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
    y = g.node_xy[:, 1]
    gr = o.node_gradient(1.0 + 2.0 * y)
    assert np.abs(gr[:, 0]).max() < 1e-12 and np.abs(gr[:, 1] - 2.0).max() < 1e-12
    g = _same_diagonal_lattice(12, 9)
    o = oracle.Oracle(g, base_params(period_x=g.period_x), synth.uniform_fields(g.nn))
    y = g.node_xy[:, 1]
    h = 1.0 / 8
    g1 = o.node_gradient(y * y)
    inner = (y > 0.5 * h) & (y < 1 - 0.5 * h)
    assert np.abs(g1[inner, 1] - 2 * y[inner]).max() < 1e-12 and np.abs(g1[:, 0]).max() < 1e-12
    g2 = o.node_gradient(g1[:, 1])
    deep = (y > 1.5 * h) & (y < 1 - 1.5 * h)
    assert np.abs(g2[deep, 1] - 2.0).max() < 1e-12


def test_derived_fields_from_statistics():
    """The fields the particles' statistics provide: <U_i>, <u_i u_j> and <omega> are the
    nodal moments; the gradient and laplacian slots are the node transfers of Eqs. 39-40
    applied once and twice; the slots of the Eulerian solves are kept."""
    w = synth.workload("channel_tiny")
    o = oracle.Oracle(w["grid"], w["params"], w["fields"])
    o.init_particles(60)
    o.step(w["dt"])
    before = o.fields()
    o.derive_fields()
    f, m = o.fields(), o.nodal_stats()
    np.testing.assert_array_equal(f[:, 0:3], m[:, 1:4])
    np.testing.assert_array_equal(f[:, 23:29], m[:, 4:10])
    np.testing.assert_array_equal(f[:, 29], m[:, 10])
    for i in range(3):
        g1 = o.node_gradient(m[:, 1 + i])
        np.testing.assert_array_equal(f[:, 5 + 2 * i:7 + 2 * i], g1)
        lap = o.node_gradient(g1[:, 0])[:, 0] + o.node_gradient(g1[:, 1])[:, 1]
        np.testing.assert_allclose(f[:, 11 + i], lap, rtol=0, atol=1e-12 * max(1.0, np.abs(lap).max()))
    for k in (3, 4, 14, 15, 16, 17, 18, 19, 20, 21, 22, 30):
        np.testing.assert_array_equal(f[:, k], before[:, k])


def test_velocity_correction_closed_form():
    """Eq. 31 (rho = 1) with a nodal pressure change linear in y, dP = b y: its gradient is
    (0, b) in every element of a jittered periodic grid, so every particle's v drops by
    exactly dt b and u, w are unchanged."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    o = oracle.Oracle(g, w["params"], w["fields"])
    o.init_particles(20)
    s0 = o.get_particles()
    b, dt = 3.0, 0.01
    o.correct_velocity(b * g.node_xy[:, 1], dt)
    s = o.get_particles()
    np.testing.assert_allclose(s["v"], s0["v"] - dt * b, rtol=0, atol=1e-13)
    np.testing.assert_allclose(s["u"], s0["u"], rtol=0, atol=1e-13)
    assert np.array_equal(s["w"], s0["w"]) and np.array_equal(s["x"], s0["x"])
