"""CUDA path vs the CPU oracle, element by element, from the same seeded inputs.

Tolerances (relative, with a per-quantity scale floor so values near zero compare on an
absolute scale):  FP64 form: particle states 1e-12, statistics 1e-10, element indices,
conditioning pointers and effective bins bit-exact.  FP32 form: states 1e-5, statistics
1e-6; particles whose element or wall decision sits within the FP32 rounding band of a
threshold are exempt, counted and bounded.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1006_0532_gb300 import synth
from helpers import STATE_KEYS, base_params, homogeneous_fields, period_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0532_gb300 import _binding as B  # noqa: E402


def gpu_ctx(grid, params, fields, precision=0, sort_every=4):
    p = dict(params)
    p.setdefault("period_x", grid.period_x)
    p.update(precision=precision, sort_every=sort_every)
    c = B.Context(p)
    c.set_grid(grid)
    c.set_fields(fields)
    return c


def scale_of(a):
    s = float(np.sqrt(np.mean(np.square(a)))) if a.size else 1.0
    return s if s > 0 else 1.0


def compare_state(g, o, L, tol, skip=None):
    """Max relative error over particles (skip: boolean mask of exempt particles)."""
    worst = {}
    for k in STATE_KEYS:
        a, b = g[k], o[k]
        if k == "x":
            d = np.abs(period_diff(a, b, L))
        else:
            d = np.abs(a - b)
        r = d / np.maximum(np.abs(b), scale_of(b))
        if skip is not None:
            r = r[~skip]
        worst[k] = float(r.max()) if r.size else 0.0
    bad = {k: v for k, v in worst.items() if v > tol}
    assert not bad, bad
    return worst


# Reynolds-stress columns of the statistics layout and the variances that bound them.
_PAIRS = {4: (4, 4), 5: (5, 5), 6: (6, 6), 7: (4, 5), 8: (4, 6), 9: (5, 6)}


def compare_stats(a, b, tol, rows=None, stats_layout=True):
    """Relative error per entry.  Floor: the column's RMS; for a covariance <u_i u_j> also
    sqrt(<u_i u_i><u_j u_j>) of the same row (the scale of a correlation coefficient)."""
    if rows is not None:
        a, b = a[rows], b[rows]
    sc = np.array([scale_of(b[:, j]) for j in range(b.shape[1])])
    den = np.maximum(np.abs(b), sc[None, :])
    if stats_layout and b.shape[1] == 13:
        for col, (i, j) in _PAIRS.items():
            den[:, col] = np.maximum(den[:, col], np.sqrt(np.abs(b[:, i] * b[:, j])))
    r = np.abs(a - b) / den
    assert r.max() <= tol, (float(r.max()), np.unravel_index(np.argmax(r), r.shape))
    return float(r.max())


def both(name, ppe=None, precision=0, **over):
    w = synth.workload(name)
    params = dict(w["params"])
    params.update(over)
    g = w["grid"]
    o = oracle.Oracle(g, params, w["fields"])
    c = gpu_ctx(g, params, w["fields"], precision=precision)
    return w, g, o, c, (ppe or w["ppe"])


# ----------------------------------------------------------------------------------------
# FP64 form
# ----------------------------------------------------------------------------------------

def test_init_matches_oracle_f64():
    w, g, o, c, ppe = both("channel_2k", ppe=25)
    o.init_particles(ppe)
    c.init_particles(ppe)
    so, sg = o.get_particles(), c.get_particles()
    assert np.array_equal(sg["elem"], so["elem"])
    compare_state(sg, so, g.period_x, 1e-12)
    assert np.array_equal(sg["cp"], so["cp"])
    vo, go = o.bins()
    vg, gg = c.bins()
    assert np.array_equal(gg, go)
    compare_stats(vg, vo, 1e-12, stats_layout=False)
    eo, co = o.element_stats()
    eg, cg = c.element_stats()
    assert np.array_equal(cg, co)
    compare_stats(eg, eo, 1e-10)
    compare_stats(c.nodal_stats(), o.nodal_stats(), 1e-10)


@pytest.mark.parametrize("name,steps", [("channel_tiny", 3), ("channel_2k", 10)])
def test_steps_match_oracle_f64(name, steps):
    """The plain FP64 workload: 211,600 particles on 2116 triangles, 10 steps."""
    w, g, o, c, ppe = both(name)
    o.init_particles(ppe)
    c.init_particles(ppe)
    for _ in range(steps):
        o.step(w["dt"])
        c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    # element indices bit-exact except for particles on a shared edge (either element)
    diff = sg["elem"] != so["elem"]
    for p in np.where(diff)[0]:
        assert o.lam(sg["elem"][p], sg["x"][p], sg["y"][p]).min() > -1e-12
    assert diff.sum() <= 2
    compare_state(sg, so, g.period_x, 1e-12)
    if diff.sum() == 0:
        assert np.array_equal(sg["cp"], so["cp"])
        vo, go = o.bins()
        vg, gg = c.bins()
        assert np.array_equal(gg, go)
        compare_stats(vg, vo, 1e-10, stats_layout=False)
        eo, co = o.element_stats()
        eg, cg = c.element_stats()
        assert np.array_equal(cg, co)
        compare_stats(eg, eo, 1e-10)
        compare_stats(c.nodal_stats(), o.nodal_stats(), 1e-10)
    dg, do = c.diag(), o.diag()
    assert dg["error"] == 0 and dg["lost"] == 0
    assert dg["wall_hits"] == do["wall_hits"]
    assert dg["hops_total"] == do["hops_total"]
    assert dg["hop_hist"] == do["hop_hist"]            # particles per number of walk hops
    if name == "channel_2k":
        assert sum(dg["hop_hist"][1:]) > 0


def _imbalanced_state(g, counts, seed):
    rng = np.random.default_rng(seed)
    xs, ys, es = [], [], []
    for e, n in enumerate(counts):
        tri = g.tri[e]
        xy = g.node_xy[tri].copy()
        for k in (1, 2):
            d = xy[k, 0] - xy[0, 0]
            if d > g.period_x / 2:
                xy[k, 0] -= g.period_x
            elif d < -g.period_x / 2:
                xy[k, 0] += g.period_x
        w = rng.dirichlet([1, 1, 1], size=n)
        p = w @ xy
        xs.append(p[:, 0] % g.period_x)
        ys.append(p[:, 1])
        es.append(np.full(n, e, dtype=np.int32))
    x, y, e = np.concatenate(xs), np.concatenate(ys), np.concatenate(es)
    n = x.size
    return dict(x=x, y=y, u=0.9 + 0.05 * rng.normal(size=n), v=0.05 * rng.normal(size=n),
                w=0.05 * rng.normal(size=n), om=rng.gamma(4, 0.25 * 3.0, size=n),
                psi=rng.uniform(size=n), elem=e)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_redistribution_matches_oracle_f64(seed):
    """Appendix B with MINNPEL above some counts: final counts, movers, their new states."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    rng = np.random.default_rng(100 + seed)
    counts = rng.integers(20, 80, g.ne)
    counts[rng.integers(0, g.ne, 6)] = rng.integers(0, 6, 6)     # includes empty elements
    counts[rng.integers(0, g.ne, 3)] = rng.integers(150, 300, 3)
    st = _imbalanced_state(g, counts, seed)
    params = dict(w["params"], minnpel=15)
    o = oracle.Oracle(g, params, w["fields"])
    c = gpu_ctx(g, params, w["fields"])
    o.set_particles(st, 7)
    c.set_particles(st, 7)
    o.step(w["dt"])
    c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    assert np.array_equal(sg["elem"], so["elem"])
    compare_state(sg, so, g.period_x, 1e-12)
    assert c.diag()["moves"] == o.diag()["moves"] > 0
    eo, co = o.element_stats()
    eg, cg = c.element_stats()
    assert np.array_equal(cg, co)
    assert cg.min() >= 15
    compare_stats(eg, eo, 1e-10)
    assert np.array_equal(sg["cp"], so["cp"])
    compare_stats(c.nodal_stats(), o.nodal_stats(), 1e-10)


def test_large_element_path_and_empty_elements():
    """Elements above the 768-particle binning tiles go through the large-element kernel."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    counts = np.full(g.ne, 30)
    counts[3] = 1500
    counts[10] = 3000
    counts[11] = 0
    counts[12] = 1
    st = _imbalanced_state(g, counts, 5)
    o = oracle.Oracle(g, w["params"], w["fields"])
    c = gpu_ctx(g, w["params"], w["fields"])
    o.set_particles(st, 0)
    c.set_particles(st, 0)
    for _ in range(2):
        o.step(w["dt"])
        c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    assert np.array_equal(sg["elem"], so["elem"])
    assert np.array_equal(sg["cp"], so["cp"])
    compare_state(sg, so, g.period_x, 1e-12)
    eo, _ = o.element_stats()
    eg, _ = c.element_stats()
    compare_stats(eg, eo, 1e-10)
    vo, go = o.bins()
    vg, gg = c.bins()
    assert np.array_equal(gg, go)
    compare_stats(vg, vo, 1e-10, stats_layout=False)


@pytest.mark.parametrize("fox", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_binning_split_changes_no_result(precision, fox):
    """Every size-class split of the binning (the tile of 256 for elements up to the split,
    tiles of 512 and 768 above it, the large-element kernels beyond; bucket ranks for the
    hierarchical bins, chunk sorts for Fox's projection)
    gives the same pointers, bins and statistics bit for bit, with the hierarchical bins and
    with Fox's projection; in FP64 they are the oracle's, and the re-ordered state keeps
    every particle's values.  Out-of-range shapes are refused."""
    w = synth.workload("channel_tiny")
    w = dict(w, params=dict(w["params"], cond_mode=1, fox_bins=16) if fox else w["params"])
    g = w["grid"]
    rng = np.random.default_rng(17)
    counts = rng.integers(1, 60, g.ne)
    counts[rng.choice(g.ne, 24, replace=False)] = np.concatenate(
        [rng.integers(100, 257, 8), rng.integers(257, 513, 8), rng.integers(513, 1025, 4),
         [768, 769, 1200, 2000]])
    st = _imbalanced_state(g, counts, 8)
    ref = None
    for split in (256, 0, 100, 192):
        c = gpu_ctx(g, w["params"], w["fields"], precision=precision)
        c.set_launch_shapes(tile_split=split)
        assert c.launch_shapes()["tile_split"] == split
        c.set_particles(st, 0)
        sg = c.get_particles()
        if precision == 0:
            for k in ("u", "v", "w", "om", "psi"):
                assert np.array_equal(sg[k], st[k]), k
        out = (sg["cp"], c.element_stats()[0], *c.bins(), c.nodal_stats())
        if ref is None:
            ref = out
        else:
            for a, b in zip(out, ref):
                assert np.array_equal(a, b)
        assert c.check() == 0
        c.close()
    if precision == 0:
        o = oracle.Oracle(g, w["params"], w["fields"])
        o.set_particles(st, 0)
        assert np.array_equal(ref[0], o.get_particles()["cp"])
        vo, go = o.bins()
        assert np.array_equal(ref[3], go)
        compare_stats(ref[2], vo, 1e-10, stats_layout=False)
        compare_stats(ref[1], o.element_stats()[0], 1e-10)
    c = gpu_ctx(g, w["params"], w["fields"], precision=precision)
    for bad in (dict(tile_split=300), dict(adv_block=96)):
        with pytest.raises(B.PdfxError):
            c.set_launch_shapes(**bad)
    c.close()


def test_empty_state():
    w = synth.workload("channel_tiny")
    g = w["grid"]
    c = gpu_ctx(g, w["params"], w["fields"])
    e = np.zeros(0)
    c.set_particles(dict(x=e, y=e, u=e, v=e, w=e, om=e, psi=e, elem=np.zeros(0, np.int32)), 0)
    c.step(w["dt"])
    em, cnt = c.element_stats()
    assert cnt.sum() == 0 and np.all(em == 0)
    assert c.check() == 0


def test_capacity_error_is_reported():
    w = synth.workload("channel_tiny")
    g = w["grid"]
    counts = np.full(g.ne, 5)
    counts[0] = 5000                       # above PDFX_MAX_PER_ELEMENT
    st = _imbalanced_state(g, counts, 6)
    c = gpu_ctx(g, w["params"], w["fields"])
    c.set_particles(st, 0)
    assert c.check() == -7


def test_homogeneous_ou_statistics_gpu():
    """The OU closed form (Eq. 27) holds for the GPU path too (FP64 form)."""
    g = synth.channel_grid(16, 9, seed=4)
    k, Om, C0, dt, n = 1.5e-4, 1.0, 2.0, 0.05, 40
    F, eps = homogeneous_fields(g, k, Om, 0.0, p_iso=0.0, dP=(-0.01, 0.0))
    P = base_params(nu=0.0, c0_mode=1, C0=C0, source_on=0, seed=21)
    c = gpu_ctx(g, P, F)
    c.init_particles(400)
    for _ in range(n):
        c.step(dt)
    st = c.get_particles()
    m = (st["y"] > 0.2) & (st["y"] < 0.8)
    a = (eps / 2) / k
    r = 1 - a * dt
    var_n = r ** (2 * n) * (2 * k / 3) + C0 * eps / (a * (2 - a * dt)) * (1 - r ** (2 * n))
    N = int(m.sum())
    for key in ("u", "v", "w"):
        assert abs(st[key][m].var() / var_n - 1) < 5 * math.sqrt(2.0 / N)


# ----------------------------------------------------------------------------------------
# FP32 form
# ----------------------------------------------------------------------------------------

def _round32(st):
    out = dict(st)
    for k in STATE_KEYS:
        out[k] = st[k].astype(np.float32).astype(np.float64)
    return out


@pytest.mark.parametrize("acc64", [0, 1])
def test_one_step_f32_matches_oracle(acc64):
    """FP32 form (acc64 = 0: compensated FP32 accumulation of moments and conditional
    means; acc64 = 1: FP64 accumulation) against the FP64 oracle."""
    w = synth.workload("channel_2k")
    g = w["grid"]
    params = dict(w["params"], acc64=acc64)
    F32 = w["fields"].astype(np.float32).astype(np.float64)
    o = oracle.Oracle(g, params, F32)
    o.init_particles(w["ppe"])
    s0 = _round32(o.get_particles())
    # geometry is rounded to FP32 on the GPU; keep particles clear of element edges there
    o.set_particles(s0, 0)
    c = gpu_ctx(g, params, F32, precision=1)
    c.set_particles(s0, 0)
    # initial statistics from identical FP32 values: exact pointers; moments within the
    # FP32-form tolerance (central products are formed in FP32)
    sg0 = c.get_particles()
    assert np.array_equal(sg0["cp"], o.get_particles()["cp"])
    compare_stats(c.element_stats()[0], o.element_stats()[0], 1e-6)
    # conditional means: FP32 sums of FP32 values over bins of a few particles
    vo, go = o.bins()
    vg, gg = c.bins()
    assert np.array_equal(gg, go)
    compare_stats(vg, vo, 1e-6, stats_layout=False)
    o.step(w["dt"])
    c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    # exemptions: element choice within the FP32 band of an edge
    diff = sg["elem"] != so["elem"]
    for p in np.where(diff)[0]:
        assert o.lam(sg["elem"][p], so["x"][p], so["y"][p]).min() > -1e-5
    assert diff.sum() <= 20
    worst = compare_state(sg, so, g.period_x, 1e-5, skip=diff)
    # nodal moments away from exempt particles
    bad_e = np.unique(np.concatenate([sg["elem"][diff], so["elem"][diff]]))
    eg, cg = c.element_stats()
    eo, co = o.element_stats()
    good_e = np.setdiff1d(np.arange(g.ne), bad_e)
    assert np.array_equal(cg[good_e], co[good_e])
    compare_stats(eg, eo, 1e-6, rows=good_e)
    vo, go = o.bins()
    vg, gg = c.bins()
    assert np.array_equal(gg[good_e], go[good_e])
    compare_stats(vg, vo, 1e-6, rows=good_e, stats_layout=False)
    bad_n = np.unique(g.tri[bad_e].ravel()) if bad_e.size else np.zeros(0, int)
    good_n = np.setdiff1d(np.arange(g.nn), bad_n)
    compare_stats(c.nodal_stats(), o.nodal_stats(), 1e-6, rows=good_n)
    assert c.check() == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_binning_with_tied_values(precision):
    """Velocities quantised to a few values per element make equal keys at every level;
    the particle id orders them (Sect. 3.5 reading).  Pointers, effective bins and the
    conditional means must equal the oracle's on the same (FP32-representable) state."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    o = oracle.Oracle(g, w["params"], w["fields"])
    o.init_particles(300)
    st = o.get_particles()
    for k in ("u", "v", "w"):
        st[k] = np.round(st[k] * 20.0) / 20.0
    st = _round32(st)
    o.set_particles(st, 0)
    c = gpu_ctx(g, w["params"], w["fields"], precision=precision)
    c.set_particles(st, 0)
    assert np.array_equal(c.get_particles()["cp"], o.get_particles()["cp"])
    vo, go = o.bins()
    vg, gg = c.bins()
    assert np.array_equal(gg, go)
    compare_stats(vg, vo, 1e-12 if precision == 0 else 1e-6, stats_layout=False)
    compare_stats(c.element_stats()[0], o.element_stats()[0], 1e-10 if precision == 0 else 1e-6)
    assert c.check() == 0


def test_street_canyon_steps_match_oracle_f64():
    """Street canyon (cavity under a periodic channel, free-slip top, walls on the floor and
    all cavity sides and corners): 38,400 particles on 1,920 triangles, 20 steps with
    particle-number control, FP64 form against the oracle."""
    w = synth.canyon_workload("canyon_2k")
    g = w["grid"]
    params = dict(w["params"], minnpel=w["ppe"] - 2)     # particle-number control fires
    o = oracle.Oracle(g, params, w["fields"])
    c = gpu_ctx(g, params, w["fields"])
    o.init_particles(w["ppe"])
    c.init_particles(w["ppe"])
    dt = 5e-4
    for _ in range(20):
        o.step(dt)
        c.step(dt)
    so, sg = o.get_particles(), c.get_particles()
    diff = sg["elem"] != so["elem"]
    for p in np.where(diff)[0]:
        assert o.lam(sg["elem"][p], sg["x"][p], sg["y"][p]).min() > -1e-12
    assert diff.sum() <= 2
    compare_state(sg, so, g.period_x, 1e-12)
    if diff.sum() == 0:
        assert np.array_equal(sg["cp"], so["cp"])
        eo, co = o.element_stats()
        eg, cg = c.element_stats()
        assert np.array_equal(cg, co)
        compare_stats(eg, eo, 1e-10)
        compare_stats(c.nodal_stats(), o.nodal_stats(), 1e-10)
    dg, do = c.diag(), o.diag()
    assert dg["error"] == 0 and dg["lost"] == 0
    assert dg["wall_hits"] == do["wall_hits"] and dg["wall_hits"] > 0
    assert dg["freeslip_hits"] == do["freeslip_hits"] and dg["freeslip_hits"] > 0
    assert dg["moves"] == do["moves"] and dg["moves"] > 0


# ----------------------------------------------------------------------------------------
# Fox's projection conditioning (Eqs. 64-66)
# ----------------------------------------------------------------------------------------

def _fox(params, nc=5):
    return dict(params, cond_mode=1, fox_bins=nc)


def test_fox_projection_steps_match_oracle_f64():
    """Conditioning on the projected velocity of Eq. 64 instead of the hierarchical
    velocity bins: pointers, effective bins (N_c, 1, 1), conditional means and the states
    they feed through Eq. 24, 10 steps on 2116 triangles (FP64 form)."""
    w = synth.workload("channel_2k")
    g = w["grid"]
    params = _fox(w["params"])
    o = oracle.Oracle(g, params, w["fields"])
    c = gpu_ctx(g, params, w["fields"])
    o.init_particles(w["ppe"])
    c.init_particles(w["ppe"])
    assert np.array_equal(c.get_particles()["cp"], o.get_particles()["cp"])
    vo, go = o.bins()
    vg, gg = c.bins()
    assert np.array_equal(gg, go)
    assert np.all(gg[:, 1:] == 1) and gg[:, 0].max() == 5
    compare_stats(vg, vo, 1e-10, stats_layout=False)
    for _ in range(10):
        o.step(w["dt"])
        c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    diff = sg["elem"] != so["elem"]
    for p in np.where(diff)[0]:
        assert o.lam(sg["elem"][p], sg["x"][p], sg["y"][p]).min() > -1e-12
    assert diff.sum() <= 2
    compare_state(sg, so, g.period_x, 1e-12)
    if diff.sum() == 0:
        assert np.array_equal(sg["cp"], so["cp"])
        vo, go = o.bins()
        vg, gg = c.bins()
        assert np.array_equal(gg, go)
        compare_stats(vg, vo, 1e-10, stats_layout=False)
    assert c.check() == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_fox_projection_large_and_degenerate_elements(precision):
    """Fox mode through the large-element kernel (1500 and 3000 particles), near-empty
    elements (N_c = 1) and elements whose scalar is constant (s_phi = 0: alpha = 0, every
    projected key ties and the particle id orders them)."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    counts = np.full(g.ne, 40)
    counts[3] = 1500
    counts[10] = 3000
    counts[11] = 0
    counts[12] = 1
    counts[13] = 7
    st = _round32(_imbalanced_state(g, counts, 8))
    # a scalar correlated with u (nonzero alpha), zero in a few elements (a zero mean and
    # variance are exact on both sides, however the sums are ordered)
    st["psi"] = np.clip(0.5 + 4.0 * (st["u"] - 0.9) + 0.1 * st["v"], 0.0, 1.0)
    for e in (5, 6, 10):
        st["psi"][st["elem"] == e] = 0.0
    st = _round32(st)
    params = _fox(w["params"], nc=8)
    o = oracle.Oracle(g, params, w["fields"])
    c = gpu_ctx(g, params, w["fields"], precision=precision)
    o.set_particles(st, 0)
    c.set_particles(st, 0)
    cg, co = c.get_particles()["cp"], o.get_particles()["cp"]
    vo, go = o.bins()
    vg, gg = c.bins()
    assert np.array_equal(gg, go)
    assert gg[11, 0] == 1 and gg[12, 0] == 1 and gg[3, 0] == 8
    if precision == 0:
        assert np.array_equal(cg, co)
        compare_stats(vg, vo, 1e-10, stats_layout=False)
    else:
        # FP32 keys: a pair of particles straddling an interval boundary may swap when
        # their projected velocities agree to FP32 rounding; such swaps move one interval
        tie_e = np.isin(st["elem"], (5, 6, 10, 11, 12))
        assert np.array_equal(cg[tie_e], co[tie_e])
        d = cg != co
        assert np.all(np.abs(cg[d].astype(int) - co[d].astype(int)) == 1)
        assert d.sum() <= 4
        rows = np.setdiff1d(np.arange(g.ne), np.unique(st["elem"][d]))
        compare_stats(vg, vo, 1e-6, rows=rows, stats_layout=False)
    # the degenerate elements are ordered by particle id alone
    for e in (5, 6, 10):
        sel = np.where(st["elem"] == e)[0]
        n, nc = sel.size, go[e, 0]
        pids = o.pids()[sel]
        rank = np.argsort(np.argsort(pids, kind="stable"), kind="stable")
        assert np.array_equal(co[sel], (nc * rank) // n)
    assert c.check() == 0


def test_cfl_steps_match_oracle_f64():
    """Steps with dt <= 0 take Eq. 26's step from the nodal means of the last statistics
    pass, on both sides: the step sizes agree to 1e-12 and the states as in the fixed-step
    parity."""
    w, g, o, c, ppe = both("channel_2k")
    o.init_particles(ppe)
    c.init_particles(ppe)
    for _ in range(5):
        o.step(0.0)
        c.step(0.0)
        assert abs(c.last_dt / o.last_dt - 1.0) <= 1e-12
        assert 0.0 < o.last_dt < 1.0
    so, sg = o.get_particles(), c.get_particles()
    diff = sg["elem"] != so["elem"]
    for p in np.where(diff)[0]:
        assert o.lam(sg["elem"][p], sg["x"][p], sg["y"][p]).min() > -1e-12
    assert diff.sum() <= 2
    compare_state(sg, so, g.period_x, 1e-12)
    assert c.check() == 0


def test_derived_fields_match_oracle_f64():
    """The fields the particles' statistics provide (Sect. 3.3-3.4, Eqs. 39-40): after two
    steps both sides derive them from their nodal statistics; the derived slots agree within
    1e-10 of each slot's RMS (they carry the statistics' summation-order rounding), the
    slots of the Eulerian solves are the values set; a step with the derived fields then
    gives states within 1e-10."""
    w, g, o, c, ppe = both("channel_2k")
    o.init_particles(ppe)
    c.init_particles(ppe)
    for _ in range(2):
        o.step(w["dt"])
        c.step(w["dt"])
    o.derive_fields()
    c.derive_fields()
    fo, fg = o.fields(), c.fields()
    derived = list(range(0, 3)) + list(range(5, 14)) + list(range(23, 30))
    for k in range(31):
        if k in derived:
            sc = max(float(np.sqrt(np.mean(fo[:, k] ** 2))), 1e-300)
            r = float(np.abs(fg[:, k] - fo[:, k]).max()) / sc
            assert r <= 1e-10, (k, r)
        else:
            assert np.array_equal(fg[:, k], w["fields"][:, k]), k
    assert np.abs(fo[:, 11:14]).max() > 0.0 and np.abs(fo[:, 5:11]).max() > 0.0
    o.step(w["dt"])
    c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    diff = sg["elem"] != so["elem"]
    assert diff.sum() <= 2
    compare_state(sg, so, g.period_x, 1e-10, skip=diff)
    assert c.check() == 0


def test_velocity_correction_matches_oracle_f64():
    """Eq. 31 applied to the particles with a random nodal pressure change (the periodic
    seam's elements included), then a step: states within 1e-12 of the oracle's."""
    w, g, o, c, ppe = both("channel_2k", ppe=40)
    o.init_particles(ppe)
    c.init_particles(ppe)
    dp = np.random.default_rng(17).normal(0.0, 1.0, g.nn)
    o.correct_velocity(dp, w["dt"])
    c.correct_velocity(dp, w["dt"])
    compare_state(c.get_particles(), o.get_particles(), g.period_x, 1e-12)
    o.step(w["dt"])
    c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    diff = sg["elem"] != so["elem"]
    assert diff.sum() <= 2
    compare_state(sg, so, g.period_x, 1e-12, skip=diff)
    assert c.check() == 0


# ----------------------------------------------------------------------------------------
# Element ids from the caller's device memory
# ----------------------------------------------------------------------------------------

def test_device_state_with_out_of_range_elements_is_refused_without_a_fault():
    """Element ids handed over in device memory are range-checked on the device: the load
    replaces an id outside the grid by element 0, counts it and raises PDFX_ERR_ELEMENT,
    which pdfx_set_particles returns.  Every later kernel sees ids inside the grid, so the
    state can still be stepped and its particles are relocated by the walk."""
    w = synth.workload("channel_tiny")
    g = w["grid"]
    c = gpu_ctx(g, w["params"], w["fields"])
    c.init_particles(w["ppe"])
    st = c.get_particles()
    dev = torch.device("cuda")
    d = {k: torch.from_numpy(np.ascontiguousarray(st[k])).to(dev) for k in STATE_KEYS}
    el = st["elem"].astype(np.int32).copy()
    el[3] = -1
    el[7] = g.ne
    d["elem"] = torch.from_numpy(el).to(dev)
    with pytest.raises(B.PdfxError) as exc:
        c.set_particles(d, 0)
    assert exc.value.code == -10
    diag = c.diag()
    assert diag["bad_element"] == 2 and diag["error"] == -10
    c.step(w["dt"])
    torch.cuda.synchronize()
    after = c.get_particles()
    assert np.all((after["elem"] >= 0) & (after["elem"] < g.ne))
    assert c.check() == -10
    c.close()
