"""Scalar statistics of probe elements (Sect. 4.1.2, Eqs. 67-69) on the GPU against the
oracle: bin counts exact, minimum and maximum exact on identical states (1e-12 after steps,
where the states agree to that); Eq. 68's phi~, the conditional diffusion and
dissipation and the moments within 1e-10 (FP64 form) or 1e-6 (FP32 form; 1e-5 for the
conditional dissipation, a running sum) relative, with each quantity's RMS as the floor."""
import numpy as np
import pytest

import oracle
from paper_1006_0532_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0532_gb300 import _binding as B  # noqa: E402


def _ctx(w, precision):
    p = dict(w["params"], precision=precision, sort_every=4, period_x=w["grid"].period_x)
    c = B.Context(p)
    c.set_grid(w["grid"])
    c.set_fields(w["fields"])
    return c


def _compare(sg, so, tol, exact_range=True, tol_cdiss=None):
    assert np.array_equal(sg["count"], so["count"])
    for k in ("phit", "cdiff", "cdiss"):
        a, b = sg[k], so[k]
        floor = max(float(np.sqrt(np.mean(b ** 2))), 1e-300)
        r = np.abs(a - b) / np.maximum(np.abs(b), floor)
        t = tol_cdiss if (k == "cdiss" and tol_cdiss is not None) else tol
        assert r.max() <= t, (k, float(r.max()))
    mg, mo = sg["mom"], so["mom"]
    if exact_range:
        assert np.array_equal(mg[:, 4:], mo[:, 4:])
    else:   # states that agree to 1e-12
        assert np.all(np.abs(mg[:, 4:] - mo[:, 4:]) <= 1e-12 * np.maximum(np.abs(mo[:, 4:]), 1.0))
    for k in range(4):
        floor = max(float(np.sqrt(np.mean(mo[:, k] ** 2))), 1e-300)
        r = np.abs(mg[:, k] - mo[:, k]) / np.maximum(np.abs(mo[:, k]), floor)
        assert r.max() <= tol, (k, float(r.max()))


def test_scalar_stats_match_oracle_f64():
    """Every element of the 2,116-triangle workload after 5 steps with the source on,
    200 bins: the particles near the source give non-trivial PDFs and conditional curves."""
    w = synth.workload("channel_2k")
    o = oracle.Oracle(w["grid"], w["params"], w["fields"])
    c = _ctx(w, 0)
    o.init_particles(w["ppe"])
    c.init_particles(w["ppe"])
    for _ in range(5):
        o.step(w["dt"])
        c.step(w["dt"])
    sp_g, sp_o = c.get_particles(), o.get_particles()
    assert np.array_equal(sp_g["elem"], sp_o["elem"]) and np.array_equal(sp_g["cp"], sp_o["cp"])
    elems = np.arange(w["grid"].ne, dtype=np.int32)
    sg, so = c.scalar_stats(elems, 200), o.scalar_stats(elems, 200)
    assert so["count"].sum() == sp_o["x"].size
    assert np.count_nonzero(so["cdiss"]) > 0           # some elements mix
    _compare(sg, so, 1e-10, exact_range=False)
    again = c.scalar_stats(elems, 200)
    for k in sg:
        assert np.array_equal(again[k], sg[k])          # fixed-point sums: bit for bit
    # the same state with psi spread over [0, 1] everywhere (every bin in use)
    st = sp_o
    st["psi"] = np.random.default_rng(9).beta(0.7, 1.3, st["psi"].size)
    o.set_particles(st, 5)
    c.set_particles(st, 5)
    assert np.array_equal(c.get_particles()["cp"], o.get_particles()["cp"])
    sg, so = c.scalar_stats(elems, 200), o.scalar_stats(elems, 200)
    assert np.count_nonzero(so["count"]) > 0.25 * so["count"].size   # ~100 particles, 200 bins
    _compare(sg, so, 1e-10)


def test_scalar_stats_match_oracle_f32_and_subset():
    """FP32 form on an FP32-representable state (identical particles on both sides): a
    subset of probe elements in a shuffled order, 64 bins."""
    w = synth.workload("channel_2k")
    o = oracle.Oracle(w["grid"], w["params"], w["fields"])
    o.init_particles(w["ppe"])
    for _ in range(3):
        o.step(w["dt"])
    st = o.get_particles()
    rng = np.random.default_rng(4)
    st["psi"] = np.clip(st["psi"] + 0.2 * rng.random(st["psi"].size), 0.0, 1.0)
    for k in ("x", "y", "u", "v", "w", "om", "psi"):
        st[k] = st[k].astype(np.float32).astype(np.float64)
    o.set_particles(st, 0)
    c = _ctx(w, 1)
    c.set_particles(st, 0)
    assert np.array_equal(c.get_particles()["cp"], o.get_particles()["cp"])
    elems = rng.permutation(w["grid"].ne)[:300].astype(np.int32)
    # the conditional dissipation is a running sum over up to N particles of psi - <phi|V>,
    # each <phi|V> carrying the FP32 form's rounding (~1e-7): 1e-5 for it
    _compare(c.scalar_stats(elems, 64), o.scalar_stats(elems, 64), 1e-6, tol_cdiss=1e-5)


def test_scalar_stats_rejects_bad_arguments():
    w = synth.workload("channel_tiny")
    c = _ctx(w, 0)
    c.init_particles(10)
    for elems, nb in (([0, 0], 10), ([-1], 10), ([w["grid"].ne], 10), ([0], 0), ([0], 5000)):
        with pytest.raises(B.PdfxError):
            c.scalar_stats(elems, nb)
