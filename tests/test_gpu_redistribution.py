"""The simplified model of the particle-redistribution test (Sect. 3.7, Eqs. 46-52) on the
GPU: parity with the oracle (FP64 form) and the closed-form ensemble statistics (FP32)."""
import math

import numpy as np
import pytest

import oracle
from paper_1006_0532_gb300 import synth
from helpers import STATE_KEYS, period_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0532_gb300 import _binding as B  # noqa: E402


def _ctx(w, params, precision):
    p = dict(params, precision=precision, sort_every=4)
    c = B.Context(p)
    c.set_grid(w["grid"])
    c.set_fields(w["fields"])
    return c


def test_simplified_model_steps_match_oracle_f64():
    """40 steps on the stretched 96-triangle grid with particle-number control firing
    (MINNPEL = ppe / 4): states 1e-12, element indices, move and reflection counts exact."""
    w = synth.redistribution_workload("redist_tiny", ratio=4)
    g = w["grid"]
    o = oracle.Oracle(g, w["params"], w["fields"])
    c = _ctx(w, w["params"], 0)
    o.init_particles(w["ppe"])
    c.init_particles(w["ppe"])
    for _ in range(40):
        o.step(w["dt"])
        c.step(w["dt"])
    so, sg = o.get_particles(), c.get_particles()
    diff = sg["elem"] != so["elem"]
    for p in np.where(diff)[0]:
        assert o.lam(sg["elem"][p], sg["x"][p], sg["y"][p]).min() > -1e-12
    assert diff.sum() <= 2
    for k in STATE_KEYS:
        d = np.abs(period_diff(sg[k], so[k], g.period_x)) if k == "x" else np.abs(sg[k] - so[k])
        assert (d / np.maximum(np.abs(so[k]), 1.0)).max() <= 1e-12, k
    dg, do = c.diag(), o.diag()
    assert dg["error"] == 0 and dg["lost"] == 0
    assert dg["moves"] == do["moves"] > 0
    assert dg["freeslip_hits"] == do["freeslip_hits"] > 0
    assert dg["wall_hits"] == 0
    if diff.sum() == 0:
        eo, co = o.element_stats()
        eg, cg = c.element_stats()
        assert np.array_equal(cg, co)
        assert cg.min() >= w["params"]["minnpel"]
        sc = np.maximum(np.abs(eo), np.sqrt(np.mean(eo ** 2, axis=0)) + 1e-300)
        assert (np.abs(eg - eo) / sc).max() <= 1e-10


def _ensemble_run(precision, minnpel, n=100):
    w = synth.redistribution_workload("redist_1k")
    params = dict(w["params"], minnpel=minnpel)
    c = _ctx(w, params, precision)
    c.init_particles(w["ppe"])
    st0 = c.get_particles()
    v0 = np.array([st0[k].var() for k in ("u", "v", "w")])
    dt = w["dt"]
    for _ in range(n):
        c.step(dt)
    st = c.get_particles()
    r = 1.0 - dt
    var = np.array([st[k].var() for k in ("u", "v", "w")])
    var_n = r ** (2 * n) * v0 + 2.0 * dt * (1.0 - r ** (2 * n)) / (1.0 - r * r)
    return c, st["u"].size, var, var_n


@pytest.mark.parametrize("precision", [1, 0])
def test_simplified_model_ensemble_statistics(precision):
    """The 1,536-triangle workload at 200 particles per element (307,200 particles), 100
    steps without particle-number control: the ensemble variance of each component follows
    the discrete OU transient toward 2 / (2 - dt); nothing is lost."""
    c, N, var, var_n = _ensemble_run(precision, 0)
    assert np.all(np.abs(var / var_n - 1.0) < 6.0 * math.sqrt(2.0 / N)), (var, var_n)
    d = c.diag()
    assert d["error"] == 0 and d["lost"] == 0 and d["moves"] == 0 and d["freeslip_hits"] > 0


def test_simplified_model_with_particle_number_control_on_the_stretched_grid():
    """Same run with MINNPEL = 20 (Eq. 51 ratio 10), FP32 form: every element keeps MINNPEL
    particles and nothing is lost.  The moved particles copy the velocities of residents of
    the thin wall cells, where a particle stays for a step only when its wall-normal velocity
    is small, so the variance falls below the closed form: the additional error of Sect. 3.7
    (measured: v 4% low after 100 steps).  It is bounded here at 10%."""
    c, N, var, var_n = _ensemble_run(1, 20)
    _, cnt = c.element_stats()
    assert cnt.min() >= 20
    d = c.diag()
    assert d["error"] == 0 and d["lost"] == 0 and d["moves"] > 0
    assert np.all(np.abs(var / var_n - 1.0) < 0.10), (var, var_n)


def test_simplified_model_refuses_no_slip_walls():
    w = synth.workload("channel_tiny")
    c = _ctx(w, dict(w["params"], model=1, period_x=w["grid"].period_x), 0)
    c.init_particles(5)
    with pytest.raises(B.PdfxError):
        c.step(1e-3)
