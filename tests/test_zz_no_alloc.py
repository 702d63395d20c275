"""The no-allocation statistics entry point gives the same results as the regular one.

pdfx_element_stats_noalloc serves callers that cannot allocate device memory while they
run; it keeps its scratch in a fixed device array of the library.  Two calls in a row on
different particle states must each match what the context computes for that state
through the regular entry points (FP64: statistics to 1e-10, pointers and bins exactly).
"""
import numpy as np
import pytest

from paper_1006_0532_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0532_gb300 import _binding as B  # noqa: E402


def _rel(a, b):
    sc = np.maximum(np.sqrt(np.mean(b * b, axis=0, keepdims=True)), 1e-300)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), sc)))


def _noalloc(c, st):
    dev = torch.device("cuda")
    d = {k: torch.from_numpy(np.ascontiguousarray(st[k])).to(dev) for k in ("u", "v", "w", "om", "psi")}
    d["elem"] = torch.from_numpy(np.ascontiguousarray(st["elem"], dtype=np.int32)).to(dev)
    emom = torch.zeros((c.ne, 13), dtype=torch.float64, device=dev)
    vcce = torch.zeros((c.ne, c.G), dtype=torch.float64, device=dev)
    gbin = torch.zeros((c.ne, 3), dtype=torch.int32, device=dev)
    cp = torch.zeros(st["u"].shape[0], dtype=torch.uint8, device=dev)
    nmom = torch.zeros((c.nn, 13), dtype=torch.float64, device=dev)
    c.element_stats_noalloc(d, emom, vcce, gbin, cp, nmom)
    torch.cuda.synchronize()
    return emom.cpu().numpy(), vcce.cpu().numpy(), gbin.cpu().numpy(), cp.cpu().numpy(), nmom.cpu().numpy()


def test_noalloc_statistics_match_regular_entry_points():
    w = synth.workload("channel_2k")
    p = dict(w["params"], precision=0, sort_every=4, period_x=w["grid"].period_x)
    c = B.Context(p)
    c.set_grid(w["grid"])
    c.set_fields(w["fields"])
    c.init_particles(w["ppe"])
    for call in range(2):
        if call == 1:
            c.step(w["dt"])          # a different state for the second call
        st = c.get_particles()
        em_ref, cnt_ref = c.element_stats()
        v_ref, g_ref = c.bins()
        nm_ref = c.nodal_stats()
        em, v, g, cp, nm = _noalloc(c, st)
        assert np.array_equal(em[:, 0].astype(np.int64), cnt_ref)
        assert _rel(em, em_ref) <= 1e-10
        assert _rel(v, v_ref) <= 1e-10
        assert np.array_equal(g, g_ref)
        assert np.array_equal(cp, st["cp"])
        assert _rel(nm, nm_ref) <= 1e-10
    assert c.check() == 0
    c.close()


def test_noalloc_follows_the_contexts_fox_projection():
    """A context conditioned on Fox's projected velocity (cond_mode 1) gets Fox's intervals
    from the no-allocation entry point too, not the hierarchical bins."""
    w = synth.workload("channel_2k")
    p = dict(w["params"], precision=0, sort_every=4, period_x=w["grid"].period_x, cond_mode=1,
             fox_bins=16)
    c = B.Context(p)
    c.set_grid(w["grid"])
    c.set_fields(w["fields"])
    c.init_particles(w["ppe"])
    c.step(w["dt"])
    st = c.get_particles()
    em_ref, _ = c.element_stats()
    v_ref, g_ref = c.bins()
    em, v, g, cp, nm = _noalloc(c, st)
    assert np.array_equal(g, g_ref)
    assert np.all(g_ref[:, 1] == 1) and np.any(g_ref[:, 0] > 4)
    assert _rel(v, v_ref) <= 1e-10
    assert np.array_equal(cp, st["cp"])
    assert _rel(em, em_ref) <= 1e-10
    assert c.check() == 0
    c.close()


def test_noalloc_skips_and_reports_element_ids_outside_the_grid():
    """An element id outside the grid is left out of every element (no write outside the
    scratch) and raises PDFX_ERR_ELEMENT in the context's error word; the other elements'
    statistics are those of the regular entry points."""
    w = synth.workload("channel_2k")
    p = dict(w["params"], precision=0, sort_every=4, period_x=w["grid"].period_x)
    c = B.Context(p)
    c.set_grid(w["grid"])
    c.set_fields(w["fields"])
    c.init_particles(w["ppe"])
    st = c.get_particles()
    em_ref, _ = c.element_stats()
    k = 12345
    home = int(st["elem"][k])
    bad = dict(st)
    bad["elem"] = st["elem"].astype(np.int32).copy()
    bad["elem"][k] = c.ne + 7
    em, v, g, cp, nm = _noalloc(c, bad)
    others = np.arange(c.ne) != home
    assert np.array_equal(em[others], em_ref[others])
    assert int(em[home, 0]) == int(em_ref[home, 0]) - 1
    assert c.check() == -10
    assert c.diag()["bad_element"] == 1
    c.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    w = synth.workload("channel_tiny")
    c = B.Context(dict(w["params"], period_x=w["grid"].period_x))
    c.set_grid(w["grid"])
    n = (1 << 20) + 1
    dev = torch.device("cuda")
    big = {k: torch.zeros(1, dtype=torch.float64, device=dev) for k in ("u", "v", "w", "om", "psi")}
    big["elem"] = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    rc = B.lib().pdfx_element_stats_noalloc(c.h, n, *[B._ptr(big[k]) for k in ("u", "v", "w", "om", "psi", "elem")],
                                            B._ptr(out), B._ptr(out), B._ptr(out), B._ptr(out), None,
                                            B._stream(None))
    assert rc == -1
    c.close()
