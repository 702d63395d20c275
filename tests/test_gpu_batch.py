"""Batched form: instances stepped together in one context must give, bit for bit, what each
instance gives alone (same grid, fields, parameters, seed and instance number)."""
import numpy as np
import pytest

from paper_1006_0532_gb300 import synth
from helpers import STATE_KEYS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
from paper_1006_0532_gb300 import _binding as B  # noqa: E402


def _instances():
    spec = [(120, 11, 30, (0.6, 0.4), 7), (300, 12, 20, (1.2, 0.5), 8), (200, 13, 40, (0.3, 0.7), 9)]
    out = []
    for k, (tri, seed, ppe, src, ps) in enumerate(spec):
        it = synth.channel_instance(tri, 392.0, seed=seed, ppe=ppe, src=src, philox_seed=ps, instance=k)
        it["params"]["minnpel"] = ppe - 1          # particle-number control fires (Appendix B)
        out.append(it)
    return out


def _mixed_instances():
    """Channel, street canyon (walls, corners, free-slip top; period 4 against 2), channel."""
    out = [synth.channel_instance(120, 392.0, seed=21, ppe=30, src=(0.6, 0.4), philox_seed=5,
                                  instance=0),
           synth.canyon_instance(1080, seed=22, ppe=20, src=(2.0, 0.5), philox_seed=6, instance=1),
           synth.channel_instance(200, 392.0, seed=23, ppe=25, src=(0.3, 0.7), philox_seed=7,
                                  instance=2)]
    for it in out:
        it["params"]["minnpel"] = it["ppe"] - 1
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mixed", [False, True])
def test_batch_matches_instances_run_alone(precision, mixed):
    """Channel instances, and a mix of channel and street-canyon instances (the ensemble's
    two kinds), stepped as one batch give each instance's results run alone bit for bit."""
    ins = _mixed_instances() if mixed else _instances()
    g, F, ef, nf = synth.union(ins)
    P = [dict(it["params"], precision=precision, sort_every=4) for it in ins]
    b = B.Context(P[0])
    b.set_instances(P, ef)
    b.set_grid(g)
    b.set_fields(F)
    b.init_particles_batch([it["ppe"] for it in ins])
    alone = []
    for it, p in zip(ins, P):
        c = B.Context(p)
        c.set_grid(it["grid"])
        c.set_fields(it["fields"])
        c.init_particles(it["ppe"])
        alone.append(c)
    dt = 1e-3 if mixed else 2e-3
    for _ in range(7):
        b.step(dt)
        for c in alone:
            c.step(dt)
    ef2, pf = b.instance_ranges()
    assert np.array_equal(ef2, ef)
    sb = b.get_particles()
    eb, cb = b.element_stats()
    nb = b.nodal_stats()
    vb, gb = b.bins()
    moves = 0
    for k, c in enumerate(alone):
        sa = c.get_particles()
        sl = slice(int(pf[k]), int(pf[k + 1]))
        assert pf[k + 1] - pf[k] == sa["x"].shape[0]
        for key in STATE_KEYS:
            assert np.array_equal(sb[key][sl], sa[key]), key
        assert np.array_equal(sb["elem"][sl] - ef[k], sa["elem"])
        assert np.array_equal(sb["cp"][sl], sa["cp"])
        ea, ca = c.element_stats()
        es = slice(int(ef[k]), int(ef[k + 1]))
        assert np.array_equal(cb[es], ca)
        assert np.array_equal(eb[es], ea)
        assert np.array_equal(nb[int(nf[k]):int(nf[k + 1])], c.nodal_stats())
        va, ga = c.bins()
        assert np.array_equal(vb[es], va)
        assert np.array_equal(gb[es], ga)
        moves += c.diag()["moves"]
        assert c.check() == 0
    assert moves > 0
    assert b.diag()["moves"] == moves
    assert b.check() == 0


def test_batch_rejects_mismatched_or_connected_instances():
    ins = _instances()
    g, F, ef, nf = synth.union(ins)
    P = [dict(it["params"]) for it in ins]
    b = B.Context(P[0])
    bad = [dict(P[0]), dict(P[1], bins=(2, 2, 2)), dict(P[2])]
    with pytest.raises(B.PdfxError):
        b.set_instances(bad, ef)
    with pytest.raises(B.PdfxError):
        b.set_instances(P, np.array([0, 5, 5, g.ne], dtype=np.int32))
    # element ranges that cut an instance's grid in two leave shared edges: a mesh error
    b.set_instances(P, np.array([0, ef[1] // 2, ef[2], g.ne], dtype=np.int32))
    with pytest.raises(B.PdfxError):
        b.set_grid(g)


def _single(it, precision, sort_every):
    c = B.Context(dict(it["params"], precision=precision, sort_every=sort_every))
    c.set_grid(it["grid"])
    c.set_fields(it["fields"])
    c.init_particles(it["ppe"])
    return c


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_plain_steps(precision):
    """Re-order cycles replayed from a CUDA graph give the plain steps' results (11 steps
    with a cycle of 4: one plain step after a first plain one, two cycles, a remainder)."""
    it = _instances()[1]
    a = _single(it, precision, 2)
    b = _single(it, precision, 2)
    dt = 2e-3
    a.step(dt)
    b.step(dt)
    for _ in range(11):
        a.step(dt)
    b.step_many(dt, 11, use_graph=True)
    assert a.step_index == b.step_index == 12
    sa, sb = a.get_particles(), b.get_particles()
    for key in STATE_KEYS + ("elem", "cp"):
        assert np.array_equal(sa[key], sb[key]), key
    assert np.array_equal(a.element_stats()[0], b.element_stats()[0])
    assert np.array_equal(a.nodal_stats(), b.nodal_stats())
    assert a.diag()["moves"] == b.diag()["moves"]
    # a further plain step continues from the replayed state
    a.step(dt)
    b.step(dt)
    assert np.array_equal(a.get_particles()["x"], b.get_particles()["x"])
    assert b.check() == 0


def test_batch_graph_equals_instances_run_alone():
    ins = _instances()
    g, F, ef, nf = synth.union(ins)
    P = [dict(it["params"], precision=1, sort_every=2) for it in ins]
    b = B.Context(P[0])
    b.set_instances(P, ef)
    b.set_grid(g)
    b.set_fields(F)
    b.init_particles_batch([it["ppe"] for it in ins])
    b.step_many(2e-3, 9, use_graph=True)
    _, pf = b.instance_ranges()
    sb = b.get_particles()
    for k, it in enumerate(ins):
        c = _single(it, 1, 2)
        for _ in range(9):
            c.step(2e-3)
        sa = c.get_particles()
        sl = slice(int(pf[k]), int(pf[k + 1]))
        for key in STATE_KEYS:
            assert np.array_equal(sb[key][sl], sa[key]), key


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_changes_no_result(precision):
    """The tuned launch shapes (advance block size, re-order period, binning split) leave
    every result as it was, and tuning leaves the state where it found it."""
    it = _instances()[2]
    a = _single(it, precision, 8)
    b = _single(it, precision, 8)
    dt = 2e-3
    for c in (a, b):
        c.step(dt)
    x_before = b.get_particles()["x"]
    tuned = b.autotune(dt)
    assert tuned["adv_block"] in (128, 256) and tuned["sort_every"] in (4, 8, 16)
    assert tuned["tile_split"] in (0, 128, 192, 256)
    assert b.launch_shapes() == tuned
    assert b.step_index == a.step_index
    assert np.array_equal(b.get_particles()["x"], x_before)
    assert b.diag()["steps"] == a.diag()["steps"]
    for _ in range(10):
        a.step(dt)
    b.step_many(dt, 10, use_graph=True)
    sa, sb = a.get_particles(), b.get_particles()
    for key in STATE_KEYS + ("elem", "cp"):
        assert np.array_equal(sa[key], sb[key]), key
    assert np.array_equal(a.nodal_stats(), b.nodal_stats())
    assert a.diag()["moves"] == b.diag()["moves"]


def test_batch_step_of_separate_contexts_equals_single_steps():
    """pdfx_batch_step over three separate contexts gives, bit for bit, what pdfx_step gives
    each of them; a repeated context is refused."""
    ins = _instances()
    a = [_single(it, 1, 4) for it in ins]
    b = [_single(it, 1, 4) for it in ins]
    dt = 2e-3
    for _ in range(5):
        B.batch_step(a, dt)
        for c in b:
            c.step(dt)
    for ca, cb in zip(a, b):
        sa, sb = ca.get_particles(), cb.get_particles()
        for key in STATE_KEYS + ("elem", "cp"):
            assert np.array_equal(sa[key], sb[key]), key
        assert np.array_equal(ca.nodal_stats(), cb.nodal_stats())
        assert ca.check() == 0
    with pytest.raises(B.PdfxError):
        B.batch_step([a[0], a[1], a[0]], dt)

