"""The synthetic workloads' recipes (host code only): the batched ensemble of config 5 and
the grids the benchmarks and parity tests use."""
import numpy as np

from paper_1006_0532_gb300 import synth


def test_ensemble_recipe():
    """64 instances, channel at even and street canyon at odd indices; triangle counts in the
    log-uniform range (the canyon's 120 k^2 and the channel's 4 rows^2 round them);
    particles per element in [50, 500]; the particle total in [2.7e8, 3.3e8]; distinct
    Philox seeds 1000 + k and instance numbers k; sources inside each domain's region."""
    ins = synth.ensemble(64)
    assert len(ins) == 64
    total = 0
    for k, it in enumerate(ins):
        g, p = it["grid"], it["params"]
        assert g.period_x == (2.0 if k % 2 == 0 else 4.0)
        assert 900 <= g.ne <= 62000
        assert 50 <= it["ppe"] <= 500
        assert p["seed"] == 1000 + k and p["instance"] == k
        if k % 2 == 0:
            assert 0.25 <= p["src_x"] <= 1.75 and 0.2 <= p["src_y"] <= 0.8
            assert np.all(g.edge_tag != 2)                       # channel: no-slip walls only
        else:
            assert 1.6 <= p["src_x"] <= 2.4 and 0.1 <= p["src_y"] <= 0.9
            assert np.any(g.edge_tag == 1) and np.any(g.edge_tag == 2)   # walls, free-slip top
            assert g.ne == 120 * synth.canyon_scale(g.ne) ** 2
        total += g.ne * it["ppe"]
    assert 2.7e8 <= total <= 3.3e8


def test_union_offsets():
    """The union of instances offsets each instance's node ids; element and node ranges
    tile the union exactly."""
    ins = [synth.channel_instance(120, 392.0, seed=1, ppe=10),
           synth.canyon_instance(1080, seed=2, ppe=10)]
    g, F, ef, nf = synth.union(ins)
    assert list(ef) == [0, ins[0]["grid"].ne, ins[0]["grid"].ne + ins[1]["grid"].ne]
    assert list(nf) == [0, ins[0]["grid"].nn, ins[0]["grid"].nn + ins[1]["grid"].nn]
    assert g.tri[ef[1]:].min() >= nf[1] and g.tri[:ef[1]].max() < nf[1]
    assert F.shape == (g.nn, synth.NF)


def test_redistribution_workload_grid():
    """Sect. 3.7's domain: periodic unit square, free-slip at y = 0 and 1 (no no-slip
    walls), rows graded toward both boundaries from the stated first row."""
    w = synth.redistribution_workload("redist_1k")
    g = w["grid"]
    assert g.ne == 1536 and g.period_x == 1.0
    assert np.all(g.edge_tag != 1) and np.count_nonzero(g.edge_tag == 2) == 2 * 24
    ys = np.sort(np.unique(np.round(g.node_xy[:, 1], 12)))
    assert ys[0] == 0.0 and ys[-1] == 1.0 and abs(ys[1] - 2e-3) < 2e-4
    assert w["params"]["model"] == 1 and w["params"]["alpha"] == 0.5
    assert w["params"]["minnpel"] == w["ppe"] // 10
