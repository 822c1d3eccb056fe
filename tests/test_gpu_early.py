"""Early compression (Sec. 7.1, Eq. early-comp) on the GPU against the oracle
(needs a GB300).  Every spawn and diagonal term is compressed on its own
before annihilation, with draws keyed by content, so the written spawn list
is bit-exact and the steps match to the same bars as late compression (FP64
1e-12, FP32 1e-5)."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import assert_same_vector, fq, pair, runs, seeded_vector, sorted_pairs
from test_gpu_parity import MODELS

pytestmark = pytest.mark.gpu

EARLY = 1


@pytest.mark.parametrize("mode", ["REAL64", "REAL32"])
@pytest.mark.parametrize("model", [MODELS[0], MODELS[2], MODELS[3], MODELS[5]],
                         ids=["real1d", "real2d", "real2d-128bit", "mom1d-63bit"])
def test_early_compression_spawns_and_steps(model, mode):
    h, m = pair(*model)
    mcode = {"REAL64": 1, "REAL32": 2}[mode]
    rtol = 1e-12 if mode == "REAL64" else 1e-5
    keys, amps = seeded_vector(m, 3000, 5, mode=mode)
    g, o = runs(h, m, mode=mcode, dt=0.003, target=1e5, seed=42, run_id=3, compression=EARLY,
                capacity_vec=400000, capacity_spawn=800000)
    g.seed(fq().keys_from_ints(keys), amps, -1.5, step=17)
    o.seed(keys, amps, -1.5, step=17)
    o.record_spawns()
    gd, gv = g.spawns()
    o.step(1)
    od, _, ov = o.spawns()
    assert len(gd) == len(od) and len(gd) > 0
    gd, gv = sorted_pairs(gd, gv)
    od, ov = sorted_pairs(od, ov)
    assert np.array_equal(gd["lo"], od["lo"]) and np.array_equal(gd["hi"], od["hi"])
    assert np.array_equal(gv, ov)
    assert np.all(np.abs(gv) >= 1.0)
    for s in range(3):
        g.step(1)
        if s:
            o.step(1)
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % s)
    gh, oh = g.history(), o.history()
    for f in ("len", "exact_steps", "inexact_steps", "n_spawns"):
        assert np.array_equal(gh[f], oh[f]), f
    for f in ("shift", "norm"):
        assert np.allclose(gh[f], oh[f], rtol=rtol, atol=0), f


@pytest.mark.parametrize("mode", ["REAL64", "REAL32"])
def test_early_compression_fifty_steps_from_default_start(mode):
    h, m = pair(*MODELS[0])
    mcode = {"REAL64": 1, "REAL32": 2}[mode]
    g, o = runs(h, m, mode=mcode, dt=0.01, target=2000.0, seed=9, compression=EARLY)
    g.seed_default(10.0)
    s = m.start()
    o.seed([s], [10.0], m.diagonal(s), 0)
    o.set_reference([s], [10.0])
    rtol = 1e-12 if mode == "REAL64" else 1e-5
    for block in range(5):
        g.step(10)
        o.step(10)
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % (10 * block + 10))
    gh, oh = g.history(), o.history()
    for f in ("step", "len", "exact_steps", "inexact_steps", "n_spawns"):
        assert np.array_equal(gh[f], oh[f]), f
    for f in ("shift", "norm", "hproj", "vproj"):
        assert np.allclose(gh[f], oh[f], rtol=rtol, atol=rtol), f
    # values below the threshold survive a sum and are counted in the norm
    k, a = g.export()
    assert O.exact_norm(a, 1.0, O.MODE_REAL64) == gh["norm"][-1] or mode == "REAL32"


def test_early_compression_energy_agrees_with_exact_diagonalisation():
    """6/6, u = 6, N_t = 1e4, early compression, seeds 1..4 pooled: the
    projected energy and the shift within 2 sigma of exact diagonalisation
    (early compression is unbiased; it only costs statistics)."""
    import oracle.blocking as BL
    import oracle.ed as ED
    h, m = pair(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e0 = ED.lowest(m, 1)[0]
    est = {"projected": [], "shift": []}
    for seed in (1, 2, 3, 4):
        g = fq().Run(h, fq().default_params(seed=seed, target=1e4, compression=EARLY))
        g.seed_default(10.0)
        g.step(6000)
        hist = g.history()
        g.close()
        r = BL.ratio_of_means(list(hist["hproj"][1000:]), list(hist["vproj"][1000:]))
        s = BL.blocking_analysis(list(hist["shift"][1000:]))
        est["projected"].append((r["ratio"], r["err"]))
        est["shift"].append((s["mean"], s["err"]))
    for name, v in est.items():
        w = np.array([1.0 / e ** 2 for _, e in v])
        mean = float(np.dot([x for x, _ in v], w) / w.sum())
        err = float(1.0 / np.sqrt(w.sum()))
        assert abs(mean - e0) < 2 * err, (name, mean, err, e0, v)
