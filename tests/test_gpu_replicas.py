"""Replica overlaps (Sec. 4.3) on the GPU against the oracle (needs a GB300).

Replicas are runs of one Hamiltonian with different run ids, stepped as one
batch; after every step the batch records c_A^T c_B and c_A^T G2(d) c_B
(Eq. g2) for every pair.  The runs follow the oracle's trajectories (draws
are keyed by content), so each row is compared with the oracle's overlaps of
the same step: FP64 to 1e-12, integer walkers to 1e-12 (the dot products of
integers are exact; the G2 terms carry the 1/M), FP32 to 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import assert_same_vector, fq, pair

pytestmark = pytest.mark.gpu


def _replicas(h, m, R, mode, seed=4, dt=0.005, target=3000.0):
    runs, oruns = [], []
    for rid in range(R):
        p = dict(mode=mode, dt=dt, target=target, seed=seed, run_id=rid)
        g = fq().Run(h, fq().default_params(**p))
        g.seed_default(10.0)
        runs.append(g)
        oruns.append(O.start_run(m, O.default_params(**p)))
    return runs, oruns


@pytest.mark.parametrize("mode,rtol", [(1, 1e-12), (0, 1e-12), (2, 1e-5)],
                         ids=["REAL64", "INT", "REAL32"])
@pytest.mark.parametrize("model,ds", [((O.REAL_1D, 8, 1, 8, 1.0, 4.0), [0, 1, 2, 3, 4]),
                                      ((O.REAL_1D, 20, 1, 20, 1.0, 2.0), [0, 5]),
                                      ((O.REAL_1D, 33, 1, 33, 1.0, 20.0), [0, 16]),
                                      ((O.REAL_2D, 4, 3, 9, 1.0, 3.0), [])],
                         ids=["real1d-8", "real1d-20", "real1d-128bit", "real2d"])
def test_overlap_rows_match_oracle(model, ds, mode, rtol):
    h, m = pair(*model)
    R = 3
    runs, oruns = _replicas(h, m, R, mode, dt=0.002 if mode == 0 else 0.005)
    b = fq().Batch(runs)
    b.set_overlaps(ds)
    pairs = [(a, c) for a in range(R) for c in range(a + 1, R)]
    width = 1 + len(pairs) * (1 + len(ds))
    for block in range(4):
        b.step(10)
        for o in oruns:
            o.step(10)
        rows = b.overlaps()
        assert rows.shape == (10, width)
        assert np.array_equal(rows[:, 0], np.arange(10 * block + 1, 10 * block + 11))
        # each replica follows the oracle's trajectory ...
        for g, o in zip(runs, oruns):
            assert_same_vector(g.export(), o.export(), rtol=rtol if mode else 0.0,
                               what="replica run_id %d step %d" % (runs.index(g), 10 * block + 10))
        # ... and the overlap row equals the oracle's overlaps of the same vectors
        want = np.concatenate([O.overlap(oruns[a], oruns[c], ds) for a, c in pairs])
        got = rows[-1, 1:]
        assert np.allclose(got, want, rtol=rtol, atol=0), (block, got, want)
        assert np.any(got[:: 1 + len(ds)] != 0)
    b.close()


def test_overlaps_are_reproducible_and_checked():
    h, m = pair(O.REAL_1D, 10, 1, 10, 1.0, 3.0)
    out = []
    for _ in range(2):
        runs, _ = _replicas(h, m, 2, 0, dt=0.002)
        b = fq().Batch(runs)
        b.set_overlaps([0, 1])
        b.step(60)
        out.append(b.overlaps())
        b.close()
    # integer walkers give identical vectors, and the per-warp sums are added
    # in a fixed order: bit-identical rows
    assert np.array_equal(out[0], out[1])
    runs, _ = _replicas(h, m, 2, 1)
    b = fq().Batch(runs)
    with pytest.raises(fq().FqError):
        b.set_overlaps([10])  # d >= M
    b.close()
    hm, mm = pair(O.MOM_1D, 8, 1, 8, 1.0, 4.0)
    runs, _ = _replicas(hm, mm, 2, 1)
    b = fq().Batch(runs)
    with pytest.raises(fq().FqError):
        b.set_overlaps([1])  # G2 is a real-space operator
    b.set_overlaps([])       # dot products alone work in momentum space
    b.step(5)
    assert b.overlaps().shape == (5, 2)
    b.close()


def test_replica_estimators_agree_with_exact_diagonalisation():
    """6/6, u = 6, two replicas, N_t = 1e3, seeds 1..3, 6000 steps (the first
    1000 dropped): the variational energy (ratio of blocked means of
    (S_A + S_B)/2 c_A^T c_B over c_A^T c_B) and <G2(d)>, each pooled over the
    seeds, within 2 sigma of the exact ground state's values."""
    import oracle.blocking as BL
    import oracle.ed as ED
    h, m = pair(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e0, basis, v0 = ED.ground_state(m)
    keys = ED.basis_ints(basis)
    ds = [0, 1, 2, 3]
    exact = [e0] + [float(np.dot(v0 * v0, [m.g2_diag(k, d) for k in keys]) / np.dot(v0, v0))
                    for d in ds]
    est = [[] for _ in exact]
    for seed in (1, 2, 3):
        runs = []
        for rid in range(2):
            g = fq().Run(h, fq().default_params(seed=seed, run_id=rid))
            g.seed_default(10.0)
            runs.append(g)
        b = fq().Batch(runs)
        b.set_overlaps(ds)
        b.step(6000)
        rows = b.overlaps()[1000:]
        ha, hb = runs[0].history()[1000:], runs[1].history()[1000:]
        assert np.array_equal(rows[:, 0], ha["step"])
        dot = rows[:, 1]
        r = BL.ratio_of_means(list(0.5 * (ha["shift"] + hb["shift"]) * dot), list(dot))
        est[0].append((r["ratio"], r["err"]))
        for i in range(len(ds)):
            r = BL.ratio_of_means(list(rows[:, 2 + i]), list(dot))
            est[1 + i].append((r["ratio"], r["err"]))
        b.close()
    for want, v in zip(exact, est):
        w = np.array([1.0 / e ** 2 for _, e in v])
        mean = float(np.dot([x for x, _ in v], w) / w.sum())
        err = float(1.0 / np.sqrt(w.sum()))
        assert abs(mean - want) < 2 * err, (mean, err, want, v)
