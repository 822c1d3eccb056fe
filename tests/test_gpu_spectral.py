"""Excited states (Sec. 2.2) on the GPU against the oracle (needs a GB300).

Runs 0..K-1 of a batch are spectral states; after every step run k is
orthogonalised to runs 0..k-1 (Gram-Schmidt) and its changed values are
compressed.  The GPU follows the oracle's trajectories: FP64 to 1e-12,
FP32 to 1e-5, the deterministic limit to 1e-12 of the vector's scale.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import assert_same_vector, fq, pair

pytestmark = pytest.mark.gpu


def _states(h, m, K, mode, seed=1, target=2000.0, dt=0.01):
    s = m.start()
    col = m.column(s)[0]
    g, o = [], []
    for k in range(K):
        keys = [s] + ([col[k - 1]] if k else [])
        amps = [10.0] * len(keys)
        p = dict(mode=mode, dt=dt, target=target, seed=seed, run_id=k)
        r = fq().Run(h, fq().default_params(**p))
        r.seed(fq().keys_from_ints(keys), amps, m.diagonal(s), 0)
        g.append(r)
        orun = O.Run(m, O.default_params(**p))
        orun.seed(keys, amps, m.diagonal(s), 0)
        o.append(orun)
    return g, o


@pytest.mark.parametrize("mode", ["REAL64", "REAL32", "DETERMINISTIC"])
@pytest.mark.parametrize("model,K", [((O.REAL_1D, 6, 1, 6, 1.0, 6.0), 2),
                                     ((O.REAL_1D, 8, 1, 8, 1.0, 4.0), 3),
                                     ((O.REAL_2D, 4, 3, 9, 1.0, 3.0), 2)],
                         ids=["real1d-6-K2", "real1d-8-K3", "real2d-K2"])
def test_spectral_states_match_oracle(model, K, mode):
    h, m = pair(*model)
    mcode = {"REAL64": 1, "REAL32": 2, "DETERMINISTIC": 3}[mode]
    g, o = _states(h, m, K, mcode)
    b = fq().Batch(g)
    b.set_spectral(K)
    for block in range(3):
        b.step(10)
        assert O.spectral_step(o, 10) == 0
        for k in range(K):
            if mode == "DETERMINISTIC":
                (gk, ga), (ok, oa) = g[k].export(), o[k].export()
                assert np.array_equal(gk, ok)
                assert np.max(np.abs(ga - oa)) <= 1e-12 * np.max(np.abs(oa))
            else:
                assert_same_vector(g[k].export(), o[k].export(),
                                   rtol=1e-12 if mode == "REAL64" else 1e-5,
                                   what="state %d step %d" % (k, 10 * block + 10))
    tol = 1e-12 if mode != "REAL32" else 1e-5
    for k in range(K):
        gh, oh = g[k].history(), o[k].history()
        assert np.array_equal(gh["len"], oh["len"]), k
        # the shift crosses zero: relative and absolute bounds, as for one run
        for f in ("shift", "norm"):
            assert np.allclose(gh[f], oh[f], rtol=tol, atol=tol), (k, f)
    b.close()


def test_spectral_deterministic_limit_reaches_the_excited_energy():
    import oracle.ed as ED
    h, m = pair(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e = ED.lowest(m, 2)
    g, _ = _states(h, m, 2, 3)
    b = fq().Batch(g)
    b.set_spectral(2)
    b.step(8000)
    assert abs(g[0].stats()["shift"] - e[0]) < 1e-8
    assert abs(g[1].stats()["shift"] - e[1]) < 1e-6
    b.close()


def test_spectral_states_reject_integer_walkers_and_mixed_sizes():
    h, m = pair(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    g, _ = _states(h, m, 2, 0)
    b = fq().Batch(g)
    with pytest.raises(fq().FqError):
        b.set_spectral(2)
    b.close()
    a = fq().Run(h, fq().default_params(target=1e3))
    c = fq().Run(h, fq().default_params(target=1e6, run_id=1))
    for r in (a, c):
        r.seed_default(10.0)
    b = fq().Batch([a, c])
    with pytest.raises(fq().FqError):
        b.set_spectral(2)  # different segment maps
    b.close()
