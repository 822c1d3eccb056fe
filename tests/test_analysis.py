"""The package's blocking analysis (used by the benchmark) against the
oracle's, on series whose answers the oracle's pins fix."""
import numpy as np
import pytest

import oracle.blocking as OB
from paper_2601_19505_gb300 import analysis as A


def _ar1(n, phi, seed):
    rng = np.random.default_rng(seed)
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0]
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    return x + 3.0


@pytest.mark.parametrize("phi,n", [(0.0, 5000), (0.9, 20000), (0.99, 40000)])
def test_blocked_mean_matches_oracle(phi, n):
    x = _ar1(n, phi, seed=int(phi * 100) + n)
    got = A.blocked_mean(x)
    want = OB.blocking_analysis(list(x))
    assert got["k"] == want["k"] and got["ok"] == want["ok"]
    assert got["mean"] == pytest.approx(want["mean"], rel=1e-13)
    assert got["err"] == pytest.approx(want["err"], rel=1e-10)


def test_ratio_estimate_matches_oracle():
    rng = np.random.default_rng(3)
    y = _ar1(8000, 0.95, 5) + 20.0
    x = -4.0 * y + 0.3 * _ar1(8000, 0.8, 6)
    got = A.ratio_estimate(x, y)
    want = OB.ratio_of_means(list(x), list(y))
    assert got["k"] == want["k"]
    assert got["ratio"] == pytest.approx(want["ratio"], rel=1e-13)
    assert got["err"] == pytest.approx(want["err"], rel=1e-9)
