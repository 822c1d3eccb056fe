"""Pins of the oracle's blocking analysis (Sec. 4.1; not GPU)."""
import math

import numpy as np

import oracle.blocking as BL
from conftest import golden


def test_printed_block_counts():
    g = golden("energies.json")
    for n, halvings, blocks in g["block_counts"]:
        lv = BL.levels(list(np.zeros(n) + np.arange(n) % 3))
        assert lv[halvings][0] == blocks


def test_iid_series_needs_no_blocking():
    rng = np.random.default_rng(1)
    x = list(rng.normal(size=4096))
    r = BL.blocking_analysis(x)
    assert r["ok"] and r["k"] <= 2
    assert abs(r["err"] - 1 / math.sqrt(4096)) < 0.15 / math.sqrt(4096)


def test_ar1_standard_error_matches_closed_form():
    """X_t = phi X_{t-1} + e_t: the variance of the mean of n points tends to
    sigma_e^2 / ((1 - phi)^2 n)."""
    phi, n = 0.9, 1 << 16
    rng = np.random.default_rng(2)
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    r = BL.blocking_analysis(list(x))
    want = 1.0 / ((1 - phi) * math.sqrt(n))
    assert r["ok"] and r["k"] > 3
    assert abs(r["err"] - want) < 0.2 * want


def test_ratio_of_means_linear_propagation():
    rng = np.random.default_rng(4)
    n = 8192
    x = 2.0 + 0.1 * rng.normal(size=n)
    y = 1.0 + 0.05 * rng.normal(size=n)
    r = BL.ratio_of_means(list(x), list(y))
    want = math.sqrt((0.1 / 2.0) ** 2 + (0.05 / 1.0) ** 2) * 2.0 / math.sqrt(n)
    assert abs(r["ratio"] - x.mean() / y.mean()) < 1e-12
    assert abs(r["err"] - want) < 0.15 * want
