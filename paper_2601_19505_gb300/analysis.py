"""Statistics of FCIQMC time series on the host (Sec. 4 of the Rimu.jl paper).

The shift and the projected-energy numerator and denominator of successive
steps are correlated, so their standard errors come from a blocking
analysis: the series is averaged pairwise again and again (Eq.
Blocking-Transformation; an odd last element is dropped), and the naive
standard error of the blocked series is taken at the first level that
passes Jonsson's M-test (Phys. Rev. E 98, 043304, 2018) at 99 % confidence.
The projected energy is the ratio of two blocked means, its error
propagated linearly with the blocked covariance at a common level.

Vectorised numpy; used by the benchmark's equal-error comparison.
"""
from __future__ import annotations

import numpy as np


def _levels(x: np.ndarray):
    """(n, variance, lag-one autocovariance) of every blocking level, both
    moments normalised by n."""
    out = []
    while x.size >= 2:
        n = x.size
        d = x - x.mean()
        out.append((n, float(np.dot(d, d)) / n, float(np.dot(d[:-1], d[1:])) / n))
        m = n // 2
        x = 0.5 * (x[0:2 * m:2] + x[1:2 * m:2])
    return out


def _first_passing_level(levels, confidence: float):
    from scipy.stats import chi2

    terms = np.array([n * (g / v) ** 2 if v > 0 else 0.0 for n, v, g in levels])
    suffix = np.cumsum(terms[::-1])[::-1]  # M_j = sum of terms j..end
    d = len(levels)
    for j in range(d):
        if suffix[j] < chi2.ppf(confidence, d - j):
            return j
    return None


def blocked_mean(x, confidence: float = 0.99) -> dict:
    """Mean and blocked standard error of a series: dict(mean, err, k, ok),
    k = number of blocking levels used counting the unblocked series as 1,
    ok = whether some level passed the M-test (else the deepest is used)."""
    x = np.asarray(x, dtype=np.float64)
    levels = _levels(x)
    j = _first_passing_level(levels, confidence)
    ok = j is not None
    if j is None:
        j = len(levels) - 1
    n, v, _ = levels[j]
    return dict(mean=float(x.mean()), err=float(np.sqrt(v / n)), k=j + 1, ok=ok)


def ratio_estimate(num, den, confidence: float = 0.99) -> dict:
    """mean(num) / mean(den) (the projected energy for num = y^T H c, den =
    y^T c) with its linearly propagated error at the deeper of the two
    series' M-test levels: dict(ratio, err, k, ok)."""
    a = np.asarray(num, dtype=np.float64)
    b = np.asarray(den, dtype=np.float64)
    la, lb = _levels(a), _levels(b)
    ja, jb = _first_passing_level(la, confidence), _first_passing_level(lb, confidence)
    ok = ja is not None and jb is not None
    j = max(len(la) - 1 if ja is None else ja, len(lb) - 1 if jb is None else jb)
    ba, bb = a, b
    for _ in range(j):
        m = ba.size // 2
        ba = 0.5 * (ba[0:2 * m:2] + ba[1:2 * m:2])
        bb = 0.5 * (bb[0:2 * m:2] + bb[1:2 * m:2])
    n = ba.size
    da, db = ba - ba.mean(), bb - bb.mean()
    va, vb, cab = np.dot(da, da) / n / n, np.dot(db, db) / n / n, np.dot(da, db) / n / n
    A, B = a.mean(), b.mean()
    if B == 0.0:
        return dict(ratio=float("nan"), err=float("inf"), k=j + 1, ok=False)
    r = A / B
    # r^2 (va/A^2 + vb/B^2 - 2 cab/(A B)) with A divided out, so A = 0 is fine
    var = (va - 2.0 * r * cab + r * r * vb) / (B * B)
    return dict(ratio=float(r), err=float(np.sqrt(max(var, 0.0))), k=j + 1, ok=ok)
