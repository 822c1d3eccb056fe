"""Blocking analysis for the oracle's time series (Sec. 4.1 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Written as plain
loops so a reader can check it against the paper by eye:

* the blocking transformation X'_i = (X_{2i-1} + X_{2i}) / 2 (Eq. Blocking-
  Transformation); an odd trailing element is dropped (the paper's printed
  block counts 10000 -> 78 after 7 halvings, 2000 -> 125 after 4 and -> 62
  after 5 fix this);
* the naive standard error at level k (k - 1 halvings),
  sigma(k)^2 = (mean(X'^2) - mean(X')^2) / Omega';
* the level is chosen by Jonsson's M-test (Phys. Rev. E 98, 043304, 2018):
  with n_i points, variance s_i^2 and lag-one autocovariance g_i at level i,
  M_j = sum_{i >= j} n_i (g_i / s_i^2)^2 is compared with the chi-squared
  quantile of (number of levels - j) degrees of freedom at 99 %; the first
  level that passes is used.
* the ratio of two means with linear error propagation and the blocked
  covariance at a common level (Sec. 4.2).
"""
from __future__ import annotations

import math

from scipy.stats import chi2


def halve(x):
    return [0.5 * (x[2 * i] + x[2 * i + 1]) for i in range(len(x) // 2)]


def levels(x):
    """Per level (n, mean, population variance, lag-one autocovariance)."""
    out = []
    cur = list(x)
    while len(cur) >= 2:
        n = len(cur)
        mu = sum(cur) / n
        var = sum((v - mu) ** 2 for v in cur) / n
        gam = sum((cur[t] - mu) * (cur[t + 1] - mu) for t in range(n - 1)) / n
        out.append((n, mu, var, gam))
        cur = halve(cur)
    return out


def mtest_level(x, confidence: float = 0.99):
    """0-based index j of the first blocking level that passes the M-test,
    or None if none does."""
    lv = levels(x)
    d = len(lv)
    terms = [n * (g / v) ** 2 if v > 0 else 0.0 for (n, _, v, g) in lv]
    for j in range(d):
        M = sum(terms[j:])
        if M < chi2.ppf(confidence, d - j):
            return j
    return None


def blocking_analysis(x, confidence: float = 0.99):
    """dict(mean, err, k, blocks, ok) of a time series."""
    lv = levels(x)
    j = mtest_level(x, confidence)
    ok = j is not None
    if j is None:
        j = len(lv) - 1
    n, mu, var, _ = lv[j]
    mean = sum(x) / len(x)
    return dict(mean=mean, err=math.sqrt(var / n), k=j + 1, blocks=n, ok=ok)


def ratio_of_means(x, y, confidence: float = 0.99):
    """r = mean(x) / mean(y) with linear error propagation at the deeper of
    the two M-test levels."""
    jx = mtest_level(x, confidence)
    jy = mtest_level(y, confidence)
    ok = jx is not None and jy is not None
    lx = levels(x)
    j = max(jx if jx is not None else len(lx) - 1, jy if jy is not None else len(lx) - 1)
    bx, by = list(x), list(y)
    for _ in range(j):
        bx, by = halve(bx), halve(by)
    n = len(bx)
    mx, my = sum(bx) / n, sum(by) / n
    vx = sum((v - mx) ** 2 for v in bx) / n / n
    vy = sum((v - my) ** 2 for v in by) / n / n
    cxy = sum((a - mx) * (b - my) for a, b in zip(bx, by)) / n / n
    X, Y = sum(x) / len(x), sum(y) / len(y)
    r = X / Y
    var_r = r * r * (vx / (X * X) + vy / (Y * Y) - 2.0 * cxy / (X * Y))
    return dict(ratio=r, err=math.sqrt(max(var_r, 0.0)), k=j + 1, blocks=n, ok=ok)
