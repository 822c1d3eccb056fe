"""Pins of the oracle's FCIQMC step (not GPU).

The step is a stochastic map, so it is pinned by what the mathematics fixes:
the deterministic limit equals the dense power-iteration step; the average of
many independently keyed steps equals T c (Eq. fciqmc-stochastic must be
unbiased); the shift update reproduces the rows the paper prints; one output
computed alone equals the full step's output; and long runs land within two
blocked standard errors of exact diagonalisation.
"""
import numpy as np
import pytest

import oracle as O
import oracle.blocking as BL
import oracle.ed as ED
from conftest import golden


def _dense_T(m, basis_keys, H, dt, S):
    return np.eye(len(basis_keys)) + dt * (S * np.eye(len(basis_keys)) - H)


def _vec(run, index, dim):
    keys, amps = run.export()
    v = np.zeros(dim)
    for k, a in zip(keys, amps):
        v[index[O.key_int(k)]] = a
    return v


@pytest.mark.parametrize("kind,Lx,N,u", [(O.REAL_1D, 6, 6, 6.0), (O.MOM_1D, 6, 5, 4.0)])
def test_deterministic_limit_is_power_iteration(kind, Lx, N, u):
    m = O.Model(kind, Lx, 1, N, 1.0, u)
    basis, H = ED.dense_hamiltonian(m)
    keys = ED.basis_ints(basis)
    index = {k: i for i, k in enumerate(keys)}
    rng = np.random.default_rng(11)
    c = rng.normal(size=len(keys)) * (rng.random(len(keys)) < 0.5)
    c[0] = 5.0
    dt, S = 0.013, -3.7
    run = O.Run(m, O.default_params(mode=O.MODE_DETERMINISTIC, dt=dt))
    nz = np.nonzero(c)[0]
    run.seed([keys[i] for i in nz], c[nz], S)
    T = _dense_T(m, keys, H, dt, S)
    v = c.copy()
    for step in range(3):
        run.step(1)
        S_now = run.state()[0]
        v = T @ v
        got = _vec(run, index, len(keys))
        assert np.allclose(got, v, rtol=1e-12, atol=1e-12 * np.abs(v).max())
        T = _dense_T(m, keys, H, dt, S_now)


@pytest.mark.parametrize("model", [(O.REAL_1D, 5, 1, 5, 4.0), (O.MOM_1D, 6, 1, 5, 4.0),
                                   (O.REAL_2D, 3, 3, 4, 3.0)], ids=["real1d", "mom1d", "real2d"])
@pytest.mark.parametrize("mode", [O.MODE_REAL64, O.MODE_REAL32, O.MODE_INT])
def test_one_step_is_unbiased(mode, model):
    """E[c^(n+1)] = (1 + dt (S - H)) c^(n) for the compressed step, averaged
    over independently keyed draws (here: different step counters)."""
    kind, Lx, Ly, N, u = model
    m = O.Model(kind, Lx, Ly, N, 1.0, u)
    basis, H = ED.dense_hamiltonian(m)
    keys = ED.basis_ints(basis)
    index = {k: i for i, k in enumerate(keys)}
    rng = np.random.default_rng(5)
    sel = rng.choice(len(keys), 25, replace=False)
    if mode == O.MODE_INT:
        amps = rng.integers(1, 40, size=25) * rng.choice([-1, 1], size=25)
        amps[0] = 900
    else:
        amps = rng.exponential(2.0, size=25) * rng.choice([-1, 1], size=25)
        amps[0] = 60.0   # an exact column
        amps[1] = -0.3   # below threshold
    c = np.zeros(len(keys))
    c[sel] = amps
    dt, S = 0.05, -1.0
    T = _dense_T(m, keys, H, dt, S)
    want = T @ c
    run = O.Run(m, O.default_params(mode=mode, dt=dt))
    R = 3000
    acc = np.zeros(len(keys))
    acc2 = np.zeros(len(keys))
    for r in range(R):
        run.seed([keys[i] for i in sel], amps.astype(float), S, step=1000 + r)
        run.step(1)
        v = _vec(run, index, len(keys))
        acc += v
        acc2 += v * v
    mean = acc / R
    var = np.maximum(acc2 / R - mean ** 2, 0)
    # A component reached only through rare survivals of Pi (quantum theta, or
    # one walker in integer mode) may never be observed in R trials; its
    # standard error is then at least that of a Bernoulli(|want|/q) q variable.
    q = 1.0
    se = np.sqrt((var + q * np.abs(want)) / R)
    touched = (var > 0) | (want != 0)
    z = np.abs(mean - want)[touched] / se[touched]
    assert np.all(z < 5.5), (np.max(z), np.argmax(z))
    # the mean agrees in aggregate too (chi-squared over touched components)
    assert np.mean(z ** 2) < 1.5


def test_printed_shift_rows():
    g = golden("shift_rows.json")
    dt, zeta = 0.01, 0.08
    xi = zeta ** 2 / 4
    for series in g["series"]:
        S, N0 = g["start_shift"], g["start_norm"]
        for step, _len, shift, norm in series["rows"]:
            S = O.shift_update(S, N0, norm, dt, zeta, xi, series["target"])
            assert S == pytest.approx(shift, abs=g["tol"])
            N0 = norm
    # the text's xi = zeta^2/2 does not reproduce the first printed row
    S = O.shift_update(0.0, 10.0, 15.0, dt, zeta, zeta ** 2 / 2, 1e5)
    assert abs(S - g["series"][0]["rows"][0][2]) > 0.5


def test_norm_is_the_exact_sum_rounded_once():
    """||c||_1 = sum |c_i| in exact arithmetic, rounded once to nearest."""
    from fractions import Fraction
    rng = np.random.default_rng(8)
    for trial in range(30):
        n = int(rng.integers(1, 5000))
        mag = np.exp(rng.uniform(0, 30, size=n)) if trial % 3 else 1.0 + rng.exponential(3, n)
        a = mag * rng.choice([-1, 1], size=n)
        if trial % 2:
            a = a.astype(np.float32).astype(np.float64)
        exact = float(sum(Fraction(abs(float(x))) for x in a))
        assert O.exact_norm(a, 1.0, O.MODE_REAL64) == exact
        half = np.where(np.abs(a) < 0.5, 0.5, a)
        exact = float(sum(Fraction(abs(float(x))) for x in half))
        assert O.exact_norm(half, 0.5, O.MODE_REAL64) == exact
    ints = rng.integers(-10**12, 10**12, size=1000).astype(np.float64)
    assert O.exact_norm(ints, 1.0, O.MODE_INT) == float(sum(abs(int(x)) for x in ints))


def test_exact_column_rule_and_counts():
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    s = m.start()                     # m_i = 12
    for amp, t_rel, exact in [(12.0, 1.0, 1), (11.9, 1.0, 0), (6.0, 2.0, 1), (5.9, 2.0, 0)]:
        run = O.Run(m, O.default_params(t_rel=t_rel))
        run.record_spawns()
        run.seed([s], [amp], 0.0)
        run.step(1)
        h = run.history()[0]
        assert (h["exact_steps"], h["inexact_steps"]) == (exact, 1 - exact)
        d, src, v = run.spawns()
        assert len(d) == (12 if exact else int(np.ceil(amp)))
        assert h["n_spawns"] == len(d)
        if exact:
            assert len(set(O.key_int(x) for x in d)) == 12
            assert np.allclose(v, 0.01 * np.sqrt(2) * amp)


def test_vector_compression_statistics():
    """Pi keeps |w| >= theta, rounds the rest to sign(w) theta with
    probability |w| / theta."""
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    s = m.start()
    theta = 0.5
    kept = 0
    R = 4000
    for r in range(R):
        run = O.Run(m, O.default_params(threshold=theta, t_rel=1e9, dt=0.01))
        run.seed([s], [-0.2], 0.0, step=r)
        run.step(1)
        k, a = run.export()
        for kk, aa in zip(k, a):
            if O.key_int(kk) == s:
                assert aa == -theta
                kept += 1
    # diagonal term is -0.2 exactly (S = H_ii = 0): kept with probability 0.4
    p = kept / R
    assert abs(p - 0.4) < 5 * np.sqrt(0.4 * 0.6 / R)


@pytest.mark.parametrize("mode", [O.MODE_REAL64, O.MODE_REAL32, O.MODE_INT])
def test_point_evaluation_equals_full_step(mode):
    m = O.Model(O.REAL_1D, 8, 1, 8, 1.0, 3.0)
    run = O.start_run(m, O.default_params(mode=mode, dt=0.01, target=3000))
    run.step(150)
    keys, amps = run.export()
    base = O.Run(m, O.default_params(mode=mode, dt=0.01, target=3000))
    base.seed(keys, amps, run.state()[0], step=run.state()[2])
    probe = O.Run(m, O.default_params(mode=mode, dt=0.01, target=3000))
    probe.seed(keys, amps, run.state()[0], step=run.state()[2])
    base.step(1)
    nk, na = base.export()
    new = {O.key_int(k): a for k, a in zip(nk, na)}
    cand = set(new)
    for k in keys[:50]:
        cand.update(m.column(O.key_int(k))[0])
    for k in sorted(cand)[:400]:
        pre, post = probe.point(k)
        assert post == new.get(k, 0.0)


def _run_energy(m, params, steps, skip, seed_weight=10.0):
    run = O.start_run(m, params, weight=seed_weight)
    rc = run.step(steps)
    assert rc == 0
    h = run.history()
    shift = BL.blocking_analysis(list(h["shift"][skip:]))
    proj = BL.ratio_of_means(list(h["hproj"][skip:]), list(h["vproj"][skip:]))
    return shift, proj, h


@pytest.mark.parametrize("mode", [O.MODE_REAL64, O.MODE_REAL32])
def test_real_run_matches_exact_energy(mode):
    """Sec. 4 example: 6/6, u = 6, default parameters, 3000 steps, skip 1000
    (FP64 amplitudes, and FP32 amplitudes with FP64 estimators)."""
    g = golden("energies.json")
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e0 = ED.lowest(m, 1)[0]
    shift, proj, h = _run_energy(m, O.default_params(mode=mode), 3000, 1000)
    assert abs(shift["mean"] - e0) < 2 * shift["err"]
    assert abs(proj["ratio"] - e0) < 2 * proj["err"]
    # the paper's printed estimates, as context: same ballpark error bars
    assert 0.2 * g["fciqmc_6x6_shift"][1] < shift["err"] < 5 * g["fciqmc_6x6_shift"][1]
    assert abs(h["norm"][1000:].mean() - 1000) < 100


def test_integer_walker_run_matches_exact_energy():
    """Integer walkers, 6/6, u = 6, target 1e3, dt = 1e-3 (longer than the
    2000-step configuration so that blocking has enough decorrelated data)."""
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e0 = ED.lowest(m, 1)[0]
    shift, proj, h = _run_energy(m, O.default_params(mode=O.MODE_INT, dt=1e-3), 40000, 4000)
    assert np.all(h["exact_steps"] == 0)
    assert abs(proj["ratio"] - e0) < 2 * proj["err"]
    assert abs(shift["mean"] - e0) < 2 * shift["err"]


def test_momentum_run_matches_exact_energy():
    """Momentum space (Sec. 6.3), 6 modes, 6 bosons, u = 4, default parameters:
    4000 steps from the condensate, blocked estimates within 2 sigma of the
    lowest eigenvalue of the same momentum sector."""
    m = O.Model(O.MOM_1D, 6, 1, 6, 1.0, 4.0)
    e0 = ED.lowest(m, 1)[0]
    shift, proj, h = _run_energy(m, O.default_params(), 4000, 1000)
    assert abs(proj["ratio"] - e0) < 2 * proj["err"], (proj, e0)
    assert abs(shift["mean"] - e0) < 2 * shift["err"], (shift, e0)


def test_two_dimensional_run_matches_exact_energy():
    """2D 3x3 periodic lattice, 4 bosons, u = 3, default parameters: 4000
    steps from near-uniform filling, blocked estimates within 2 sigma of
    exact diagonalisation."""
    m = O.Model(O.REAL_2D, 3, 3, 4, 1.0, 3.0)
    e0 = ED.lowest(m, 1)[0]
    shift, proj, h = _run_energy(m, O.default_params(), 4000, 1000)
    assert abs(proj["ratio"] - e0) < 2 * proj["err"], (proj, e0)
    assert abs(shift["mean"] - e0) < 2 * shift["err"], (shift, e0)
