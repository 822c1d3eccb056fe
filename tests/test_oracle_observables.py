"""Pins of the oracle's replica overlaps and early compression (not GPU).

Replica overlaps (Sec. 4.3): c_A^T c_B and c_A^T G2(d) c_B, with the
density-density correlator G2(d) of Eq. g2.  Pinned by a combinatorial
reading of G2 (ordered pairs of distinct bosons d sites apart), its sum rule
over d, its d = 0 relation to the interaction energy, brute-force sums over
exported vectors, and two-replica runs whose variational energy and <G2(d)>
land within 2 sigma of exact diagonalisation.

Early compression (Sec. 7.1, Eq. early-comp): every spawn and diagonal term is
compressed on its own before annihilation.  Pinned by unbiasedness of one
step, the absence of any sub-threshold term, and equality with late
compression when the threshold compresses nothing.
"""
import itertools

import numpy as np
import pytest

import oracle as O
import oracle.blocking as BL
import oracle.ed as ED
from conftest import golden


def _pairs_at_distance(occ, d):
    """Ordered pairs of distinct bosons whose sites differ by d around the ring."""
    pos = [s for s, n in enumerate(occ) for _ in range(int(n))]
    M = len(occ)
    return sum(1 for a, b in itertools.permutations(range(len(pos)), 2)
               if (pos[b] - pos[a]) % M == d)


def test_g2_counts_boson_pairs_and_obeys_its_sum_rule():
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    basis = ED.basis_ints(ED.sparse_hamiltonian(m)[0])
    assert len(basis) == 462
    for k in basis:
        occ = m.decode(k)
        vals = [m.g2_diag(k, d) for d in range(6)]
        for d in range(6):
            assert vals[d] * 6 == pytest.approx(_pairs_at_distance(occ, d), abs=1e-12)
        # sum over d of n_{i+d} is N: sum_d G2(d) = N (N - 1) / M
        assert sum(vals) == pytest.approx(6 * 5 / 6, abs=1e-12)
        # d = 0 counts on-site pairs: G2(0) = 2 H_jj / (u M) in real space
        assert vals[0] == pytest.approx(2.0 * m.diagonal(k) / (6.0 * 6), abs=1e-12)


def test_overlaps_equal_brute_force_sums():
    m = O.Model(O.REAL_1D, 7, 1, 5, 1.0, 3.0)
    ra = O.start_run(m, O.default_params(seed=3, run_id=0))
    rb = O.start_run(m, O.default_params(seed=3, run_id=1))
    ra.step(300)
    rb.step(300)
    ds = [0, 1, 2, 3]
    got = O.overlap(ra, rb, ds)
    (ka, aa), (kb, ab) = ra.export(), rb.export()
    da = {O.key_int(k): a for k, a in zip(ka, aa)}
    db = {O.key_int(k): a for k, a in zip(kb, ab)}
    common = sorted(set(da) & set(db))
    assert len(common) > 20
    want = [sum(da[k] * db[k] for k in common)]
    for d in ds:
        want.append(sum(_pairs_at_distance(m.decode(k), d) / 7.0 * da[k] * db[k]
                        for k in common))
    assert np.allclose(got, want, rtol=1e-12)
    # symmetric in the two replicas; a vector with itself gives sum c^2
    assert np.allclose(O.overlap(rb, ra, ds), got, rtol=1e-13)
    assert O.overlap(ra, ra)[0] == pytest.approx(float(np.dot(aa, aa)), rel=1e-13)
    with pytest.raises(ValueError):
        O.overlap(ra, rb, [7])


def test_two_replicas_give_exact_variational_energy_and_g2():
    """6/6, u = 6, two replicas (run ids 0 and 1), N_t = 1e3, seeds 1..3:
    after 1000 steps, the variational energy (ratio of blocked means of
    (S_A + S_B)/2 c_A^T c_B over c_A^T c_B, Sec. 4.3) and <G2(d)>
    (Eq. RayleighQuotientReplica), each pooled over the seeds by
    inverse-variance weights, lie within 2 sigma of the exact ground state's
    values."""
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e0, basis, v0 = ED.ground_state(m)
    keys = ED.basis_ints(basis)
    ds = [0, 1, 2, 3]
    exact = [e0] + [float(np.dot(v0 * v0, [m.g2_diag(k, d) for k in keys]) / np.dot(v0, v0))
                    for d in ds]
    est = [[] for _ in exact]
    for seed in (1, 2, 3):
        ra = O.start_run(m, O.default_params(seed=seed, run_id=0))
        rb = O.start_run(m, O.default_params(seed=seed, run_id=1))
        rows = []
        for _ in range(6000):
            ra.step(1)
            rb.step(1)
            rows.append(O.overlap(ra, rb, ds).tolist() + [ra.state()[0], rb.state()[0]])
        rows = np.array(rows)[1000:]
        dot = rows[:, 0]
        r = BL.ratio_of_means(list(0.5 * (rows[:, -2] + rows[:, -1]) * dot), list(dot))
        est[0].append((r["ratio"], r["err"]))
        for i in range(len(ds)):
            r = BL.ratio_of_means(list(rows[:, 1 + i]), list(dot))
            est[1 + i].append((r["ratio"], r["err"]))
    for want, v in zip(exact, est):
        w = np.array([1.0 / e ** 2 for _, e in v])
        mean = float(np.dot([x for x, _ in v], w) / w.sum())
        err = float(1.0 / np.sqrt(w.sum()))
        assert abs(mean - want) < 2 * err, (mean, err, want, v)
    # the paper's printed variational estimate (same model and N_t), as context
    g = golden("observables.json")
    assert abs(g["variational_6x6"][0] - e0) < 2 * g["variational_6x6"][1]


@pytest.mark.parametrize("mode", [O.MODE_REAL64, O.MODE_REAL32])
def test_early_compression_step_is_unbiased(mode):
    """E[c^(n+1)] = (1 + dt (S - H)) c^(n) also when every spawn and diagonal
    term is compressed on its own (Eq. early-comp), over independently keyed
    draws."""
    m = O.Model(O.REAL_1D, 5, 1, 5, 1.0, 4.0)
    basis, H = ED.dense_hamiltonian(m)
    keys = ED.basis_ints(basis)
    index = {k: i for i, k in enumerate(keys)}
    rng = np.random.default_rng(7)
    sel = rng.choice(len(keys), 25, replace=False)
    amps = rng.exponential(2.0, size=25) * rng.choice([-1, 1], size=25)
    amps[0] = 60.0   # an exact column
    amps[1] = -0.3
    c = np.zeros(len(keys))
    c[sel] = amps
    dt, S = 0.05, -1.0
    want = (np.eye(len(keys)) + dt * (S * np.eye(len(keys)) - H)) @ c
    run = O.Run(m, O.default_params(mode=mode, dt=dt, compression=O.COMPRESS_EARLY))
    R = 3000
    acc = np.zeros(len(keys))
    acc2 = np.zeros(len(keys))
    for r in range(R):
        run.seed([keys[i] for i in sel], amps, S, step=1000 + r)
        run.step(1)
        k, a = run.export()
        v = np.zeros(len(keys))
        for kk, aa in zip(k, a):
            v[index[O.key_int(kk)]] = aa
        acc += v
        acc2 += v * v
    mean = acc / R
    var = np.maximum(acc2 / R - mean ** 2, 0)
    se = np.sqrt((var + np.abs(want)) / R)
    touched = (var > 0) | (want != 0)
    z = np.abs(mean - want)[touched] / se[touched]
    assert np.all(z < 5.5), (np.max(z), np.argmax(z))
    assert np.mean(z ** 2) < 1.5


def test_early_compression_terms_and_no_compression_limit():
    m = O.Model(O.REAL_1D, 8, 1, 8, 1.0, 2.0)
    rng = np.random.default_rng(2)
    basis = ED.basis_ints(ED.sparse_hamiltonian(m)[0])
    sel = rng.choice(len(basis), 300, replace=False)
    keys = [basis[i] for i in sel]
    amps = (1.0 + rng.exponential(2.0, 300)) * rng.choice([-1, 1], 300)
    # every spawn written under early compression is at least theta
    run = O.Run(m, O.default_params(dt=0.01, compression=O.COMPRESS_EARLY))
    run.seed(keys, amps, -1.0, step=5)
    run.record_spawns()
    run.step(1)
    _, _, val = run.spawns()
    assert len(val) > 0 and np.all(np.abs(val) >= 1.0)
    late = O.Run(m, O.default_params(dt=0.01))
    late.seed(keys, amps, -1.0, step=5)
    late.record_spawns()
    late.step(1)
    assert len(late.spawns()[2]) > len(val)  # most small spawns are dropped
    # with a threshold below every value nothing is compressed: early = late
    tiny = dict(dt=0.01, threshold=2.0 ** -40)
    a = O.Run(m, O.default_params(compression=O.COMPRESS_EARLY, **tiny))
    b = O.Run(m, O.default_params(**tiny))
    for r in (a, b):
        r.seed(keys, amps, -1.0, step=5)
        r.step(1)
    (ka, va), (kb, vb) = a.export(), b.export()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    # the one-norm stays the exact sum although values below theta survive
    e = O.Run(m, O.default_params(dt=0.01, compression=O.COMPRESS_EARLY))
    e.seed(keys, amps, -1.0, step=5)
    e.step(3)
    k, v = e.export()
    assert np.any(np.abs(v) < 1.0)
    assert O.exact_norm(v, 1.0, O.MODE_REAL64) == e.state()[1]


def _spectral_pair(m, mode, seed, target):
    s = m.start()
    nb = m.column(s)[0][0]
    a = O.Run(m, O.default_params(mode=mode, dt=0.01, target=target, seed=seed))
    a.seed([s], [10.0], m.diagonal(s), 0)
    b = O.Run(m, O.default_params(mode=mode, dt=0.01, target=target, seed=seed, run_id=1))
    b.seed([s, nb], [10.0, 10.0], m.diagonal(s), 0)
    return a, b


def test_gram_schmidt_deterministic_limit_gives_the_first_excited_state():
    """Excited states (Sec. 2.2): in the deterministic limit the first run is
    the power iteration of Eq. fciqmc and the second, orthogonalised to it
    after every step, converges to the next eigenvector; the shifts then equal
    the two lowest eigenvalues of exact diagonalisation."""
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e = ED.lowest(m, 2)
    a, b = _spectral_pair(m, O.MODE_DETERMINISTIC, 1, 1e3)
    assert O.spectral_step([a, b], 8000) == 0
    assert abs(a.state()[0] - e[0]) < 1e-8
    assert abs(b.state()[0] - e[1]) < 1e-6
    # the two vectors are orthogonal after the last step
    (ka, va), (kb, vb) = a.export(), b.export()
    da = {O.key_int(k): x for k, x in zip(ka, va)}
    dot = sum(da.get(O.key_int(k), 0.0) * x for k, x in zip(kb, vb))
    assert abs(dot) < 1e-12 * np.linalg.norm(va) * np.linalg.norm(vb)
    with pytest.raises(Exception):
        ai, bi = _spectral_pair(m, O.MODE_INT, 1, 1e3)
        assert O.spectral_step([ai, bi], 1) == 0


def test_gram_schmidt_stochastic_excited_energy_within_two_sigma():
    """Two compressed FP64 runs (N_t = 1e4, seeds 1..3): the blocked shift of
    the orthogonalised run, pooled over the seeds, lies within 2 sigma of the
    first excited energy, and the first run's within 2 sigma of the ground
    energy."""
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e = ED.lowest(m, 2)
    est = [[], []]
    for seed in (1, 2, 3):
        a, b = _spectral_pair(m, O.MODE_REAL64, seed, 1e4)
        assert O.spectral_step([a, b], 6000) == 0
        for i, r in enumerate((a, b)):
            s = BL.blocking_analysis(list(r.history()["shift"][1000:]))
            est[i].append((s["mean"], s["err"]))
    for i in range(2):
        w = np.array([1.0 / x[1] ** 2 for x in est[i]])
        mean = float(np.dot([x[0] for x in est[i]], w) / w.sum())
        err = float(1.0 / np.sqrt(w.sum()))
        assert abs(mean - e[i]) < 2 * err, (i, mean, err, e[i])
