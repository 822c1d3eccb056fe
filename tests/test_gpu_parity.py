"""GPU path vs CPU oracle, through the C ABI (needs a GB300).

Bars (the method's own): addresses, occupied sets and integer-walker runs
bit-exact; FP64 amplitudes within 1e-12 relative over the first 50 steps;
FP32 amplitudes within 1e-5 relative (FP32 sums of two or more contributions
are taken in a different order on the GPU; a few ulps of a cancelling sum);
spawn lists bit-exact (draws are keyed by content, so order does not matter).
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import assert_same_vector, fq, pair, runs, seeded_vector, sorted_pairs

pytestmark = pytest.mark.gpu

MODELS = [
    (O.REAL_1D, 6, 1, 6, 1.0, 6.0),
    (O.REAL_1D, 20, 1, 20, 1.0, 2.0),
    (O.REAL_2D, 4, 3, 9, 1.0, 3.0),
    (O.REAL_2D, 8, 8, 64, 1.0, 8.0),      # 127-bit addresses
    (O.MOM_1D, 8, 1, 8, 1.0, 4.0),
    (O.MOM_1D, 32, 1, 32, 1.0, 4.0),      # 63-bit addresses
    (O.MOM_1D, 7, 1, 9, 1.0, 2.0),        # odd M
    (O.REAL_1D, 70, 1, 30, 1.0, 2.0),     # 99-bit, real space
    (O.REAL_1D, 33, 1, 33, 1.0, 20.0),    # 65-bit, real space, Mott-like
]


@pytest.mark.parametrize("model", MODELS)
def test_column_bit_exact(model):
    h, m = pair(*model)
    rng = np.random.default_rng(3)
    keys = [m.start()] + seeded_vector(m, 60, 11)[0]
    for k in keys[:61]:
        d, dk, dv = h.column(k)
        ok, ov = m.column(k)
        assert d == m.diagonal(k)
        assert dk == ok
        assert np.array_equal(dv, ov)
    del rng


@pytest.mark.parametrize("mode", ["REAL64", "REAL32", "INT"])
@pytest.mark.parametrize("model", MODELS)
def test_spawn_list_bit_exact(model, mode):
    h, m = pair(*model)
    mcode = {"REAL64": 1, "REAL32": 2, "INT": 0}[mode]
    keys, amps = seeded_vector(m, 3000, 5, mode=mode)
    g, o = runs(h, m, mode=mcode, dt=0.003, target=1e5, seed=42, run_id=3,
                capacity_vec=20000, capacity_spawn=400000)
    g.seed(fq().keys_from_ints(keys), amps, -1.5, step=17)
    o.seed(keys, amps, -1.5, step=17)
    o.record_spawns()
    gd, gv = g.spawns()
    o.step(1)
    od, osrc, ov = o.spawns()
    assert len(gd) == len(od)
    gd, gv = sorted_pairs(gd, gv)
    od, ov = sorted_pairs(od, ov)
    assert np.array_equal(gd["lo"], od["lo"]) and np.array_equal(gd["hi"], od["hi"])
    assert np.array_equal(gv, ov)
    # the spawning stage leaves the run untouched
    g.step(1)
    assert_same_vector(g.export(), o.export(), rtol=1e-12 if mode != "REAL32" else 1e-5,
                       what="after one step")


@pytest.mark.parametrize("mode", ["REAL64", "REAL32", "INT", "DETERMINISTIC"])
@pytest.mark.parametrize("model", [MODELS[0], MODELS[2], MODELS[4], MODELS[6], MODELS[8]])
def test_fifty_steps_from_default_start(model, mode):
    if model is MODELS[8] and mode == "DETERMINISTIC":
        pytest.skip("the exact power iteration of a 65-bit space outgrows any capacity")
    h, m = pair(*model)
    mcode = {"REAL64": 1, "REAL32": 2, "INT": 0, "DETERMINISTIC": 3}[mode]
    dt = (0.01 if mode != "INT" else 0.002) if model is not MODELS[8] else 0.002
    g, o = runs(h, m, mode=mcode, dt=dt, target=2000.0, seed=9)
    g.seed_default(10.0)
    s = m.start()
    o.seed([s], [10.0], m.diagonal(s), 0)
    o.set_reference([s], [10.0])
    rtol = {"REAL64": 1e-12, "REAL32": 1e-5, "INT": 0.0, "DETERMINISTIC": 1e-12}[mode]
    for block in range(5):
        g.step(10)
        o.step(10)
        if mode == "DETERMINISTIC":
            # no compression: amplitudes far below the vector's scale come out
            # of cancelling sums, whose rounding depends on the summation
            # order; the bound is relative to the vector's largest amplitude
            (gk, ga), (ok, oa) = g.export(), o.export()
            assert np.array_equal(gk, ok)
            assert np.max(np.abs(ga - oa)) <= 1e-12 * np.max(np.abs(oa))
            continue
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % (10 * block + 10))
    gh, oh = g.history(), o.history()
    assert len(gh) == 50
    for f in ("step", "len", "exact_steps", "inexact_steps", "n_spawns"):
        assert np.array_equal(gh[f], oh[f]), f
    tol = 1e-12 if mode != "REAL32" else 1e-5
    for f in ("shift", "norm", "hproj", "vproj"):
        assert np.allclose(gh[f], oh[f], rtol=tol, atol=tol), f


@pytest.mark.parametrize("mode", ["REAL64", "REAL32", "INT"])
@pytest.mark.parametrize("model", [MODELS[1], MODELS[3], MODELS[5]])
def test_large_seeded_vector_steps(model, mode):
    """A 20k-entry seeded vector (many segments, ragged segment fills) for
    three steps."""
    h, m = pair(*model)
    mcode = {"REAL64": 1, "REAL32": 2, "INT": 0}[mode]
    keys, amps = seeded_vector(m, 20000, 21, mode=mode)
    g, o = runs(h, m, mode=mcode, dt=0.001, target=float(np.abs(amps).sum()), seed=5,
                capacity_vec=200000, capacity_spawn=2000000)
    g.seed(fq().keys_from_ints(keys), amps, -2.0, step=100)
    o.seed(keys, amps, -2.0, step=100)
    refs = keys[:5]
    g.set_reference(fq().keys_from_ints(refs), [1.0, 2.0, 3.0, -1.0, 0.5])
    o.set_reference(refs, [1.0, 2.0, 3.0, -1.0, 0.5])
    rtol = {"REAL64": 1e-12, "REAL32": 1e-5, "INT": 0.0}[mode]
    for s in range(3):
        g.step(1)
        o.step(1)
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % s)
    gh, oh = g.history(), o.history()
    for f in ("len", "exact_steps", "inexact_steps", "n_spawns"):
        assert np.array_equal(gh[f], oh[f]), f
    tol = 1e-11 if mode != "REAL32" else 1e-5
    for f in ("shift", "norm", "hproj", "vproj"):
        assert np.allclose(gh[f], oh[f], rtol=tol, atol=tol), f


def test_empty_vector_and_population_death():
    h, m = pair(*MODELS[0])
    g, o = runs(h, m, seed=2)
    g.seed([], [], 0.0)
    st = g.stats()
    assert st["len"] == 0 and st["norm"] == 0.0
    # one boson in two momentum modes has no off-diagonal elements; with
    # S = H_ii - 1/dt the diagonal factor is exactly 0 and the walker dies
    h1 = fq().Hamiltonian(fq().BH_MOM_1D, 2, 1, 1, 1.0, 1.0)
    r = fq().Run(h1, fq().default_params(dt=0.01))
    s = h1.starting_address()
    diag = h1.column(s)[0]
    r.seed([s], [3.0], diag - 100.0)
    r.step(1)
    with pytest.raises(fq().FqError) as e:
        r.stats()
    assert e.value.code == -5
    # rolled back: the run is still at step 0 with its vector, and continues
    assert r.stats()["step"] == 0
    r.set_shift(diag)
    r.step(1)
    st = r.stats()
    assert st["step"] == 1 and st["len"] == 1 and st["norm"] == 3.0


def test_capacity_overflow_rolls_back():
    h, m = pair(*MODELS[1])
    g = fq().Run(h, fq().default_params(dt=0.001, target=1e6, capacity_vec=4096,
                                        capacity_spawn=4096))
    g.seed_default(10.0)
    rc = 0
    for _ in range(400):
        g.step(10)
        rc = g.sync()
        if rc:
            break
    assert rc == -3
    st = g.stats()
    k, a = g.export()
    assert len(k) == st["len"] and np.isclose(np.abs(a).sum(), st["norm"], rtol=1e-12)


@pytest.mark.parametrize("mode", [0, 1])
def test_reserve_after_overflow_continues_the_same_run(mode):
    """A run that overflows a small capacity is rolled back to its last
    completed step; after fq_run_reserve it continues exactly as a run
    created large enough from the start (integer walkers: bit-exact; FP64:
    the same addresses, amplitudes to 1e-12)."""
    h, m = pair(*MODELS[1])
    prm = dict(mode=mode, dt=0.001, target=2e5, seed=5)
    small = fq().Run(h, fq().default_params(capacity_vec=4096, capacity_spawn=4096, **prm))
    big = fq().Run(h, fq().default_params(capacity_vec=1 << 20, capacity_spawn=1 << 21, **prm))
    small.seed_default(10.0)
    big.seed_default(10.0)
    grows = small.advance(600, chunk=50)
    big.step(600)
    assert grows >= 1
    assert small.stats()["step"] == big.stats()["step"] == 600
    (ks, as_), (kb, ab) = small.export(), big.export()
    assert np.array_equal(ks, kb)
    if mode == 0:
        assert np.array_equal(as_, ab)
    else:
        assert np.allclose(as_, ab, rtol=1e-12, atol=0)
    hs, hb = small.history(), big.history()
    assert np.array_equal(hs["len"], hb["len"])
    assert np.array_equal(hs["step"], hb["step"])


def test_launch_shape_and_profile():
    h, m = pair(*MODELS[1])
    g = fq().Run(h, fq().default_params(dt=0.001, target=1e5, seed=3))
    g.seed_default(10.0)
    g.step(300)
    g.autotune(1)
    shp = g.shape()
    assert shp["spawn_wpb"] in (4, 8) and shp["merge_wpb"] in (4, 8)
    assert shp["spawn_grid"] > 0 and shp["merge_grid"] > 0 and shp["slots"] >= 64
    before = g.stats()["step"]
    ms = g.profile(5)
    assert g.stats()["step"] == before + 5
    assert ms[0] > 0 and ms[1] > 0 and ms[2] > 0


@pytest.mark.parametrize("case", [
    (O.REAL_1D, 6, 1, 6, 6.0, 1), (O.REAL_1D, 6, 1, 6, 6.0, 2),
    (O.MOM_1D, 6, 1, 6, 4.0, 1), (O.REAL_2D, 3, 3, 4, 3.0, 1)],
    ids=["real1d-f64", "real1d-f32", "mom1d-f64", "real2d-f64"])
def test_energy_agrees_with_exact_diagonalisation(case):
    """GPU runs with N_t = 1e4 and seeds 1..4: after 1000 steps of
    equilibration, the blocked projected energy (ratio of means, Sec. 4.2)
    and the blocked shift of the next 5000 steps, each pooled over the four
    seeds by inverse-variance weights, lie within 2 sigma of exact
    diagonalisation.  (At the default N_t = 1e3 the 6/6 projected energy
    carries a population-control bias of about 2 pooled sigma, Sec. 3.3; ten
    times the walkers shrink it by about sqrt(10) relative to the error.)"""
    import oracle.blocking as BL
    import oracle.ed as ED
    kind, Lx, Ly, N, u, mode = case
    h, m = pair(kind, Lx, Ly, N, 1.0, u)
    e0 = ED.lowest(m, 1)[0]
    est = {"projected": [], "shift": []}
    for seed in (1, 2, 3, 4):
        g = fq().Run(h, fq().default_params(mode=mode, seed=seed, target=1e4))
        g.seed_default(10.0)
        g.step(6000)
        hist = g.history()
        g.close()
        assert len(hist) == 6000
        r = BL.ratio_of_means(list(hist["hproj"][1000:]), list(hist["vproj"][1000:]))
        s = BL.blocking_analysis(list(hist["shift"][1000:]))
        est["projected"].append((r["ratio"], r["err"]))
        est["shift"].append((s["mean"], s["err"]))
    for name, v in est.items():
        w = np.array([1.0 / e ** 2 for _, e in v])
        mean = float(np.dot([x for x, _ in v], w) / w.sum())
        err = float(1.0 / np.sqrt(w.sum()))
        assert abs(mean - e0) < 2 * err, (name, mean, err, e0, v)


@pytest.mark.parametrize("mode", ["REAL64", "REAL32", "INT"])
@pytest.mark.parametrize("model", [MODELS[1], MODELS[3]], ids=["real1d-64bit", "real2d-128bit"])
def test_scratch_table_path_matches_oracle(model, mode):
    """Buckets whose spawns fill more than 0.7 of a merge warp's on-chip table
    are summed in that warp's table in device memory.  A small target (few
    buckets) and a 20k-entry seeded vector put thousands of spawns in every
    bucket, so every bucket takes that path (counted by the library); the
    steps still match the oracle (FP64 to 1e-12, integers bit-exact)."""
    h, m = pair(*model)
    mcode = {"REAL64": 1, "REAL32": 2, "INT": 0}[mode]
    keys, amps = seeded_vector(m, 20000, 31, mode=mode)
    g, o = runs(h, m, mode=mcode, dt=0.001, target=1000.0, seed=6,
                capacity_vec=200000, capacity_spawn=2000000)
    g.seed(fq().keys_from_ints(keys), amps, -2.0, step=100)
    o.seed(keys, amps, -2.0, step=100)
    rtol = {"REAL64": 1e-12, "REAL32": 1e-5, "INT": 0.0}[mode]
    for s in range(3):
        g.step(1)
        o.step(1)
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % s)
    onchip, scratch = g.merge_paths()
    assert scratch > 0 and scratch >= 3 * onchip, (onchip, scratch)
    gh, oh = g.history(), o.history()
    for f in ("len", "exact_steps", "inexact_steps", "n_spawns"):
        assert np.array_equal(gh[f], oh[f]), f


def test_scratch_table_overflow_rolls_back():
    """A bucket beyond 0.9 of the scratch table fails the step: FQ_ERR_CAPACITY
    with error bit 2 (a full annihilation table), the run rolled back to its
    last completed step; with the default tables it then steps like the
    oracle."""
    h, m = pair(*MODELS[1])
    keys, amps = seeded_vector(m, 20000, 31)
    g, o = runs(h, m, dt=0.001, target=1000.0, seed=6, capacity_vec=200000,
                capacity_spawn=2000000)
    g.seed(fq().keys_from_ints(keys), amps, -2.0, step=100)
    o.seed(keys, amps, -2.0, step=100)
    g.set_tables(64, 64)  # 57 spawns at most per bucket; these buckets hold thousands
    g.step(1)
    assert g.sync() == -3
    assert g.error_bits() & 4
    st = g.stats()
    assert st["step"] == 100 and st["len"] == len(keys)
    assert_same_vector(g.export(), o.export(), rtol=0.0, what="after the rollback")
    with pytest.raises(fq().FqError):
        g.set_tables(100, 0)  # not a power of two
    g.set_tables(0, 0)
    g.step(1)
    o.step(1)
    assert_same_vector(g.export(), o.export(), rtol=1e-12, what="after the failed step")
    assert g.merge_paths()[1] > 0


@pytest.mark.parametrize("primary", [0, 32, 64])
@pytest.mark.parametrize("mode", ["REAL64", "INT"])
@pytest.mark.parametrize("model", [MODELS[1], MODELS[3]], ids=["real1d-64bit", "real2d-128bit"])
def test_spawn_split_matches_oracle(model, mode, primary):
    """The spawn buffers keep the first `primary` slots of every bucket in a
    dense region and the rest in a second one.  With a 20k-entry seeded vector
    the buckets fill past 32 and 64 slots, so spawns land in both regions (0:
    all in the second); the spawn list and three steps still match the
    oracle, and an invalid split is rejected.  (A target of an eighth of
    the seeded norm gives buckets of about 390 to 530 spawns in REAL64 and 34
    to 130 for integer walkers.)"""
    h, m = pair(*model)
    mcode = {"REAL64": 1, "INT": 0}[mode]
    keys, amps = seeded_vector(m, 20000, 41, mode=mode)
    g, o = runs(h, m, mode=mcode, dt=0.001, target=float(np.abs(amps).sum()) / 8, seed=7,
                capacity_vec=200000, capacity_spawn=2000000)
    g.set_spawn_split(primary)
    with pytest.raises(fq().FqError):
        g.set_spawn_split(primary + 16)  # not a multiple of 32
    g.seed(fq().keys_from_ints(keys), amps, -2.0, step=100)
    o.seed(keys, amps, -2.0, step=100)
    o.record_spawns()
    gd, gv = g.spawns()
    o.step(1)
    od, osrc, ov = o.spawns()
    assert len(gd) == len(od)
    gd, gv = sorted_pairs(gd, gv)
    od, ov = sorted_pairs(od, ov)
    assert np.array_equal(gd["lo"], od["lo"]) and np.array_equal(gd["hi"], od["hi"])
    assert np.array_equal(gv, ov)
    rtol = {"REAL64": 1e-12, "INT": 0.0}[mode]
    g.step(1)
    assert_same_vector(g.export(), o.export(), rtol=rtol, what="step 0")
    for s in range(1, 3):
        g.step(1)
        o.step(1)
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % s)
    gh, oh = g.history(), o.history()
    for f in ("len", "exact_steps", "inexact_steps", "n_spawns"):
        assert np.array_equal(gh[f], oh[f]), f
