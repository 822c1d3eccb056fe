"""Annihilation by sorting (FQ_ANN_SORT) on the GPU (needs a GB300).

The sort arm sums each address's contributions after a per-bucket radix sort
instead of an on-chip hash table.  It reaches the same addresses and takes
every random decision on the same keyed draws, so it meets the same bars
against the oracle (integers bit-exact, FP64 1e-12, FP32 1e-5), in the
on-chip workspace and in the device-memory workspace that larger buckets use.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import assert_same_vector, fq, pair, runs, seeded_vector
from test_gpu_parity import MODELS

pytestmark = pytest.mark.gpu

SORT, HASH, AUTO = 1, 2, 0


@pytest.mark.parametrize("mode", ["REAL64", "REAL32", "INT", "DETERMINISTIC"])
@pytest.mark.parametrize("model", [MODELS[0], MODELS[2], MODELS[4], MODELS[8]],
                         ids=["real1d", "real2d", "mom1d", "real1d-65bit"])
def test_sort_arm_fifty_steps_from_default_start(model, mode):
    if model is MODELS[8] and mode == "DETERMINISTIC":
        pytest.skip("the exact power iteration of a 65-bit space outgrows any capacity")
    h, m = pair(*model)
    mcode = {"REAL64": 1, "REAL32": 2, "INT": 0, "DETERMINISTIC": 3}[mode]
    dt = (0.01 if mode != "INT" else 0.002) if model is not MODELS[8] else 0.002
    g, o = runs(h, m, mode=mcode, dt=dt, target=2000.0, seed=9, annihilation=SORT)
    g.seed_default(10.0)
    s = m.start()
    o.seed([s], [10.0], m.diagonal(s), 0)
    o.set_reference([s], [10.0])
    g.step(1)
    assert g.shape()["annihilation"] == "sort"
    o.step(1)
    rtol = {"REAL64": 1e-12, "REAL32": 1e-5, "INT": 0.0, "DETERMINISTIC": 1e-12}[mode]
    for block in range(5):
        g.step(10 if block else 9)
        o.step(10 if block else 9)
        if mode == "DETERMINISTIC":
            (gk, ga), (ok, oa) = g.export(), o.export()
            assert np.array_equal(gk, ok)
            assert np.max(np.abs(ga - oa)) <= 1e-12 * np.max(np.abs(oa))
            continue
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % (10 * block + 10))
    gh, oh = g.history(), o.history()
    for f in ("step", "len", "exact_steps", "inexact_steps", "n_spawns"):
        assert np.array_equal(gh[f], oh[f]), f
    tol = 1e-12 if mode != "REAL32" else 1e-5
    for f in ("shift", "norm", "hproj", "vproj"):
        assert np.allclose(gh[f], oh[f], rtol=tol, atol=tol), f


@pytest.mark.parametrize("mode", ["REAL64", "INT"])
@pytest.mark.parametrize("tables", [(0, 0), (64, 0)], ids=["on-chip", "device-memory"])
@pytest.mark.parametrize("model", [MODELS[1], MODELS[3]], ids=["real1d", "real2d-128bit"])
def test_sort_arm_large_vector(model, mode, tables):
    """A 20k-entry seeded vector over many buckets; with a 64-element on-chip
    workspace the larger buckets are sorted in the warp's device-memory
    workspace."""
    h, m = pair(*model)
    mcode = {"REAL64": 1, "INT": 0}[mode]
    keys, amps = seeded_vector(m, 20000, 21, mode=mode)
    # a small target (few buckets) when the device-memory workspace is wanted
    target = float(np.abs(amps).sum()) if not tables[0] else 1000.0
    g, o = runs(h, m, mode=mcode, dt=0.001, target=target, seed=5,
                capacity_vec=200000, capacity_spawn=2000000, annihilation=SORT)
    g.set_tables(*tables)
    g.seed(fq().keys_from_ints(keys), amps, -2.0, step=100)
    o.seed(keys, amps, -2.0, step=100)
    rtol = {"REAL64": 1e-12, "INT": 0.0}[mode]
    for s in range(3):
        g.step(1)
        o.step(1)
        assert_same_vector(g.export(), o.export(), rtol=rtol, what="step %d" % s)
    onchip, scratch = g.merge_paths()
    if tables[0]:
        assert scratch > 0, (onchip, scratch)
    else:
        assert onchip > 0


def test_sort_and_hash_arms_agree_and_autotuner_picks_one():
    """The same run with either arm: integer walkers give identical vectors
    and histories; with AUTO the autotuner times both arms and keeps one."""
    h, m = pair(*MODELS[1])
    out = []
    for ann in (SORT, HASH):
        g = fq().Run(h, fq().default_params(mode=0, dt=0.002, target=3e4, seed=8,
                                            annihilation=ann))
        g.seed_default(10.0)
        g.step(400)
        out.append((g.export(), g.history()))
        g.close()
    (ka, aa), ha = out[0]
    (kb, ab), hb = out[1]
    assert np.array_equal(ka, kb) and np.array_equal(aa, ab)
    assert np.array_equal(ha["len"], hb["len"]) and np.array_equal(ha["norm"], hb["norm"])
    g = fq().Run(h, fq().default_params(dt=0.001, target=1e5, seed=3, annihilation=AUTO))
    g.seed_default(10.0)
    g.step(300)
    g.autotune(1)
    assert g.shape()["annihilation"] in ("hash", "sort")
    g.close()
