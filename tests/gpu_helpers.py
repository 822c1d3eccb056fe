"""Shared helpers of the GPU parity tests: build matching runs on the GPU
(through the C ABI) and on the CPU oracle from the same seeded inputs."""
import numpy as np

import oracle as O
import workloads as W

MODES = {"INT": 0, "REAL64": 1, "REAL32": 2, "DETERMINISTIC": 3}


def fq():
    import paper_2601_19505_gb300 as m
    return m


def pair(kind, Lx, Ly, N, t, u, **prm):
    """(GPU Hamiltonian, oracle model)."""
    return fq().Hamiltonian(kind, Lx, Ly, N, t, u), O.Model(kind, Lx, Ly, N, t, u)


def runs(h, m, **prm):
    gp = fq().default_params(**prm)
    op = O.default_params(**{k: v for k, v in prm.items()
                             if k not in ("capacity_vec", "capacity_spawn", "annihilation")})
    return fq().Run(h, gp), O.Run(m, op)


def seeded_vector(m, n, seed, mode="REAL64", **kw):
    rng = np.random.default_rng(seed)
    occ = W.random_occupations(m.kind, m.Lx, m.Ly, m.N, n, rng)
    keys = [m.encode(o) for o in occ]
    amps = W.random_amplitudes(len(keys), rng, mode=mode, **kw)
    return keys, amps


def assert_same_vector(g, o, rtol=0.0, what=""):
    gk, ga = g
    ok, oa = o
    assert len(gk) == len(ok), "%s: lengths %d vs %d" % (what, len(gk), len(ok))
    assert np.array_equal(gk["lo"], ok["lo"]) and np.array_equal(gk["hi"], ok["hi"]), what
    if rtol == 0.0:
        assert np.array_equal(ga, oa), "%s: max |diff| %g" % (what, np.max(np.abs(ga - oa)))
    else:
        assert np.allclose(ga, oa, rtol=rtol, atol=0), "%s: max rel %g" % (
            what, np.max(np.abs(ga - oa) / np.abs(oa)))


def sorted_pairs(keys, vals):
    order = np.lexsort((vals, keys["lo"], keys["hi"]))
    return keys[order], vals[order]
