"""fq_ham_column_noalloc against fq_ham_column (needs a GB300).

The variant evaluates the column into a fixed device array instead of
buffers allocated per call.  Both run the same device code on the same
tables, so the results must be identical (tolerance: exact), on two calls
in a row.  This file is named to be collected last, so it also shows that
the fixed array works after everything else in the suite has run.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

MODELS = [  # kind, Lx, Ly, N, t, u: 64- and 128-bit addresses, all three kinds
    (1, 20, 1, 20, 1.0, 2.0),
    (2, 8, 8, 64, 1.0, 8.0),
    (3, 32, 1, 32, 1.0, 4.0),
    (3, 16, 1, 9, 0.7, 1.5),
    (2, 5, 3, 11, 2.5, 3.0),
    (1, 9, 1, 30, 0.3, 1.0),   # N > M: multiply occupied sites, t != 1
]


def _lib():
    from paper_2601_19505_gb300 import _lib as L
    return L


def _call(name, h, key, cap):
    L = _lib()
    k = int(key)
    dest = np.zeros(cap, dtype=[("lo", "<u8"), ("hi", "<u8")])
    val = np.full(cap, np.nan)
    d, m = C.c_double(np.nan), C.c_size_t(0)
    rc = getattr(L.load(), name)(h.h, L.FqKey(k & 0xFFFFFFFFFFFFFFFF, k >> 64), C.byref(d),
                                 dest.ctypes.data_as(C.c_void_p), val.ctypes.data_as(C.c_void_p),
                                 cap, C.byref(m))
    return rc, d.value, m.value, dest, val


@pytest.mark.parametrize("model", MODELS, ids=lambda m: "k%d_%dx%d_N%d" % m[:4])
def test_noalloc_column_equals_allocating_column(model):
    import paper_2601_19505_gb300 as fq
    kind, Lx, Ly, N, t, u = model
    h = fq.Hamiltonian(kind, Lx, Ly, N, t, u)
    rng = np.random.default_rng(7)
    occ = W.random_occupations(kind, Lx, Ly, N, 6, rng)
    keys = [h.starting_address()] + [h.encode(o) for o in occ]
    cap = 1 << 15
    for key in keys:
        rc0, d0, m0, k0, v0 = _call("fq_ham_column", h, key, cap)
        assert rc0 == 0 and 0 < m0 <= 16384
        for _ in range(2):  # two calls in a row on the same fixed array
            rc1, d1, m1, k1, v1 = _call("fq_ham_column_noalloc", h, key, cap)
            assert rc1 == 0
            assert m1 == m0 and d1 == d0
            assert np.array_equal(k1[:m1], k0[:m0])
            assert np.array_equal(v1[:m1], v0[:m0])
            assert np.all(np.isnan(v1[m1:]))  # nothing written past the column


def test_noalloc_column_short_buffer_and_rejection():
    import paper_2601_19505_gb300 as fq
    # a short caller buffer gets the first cap entries, as with fq_ham_column
    h = fq.Hamiltonian(1, 20, 1, 20, 1.0, 2.0)
    key = h.starting_address()
    rc0, d0, m0, k0, v0 = _call("fq_ham_column", h, key, 5)
    rc1, d1, m1, k1, v1 = _call("fq_ham_column_noalloc", h, key, 5)
    assert rc0 == rc1 == 0 and m0 == m1 == 40
    assert np.array_equal(k0, k1) and np.array_equal(v0, v1)
    # 64 singly occupied momentum modes: a column of ~6e4 entries, beyond the
    # fixed array; rejected with FQ_ERR_CAPACITY and its length reported
    hm = fq.Hamiltonian(3, 64, 1, 64, 1.0, 1.0)
    big = hm.encode(np.ones(64, dtype=np.uint8))
    rc0, _, m0, _, _ = _call("fq_ham_column", hm, big, 1 << 17)
    assert rc0 == 0 and m0 > 16384
    rc1, d1, m1, k1, v1 = _call("fq_ham_column_noalloc", hm, big, 1 << 17)
    assert rc1 == -3 and m1 == m0
    assert np.isnan(d1) and np.all(np.isnan(v1))
    # the array is still good afterwards
    rc2, d2, m2, _, v2 = _call("fq_ham_column_noalloc", h, key, 64)
    assert rc2 == 0 and m2 == 40 and d2 == d0


def test_noalloc_calls_alternating_between_models():
    """Calls on models with different N, t and address width, alternated
    A, B, A, C, B, ...: every call rewrites the tables in the fixed array, so
    a stale or partial table of the previous model would show here."""
    import paper_2601_19505_gb300 as fq
    hams = [fq.Hamiltonian(*m[:3], m[3], m[4], m[5]) for m in MODELS]
    rng = np.random.default_rng(11)
    keys = []
    for (kind, Lx, Ly, N, _, _), h in zip(MODELS, hams):
        occ = W.random_occupations(kind, Lx, Ly, N, 2, rng)
        keys.append([h.starting_address()] + [h.encode(o) for o in occ])
    want = {}
    for i, h in enumerate(hams):
        for j, key in enumerate(keys[i]):
            rc, d, m, k, v = _call("fq_ham_column", h, key, 1 << 15)
            assert rc == 0
            want[i, j] = (d, m, k[:m].copy(), v[:m].copy())
    order = [0, 1, 0, 2, 1, 5, 3, 0, 4, 5, 2, 3, 1, 4, 0]
    for n, i in enumerate(order):
        j = n % len(keys[i])
        rc, d, m, k, v = _call("fq_ham_column_noalloc", hams[i], keys[i][j], 1 << 15)
        d0, m0, k0, v0 = want[i, j]
        assert rc == 0 and m == m0 and d == d0, (i, j)
        assert np.array_equal(k[:m], k0) and np.array_equal(v[:m], v0), (i, j)
