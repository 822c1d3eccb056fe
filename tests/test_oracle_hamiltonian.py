"""Pins of the oracle's Hamiltonians (not GPU): printed matrices and columns,
exact diagonalisation, closed forms and invariants."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.ed as ED
from conftest import golden


def test_three_site_matrix_as_printed():
    g = golden("real_3site_matrix.json")
    md = g["model"]
    m = O.Model(md["kind"], md["Lx"], 1, md["N"], md["t"], md["u"])
    basis = [m.encode(o) for o in g["basis_occ"]]
    idx = {k: i for i, k in enumerate(basis)}
    H = np.zeros((6, 6))
    for j, k in enumerate(basis):
        H[j, j] = m.diagonal(k)
        for d, v in zip(*m.column(k)):
            H[idx[d], j] += v
    assert np.allclose(H, np.array(g["matrix"]), atol=g["tol"], rtol=0)
    # a scaled Hamiltonian (alpha H) is printed beside it: u and t scale together
    a = g["scaled_alpha"]
    ms = O.Model(md["kind"], md["Lx"], 1, md["N"], a * md["t"], a * md["u"])
    Hs = np.zeros((6, 6))
    for j, k in enumerate(basis):
        Hs[j, j] = ms.diagonal(k)
        for d, v in zip(*ms.column(k)):
            Hs[idx[d], j] += v
    assert np.allclose(Hs, a * np.array(g["matrix"]), atol=2 * g["tol"], rtol=0)


def test_column_of_uniform_12x12_as_printed():
    g = golden("column_12x12.json")
    md = g["model"]
    m = O.Model(md["kind"], md["Lx"], 1, md["N"], md["t"], md["u"])
    s = m.start()
    assert list(m.decode(s)) == [1] * 12
    assert m.diagonal(s) == g["diagonal"]
    keys, vals = m.column(s)
    assert len(keys) == g["m"]
    assert np.all(vals == g["value"])
    assert 1.0 / len(keys) == g["random_offdiagonal_probability"]
    first = [list(m.decode(k)) for k in keys[:4]]
    last = [list(m.decode(k)) for k in keys[-3:]]
    assert first == g["first"] and last == g["last"]
    assert m.encode(g["random_offdiagonal_example"]) in keys


def _assert_hermitian_columns(m, keys):
    for k in keys:
        ck, cv = m.column(k)
        assert len(set(ck)) == len(ck)  # distinct destinations within a column
        for j, v in zip(ck, cv):
            bk, bv = m.column(j)
            pos = bk.index(k)
            assert bv[pos] == v


@pytest.mark.parametrize("kind,Lx,Ly,N,u", [(O.REAL_1D, 7, 1, 9, 3.0), (O.REAL_2D, 3, 4, 6, 2.0),
                                            (O.MOM_1D, 8, 1, 6, 4.0), (O.MOM_1D, 7, 1, 5, 1.5)])
def test_hermiticity(kind, Lx, Ly, N, u):
    m = O.Model(kind, Lx, Ly, N, 1.0, u)
    rng = np.random.default_rng(3)
    keys = [m.encode(np.bincount(rng.integers(0, m.M, N), minlength=m.M)) for _ in range(40)]
    _assert_hermitian_columns(m, keys)


@pytest.mark.parametrize("M,N", [(4, 4), (5, 3), (6, 6), (7, 4), (8, 5)])
def test_momentum_column_equals_second_quantised_sum(M, N):
    m = O.Model(O.MOM_1D, M, 1, N, 1.0, 2.5)
    eps = m.eps()
    for occ in ED.all_compositions(N, M)[:: max(1, math.comb(N + M - 1, N) // 60)]:
        k = m.encode(occ)
        ek, ev = m.column(k)
        bk, bv, bdiag = m.column_bruteforce(k)
        got = dict(zip(ek, ev))
        want = {d: v for d, v in zip(bk, bv) if abs(v) > 1e-14}
        assert set(got) == set(want)
        for d in want:
            assert got[d] == pytest.approx(want[d], rel=1e-13, abs=1e-14)
        kin = float(np.dot(eps, occ.astype(float)))
        assert m.diagonal(k) == pytest.approx(kin + bdiag, rel=1e-13, abs=1e-13)


def test_momentum_worked_example_as_printed():
    g = golden("momentum_h1111.json")
    md = g["model"]
    m = O.Model(md["kind"], md["Lx"], 1, md["N"], md["t"], md["u"])

    def apply(vec):
        out = {}
        for k, c in vec.items():
            out[k] = out.get(k, 0.0) + m.diagonal(k) * c
            for j, v in zip(*m.column(k)):
                out[j] = out.get(j, 0.0) + v * c
        return out

    dvec1 = {m.encode(o): c for o, c in g["dvec1"]}
    dvec2 = apply(dvec1)
    want = {m.encode(o): v for o, v in g["dvec2"]}
    got = {k: v for k, v in dvec2.items() if v != 0.0}
    assert set(got) == set(want)
    for k in want:
        assert got[k] == pytest.approx(want[k], abs=g["tol"])
    s = g["scalars_of_H_1111"]
    one = m.encode([1, 1, 1, 1])
    h1 = apply({one: 1.0})
    vals = np.array(list(h1.values()))
    assert h1[one] == s["dot"] == s["dot_vHv"]
    assert np.linalg.norm(vals) == pytest.approx(s["norm2"], rel=1e-15)
    assert vals.sum() == pytest.approx(s["sum"], rel=1e-14)


@pytest.mark.parametrize("M,N", [(4, 4), (5, 3), (6, 4)])
def test_momentum_spectrum_equals_real_space(M, N):
    """The momentum-space Hamiltonian is the Fourier transform of the
    real-space one: same full spectrum over every sector."""
    r = O.Model(O.REAL_1D, M, 1, N, 1.0, 3.0)
    k = O.Model(O.MOM_1D, M, 1, N, 1.0, 3.0)
    Hr, Hk = ED.full_dense(r), ED.full_dense(k)
    assert np.allclose(Hr, Hr.T) and np.allclose(Hk, Hk.T)
    assert np.allclose(np.linalg.eigvalsh(Hr), np.linalg.eigvalsh(Hk), atol=1e-10)


@pytest.mark.parametrize("kind,Lx,Ly,N", [(O.REAL_1D, 6, 1, 6), (O.REAL_1D, 5, 1, 7),
                                          (O.REAL_2D, 3, 3, 4), (O.MOM_1D, 6, 1, 6)])
def test_dimension_closed_form(kind, Lx, Ly, N):
    m = O.Model(kind, Lx, Ly, N, 1.0, 1.0)
    if kind == O.MOM_1D:
        # the start sector is one of M total-momentum sectors; all of them
        # together fill the Fock space
        occs = ED.all_compositions(N, m.M)
        sectors = {}
        for o in occs:
            sectors.setdefault(int(np.dot(np.arange(m.M), o)) % m.M, o)
        total = sum(len(ED.sparse_hamiltonian(m, m.encode(o))[0]) for o in sectors.values())
        assert total == math.comb(N + m.M - 1, N)
    else:
        basis, H = ED.sparse_hamiltonian(m)
        assert len(basis) == math.comb(N + m.M - 1, N)


@pytest.mark.parametrize("kind,Lx,Ly,N,z", [(O.REAL_1D, 7, 1, 3, 2), (O.REAL_2D, 3, 3, 2, 4),
                                            (O.REAL_2D, 4, 3, 3, 4)])
def test_noninteracting_ground_energy(kind, Lx, Ly, N, z):
    """U = 0: all bosons in the k = 0 orbital, E0 = -z t N."""
    t = 0.7
    m = O.Model(kind, Lx, Ly, N, t, 0.0)
    assert ED.lowest(m, 1)[0] == pytest.approx(-z * t * N, abs=1e-10)
    mk = O.Model(O.MOM_1D, 7, 1, 3, t, 0.0)
    assert ED.lowest(mk, 1)[0] == pytest.approx(-2 * t * 3, abs=1e-10)


def test_ed_6x6_small():
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    e = ED.lowest(m, 1)[0]
    assert e == pytest.approx(-4.02150241, abs=1e-8)


@pytest.mark.slow
def test_ed_12x12_as_printed():
    g = golden("energies.json")
    gc = golden("column_12x12.json")
    m = O.Model(O.REAL_1D, 12, 1, 12, 1.0, 6.0)
    basis, H = ED.sparse_hamiltonian(m)
    assert len(basis) == gc["dimension"]
    e = ED.lowest(m, 2)
    assert np.allclose(e, g["ed_12x12_u6"], atol=g["ed_tol"])
    # Sec. 2.3: the on-site correlation <G2(0)> of this ground state is
    # about one fifth (Sec. 2.3); G2(0) is diagonal, (1/M) sum_i n_i (n_i - 1) (Eq. g2)
    go = golden("observables.json")
    e0, basis, v0 = ED.ground_state(m)
    g20 = np.array([m.g2_diag(b, 0) for b in ED.basis_ints(basis)])
    expect = float(np.dot(v0 * v0, g20) / np.dot(v0, v0))
    assert abs(expect - go["g2_0_12x12_u6_about"]) < go["g2_0_tol"], expect
