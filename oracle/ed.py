"""Exact diagonalisation for the oracle (Sec. 5 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The sparse matrix is
assembled by a breadth-first search over the column graph of H, starting from
a given address (``or_build_sparse`` in ``fq_oracle.c``); the spectrum comes
from numpy's dense ``eigh`` for small dimensions or scipy's Lanczos ``eigsh``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import KEY_DT, Model, key_int


def sparse_hamiltonian(model: Model, start=None, max_dim: int = 2_000_000, nnz_per_row: int = 64):
    """(basis as Python ints, csr_matrix H) over the sector reachable from
    ``start`` (default: the model's starting address)."""
    basis, rows, cols, vals = model.build_sparse(start, max_dim=max_dim, nnz_per_row=nnz_per_row)
    dim = len(basis)
    H = sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim))
    return basis, H


def basis_ints(basis: np.ndarray):
    return [key_int(b) for b in basis]


def dense_hamiltonian(model: Model, start=None):
    basis, H = sparse_hamiltonian(model, start, max_dim=20000)
    return basis, H.toarray()


def lowest(model: Model, k: int = 1, start=None) -> np.ndarray:
    """The k lowest eigenvalues of H in the sector of ``start``."""
    basis, H = sparse_hamiltonian(model, start)
    if H.shape[0] <= 4000:
        return np.linalg.eigvalsh(H.toarray())[:k]
    vals = spla.eigsh(H, k=k, which="SA", tol=1e-12, ncv=max(2 * k + 1, 40),
                      return_eigenvectors=False)
    return np.sort(vals)


def ground_state(model: Model, start=None):
    """(E0, basis, v0) with v0 normalised to one-norm 1 and positive sum."""
    basis, H = sparse_hamiltonian(model, start)
    if H.shape[0] <= 4000:
        w, v = np.linalg.eigh(H.toarray())
        e0, v0 = w[0], v[:, 0]
    else:
        w, v = spla.eigsh(H, k=1, which="SA", tol=1e-12)
        e0, v0 = w[0], v[:, 0]
    v0 = v0 / np.sum(np.abs(v0))
    if v0.sum() < 0:
        v0 = -v0
    return e0, basis, v0


def all_compositions(N: int, M: int):
    """Every occupation vector of N bosons in M modes (the full Fock space)."""
    out = []

    def rec(prefix, left, modes):
        if modes == 1:
            out.append(prefix + [left])
            return
        for n in range(left, -1, -1):
            rec(prefix + [n], left - n, modes - 1)

    rec([], N, M)
    return np.array(out, dtype=np.uint8)


def full_dense(model: Model) -> np.ndarray:
    """Dense H over the whole Fock space (every sector), from the columns."""
    occs = all_compositions(model.N, model.M)
    keys = [model.encode(o) for o in occs]
    index = {k: i for i, k in enumerate(keys)}
    D = len(keys)
    H = np.zeros((D, D))
    for i, k in enumerate(keys):
        H[i, i] = model.diagonal(k)
        ck, cv = model.column(k)
        for j, v in zip(ck, cv):
            H[index[j], i] += v
    return H


__all__ = ["sparse_hamiltonian", "dense_hamiltonian", "lowest", "ground_state",
           "all_compositions", "full_dense", "basis_ints", "KEY_DT"]
