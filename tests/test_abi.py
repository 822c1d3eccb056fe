"""The C ABI library loads and exports every declared entry point; host-side
calls that do no GPU work behave as declared (not GPU)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "fciqmc.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(fq_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2601_19505_gb300 import _lib
    lib = ctypes.CDLL(_lib._build.build())
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SYMBOLS), set(names) ^ set(_lib.SYMBOLS)


def test_struct_layouts_match_header():
    from paper_2601_19505_gb300 import _lib
    assert ctypes.sizeof(_lib.FqKey) == 16
    assert ctypes.sizeof(_lib.FqStats) == 72
    assert ctypes.sizeof(_lib.FqParams) == 88


def test_host_side_calls_without_gpu():
    import paper_2601_19505_gb300 as fq
    p = fq.default_params()
    assert (p.dt, p.zeta, p.threshold, p.t_rel, p.target) == (0.01, 0.08, 1.0, 1.0, 1000.0)
    assert p.xi == pytest.approx(0.08 ** 2 / 4)
    # the library sets the forcing of a given damping (xi = zeta^2 / 4); an
    # explicit xi overrides it
    p = fq.default_params(zeta=0.3)
    assert (p.zeta, p.xi) == (0.3, 0.3 * 0.3 / 4.0)
    p = fq.default_params(zeta=0.3, xi=0.01)
    assert (p.zeta, p.xi) == (0.3, 0.01)
    with pytest.raises(fq.FqError):
        fq.default_params(zeta=-1.0)
    for kind, Lx, Ly, N in [(1, 6, 1, 6), (1, 20, 1, 20), (3, 32, 1, 32), (2, 8, 8, 64)]:
        h = fq.Hamiltonian(kind, Lx, Ly, N, 1.0, 2.0)
        m = O.Model(kind, Lx, Ly, N, 1.0, 2.0)
        assert h.M == m.M and h.nbits == m.nbits
        assert h.key_words == (1 if m.nbits <= 64 else 2)
        assert h.starting_address() == m.start()
        assert h.dimension() == pytest.approx(math.comb(N + m.M - 1, N), rel=1e-15)
        rng = np.random.default_rng(1)
        for _ in range(50):
            occ = np.bincount(rng.integers(0, m.M, N), minlength=m.M).astype(np.uint8)
            k = h.encode(occ)
            assert k == m.encode(occ)
            assert np.array_equal(h.decode(k), occ)
    with pytest.raises(fq.FqError):
        fq.Hamiltonian(1, 2, 1, 4, 1.0, 1.0)      # ring of 2 sites: neighbours coincide
    with pytest.raises(fq.FqError):
        fq.Hamiltonian(3, 65, 1, 4, 1.0, 1.0)     # momentum space up to 64 modes
    with pytest.raises(fq.FqError):
        fq.Hamiltonian(1, 100, 1, 40, 1.0, 1.0)   # 139 bits
    h = fq.Hamiltonian(1, 6, 1, 6, 1.0, 1.0)
    with pytest.raises(fq.FqError):
        h.encode([1, 1, 1, 1, 1, 0])
    with pytest.raises(fq.FqError):
        h.decode(1 << 11)


def test_run_creation_fails_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2601_19505_gb300 as fq
    h = fq.Hamiltonian(1, 6, 1, 6, 1.0, 6.0)
    with pytest.raises(Exception):
        fq.Run(h, fq.default_params(), stream=0, torch_allocator=False)
