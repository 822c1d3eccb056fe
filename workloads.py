"""Seeded synthetic workloads for tests and benchmarks.

This module holds no arithmetic of the method: it only names the benchmark
configurations and draws random occupation-number vectors and amplitudes
(numpy ``default_rng``).  Both the CPU oracle and the GPU path encode the
occupations into addresses with their own codecs.

Configurations (the paper's workloads are synthetic Bose-Hubbard models; no
dataset is involved):
  c1  1D real space M = N = 6, U = 6, integer walkers, N_t = 1e3, dt = 1e-3
  c2  1D real space M = N = 20, U = 2, FP64, N_t = 1e7, dt = 1e-3 (39-bit keys)
  c3  1D momentum space M = N = 32, U = 4, FP32, N_t = 1e8, dt = 5e-4 (63-bit)
  c4  64 runs, 1D real space, M = N ~ U{10..30}, U/t ~ U[1, 10],
      N_t log-uniform in [1e4, 1e6], FP32, dt = 1e-3
  c5  2D 8 x 8 real space, N = 64, U = 8, FP32, N_t = 5e8, dt = 2e-4 (127-bit)
Every run starts from N_w = 10 walkers on the starting address.
"""
from __future__ import annotations

import numpy as np

CONFIGS = {
    "c1": dict(kind=1, Lx=6, Ly=1, N=6, t=1.0, u=6.0, mode="INT", target=1e3, dt=1e-3,
               steps=2000, seed=1),
    "c2": dict(kind=1, Lx=20, Ly=1, N=20, t=1.0, u=2.0, mode="REAL64", target=1e7, dt=1e-3,
               steps=10000, seed=1),
    # momentum space has positive off-diagonal elements (a sign problem): the
    # population overshoots the target several-fold before the shift controls it
    "c3": dict(kind=3, Lx=32, Ly=1, N=32, t=1.0, u=4.0, mode="REAL32", target=1e8, dt=5e-4,
               steps=5000, seed=1),
    "c5": dict(kind=2, Lx=8, Ly=8, N=64, t=1.0, u=8.0, mode="REAL32", target=5e8, dt=2e-4,
               steps=2000, seed=1),
}
START_WEIGHT = 10.0


def batch_configs(n: int = 64, seed: int = 1):
    """The c4 parameter points, drawn once with default_rng(seed)."""
    rng = np.random.default_rng(seed)
    M = rng.integers(10, 31, size=n)
    U = rng.uniform(1.0, 10.0, size=n)
    Nt = 10.0 ** rng.uniform(4.0, 6.0, size=n)
    return [dict(kind=1, Lx=int(M[i]), Ly=1, N=int(M[i]), t=1.0, u=float(U[i]), mode="REAL32",
                 target=float(Nt[i]), dt=1e-3, steps=5000, seed=1, run_id=i)
            for i in range(n)]


def _neighbours(kind: int, Lx: int, Ly: int, s: int):
    if kind == 2:
        x, y = s % Lx, s // Lx
        return [((x + 1) % Lx) + Lx * y, ((x - 1) % Lx) + Lx * y,
                x + Lx * ((y + 1) % Ly), x + Lx * ((y - 1) % Ly)]
    M = Lx * Ly
    return [(s + 1) % M, (s - 1) % M]


def random_occupations(kind: int, Lx: int, Ly: int, N: int, n: int, rng, max_moves: int = 12):
    """n distinct occupation vectors of N bosons in M modes.  Real space: random
    walks of single-boson hops from near-uniform filling (the support of a
    ground state spreads this way).  Momentum space: random pair moves that
    keep the total momentum, from the k = 0 condensate."""
    M = Lx * Ly
    if kind == 3:
        base = np.zeros(M, dtype=np.int64)
        base[M // 2 - 1] = N
    else:
        base = np.array([N // M + (1 if m < N % M else 0) for m in range(M)], dtype=np.int64)
    seen = set()
    out = []
    attempts = 0
    while len(out) < n and attempts < 50 * n + 1000:
        attempts += 1
        occ = base.copy()
        for _ in range(int(rng.integers(0, max_moves + 1))):
            if kind == 3:
                occupied = np.flatnonzero(occ)
                p = int(rng.choice(occupied))
                occ[p] -= 1
                occupied = np.flatnonzero(occ)
                if len(occupied) == 0:
                    occ[p] += 1
                    continue
                q = int(rng.choice(occupied))
                occ[q] -= 1
                r = int(rng.integers(0, M))
                s = (p + q - r) % M
                occ[r] += 1
                occ[s] += 1
            else:
                s = int(rng.choice(np.flatnonzero(occ)))
                t = int(rng.choice(_neighbours(kind, Lx, Ly, s)))
                occ[s] -= 1
                occ[t] += 1
        if occ.max() > 255:
            continue
        key = occ.tobytes()
        if key in seen:
            continue
        seen.add(key)
        out.append(occ.astype(np.uint8))
    return np.array(out, dtype=np.uint8).reshape(-1, M)


def random_amplitudes(n: int, rng, mode: str = "REAL64", big: float = 200.0, neg: float = 0.1):
    """Amplitudes shaped like an equilibrated walker vector: most near the
    compression threshold, a heavy tail of large ones (exact columns), a few
    below threshold, a fraction negative."""
    mag = 1.0 + rng.exponential(1.5, size=n)
    tail = rng.random(n) < 0.02
    mag[tail] = rng.uniform(20.0, big, size=int(tail.sum()))
    low = rng.random(n) < 0.05
    mag[low] = rng.uniform(0.05, 1.0, size=int(low.sum()))
    sign = np.where(rng.random(n) < neg, -1.0, 1.0)
    a = sign * mag
    if mode == "INT":
        a = np.where(a > 0, np.ceil(a), np.floor(a))
    return a
