"""CPU oracle for the FCIQMC step (Rimu.jl paper, arXiv 2601.19505).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2601_19505_gb300``) never imports it, and it
never imports the product path: the two share no code.

The arithmetic lives in ``fq_oracle.c`` (plain single-threaded C, compiled with
``-ffp-contract=off``); this module only marshals arguments.  ``ed.py`` holds
exact diagonalisation (Sec. 5) and ``blocking.py`` the blocking analysis
(Sec. 4.1) used to check the oracle against exact energies.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against values the paper prints (bit strings, the 6x6 matrix, the 24-entry
column, the momentum-space H|1111> table, the printed shift rows), against
exact diagonalisation, closed forms (dimension, U = 0 energy), invariants
(Hermiticity, unbiasedness of one step) and the published Philox4x32-10
known-answer vectors.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fq_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libfqoracle.so")

REAL_1D, REAL_2D, MOM_1D = 1, 2, 3
MODE_INT, MODE_REAL64, MODE_REAL32, MODE_DETERMINISTIC = 0, 1, 2, 3
COMPRESS_LATE, COMPRESS_EARLY = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libfqoracle.so`` (gcc, no FMA)."""
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


class Key(C.Structure):
    _fields_ = [("lo", C.c_uint64), ("hi", C.c_uint64)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("target", C.c_double), ("zeta", C.c_double),
                ("xi", C.c_double), ("threshold", C.c_double), ("t_rel", C.c_double),
                ("mode", C.c_int32), ("pad0", C.c_int32), ("seed", C.c_uint64),
                ("run_id", C.c_uint32), ("compression", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("len", C.c_int64), ("exact_steps", C.c_int64),
                ("inexact_steps", C.c_int64), ("n_spawns", C.c_int64), ("shift", C.c_double),
                ("norm", C.c_double), ("hproj", C.c_double), ("vproj", C.c_double)]


KEY_DT = np.dtype([("lo", "<u8"), ("hi", "<u8")])
STATS_FIELDS = [f for f, _ in Stats._fields_]

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, dp, kp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(Key)
        L.or_model_new.restype = vp
        L.or_model_new.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]
        L.or_model_free.argtypes = [vp]
        L.or_model_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.or_model_eps.restype = C.c_double
        L.or_model_eps.argtypes = [vp, C.c_int]
        L.or_encode.argtypes = [vp, C.c_void_p, kp]
        L.or_decode.argtypes = [vp, kp, C.c_void_p]
        L.or_start.argtypes = [vp, kp]
        L.or_diagonal.restype = C.c_double
        L.or_diagonal.argtypes = [vp, kp]
        L.or_column.restype = C.c_long
        L.or_column.argtypes = [vp, kp, C.c_void_p, C.c_void_p, C.c_long]
        L.or_column_bruteforce.restype = C.c_long
        L.or_column_bruteforce.argtypes = [vp, kp, C.c_void_p, C.c_void_p, C.c_long, dp]
        L.or_philox.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_run_new.restype = vp
        L.or_run_new.argtypes = [vp, C.POINTER(Params)]
        L.or_run_free.argtypes = [vp]
        L.or_run_seed.argtypes = [vp, C.c_void_p, C.c_void_p, C.c_long, C.c_double, C.c_int64]
        L.or_run_set_reference.argtypes = [vp, C.c_void_p, C.c_void_p, C.c_long]
        L.or_run_set.argtypes = [vp, C.c_double, C.c_double, C.c_double]
        L.or_run_record_spawns.argtypes = [vp, C.c_int]
        L.or_run_step.argtypes = [vp, C.c_long]
        L.or_run_len.restype = C.c_long
        L.or_run_len.argtypes = [vp]
        L.or_run_export.restype = C.c_long
        L.or_run_export.argtypes = [vp, C.c_void_p, C.c_void_p, C.c_long]
        L.or_run_state.argtypes = [vp, dp, dp, C.POINTER(C.c_int64)]
        L.or_run_history.restype = C.c_long
        L.or_run_history.argtypes = [vp, C.c_void_p, C.c_long]
        L.or_run_spawns.restype = C.c_long
        L.or_run_spawns.argtypes = [vp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_long]
        L.or_point.argtypes = [vp, kp, dp, dp]
        L.or_exact_norm_of.restype = C.c_double
        L.or_exact_norm_of.argtypes = [C.c_void_p, C.c_long, C.c_double, C.c_int]
        L.or_shift_update.restype = C.c_double
        L.or_shift_update.argtypes = [C.c_double] * 7
        L.or_overlap.argtypes = [vp, vp, C.c_void_p, C.c_int, dp]
        L.or_spectral_step.argtypes = [C.c_void_p, C.c_int, C.c_long]
        L.or_g2_diag.restype = C.c_double
        L.or_g2_diag.argtypes = [vp, kp, C.c_int]
        L.or_build_sparse.restype = C.c_long
        L.or_build_sparse.argtypes = [vp, kp, C.c_long, C.c_void_p, C.c_long, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def key_of(k) -> Key:
    if isinstance(k, Key):
        return k
    if isinstance(k, (tuple, list)):
        return Key(int(k[0]), int(k[1]))
    if isinstance(k, np.void):
        return Key(int(k["lo"]), int(k["hi"]))
    v = int(k)
    return Key(v & 0xFFFFFFFFFFFFFFFF, v >> 64)


def key_int(k) -> int:
    return int(k["lo"]) | (int(k["hi"]) << 64) if not isinstance(k, Key) else k.lo | (k.hi << 64)


def keys_array(keys) -> np.ndarray:
    """Python ints or (lo, hi) pairs -> structured array of KEY_DT."""
    out = np.zeros(len(keys), dtype=KEY_DT)
    for i, k in enumerate(keys):
        kk = key_of(k)
        out[i] = (kk.lo, kk.hi)
    return out


def philox4x32_10(ctr, key) -> tuple:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_ptr(c), _ptr(k), _ptr(o))
    return tuple(int(x) for x in o)


def exact_norm(amps, threshold: float = 1.0, mode: int = MODE_REAL64) -> float:
    """The oracle's one-norm of a vector with these amplitudes."""
    a = np.ascontiguousarray(amps, dtype=np.float64)
    return lib().or_exact_norm_of(_ptr(a), len(a), threshold, mode)


def shift_update(S, N0, N1, dt, zeta, xi, target) -> float:
    """The oracle's shift update (Eq. shift-update)."""
    return lib().or_shift_update(S, N0, N1, dt, zeta, xi, target)


class Model:
    """A Bose-Hubbard Hamiltonian: kind REAL_1D (Lx sites), REAL_2D (Lx x Ly,
    periodic) or MOM_1D (Lx momentum modes)."""

    def __init__(self, kind: int, Lx: int, Ly: int, N: int, t: float, u: float):
        self.kind, self.Lx, self.Ly, self.N, self.t, self.u = kind, Lx, Ly, N, t, u
        self.h = lib().or_model_new(kind, Lx, Ly, N, t, u)
        if not self.h:
            raise ValueError("invalid model parameters")
        M, nb = C.c_int(), C.c_int()
        lib().or_model_info(self.h, C.byref(M), C.byref(nb))
        self.M, self.nbits = M.value, nb.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_model_free(self.h)
            self.h = None

    def eps(self) -> np.ndarray:
        return np.array([lib().or_model_eps(self.h, m) for m in range(self.M)])

    def encode(self, occ) -> int:
        o = np.ascontiguousarray(occ, dtype=np.uint8)
        assert o.size == self.M
        k = Key()
        if lib().or_encode(self.h, _ptr(o), C.byref(k)):
            raise ValueError("occupation does not hold N bosons")
        return k.lo | (k.hi << 64)

    def decode(self, key) -> np.ndarray:
        o = np.zeros(self.M, dtype=np.uint8)
        if lib().or_decode(self.h, C.byref(key_of(key)), _ptr(o)):
            raise ValueError("not a valid address")
        return o

    def start(self) -> int:
        k = Key()
        lib().or_start(self.h, C.byref(k))
        return k.lo | (k.hi << 64)

    def diagonal(self, key) -> float:
        return lib().or_diagonal(self.h, C.byref(key_of(key)))

    def column(self, key):
        """Off-diagonal entries of the column at ``key`` in enumeration order:
        (list of int addresses, np.ndarray of values)."""
        kk = key_of(key)
        m = lib().or_column(self.h, C.byref(kk), None, None, 0)
        keys = np.zeros(max(m, 1), dtype=KEY_DT)
        vals = np.zeros(max(m, 1))
        lib().or_column(self.h, C.byref(kk), _ptr(keys), _ptr(vals), m)
        return [key_int(keys[i]) for i in range(m)], vals[:m].copy()

    def g2_diag(self, key, d: int) -> float:
        """G2(d) on one address (Eq. g2), 1D real space."""
        return lib().or_g2_diag(self.h, C.byref(key_of(key)), int(d))

    def column_bruteforce(self, key, cap: int = 1 << 16):
        kk = key_of(key)
        keys = np.zeros(cap, dtype=KEY_DT)
        vals = np.zeros(cap)
        d = C.c_double()
        n = lib().or_column_bruteforce(self.h, C.byref(kk), _ptr(keys), _ptr(vals), cap, C.byref(d))
        if n < 0:
            raise RuntimeError("capacity")
        return [key_int(keys[i]) for i in range(n)], vals[:n].copy(), d.value

    def build_sparse(self, start=None, max_dim: int = 2_000_000, nnz_per_row: int = 64):
        """BFS basis and COO nonzeros of H (Sec. 5)."""
        s = key_of(self.start() if start is None else start)
        basis = np.zeros(max_dim, dtype=KEY_DT)
        cap = max_dim * nnz_per_row
        rows = np.zeros(cap, dtype=np.int64)
        cols = np.zeros(cap, dtype=np.int64)
        vals = np.zeros(cap)
        nnz = C.c_int64()
        dim = lib().or_build_sparse(self.h, C.byref(s), max_dim, _ptr(basis), cap, _ptr(rows),
                                    _ptr(cols), _ptr(vals), C.byref(nnz))
        if dim < 0:
            raise RuntimeError("basis or nonzero capacity exceeded")
        n = nnz.value
        return basis[:dim].copy(), rows[:n].copy(), cols[:n].copy(), vals[:n].copy()


def default_params(**kw) -> Params:
    """Defaults recovered from the paper's printed time series: dt = 0.01,
    zeta = 0.08, xi = zeta^2 / 4, threshold 1, t_rel 1, target 1000."""
    p = Params(dt=0.01, target=1000.0, zeta=0.08, xi=0.08 ** 2 / 4, threshold=1.0, t_rel=1.0,
               mode=MODE_REAL64, pad0=0, seed=1, run_id=0, compression=COMPRESS_LATE)
    for k, v in kw.items():
        setattr(p, k, v)
    if "zeta" in kw and "xi" not in kw:
        p.xi = p.zeta ** 2 / 4
    return p


class Run:
    """One FCIQMC run on the oracle."""

    def __init__(self, model: Model, params: Params):
        self.model = model
        self.params = params
        self.h = lib().or_run_new(model.h, C.byref(params))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_run_free(self.h)
            self.h = None

    def seed(self, keys, amps, shift: float, step: int = 0):
        ka = keys if isinstance(keys, np.ndarray) and keys.dtype == KEY_DT else keys_array(keys)
        aa = np.ascontiguousarray(amps, dtype=np.float64)
        if lib().or_run_seed(self.h, _ptr(ka), _ptr(aa), len(aa), shift, step):
            raise ValueError("duplicate addresses in seed")

    def set_reference(self, keys, y):
        ka = keys if isinstance(keys, np.ndarray) and keys.dtype == KEY_DT else keys_array(keys)
        ya = np.ascontiguousarray(y, dtype=np.float64)
        lib().or_run_set_reference(self.h, _ptr(ka), _ptr(ya), len(ya))

    def set(self, dt=0.0, shift=None, target=0.0):
        if shift is None:
            shift = self.state()[0]
        lib().or_run_set(self.h, dt, shift, target)

    def record_spawns(self, on=True):
        lib().or_run_record_spawns(self.h, 1 if on else 0)

    def step(self, n: int = 1) -> int:
        return lib().or_run_step(self.h, n)

    def export(self):
        n = lib().or_run_len(self.h)
        keys = np.zeros(max(n, 1), dtype=KEY_DT)
        amps = np.zeros(max(n, 1))
        lib().or_run_export(self.h, _ptr(keys), _ptr(amps), n)
        return keys[:n].copy(), amps[:n].copy()

    def state(self):
        s, nm, st = C.c_double(), C.c_double(), C.c_int64()
        lib().or_run_state(self.h, C.byref(s), C.byref(nm), C.byref(st))
        return s.value, nm.value, st.value

    def history(self) -> np.ndarray:
        n = lib().or_run_history(self.h, None, 0)
        rows = (Stats * max(n, 1))()
        lib().or_run_history(self.h, C.cast(rows, C.c_void_p), n)
        dt = np.dtype([(f, "<i8") if i < 5 else (f, "<f8") for i, f in enumerate(STATS_FIELDS)])
        return np.frombuffer(bytes(rows), dtype=dt, count=n).copy()

    def spawns(self):
        n = lib().or_run_spawns(self.h, None, None, None, 0)
        d = np.zeros(max(n, 1), dtype=KEY_DT)
        s = np.zeros(max(n, 1), dtype=KEY_DT)
        v = np.zeros(max(n, 1))
        lib().or_run_spawns(self.h, _ptr(d), _ptr(s), _ptr(v), n)
        return d[:n].copy(), s[:n].copy(), v[:n].copy()

    def point(self, key):
        pre, post = C.c_double(), C.c_double()
        lib().or_point(self.h, C.byref(key_of(key)), C.byref(pre), C.byref(post))
        return pre.value, post.value


def overlap(a: Run, b: Run, g2_d=()) -> np.ndarray:
    """[c_A^T c_B, c_A^T G2(d) c_B for d in g2_d] of two runs of one model (Sec. 4.3)."""
    d = np.ascontiguousarray(g2_d, dtype=np.int32)
    out = np.zeros(1 + len(d))
    if lib().or_overlap(a.h, b.h, _ptr(d), len(d), out.ctypes.data_as(C.POINTER(C.c_double))):
        raise ValueError("G2 needs 1D real space and 0 <= d < M")
    return out


def spectral_step(runs, n: int = 1) -> int:
    """n steps of runs of one model, each run after the first orthogonalised to
    the ones before it (Gram-Schmidt, Sec. 2.2); 0, or -5 if a population died."""
    arr = (C.c_void_p * len(runs))(*[r.h for r in runs])
    rc = lib().or_spectral_step(arr, len(runs), n)
    if rc == -1:
        raise ValueError("Gram-Schmidt needs 1 to 8 runs of real-valued walkers")
    return rc


def start_run(model: Model, params: Params, weight: float = 10.0, shift=None) -> Run:
    """A run seeded like the paper's default: ``weight`` (N_w = 10) on the
    starting address, shift = its diagonal element, y = N_w e_start."""
    r = Run(model, params)
    s = model.start()
    r.seed([s], [weight], model.diagonal(s) if shift is None else shift, 0)
    r.set_reference([s], [weight])
    return r
