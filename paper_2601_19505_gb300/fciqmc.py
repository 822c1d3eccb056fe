"""Python objects over the C ABI of libfciqmc (include/fciqmc.h).

Every call forwards to the function of the same name in the C ABI; nothing
here computes any part of the step.  Device memory comes from PyTorch's
caching allocator and work is queued on PyTorch's current CUDA stream unless
told otherwise.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

BH_REAL_1D, BH_REAL_2D, BH_MOM_1D = 1, 2, 3
MODE_INT, MODE_REAL64, MODE_REAL32, MODE_DETERMINISTIC = 0, 1, 2, 3
ANN_AUTO, ANN_SORT, ANN_HASH = 0, 1, 2
COMPRESS_LATE, COMPRESS_EARLY = 0, 1

KEY_DTYPE = np.dtype([("lo", "<u8"), ("hi", "<u8")])
STATS_DTYPE = np.dtype([("step", "<i8"), ("len", "<i8"), ("exact_steps", "<i8"),
                        ("inexact_steps", "<i8"), ("n_spawns", "<i8"), ("shift", "<f8"),
                        ("norm", "<f8"), ("hproj", "<f8"), ("vproj", "<f8")])


class FqError(RuntimeError):
    """A negative status code of the C ABI (FQ_ERR_*), with the call that returned it."""
    def __init__(self, code: int, what: str):
        self.code = code
        msg = L.load().fq_strerror(code).decode()
        super().__init__("%s: %s (%d)" % (what, msg, code))


class RunError(FqError):
    """A device-side error of a run, with the cause bits of fq_run_error_bits."""

    def __init__(self, code: int, what: str, bits: int):
        super().__init__(code, what)
        self.bits = bits
        self.args = (self.args[0] + " [device bits 0x%x]" % bits,)


def _check(code: int, what: str):
    if code:
        raise FqError(code, what)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def version() -> str:
    """fq_version: the library version string."""
    return L.load().fq_version().decode()


def keys_from_ints(keys) -> np.ndarray:
    """Python integers (addresses up to 128 bits) as an fq_key array (lo, hi)."""
    out = np.zeros(len(keys), dtype=KEY_DTYPE)
    for i, k in enumerate(keys):
        k = int(k)
        out[i] = (k & 0xFFFFFFFFFFFFFFFF, k >> 64)
    return out


def keys_to_ints(keys: np.ndarray):
    """An fq_key array as Python integers."""
    return [int(k["lo"]) | (int(k["hi"]) << 64) for k in keys]


def _as_keys(keys) -> np.ndarray:
    if isinstance(keys, np.ndarray) and keys.dtype == KEY_DTYPE:
        return np.ascontiguousarray(keys)
    if isinstance(keys, np.ndarray) and keys.dtype.names == ("lo", "hi"):
        return np.ascontiguousarray(keys).view(KEY_DTYPE)
    return keys_from_ints(keys)


def default_params(**kw) -> L.FqParams:
    """fq_params_default, then the given fields; zeta goes through
    fq_params_set_zeta (which also sets its forcing xi) before an explicit xi."""
    p = L.FqParams()
    lib = L.load()
    _check(lib.fq_params_default(C.byref(p)), "fq_params_default")
    if "zeta" in kw:
        _check(lib.fq_params_set_zeta(C.byref(p), float(kw["zeta"])), "fq_params_set_zeta")
    for k, v in kw.items():
        if k == "zeta":
            continue
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Hamiltonian:
    """fq_ham_create(kind, Lx, Ly, N, t, u)."""

    def __init__(self, kind: int, Lx: int, Ly: int, N: int, t: float, u: float):
        self._lib = L.load()
        h = C.c_void_p()
        _check(self._lib.fq_ham_create(C.byref(h), kind, Lx, Ly, N, t, u), "fq_ham_create")
        self.h = h
        self.kind, self.Lx, self.Ly, self.N, self.t, self.u = kind, Lx, Ly, N, t, u
        M, nb, kw = C.c_int(), C.c_int(), C.c_int()
        self._lib.fq_ham_info(h, C.byref(M), C.byref(nb), C.byref(kw))
        self.M, self.nbits, self.key_words = M.value, nb.value, kw.value

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.fq_ham_destroy(self.h)
            self.h = None

    def dimension(self) -> float:
        """fq_ham_dimension: the Fock-space dimension C(N + M - 1, N), as a float."""
        d = C.c_double()
        _check(self._lib.fq_ham_dimension(self.h, C.byref(d)), "fq_ham_dimension")
        return d.value

    def starting_address(self) -> int:
        """fq_ham_starting_address: near-uniform filling (real space) or the k = 0 condensate."""
        k = L.FqKey()
        _check(self._lib.fq_ham_starting_address(self.h, C.byref(k)), "fq_ham_starting_address")
        return k.lo | (k.hi << 64)

    def encode(self, occ) -> int:
        """fq_encode: occupation numbers of the M modes to an address (an int)."""
        o = np.ascontiguousarray(occ, dtype=np.uint8)
        k = L.FqKey()
        _check(self._lib.fq_encode(self.h, _ptr(o), C.byref(k)), "fq_encode")
        return k.lo | (k.hi << 64)

    def decode(self, key) -> np.ndarray:
        """fq_decode: an address to the occupation numbers of the M modes."""
        o = np.zeros(self.M, dtype=np.uint8)
        k = int(key)
        _check(self._lib.fq_decode(self.h, L.FqKey(k & 0xFFFFFFFFFFFFFFFF, k >> 64), _ptr(o)),
               "fq_decode")
        return o

    def column(self, key, cap: int = 1 << 16):
        """(diagonal, [destination ints], values) from the device code."""
        k = int(key)
        dest = np.zeros(cap, dtype=KEY_DTYPE)
        val = np.zeros(cap)
        d, m = C.c_double(), C.c_size_t()
        _check(self._lib.fq_ham_column(self.h, L.FqKey(k & 0xFFFFFFFFFFFFFFFF, k >> 64),
                                       C.byref(d), _ptr(dest), _ptr(val), cap, C.byref(m)),
               "fq_ham_column")
        n = min(m.value, cap)
        return d.value, keys_to_ints(dest[:n]), val[:n].copy()


class _TorchAllocator:
    """Routes device allocations through torch.cuda's caching allocator."""

    def __init__(self):
        import torch

        self.torch = torch
        self.device = torch.cuda.current_device()
        self._alloc = L.ALLOC_FN(self.alloc)
        self._free = L.FREE_FN(self.free)
        self.struct = L.FqAllocator(None, self._alloc, self._free)

    def alloc(self, ctx, nbytes, stream):
        """Device allocation for the C library, from the caching allocator (None on failure)."""
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                           int(stream or 0))
        except Exception:  # noqa: BLE001 - the C side reports FQ_ERR_NOMEM
            return None

    def free(self, ctx, ptr, nbytes, stream):
        """Release an allocation made by alloc."""
        self.torch.cuda.caching_allocator_delete(int(ptr))


def _current_stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


class Run:
    """fq_run_create(h, params, stream, allocator)."""

    def __init__(self, ham: Hamiltonian, params: L.FqParams | None = None, stream=None,
                 torch_allocator: bool = True):
        self._lib = L.load()
        self.ham = ham
        self.params = params if params is not None else default_params()
        self.stream = _current_stream() if stream is None else int(stream)
        self._alloc = _TorchAllocator() if torch_allocator else None
        r = C.c_void_p()
        _check(self._lib.fq_run_create(C.byref(r), ham.h, C.byref(self.params),
                                       C.c_void_p(self.stream),
                                       C.byref(self._alloc.struct) if self._alloc else None),
               "fq_run_create")
        self.r = r

    def close(self):
        """Release the handle and its device memory (also done on garbage collection)."""
        if getattr(self, "r", None):
            self._lib.fq_run_destroy(self.r)
            self.r = None

    def _chk(self, code: int, what: str):
        if code:
            b = C.c_uint()
            self._lib.fq_run_error_bits(self.r, C.byref(b))
            raise RunError(code, what, b.value)

    def __del__(self):
        self.close()

    def seed(self, keys, amps, shift: float, step: int = 0):
        """fq_run_seed: replace the vector by (keys, amps); set the shift and the step counter."""
        k = _as_keys(keys)
        a = np.ascontiguousarray(amps, dtype=np.float64)
        _check(self._lib.fq_run_seed(self.r, _ptr(k), _ptr(a), len(a), float(shift), int(step)),
               "fq_run_seed")

    def seed_default(self, weight: float = 10.0):
        """fq_run_seed_default: `weight` walkers on the starting address, shift = its diagonal."""
        _check(self._lib.fq_run_seed_default(self.r, float(weight)), "fq_run_seed_default")

    def set_reference(self, keys, y):
        """fq_run_set_reference: the projected-energy reference y (addresses, coefficients)."""
        k = _as_keys(keys)
        a = np.ascontiguousarray(y, dtype=np.float64)
        _check(self._lib.fq_run_set_reference(self.r, _ptr(k), _ptr(a), len(a)),
               "fq_run_set_reference")

    def set_dt(self, dt: float):
        """fq_run_set_dt: the time step of the following steps."""
        _check(self._lib.fq_run_set_dt(self.r, float(dt)), "fq_run_set_dt")

    def set_shift(self, s: float):
        """fq_run_set_shift: the current shift."""
        _check(self._lib.fq_run_set_shift(self.r, float(s)), "fq_run_set_shift")

    def set_target(self, t: float):
        """fq_run_set_target: the target one-norm N_t."""
        _check(self._lib.fq_run_set_target(self.r, float(t)), "fq_run_set_target")

    def step(self, n: int = 1):
        """Enqueue n steps (asynchronous; errors surface at the next synchronising call)."""
        _check(self._lib.fq_run_step(self.r, int(n)), "fq_run_step")

    def sync(self) -> int:
        """Wait for queued steps; the status code (0, or a negative FQ_ERR_* after a rollback)."""
        return self._lib.fq_run_sync(self.r)

    def error_bits(self) -> int:
        """fq_run_error_bits: the device-side cause of the last reported error."""
        b = C.c_uint()
        _check(self._lib.fq_run_error_bits(self.r, C.byref(b)), "fq_run_error_bits")
        return b.value

    def stats(self) -> dict:
        """fq_run_stats: the row of the last completed step as a dict (synchronises)."""
        s = L.FqStats()
        self._chk(self._lib.fq_run_stats(self.r, C.byref(s)), "fq_run_stats")
        return {f: getattr(s, f) for f, _ in L.FqStats._fields_}

    def history(self, cap: int = 1 << 16) -> np.ndarray:
        """fq_run_history: the rows recorded since the last call (STATS_DTYPE array)."""
        out = np.zeros(cap, dtype=STATS_DTYPE)
        n = C.c_size_t()
        self._chk(self._lib.fq_run_history(self.r, _ptr(out), cap, C.byref(n)), "fq_run_history")
        return out[: n.value].copy()

    def export(self):
        """fq_run_export: (keys, amplitudes) of the vector, sorted by address."""
        n = C.c_size_t()
        self._chk(self._lib.fq_run_export(self.r, None, None, 0, C.byref(n)), "fq_run_export")
        cap = n.value
        k = np.zeros(max(cap, 1), dtype=KEY_DTYPE)
        a = np.zeros(max(cap, 1))
        _check(self._lib.fq_run_export(self.r, _ptr(k), _ptr(a), cap, C.byref(n)), "fq_run_export")
        return k[: n.value].copy(), a[: n.value].copy()

    def set_tables(self, slots: int = 0, scratch_slots: int = 0):
        """fq_run_set_tables: override the merge's on-chip and scratch table sizes (0 = default)."""
        _check(self._lib.fq_run_set_tables(self.r, int(slots), int(scratch_slots)),
               "fq_run_set_tables")

    def set_spawn_split(self, primary: int):
        """fq_run_set_spawn_split: spawn slots per bucket in the dense primary region."""
        _check(self._lib.fq_run_set_spawn_split(self.r, int(primary)), "fq_run_set_spawn_split")

    def merge_paths(self):
        """fq_run_merge_paths: (on-chip, scratch) bucket counts since seeding."""
        a, b = C.c_uint64(), C.c_uint64()
        self._chk(self._lib.fq_run_merge_paths(self.r, C.byref(a), C.byref(b)),
                  "fq_run_merge_paths")
        return a.value, b.value

    def lookup(self, keys) -> np.ndarray:
        """Amplitudes of the given addresses (0 when not stored)."""
        k = _as_keys(keys)
        out = np.zeros(max(len(k), 1))
        self._chk(self._lib.fq_run_lookup(self.r, _ptr(k), len(k), _ptr(out)), "fq_run_lookup")
        return out[: len(k)].copy()

    def sample(self, want: int, seed: int = 0):
        """Entries of randomly chosen whole segments, at least `want` of them."""
        cap = int(want) + 4 * 4096
        k = np.zeros(cap, dtype=KEY_DTYPE)
        a = np.zeros(cap)
        n = C.c_size_t()
        self._chk(self._lib.fq_run_sample(self.r, int(seed), int(want), _ptr(k), _ptr(a), cap,
                                          C.byref(n)), "fq_run_sample")
        m = min(n.value, cap)
        return k[:m].copy(), a[:m].copy()

    def spawns(self, cap: int | None = None):
        """fq_run_spawns: (destinations, values) of the next step's spawns; the run does not change."""
        n = C.c_size_t()
        if cap is None:
            cap = 1 << 22
        d = np.zeros(cap, dtype=KEY_DTYPE)
        v = np.zeros(cap)
        self._chk(self._lib.fq_run_spawns(self.r, _ptr(d), _ptr(v), cap, C.byref(n)), "fq_run_spawns")
        if n.value > cap:
            raise FqError(-3, "fq_run_spawns: %d spawns exceed the buffer" % n.value)
        return d[: n.value].copy(), v[: n.value].copy()

    def autotune(self, steps: int = 3):
        """Time the launch shapes on real steps and keep the fastest (the run advances)."""
        _check(self._lib.fq_run_autotune(self.r, int(steps)), "fq_run_autotune")

    def reserve(self, capacity_vec: int, capacity_spawn: int):
        """fq_run_reserve: grow the vector and spawn capacities, keeping the vector."""
        _check(self._lib.fq_run_reserve(self.r, int(capacity_vec), int(capacity_spawn)),
               "fq_run_reserve")

    def capacity(self):
        """fq_run_capacity: (vector entries, spawns per step) the run can hold."""
        v, s = C.c_size_t(), C.c_size_t()
        _check(self._lib.fq_run_capacity(self.r, C.byref(v), C.byref(s)), "fq_run_capacity")
        return v.value, s.value

    def advance(self, n: int, chunk: int = 200, grow: float = 1.5, max_grows: int = 12):
        """Step until n more steps are done.  Every `chunk` steps the run is
        synchronised; after a capacity error (the run is rolled back to its
        last completed step) both capacities grow by `grow` and stepping goes on."""
        target = self.stats()["step"] + int(n)
        grows = 0
        while True:
            done = self.stats()["step"]
            if done >= target:
                return grows
            self.step(min(chunk, target - done))
            rc = self.sync()
            if rc == -3 and grows < max_grows:
                v, s = self.capacity()
                if self._alloc is not None:
                    # hand cached blocks back to the CUDA driver before the copy
                    self._alloc.torch.cuda.empty_cache()
                self.reserve(int(v * grow), int(s * grow))
                grows += 1
            elif rc:
                raise RunError(rc, "advance", self.error_bits())

    def shape(self) -> dict:
        """The launch shape the run steps with (fq_run_shape)."""
        v = (C.c_int * 7)()
        _check(self._lib.fq_run_shape(self.r, v), "fq_run_shape")
        keys = ("spawn_wpb", "spawn_grid", "merge_wpb", "merge_grid", "slots", "scratch_slots",
                "annihilation")
        out = dict(zip(keys, [int(x) for x in v]))
        out["annihilation"] = {ANN_HASH: "hash", ANN_SORT: "sort"}.get(out["annihilation"], "?")
        return out

    def arm_times(self):
        """fq_run_arm_times: the autotuner's best merge ms per arm, {"hash": ..., "sort": ...}."""
        a, b = C.c_float(), C.c_float()
        _check(self._lib.fq_run_arm_times(self.r, C.byref(a), C.byref(b)), "fq_run_arm_times")
        return {"hash": a.value, "sort": b.value}

    def profile(self, n: int):
        """Mean ms per step of (spawn, merge, shift) over n eagerly launched steps."""
        ms = (C.c_float * 3)()
        _check(self._lib.fq_run_profile(self.r, int(n), ms), "fq_run_profile")
        return tuple(float(x) for x in ms)


class Batch:
    """fq_batch_create(runs): the runs step together, one launch per kernel."""

    def __init__(self, runs):
        self._lib = L.load()
        self.runs = list(runs)
        arr = (C.c_void_p * len(self.runs))(*[r.r.value for r in self.runs])
        b = C.c_void_p()
        _check(self._lib.fq_batch_create(C.byref(b), arr, len(self.runs)), "fq_batch_create")
        self.b = b

    def close(self):
        """Release the handle and its device memory (also done on garbage collection)."""
        if getattr(self, "b", None):
            self._lib.fq_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1):
        """Enqueue n steps (asynchronous; errors surface at the next synchronising call)."""
        _check(self._lib.fq_batch_step(self.b, int(n)), "fq_batch_step")

    def sync(self):
        """fq_batch_sync: wait and report the first error of the batch's runs."""
        _check(self._lib.fq_batch_sync(self.b), "fq_batch_sync")

    def autotune(self, steps: int = 3):
        """Time the launch shapes on real steps and keep the fastest (the run advances)."""
        _check(self._lib.fq_batch_autotune(self.b, int(steps)), "fq_batch_autotune")

    def set_overlaps(self, g2_d=()):
        """fq_batch_set_overlaps: record c_A^T c_B and c_A^T G2(d) c_B after every step."""
        d = np.ascontiguousarray(g2_d, dtype=np.int32)
        _check(self._lib.fq_batch_set_overlaps(self.b, _ptr(d), len(d)), "fq_batch_set_overlaps")

    def set_spectral(self, K: int):
        """fq_batch_set_spectral: runs 0..K-1 as spectral states, orthogonalised every step."""
        _check(self._lib.fq_batch_set_spectral(self.b, int(K)), "fq_batch_set_spectral")

    def overlaps(self, cap: int = 1 << 16) -> np.ndarray:
        """fq_batch_overlaps: the rows recorded since the last call, shape (rows, width)."""
        w = C.c_int()
        n = C.c_size_t()
        _check(self._lib.fq_batch_overlaps(self.b, None, 0, C.byref(n), C.byref(w)),
               "fq_batch_overlaps")
        out = np.zeros((cap, w.value))
        _check(self._lib.fq_batch_overlaps(self.b, _ptr(out), cap, C.byref(n), C.byref(w)),
               "fq_batch_overlaps")
        return out[: n.value].copy()
