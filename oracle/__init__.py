"""CPU oracle for the checkerboard Metropolis method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the CUDA library: the two share no code.

The chains themselves are plain C (``spin_oracle.c``, one site at a time, in
the paper's order: Alg. 1 with the checkerboard colours), built here with gcc
on first use.  The fluctuation estimator (``estimator.py``) and the MLP
surrogate reference (``mlp.py``) are plain numpy in float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spin_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


_LIB_SAN = os.path.join(_HERE, "liboracle_san.so")
# AddressSanitizer + UndefinedBehaviorSanitizer build of the same source: any
# out-of-bounds access or undefined operation aborts the process.
_SAN_FLAGS = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
              "-fno-sanitize-recover=all"]


def build(force: bool = False, sanitize: bool = False) -> str:
    """Compile spin_oracle.c into liboracle.so (plain C, -O2, no fast-math),
    or with sanitize=True into liboracle_san.so (ASan + UBSan, for the
    sanitizer tests; loaded instead when SPINMC_ORACLE_SANITIZE=1)."""
    out = _LIB_SAN if sanitize else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        opt = _SAN_FLAGS if sanitize else ["-O2"]
        subprocess.check_call(
            ["gcc", *opt, "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
             "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build(sanitize=os.environ.get("SPINMC_ORACLE_SANITIZE") == "1"))
            _declare(_lib)
    return _lib


_u32p = ctypes.POINTER(ctypes.c_uint32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f = ctypes.c_float
_i = ctypes.c_int
_d = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64


def _declare(L):
    sig = {
        "or_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
        "or_philox_xor": (_u32, [_u64, _u32, _u32, _u32, _u32, _u32]),
        "or_accept_count": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
        "or_accept": (_i, [ctypes.c_double, ctypes.c_double, _u32]),
        "or_init_ising": (None, [_i, _u64, _u32, _i8p]),
        "or_init_potts": (None, [_i, _i, _u64, _u32, _u8p]),
        "or_ising_substep": (None, [_i, _f, _f, _f, _u64, _u32, _u32, _i, _i8p]),
        "or_ising_sweep": (None, [_i, _f, _f, _f, _u64, _u32, _u32, _i8p]),
        "or_ising_stats": (None, [_i, _i8p, _i64p]),
        "or_ising_run": (None, [_i, _f, _f, _f, _u64, _u32, _u32, _i, _i8p, _i64p]),
        "or_potts_substep": (None, [_i, _i, _f, _f, _u64, _u32, _u32, _i, _u8p]),
        "or_potts_sweep": (None, [_i, _i, _f, _f, _u64, _u32, _u32, _u8p]),
        "or_potts_stats": (None, [_i, _i, _u8p, _i64p]),
        "or_potts_run": (None, [_i, _i, _f, _f, _u64, _u32, _u32, _i, _u8p, _i64p]),
        "or_cpm_substep": (None, [_i, _i, _i32p, _i, _i, _i, _u8p, _f, _u64, _u32, _u32, _i,
                                  _i32p, _i32p]),
        "or_cpm_sweep": (None, [_i, _i, _i32p, _i, _i, _i, _u8p, _f, _u64, _u32, _u32,
                                _i32p, _i32p]),
        "or_cpm_stats": (None, [_i, _i, _i, _i, _u8p, _i32p, _i32p, _i64p]),
        "or_cpm_init": (_i, [_i, _i, _i, _i, _u64, _u32, _i32p, _u8p, _i32p]),
        "or_cpm_run": (None, [_i, _i, _i32p, _i, _i, _i, _u8p, _f, _u64, _u32, _u32, _i,
                              _i32p, _i32p, _i64p]),
        "or_cpm_energy": (ctypes.c_int64, [_i, _i, _i32p, _i, _i, _i, _u8p, _i32p]),
        "or_tri_substep": (None, [_i, _f, _f, _f, _u64, _u32, _u32, _i, _i8p]),
        "or_tri_sweep": (None, [_i, _f, _f, _f, _u64, _u32, _u32, _i8p]),
        "or_tri_stats": (None, [_i, _i8p, _i64p]),
        "or_tri_run": (None, [_i, _f, _f, _f, _u64, _u32, _u32, _i, _i8p, _i64p]),
        "or_nnn_substep": (None, [_i, _f, _f, _f, _f, _u64, _u32, _u32, _i, _i8p]),
        "or_nnn_sweep": (None, [_i, _f, _f, _f, _f, _u64, _u32, _u32, _i8p]),
        "or_nnn_stats": (None, [_i, _i8p, _i64p]),
        "or_nnn_run": (None, [_i, _f, _f, _f, _f, _u64, _u32, _u32, _i, _i8p, _i64p]),
        "or_dmc_substep": (None, [_i, _dp, _dp, _d, _d, _d, _u64, _u32, _u32, _i, _dp]),
        "or_dmc_run": (None, [_i, _dp, _dp, _d, _d, _d, _u64, _u32, _u32, _i, _dp, _dp]),
        "or_dmc_backward": (None, [_i, _dp, _dp, _d, _d, _d, _u64, _u32, _u32, _i, _dp, _dp, _dp, _dp]),
        "or_dmc_loss": (_d, [_i, _dp, _dp, _dp]),
        "or_dmc_discretize": (None, [_i, _dp]),
        "or_dmc_energy": (_d, [_i, _dp, _dp, _d, _dp, _dp]),
        "or_dmc_spin_step": (None, [_i, _dp, _dp, _d]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _p(a, ct):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ct))


# --------------------------------------------------------------------------
# Philox and acceptance
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                           _p(out, ctypes.c_uint32))
    return out


def philox_xor(seed, lattice, sweep, colour, g0, n):
    """XOR of every word of the Philox blocks for counters (g, lattice, sweep,
    colour), g in [g0, g0 + n), under the seed's key."""
    return int(lib().or_philox_xor(seed, lattice, sweep, colour, g0, n))


def accept_count(beta: float, dE: float) -> float:
    """How many of the 2^32 values of a uniform uint32 draw accept the move."""
    return lib().or_accept_count(float(beta), float(dE))


# --------------------------------------------------------------------------
# Ising
# --------------------------------------------------------------------------
def init_ising(L: int, seed: int, lattice: int = 0) -> np.ndarray:
    s = np.zeros(L * L, dtype=np.int8)
    lib().or_init_ising(L, seed, lattice, _p(s, ctypes.c_int8))
    return s.reshape(L, L)


def ising_sweep(s: np.ndarray, beta, J, h, seed, lattice, sweep):
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    lib().or_ising_sweep(s.shape[0], beta, J, h, seed, lattice, sweep, _p(s, ctypes.c_int8))


def ising_substep(s, beta, J, h, seed, lattice, sweep, colour):
    lib().or_ising_substep(s.shape[0], beta, J, h, seed, lattice, sweep, colour,
                           _p(s, ctypes.c_int8))


def ising_stats(s: np.ndarray) -> np.ndarray:
    out = np.zeros(2, dtype=np.int64)
    lib().or_ising_stats(s.shape[0], _p(np.ascontiguousarray(s), ctypes.c_int8),
                         _p(out, ctypes.c_int64))
    return out


def ising_run(s, beta, J, h, seed, lattice, sweep0, nsweeps, record=True):
    """Run nsweeps in place; return stats [nsweeps, 2] = (M, B) after each sweep."""
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    st = np.zeros((nsweeps, 2), dtype=np.int64) if record else None
    lib().or_ising_run(s.shape[0], beta, J, h, seed, lattice, sweep0, nsweeps,
                       _p(s, ctypes.c_int8), _p(st, ctypes.c_int64) if record else None)
    return st


# --------------------------------------------------------------------------
# Potts
# --------------------------------------------------------------------------
def tri_substep(s, beta, J, h, seed, lattice, sweep, colour):
    """Triangular-lattice Ising colour sub-step in place (s int8 [L, L], L % 3 == 0)."""
    lib().or_tri_substep(s.shape[0], beta, J, h, seed, lattice, sweep, colour, _p(s, ctypes.c_int8))


def tri_sweep(s, beta, J, h, seed, lattice, sweep):
    lib().or_tri_sweep(s.shape[0], beta, J, h, seed, lattice, sweep, _p(s, ctypes.c_int8))


def tri_stats(s):
    out = np.zeros(2, dtype=np.int64)
    lib().or_tri_stats(s.shape[0], _p(np.ascontiguousarray(s), ctypes.c_int8), _p(out, ctypes.c_int64))
    return out


def tri_run(s, beta, J, h, seed, lattice, sweep0, nsweeps, record=True):
    """Run nsweeps in place; stats [nsweeps, 2] = (M, B) after each sweep."""
    st = np.zeros((nsweeps, 2), dtype=np.int64) if record else None
    lib().or_tri_run(s.shape[0], beta, J, h, seed, lattice, sweep0, nsweeps, _p(s, ctypes.c_int8),
                     _p(st, ctypes.c_int64) if record else None)
    return st


def nnn_substep(s, beta, J, J2, h, seed, lattice, sweep, colour):
    """First-and-second-neighbour Ising colour sub-step in place (s int8 [L, L], L even)."""
    lib().or_nnn_substep(s.shape[0], beta, J, J2, h, seed, lattice, sweep, colour, _p(s, ctypes.c_int8))


def nnn_sweep(s, beta, J, J2, h, seed, lattice, sweep):
    lib().or_nnn_sweep(s.shape[0], beta, J, J2, h, seed, lattice, sweep, _p(s, ctypes.c_int8))


def nnn_stats(s):
    """(M, B, B2): magnetisation, nearest- and diagonal-bond sums."""
    out = np.zeros(3, dtype=np.int64)
    lib().or_nnn_stats(s.shape[0], _p(np.ascontiguousarray(s), ctypes.c_int8), _p(out, ctypes.c_int64))
    return out


def nnn_run(s, beta, J, J2, h, seed, lattice, sweep0, nsweeps, record=True):
    """Run nsweeps in place; stats [nsweeps, 3] = (M, B, B2) after each sweep."""
    st = np.zeros((nsweeps, 3), dtype=np.int64) if record else None
    lib().or_nnn_run(s.shape[0], beta, J, J2, h, seed, lattice, sweep0, nsweeps, _p(s, ctypes.c_int8),
                     _p(st, ctypes.c_int64) if record else None)
    return st


def init_potts(L, q, seed, lattice=0):
    s = np.zeros(L * L, dtype=np.uint8)
    lib().or_init_potts(L, q, seed, lattice, _p(s, ctypes.c_uint8))
    return s.reshape(L, L)


def potts_sweep(s, q, beta, J, seed, lattice, sweep):
    lib().or_potts_sweep(s.shape[0], q, beta, J, seed, lattice, sweep, _p(s, ctypes.c_uint8))


def potts_substep(s, q, beta, J, seed, lattice, sweep, colour):
    lib().or_potts_substep(s.shape[0], q, beta, J, seed, lattice, sweep, colour,
                           _p(s, ctypes.c_uint8))


def potts_stats(s, q):
    out = np.zeros(q + 1, dtype=np.int64)
    lib().or_potts_stats(s.shape[0], q, _p(np.ascontiguousarray(s), ctypes.c_uint8),
                         _p(out, ctypes.c_int64))
    return out


def potts_run(s, q, beta, J, seed, lattice, sweep0, nsweeps, record=True):
    """Run nsweeps in place; stats [nsweeps, q+1] = (B_eq, n_0..n_{q-1})."""
    st = np.zeros((nsweeps, q + 1), dtype=np.int64) if record else None
    lib().or_potts_run(s.shape[0], q, beta, J, seed, lattice, sweep0, nsweeps,
                       _p(s, ctypes.c_uint8), _p(st, ctypes.c_int64) if record else None)
    return st


# --------------------------------------------------------------------------
# Cellular Potts
# --------------------------------------------------------------------------
class CPM:
    """Parameters of one cellular Potts lattice (Eq. "h" of the paper)."""

    def __init__(self, L, J, lam, target, n_cells, T, side, cols):
        self.L = int(L)
        self.J = np.ascontiguousarray(np.asarray(J, dtype=np.int32))
        self.n_types = self.J.shape[0]
        self.lam = int(lam)
        self.target = int(target)
        self.n_cells = int(n_cells)
        self.T = float(T)
        self.side = int(side)
        self.cols = int(cols)

    @property
    def n_stats(self):
        return self.n_types * (self.n_types + 1) // 2 + 2

    def init(self, seed, lattice=0):
        ids = np.zeros(self.L * self.L, dtype=np.int32)
        types = np.zeros(self.n_cells + 1, dtype=np.uint8)
        vol = np.zeros(self.n_cells + 1, dtype=np.int32)
        rc = lib().or_cpm_init(self.L, self.n_cells, self.side, self.cols, seed, lattice,
                               _p(ids, ctypes.c_int32), _p(types, ctypes.c_uint8),
                               _p(vol, ctypes.c_int32))
        if rc != 0:
            raise ValueError("initial cell block does not fit the lattice")
        return ids.reshape(self.L, self.L), types, vol

    def _args(self, types):
        return (self.L, self.n_types, _p(self.J, ctypes.c_int32), self.lam, self.target,
                self.n_cells, _p(types, ctypes.c_uint8), self.T)

    def substep(self, ids, vol, types, seed, lattice, sweep, colour):
        lib().or_cpm_substep(*self._args(types), seed, lattice, sweep, colour,
                             _p(ids, ctypes.c_int32), _p(vol, ctypes.c_int32))

    def sweep(self, ids, vol, types, seed, lattice, sweep):
        lib().or_cpm_sweep(*self._args(types), seed, lattice, sweep,
                           _p(ids, ctypes.c_int32), _p(vol, ctypes.c_int32))

    def run(self, ids, vol, types, seed, lattice, sweep0, nsweeps, record=True):
        st = np.zeros((nsweeps, self.n_stats), dtype=np.int64) if record else None
        lib().or_cpm_run(*self._args(types), seed, lattice, sweep0, nsweeps,
                         _p(ids, ctypes.c_int32), _p(vol, ctypes.c_int32),
                         _p(st, ctypes.c_int64) if record else None)
        return st

    def stats(self, ids, vol, types):
        out = np.zeros(self.n_stats, dtype=np.int64)
        lib().or_cpm_stats(self.L, self.n_types, self.target, self.n_cells,
                           _p(types, ctypes.c_uint8), _p(np.ascontiguousarray(ids), ctypes.c_int32),
                           _p(vol, ctypes.c_int32), _p(out, ctypes.c_int64))
        return out

    def energy(self, ids, types):
        return int(lib().or_cpm_energy(*self._args(types)[:7],
                                       _p(np.ascontiguousarray(ids), ctypes.c_int32)))
