"""Python binding of libspinmc.so (include/spinmc.h): argument marshalling only.

Every Monte Carlo step, reduction and gradient runs in the library's CUDA
kernels; this module turns torch tensors and Python numbers into pointers and
sizes, checks return codes, and raises on any error.  There is no CPU path:
if the library cannot be loaded, every call raises.

Names follow the C ABI: ``spin_init`` .. ``spin_mlp_adam`` are exposed as the
raw ctypes functions on ``lib()``; :class:`Sim` wraps one context.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SPINMC_LIBRARY: path of a test build to load instead (libspinmc_check.so,
# libspinmc_san.so: see build.py); the default is the in-tree libspinmc.so.
_LIB_PATH = os.environ.get("SPINMC_LIBRARY") or os.path.join(_HERE, "libspinmc.so")
_lib = None
_lock = threading.Lock()

SPIN_ISING, SPIN_POTTS, SPIN_CPM = 0, 1, 2
ERRORS = {-1: "SPIN_EINVAL", -2: "SPIN_ENOMEM", -3: "SPIN_ECUDA", -4: "SPIN_ETIMEOUT", -5: "SPIN_ESTATE"}


class SpinError(RuntimeError):
    pass


class LatticeDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("q", ctypes.c_int32), ("beta", ctypes.c_float),
                ("J", ctypes.c_float), ("h", ctypes.c_float), ("geometry", ctypes.c_int32),
                ("J2", ctypes.c_float), ("lattice_id", ctypes.c_uint32), ("spin_offset", ctypes.c_uint64)]


class CpmParams(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int32), ("lambda_", ctypes.c_int32),
                ("target_area", ctypes.c_int32), ("n_cells", ctypes.c_int32),
                ("J_type", ctypes.POINTER(ctypes.c_int32)), ("cell_type", ctypes.POINTER(ctypes.c_uint8)),
                ("T", ctypes.c_float), ("init_side", ctypes.c_int32), ("init_cols", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_SIGS = {
    "spin_init": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.c_uint64, _i32, ctypes.POINTER(LatticeDesc),
                         ctypes.POINTER(CpmParams), _vp, _i32, _i32, _vp]),
    "spin_sweep": (_i32, [_vp, _i32, _i32, _vp]),
    "spin_stats_width": (_i32, [_vp]),
    "spin_num_records": (_i64, [_vp]),
    "spin_observables": (_i32, [_vp, _i64, _i32, _vp, _vp, _vp, _vp]),
    "spin_current_stats": (_i32, [_vp, _vp, _vp]),
    "spin_moments": (_i32, [_vp, _i64, _i32, _vp, _vp]),
    "spin_num_moments": (_i32, [_vp]),
    "spin_grad": (_i32, [_vp, _i64, _i32, _i32, _i32, _vp, _vp]),
    "spin_num_grad": (_i32, [_vp]),
    "spin_expectations": (_i32, [_vp, _i64, _i32, _i32, _vp, _vp]),
    "spin_set_params": (_i32, [_vp, ctypes.POINTER(LatticeDesc), ctypes.POINTER(CpmParams)]),
    "spin_set_launch": (_i32, [_vp, _i32, _i32, _i32, _i32]),
    "spin_autotune": (_i32, [_vp, _i32, _vp]),
    "spin_get_launch": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "spin_load_spins": (_i32, [_vp, _vp, _vp]),
    "spin_store_spins": (_i32, [_vp, _vp, _vp]),
    "spin_checkpoint": (_i32, [_vp, _vp, ctypes.POINTER(ctypes.c_size_t), _vp]),
    "spin_restore": (_i32, [_vp, _vp, ctypes.c_size_t, _vp]),
    "spin_profile": (_i32, [_vp, _i32, _i32]),
    "spin_profile_read": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _vp]),
    "spin_barrier_selftest": (_i32, [_i32, _i32, _i32, _vp]),
    "spin_packed_words": (_i32, [_vp]),
    "spin_load_spins_packed": (_i32, [_vp, _vp, _vp]),
    "spin_store_spins_packed": (_i32, [_vp, _vp, _vp]),
    "spin_sweep_packed": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp]),
    "spin_sweep_index": (ctypes.c_uint32, [_vp]),
    "spin_gpu_launches": (_i32, [_vp]),
    "spin_last_error": (ctypes.c_char_p, [_vp]),
    "spin_destroy": (None, [_vp]),
    "spin_version": (_i32, []),
    "spin_check_status": (_i32, [ctypes.POINTER(ctypes.c_uint32)]),
    "spin_philox_xor": (_i32, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                               ctypes.c_uint32, _vp, _vp]),
    "spin_ising_sweep_noalloc": (_i32, [ctypes.c_uint64, _i32, ctypes.POINTER(LatticeDesc), _vp, ctypes.c_uint32,
                                        _i32, _vp, _vp]),
    "spin_adam": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                         ctypes.c_float, _vp]),
    "spin_dmc_tape_floats": (ctypes.c_int64, [_i32, _i32, _i32]),
    "spin_dmc_forward": (_i32, [ctypes.c_uint64, _i32, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                _vp, _vp, ctypes.c_uint32, _i32, _vp, _vp]),
    "spin_dmc_backward": (_i32, [ctypes.c_uint64, _i32, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 _vp, _vp, _vp, ctypes.c_uint32, _i32, _vp, _vp, _vp]),
    "spin_dmc_loss": (_i32, [_i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    "spin_dmc_discretize": (_i32, [ctypes.c_int64, _vp, _vp]),
    "spin_dmc_step_max_sweeps": (_i32, [_i32]),
    "spin_dmc_spin_iter": (_i32, [ctypes.c_uint64, _i32, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_uint32, _i32, _vp, _vp, _vp, _vp]),
    "spin_dmc_spin_iter_max_sweeps": (_i32, [_i32]),
    "spin_dmc_energy": (_i32, [_i32, _i32, ctypes.c_float, _vp, _vp, _vp, _vp, _vp]),
    "spin_dmc_spin_step": (_i32, [ctypes.c_int64, _vp, _vp, ctypes.c_float, _vp]),
    "spin_dmc_step": (_i32, [ctypes.c_uint64, _i32, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_uint32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp]),
    "spin_cpm_batch_workspace_bytes": (ctypes.c_int64, [ctypes.POINTER(CpmParams)]),
    "spin_cpm_batch_init": (_i32, [ctypes.c_uint64, _i32, _i32, ctypes.POINTER(CpmParams), _vp, _vp, _vp, _vp]),
    "spin_cpm_batch_run": (_i32, [ctypes.c_uint64, _i32, _i32, ctypes.POINTER(CpmParams), _vp, _vp, _vp,
                                  ctypes.c_uint32, _i32, _vp, _vp, _vp]),
    "spin_pooled_limbs": (_i32, [_vp, ctypes.c_int64, _i32, _vp, _vp]),
    "spin_grad_from_limbs": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp]),
    "spin_mlp_param_count": (_i32, []),
    "spin_mlp_forward": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "spin_mlp_backward": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "spin_mlp_adam": (_i32, [_vp, _vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, _vp]),
}


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libspinmc.so (building it in-tree first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                if os.environ.get("SPINMC_LIBRARY"):
                    raise OSError(f"SPINMC_LIBRARY names a missing library: {_LIB_PATH}")
                from . import build as _build
                _build.build()
            L = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(t):
    """Device (torch) or host (numpy / torch CPU) buffer -> void*."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc, ctx=None, what=""):
    if rc < 0:
        msg = lib().spin_last_error(ctx).decode() if ctx else ""
        raise SpinError(f"{what}: {ERRORS.get(rc, rc)} {msg}")
    return rc


def pack_offsets(sizes, elem=1, align=256):
    """Element offsets of lattices of side L packed into one buffer, each
    starting on an `align`-byte boundary; returns (offsets, total elements)."""
    off, cur = [], 0
    step = max(1, align // elem)
    for L in sizes:
        cur = (cur + step - 1) // step * step
        off.append(cur)
        cur += L * L
    return off, cur


class Sim:
    """One context: a batch of lattices of one model on the current CUDA device.

    lattices: list of dicts with L, beta, J, h (Ising), q (Potts).
    spins: optional caller tensor (int8 / uint8 / int32, CUDA) holding every
    lattice at its offset; allocated here when omitted.
    """

    def __init__(self, model, lattices, seed=0, spins=None, offsets=None, init_mode=None,
                 max_record=0, cpm=None, stream=None):
        import torch
        self.model = model
        self.n = len(lattices)
        elem = 4 if model == SPIN_CPM else 1
        if offsets is None:
            offsets, total = pack_offsets([d["L"] for d in lattices], elem)
        else:
            total = max(o + d["L"] ** 2 for o, d in zip(offsets, lattices))
        self.offsets = list(offsets)
        self.sizes = [int(d["L"]) for d in lattices]
        dtype = {SPIN_ISING: torch.int8, SPIN_POTTS: torch.uint8, SPIN_CPM: torch.int32}[model]
        if spins is None:
            spins = torch.zeros(total, dtype=dtype, device="cuda")
        assert spins.is_cuda and spins.dtype == dtype and spins.numel() >= total
        self.spins = spins
        arr = (LatticeDesc * self.n)()
        for i, d in enumerate(lattices):
            arr[i] = LatticeDesc(int(d["L"]), int(d.get("q", 2)), float(d.get("beta", 0.0)),
                                 float(d.get("J", 1.0)), float(d.get("h", 0.0)), int(d.get("geometry", 0)),
                                 float(d.get("J2", 0.0)), int(d.get("lattice_id", 0)), int(offsets[i]))
        self._desc = arr
        self.lattices = [dict(d) for d in lattices]
        cp = None
        if model == SPIN_CPM:
            cp = self._cpm_struct(cpm)
            if init_mode is None:
                init_mode = 2
        elif init_mode is None:
            init_mode = 0
        ctx = ctypes.c_void_p()
        rc = lib().spin_init(ctypes.byref(ctx), model, ctypes.c_uint64(seed), self.n, arr,
                             ctypes.byref(cp) if cp is not None else None, _ptr(spins),
                             init_mode, int(max_record), _stream(stream))
        if rc < 0:
            raise SpinError(f"spin_init: {ERRORS.get(rc, rc)}")
        self.ctx = ctx
        self.width = lib().spin_stats_width(ctx)

    def _cpm_struct(self, cpm):
        J = np.ascontiguousarray(np.asarray(cpm["J"], dtype=np.int32))
        self._cpm_J = J
        ct = cpm.get("cell_type")
        self._cpm_types = None if ct is None else np.ascontiguousarray(np.asarray(ct, dtype=np.uint8))
        return CpmParams(J.shape[0], int(cpm["lambda"]), int(cpm["target"]), int(cpm["n_cells"]),
                         J.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         None if self._cpm_types is None else
                         self._cpm_types.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                         float(cpm["T"]), int(cpm.get("side", 0)), int(cpm.get("cols", 0)), 0)

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            lib().spin_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- sweeping ----------------------------------------------------------
    def sweep(self, n=1, record=False, stream=None):
        _check(lib().spin_sweep(self.ctx, int(n), 1 if record else 0, _stream(stream)), self.ctx, "spin_sweep")

    @property
    def t(self):
        return int(lib().spin_sweep_index(self.ctx))

    @property
    def n_records(self):
        return int(lib().spin_num_records(self.ctx))

    @property
    def gpu_launches(self):
        return int(lib().spin_gpu_launches(self.ctx))

    def lattice(self, i):
        """View of lattice i in the caller's buffer, shape [L, L]."""
        L = self.sizes[i]
        return self.spins[self.offsets[i]:self.offsets[i] + L * L].view(L, L)

    # -- observables -------------------------------------------------------
    def observables(self, first=0, n=None, stream=None):
        """(stats [n, n_lat, width] int64, E [n, n_lat] f32, M [n, n_lat] f32), on the device."""
        import torch
        if n is None:
            n = self.n_records - first
        st = torch.empty((n, self.n, self.width), dtype=torch.int64, device="cuda")
        E = torch.empty((n, self.n), dtype=torch.float32, device="cuda")
        M = torch.empty((n, self.n), dtype=torch.float32, device="cuda")
        _check(lib().spin_observables(self.ctx, int(first), int(n), _ptr(st), _ptr(E), _ptr(M),
                                      _stream(stream)), self.ctx, "spin_observables")
        return st, E, M

    def observables_host(self, first=0, n=None, stream=None):
        """The same, written straight into host (numpy) buffers."""
        if n is None:
            n = self.n_records - first
        st = np.empty((n, self.n, self.width), dtype=np.int64)
        E = np.empty((n, self.n), dtype=np.float32)
        M = np.empty((n, self.n), dtype=np.float32)
        _check(lib().spin_observables(self.ctx, int(first), int(n), _ptr(st), _ptr(E), _ptr(M),
                                      _stream(stream)), self.ctx, "spin_observables")
        return st, E, M

    def current_stats(self, stream=None):
        import torch
        out = torch.empty((self.n, self.width), dtype=torch.int64, device="cuda")
        _check(lib().spin_current_stats(self.ctx, _ptr(out), _stream(stream)), self.ctx, "spin_current_stats")
        return out

    def moments(self, first=0, n=None, stream=None):
        import torch
        if n is None:
            n = self.n_records - first
        nm = lib().spin_num_moments(self.ctx)
        out = torch.empty((self.n, nm), dtype=torch.int64, device="cuda")
        _check(lib().spin_moments(self.ctx, int(first), int(n), _ptr(out), _stream(stream)), self.ctx,
               "spin_moments")
        return out

    def grad(self, first=0, n=None, observable=0, pool=False, stream=None):
        import torch
        if n is None:
            n = self.n_records - first
        ng = lib().spin_num_grad(self.ctx)
        rows = 1 if pool else self.n
        out = torch.empty((rows, ng), dtype=torch.float64, device="cuda")
        _check(lib().spin_grad(self.ctx, int(first), int(n), int(observable), 1 if pool else 0, _ptr(out),
                               _stream(stream)), self.ctx, "spin_grad")
        return out

    def pooled_limbs(self, first=0, n=None, stream=None):
        """[n_mom, 4] int64 device tensor: this context's pooled moments as limbs
        whose element-wise sum over processes is exact (see spin_pooled_limbs)."""
        import torch
        if n is None:
            n = self.n_records - first
        out = torch.empty((lib().spin_num_moments(self.ctx), 4), dtype=torch.int64, device="cuda")
        _check(lib().spin_pooled_limbs(self.ctx, int(first), int(n), _ptr(out), _stream(stream)), self.ctx,
               "spin_pooled_limbs")
        return out

    def grad_from_limbs(self, limbs, observable=0, stream=None):
        """(pooled gradient [1, n_grad], pooled expectations [1, 2]) from summed limbs."""
        import torch
        g = torch.empty((1, lib().spin_num_grad(self.ctx)), dtype=torch.float64, device="cuda")
        e = torch.empty((1, 2), dtype=torch.float64, device="cuda")
        _check(lib().spin_grad_from_limbs(self.ctx, _ptr(limbs.contiguous()), int(observable), _ptr(g), _ptr(e),
                                          _stream(stream)), self.ctx, "spin_grad_from_limbs")
        return g, e

    def expectations(self, first=0, n=None, pool=False, stream=None):
        """[rows, 2] float64 on the device: (<E>/N, <M>/N) per lattice or pooled."""
        import torch
        if n is None:
            n = self.n_records - first
        out = torch.empty((1 if pool else self.n, 2), dtype=torch.float64, device="cuda")
        _check(lib().spin_expectations(self.ctx, int(first), int(n), 1 if pool else 0, _ptr(out),
                                       _stream(stream)), self.ctx, "spin_expectations")
        return out

    # -- parameters / launch form -----------------------------------------
    def set_params(self, lattices=None, cpm=None):
        arr = None
        if lattices is not None:
            arr = (LatticeDesc * self.n)()
            for i, d in enumerate(lattices):
                arr[i] = LatticeDesc(int(d["L"]), int(d.get("q", 2)), float(d.get("beta", 0.0)),
                                     float(d.get("J", 1.0)), float(d.get("h", 0.0)), int(d.get("geometry", 0)),
                                     float(d.get("J2", 0.0)), int(d.get("lattice_id", 0)), int(self.offsets[i]))
            self._desc = arr
            self.lattices = [dict(d) for d in lattices]
        cp = self._cpm_struct(cpm) if cpm is not None else None
        _check(lib().spin_set_params(self.ctx, arr, ctypes.byref(cp) if cp is not None else None), self.ctx,
               "spin_set_params")

    def set_launch(self, mode=0, use_graph=True, tile_rows=0, threads=0):
        _check(lib().spin_set_launch(self.ctx, int(mode), 1 if use_graph else 0, int(tile_rows), int(threads)),
               self.ctx, "spin_set_launch")

    def get_launch(self):
        out = (ctypes.c_int32 * 4)()
        _check(lib().spin_get_launch(self.ctx, out), self.ctx, "spin_get_launch")
        return {"mode": out[0], "use_graph": out[1], "tile_rows": out[2], "threads": out[3]}

    def autotune(self, sweeps_per_trial=4, stream=None):
        _check(lib().spin_autotune(self.ctx, int(sweeps_per_trial), _stream(stream)), self.ctx, "spin_autotune")
        return self.get_launch()

    # -- kernel timing -----------------------------------------------------
    def profile(self, enable=True, max_launches=4096):
        _check(lib().spin_profile(self.ctx, 1 if enable else 0, int(max_launches)), self.ctx, "spin_profile")

    def profile_read(self, stream=None):
        """[(ms, launches)] for kernel classes 0 (tile), 1 (row strip), 2 (plain)."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        _check(lib().spin_profile_read(self.ctx, ms, n, _stream(stream)), self.ctx, "spin_profile_read")
        return [(ms[i], n[i]) for i in range(3)]

    # -- host transfers / checkpoint ---------------------------------------
    def load_spins(self, host, stream=None):
        _check(lib().spin_load_spins(self.ctx, _ptr(host), _stream(stream)), self.ctx, "spin_load_spins")

    def store_spins(self, host, stream=None):
        _check(lib().spin_store_spins(self.ctx, _ptr(host), _stream(stream)), self.ctx, "spin_store_spins")

    @property
    def packed_words(self):
        """Words of the bit-packed host buffer (Ising contexts)."""
        return int(lib().spin_packed_words(self.ctx))

    def load_spins_packed(self, host, stream=None):
        """Load from one bit per spin (bit e = element e is -1; uint32 / int32 words)."""
        _check(lib().spin_load_spins_packed(self.ctx, _ptr(host), _stream(stream)), self.ctx, "spin_load_spins_packed")

    def store_spins_packed(self, host, stream=None):
        _check(lib().spin_store_spins_packed(self.ctx, _ptr(host), _stream(stream)), self.ctx,
               "spin_store_spins_packed")

    def sweep_packed(self, host_in, host_out, n=1, record=False, stream=None):
        """load_spins_packed(host_in) + sweep(n, record) + store_spins_packed(host_out)
        in one call (either buffer may be None)."""
        _check(lib().spin_sweep_packed(self.ctx, None if host_in is None else _ptr(host_in),
                                       None if host_out is None else _ptr(host_out), int(n),
                                       1 if record else 0, _stream(stream)), self.ctx, "spin_sweep_packed")

    def checkpoint(self, stream=None):
        size = ctypes.c_size_t(0)
        _check(lib().spin_checkpoint(self.ctx, None, ctypes.byref(size), _stream(stream)), self.ctx, "ckpt")
        buf = np.zeros(size.value, dtype=np.uint8)
        _check(lib().spin_checkpoint(self.ctx, _ptr(buf), ctypes.byref(size), _stream(stream)), self.ctx, "ckpt")
        return buf

    def restore(self, blob, stream=None):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().spin_restore(self.ctx, _ptr(blob), blob.size, _stream(stream)), self.ctx, "restore")


def barrier_selftest(blocks, missing=0, rounds=1, stream=None):
    """Run the bounded grid barrier of the CPM persistent form as a self-test;
    returns SPIN_OK (0) or SPIN_ETIMEOUT (-4) (see spin_barrier_selftest)."""
    return int(lib().spin_barrier_selftest(int(blocks), int(missing), int(rounds), _stream(stream)))


def check_status():
    """(built_with_checks, first recorded check code or 0); see spin_check_status."""
    code = ctypes.c_uint32(0)
    rc = lib().spin_check_status(ctypes.byref(code))
    _check(rc, None, "spin_check_status")
    return bool(rc == 1), int(code.value)


def philox_xor(seed, lattice, sweep, colour, g0, n_groups, out=None, stream=None):
    """XOR digest of the Philox blocks (g, lattice, sweep, colour), g in
    [g0, g0 + n_groups), computed on the device (see spin_philox_xor).
    Returns the one-element uint32-in-int32 device tensor it wrote."""
    import torch
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device="cuda")
    _check(lib().spin_philox_xor(int(seed), int(lattice), int(sweep), int(colour), int(g0), int(n_groups),
                                 _ptr(out), _stream(stream)), None, "spin_philox_xor")
    return out


# --------------------------------------------------------------------------
# BF16 MLP surrogate
# --------------------------------------------------------------------------
def mlp_param_count():
    return int(lib().spin_mlp_param_count())


def mlp_forward(params, mu, inv_sigma, X, stream=None):
    import torch
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
    _check(lib().spin_mlp_forward(_ptr(params), _ptr(mu), _ptr(inv_sigma), _ptr(X), X.shape[0], _ptr(Y),
                                  _stream(stream)), None, "spin_mlp_forward")
    return Y


def mlp_backward(params, mu, inv_sigma, X, T, want_dx=False, stream=None):
    import torch
    grad = torch.empty(mlp_param_count(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dX = torch.empty_like(X) if want_dx else None
    _check(lib().spin_mlp_backward(_ptr(params), _ptr(mu), _ptr(inv_sigma), _ptr(X), _ptr(T), X.shape[0],
                                   _ptr(grad), _ptr(loss), _ptr(dX), _stream(stream)), None, "spin_mlp_backward")
    return grad, loss, dX


def adam(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    """Adam update of a float32 device tensor in place (library kernel)."""
    _check(lib().spin_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(step), float(lr),
                           float(b1), float(b2), float(eps), _stream(stream)), None, "spin_adam")


def mlp_adam(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _check(lib().spin_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), float(b1),
                               float(b2), float(eps), _stream(stream)), None, "spin_mlp_adam")


# --------------------------------------------------------------------------
# differentiable Monte Carlo (Alg. 2): argument marshalling only
# --------------------------------------------------------------------------
def dmc_tape_floats(n_lattices, L, n_sweeps):
    n = int(lib().spin_dmc_tape_floats(int(n_lattices), int(L), int(n_sweeps)))
    if n < 0:
        raise ValueError(f"spin_dmc_tape_floats: invalid geometry (L={L}, n_sweeps={n_sweeps})")
    return n


def dmc_forward(seed, J, spins, beta, h, alpha, first_sweep, n_sweeps, tape, stream=None):
    """Relaxed sweeps in place on spins [B, L, L] (float32, device) with
    couplings J [B, 2, L, L]; tape receives the active sites' old values."""
    B, L = spins.shape[0], spins.shape[-1]
    _check(lib().spin_dmc_forward(int(seed), B, L, float(beta), float(h), float(alpha), _ptr(J), _ptr(spins),
                                  int(first_sweep), int(n_sweeps), _ptr(tape), _stream(stream)),
           None, "spin_dmc_forward")


def dmc_backward(seed, J, spins, tape, beta, h, alpha, first_sweep, n_sweeps, grad_spins, grad_J, stream=None):
    """Reverse pass: grad_spins (in: dL/ds after, out: dL/ds before), grad_J out."""
    B, L = spins.shape[0], spins.shape[-1]
    _check(lib().spin_dmc_backward(int(seed), B, L, float(beta), float(h), float(alpha), _ptr(J), _ptr(spins),
                                   _ptr(tape), int(first_sweep), int(n_sweeps), _ptr(grad_spins), _ptr(grad_J),
                                   _stream(stream)), None, "spin_dmc_backward")


def dmc_loss(spins, target, grad_spins, loss, stream=None):
    B, L = spins.shape[0], spins.shape[-1]
    _check(lib().spin_dmc_loss(B, L, _ptr(spins), _ptr(target), _ptr(grad_spins), _ptr(loss), _stream(stream)),
           None, "spin_dmc_loss")


def dmc_discretize(spins, stream=None):
    _check(lib().spin_dmc_discretize(spins.numel(), _ptr(spins), _stream(stream)), None, "spin_dmc_discretize")


def dmc_step_max_sweeps(L):
    return int(lib().spin_dmc_step_max_sweeps(int(L)))


def dmc_step(seed, J, spins, m, v, target, loss, beta, h, alpha, first_sweep, n_sweeps, step, lr,
             b1=0.9, b2=0.999, eps=1e-8, stream=None):
    """One fused optimisation iteration (forward, loss, reverse pass, Adam on J,
    discretisation) in a single launch."""
    B, L = spins.shape[0], spins.shape[-1]
    _check(lib().spin_dmc_step(int(seed), B, L, float(beta), float(h), float(alpha), int(first_sweep),
                               int(n_sweeps), _ptr(spins), _ptr(J), _ptr(m), _ptr(v), _ptr(target), _ptr(loss),
                               int(step), float(lr), float(b1), float(b2), float(eps), _stream(stream)),
           None, "spin_dmc_step")


def dmc_energy(J, spins, h, energy, grad_spins=None, stream=None):
    B, L = spins.shape[0], spins.shape[-1]
    _check(lib().spin_dmc_energy(B, L, float(h), _ptr(J), _ptr(spins), _ptr(grad_spins), _ptr(energy),
                                 _stream(stream)), None, "spin_dmc_energy")


def dmc_spin_step(spins, grad, eta, stream=None):
    _check(lib().spin_dmc_spin_step(spins.numel(), _ptr(spins), _ptr(grad), float(eta), _stream(stream)),
           None, "spin_dmc_spin_step")


# --------------------------------------------------------------------------
# batched cellular Potts: argument marshalling only
# --------------------------------------------------------------------------
class CPMBatch:
    """n_lattices independent cellular Potts lattices of side L sharing the
    parameters `cpm` (dict: J, lambda, target, n_cells, T, side, cols and
    optionally cell_type).  Holds the caller-owned buffers of the batched ABI:
    ids [B, L, L] int32, types [B, n_cells + 1] uint8, areas [B, n_cells + 1]
    int32 and the workspace."""

    def __init__(self, n_lattices, L, cpm, seed=0, stream=None):
        import torch
        J = np.ascontiguousarray(np.asarray(cpm["J"], dtype=np.int32))
        ct = cpm.get("cell_type")
        self._J = J
        self._types_host = None if ct is None else np.ascontiguousarray(np.asarray(ct, dtype=np.uint8))
        self.params = CpmParams(J.shape[0], int(cpm["lambda"]), int(cpm["target"]), int(cpm["n_cells"]),
                                J.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                None if self._types_host is None else
                                self._types_host.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                float(cpm["T"]), int(cpm.get("side", 0)), int(cpm.get("cols", 0)), 0)
        self.B, self.L, self.seed = int(n_lattices), int(L), int(seed)
        nc1 = int(cpm["n_cells"]) + 1
        self.width = J.shape[0] * (J.shape[0] + 1) // 2 + 2
        self.ids = torch.empty((self.B, L, L), dtype=torch.int32, device="cuda")
        self.types = torch.empty((self.B, nc1), dtype=torch.uint8, device="cuda")
        self.areas = torch.empty((self.B, nc1), dtype=torch.int32, device="cuda")
        nbytes = int(lib().spin_cpm_batch_workspace_bytes(ctypes.byref(self.params)))
        if nbytes < 0:
            raise SpinError("spin_cpm_batch_workspace_bytes: invalid parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.step = 0
        _check(lib().spin_cpm_batch_init(self.seed, self.B, self.L, ctypes.byref(self.params), _ptr(self.ids),
                                         _ptr(self.types), _ptr(self.areas), _stream(stream)), None,
               "spin_cpm_batch_init")

    def run(self, n_steps, record=False, stream=None):
        """n_steps Monte Carlo steps; with record=True returns the statistics
        [n_steps, B, width] (int64, device)."""
        import torch
        stats = (torch.empty((n_steps, self.B, self.width), dtype=torch.int64, device="cuda") if record else None)
        _check(lib().spin_cpm_batch_run(self.seed, self.B, self.L, ctypes.byref(self.params), _ptr(self.ids),
                                        _ptr(self.types), _ptr(self.areas), self.step, int(n_steps), _ptr(stats),
                                        _ptr(self.workspace), _stream(stream)), None, "spin_cpm_batch_run")
        self.step += int(n_steps)
        return stats


def dmc_spin_iter(seed, J, spins, energy, beta, h, alpha, eta, first_sweep, n_sweeps, stream=None):
    """One fused spin-value iteration of the differentiable Monte Carlo."""
    B, L = spins.shape[0], spins.shape[-1]
    _check(lib().spin_dmc_spin_iter(int(seed), B, L, float(beta), float(h), float(alpha), float(eta),
                                    int(first_sweep), int(n_sweeps), _ptr(J), _ptr(spins), _ptr(energy),
                                    _stream(stream)), None, "spin_dmc_spin_iter")


def dmc_spin_iter_max_sweeps(L):
    return int(lib().spin_dmc_spin_iter_max_sweeps(int(L)))

