"""GB300-native micromagnetic-ensemble Wang-Landau (arXiv:1302.2320).

Thin ctypes binding over the C ABI in ``include/wl.h``: every function here
marshals arguments and calls the CUDA library ``_build/libwl.so``; all of the
walk (initialisation, moves, flatness tests, stage steps, assembly) runs in its
kernels.  There is no CPU fallback: if the library is missing or fails to load,
``lib()`` raises.

The C names are kept: ``wl_create``, ``wl_set_option``, ``wl_run``,
``wl_assemble``, ``wl_get_lng``, ``wl_get_surface``, ``wl_get_stats``,
``wl_get_line_state``, ``wl_get_exp_table``, ``wl_philox``, ``wl_accept_threshold``, ``wl_reset``,
``wl_abort``, ``wl_destroy``, ``wl_last_error``.  ``Handle`` wraps a handle
with the same calls as methods.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwl.so")

WL_SQUARE, WL_TRIANGULAR, WL_SIMPLE_CUBIC, WL_SQUARE_OPEN = 0, 1, 2, 3
LATTICES = {"square": WL_SQUARE, "triangular": WL_TRIANGULAR, "cubic": WL_SIMPLE_CUBIC,
            "square_open": WL_SQUARE_OPEN}
STATUS = {0: "WL_OK", 1: "WL_EINVAL", 2: "WL_ENOMEM", 3: "WL_ECUDA", 4: "WL_ETIMEOUT",
          5: "WL_EABORTED", 6: "WL_ENOTCONVERGED", 7: "WL_EMISMATCH", 8: "WL_ESTATE",
          9: "WL_EOVERFLOW"}
WL_OK, WL_EINVAL, WL_ENOTCONVERGED, WL_ETIMEOUT, WL_EABORTED = 0, 1, 6, 4, 5

EXPORTED = ["wl_create", "wl_required_bytes", "wl_set_option", "wl_get_option", "wl_run",
            "wl_abort", "wl_reset", "wl_assemble", "wl_get_lng", "wl_get_surface",
            "wl_get_stats", "wl_get_line_state", "wl_get_exp_table", "wl_philox", "wl_accept_threshold", "wl_destroy",
            "wl_last_error", "wl_walk_noalloc", "wl_server_create", "wl_server_submit",
            "wl_server_info", "wl_server_wait", "wl_server_result", "wl_server_release",
            "wl_server_destroy", "wl_thermo", "wl_measure_peaks", "wl_select_lines"]


class WLError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class wl_stats(ctypes.Structure):
    _fields_ = [("moves", ctypes.c_int64), ("accepts", ctypes.c_int64), ("checks", ctypes.c_int64),
                ("batches", ctypes.c_int64),
                ("lines", ctypes.c_int32), ("lines_converged", ctypes.c_int32),
                ("min_stage", ctypes.c_int32), ("max_stage", ctypes.c_int32),
                ("mapping", ctypes.c_int32), ("form", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("walk_ms", ctypes.c_double),
                ("init_ms", ctypes.c_double), ("assemble_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """Load libwl.so (raises if it is absent: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build() or python -m paper_1302_2320_gb300.buildlib)")
        L = ctypes.CDLL(LIB_PATH)
        i32, i64, u32, dbl, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_size_t
        vp, cp = ctypes.c_void_p, ctypes.c_char_p
        for name in EXPORTED:
            getattr(L, name).restype = i32
        L.wl_create.argtypes = [i32, i32, vp]
        L.wl_required_bytes.argtypes = [i32, i32]
        L.wl_required_bytes.restype = sz
        L.wl_set_option.argtypes = [vp, cp, i64]
        L.wl_get_option.argtypes = [vp, cp, vp]
        L.wl_run.argtypes = [vp, dbl, dbl]
        L.wl_abort.argtypes = [vp]
        L.wl_reset.argtypes = [vp]
        L.wl_assemble.argtypes = [vp]
        L.wl_get_lng.argtypes = [vp, i32, vp, sz, vp, vp, vp]
        L.wl_get_surface.argtypes = [vp, vp, sz, vp, sz, vp]
        L.wl_get_stats.argtypes = [vp, vp]
        L.wl_get_line_state.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.wl_get_exp_table.argtypes = [vp, vp, vp]
        L.wl_philox.argtypes = [sz, vp, vp, vp]
        L.wl_accept_threshold.argtypes = [dbl, i32, sz, vp, vp]
        L.wl_measure_peaks.argtypes = [vp]
        L.wl_select_lines.argtypes = [vp, vp, i32]
        L.wl_destroy.argtypes = [vp]
        L.wl_last_error.argtypes = []
        L.wl_last_error.restype = cp
        L.wl_thermo.argtypes = [vp, vp, i32, vp, i32, vp]
        L.wl_server_create.argtypes = [i64, i32, vp]
        L.wl_server_submit.argtypes = [vp, i32, i32, u32, dbl, dbl, i64, i64, vp]
        L.wl_server_info.argtypes = [vp, i64, vp]
        L.wl_server_wait.argtypes = [vp, i64, dbl]
        L.wl_server_result.argtypes = [vp, i64, vp, sz, vp]
        L.wl_server_release.argtypes = [vp, i64]
        L.wl_server_destroy.argtypes = [vp]
        _lib = L
        return L


def wl_last_error() -> str:
    return lib().wl_last_error().decode()


def _check(rc: int, where: str, ok=(WL_OK,)) -> int:
    if rc not in ok:
        raise WLError(rc, where, wl_last_error())
    return rc


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def wl_required_bytes(lattice: int, L: int) -> int:
    return int(lib().wl_required_bytes(lattice, L))


def wl_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Device Philox4x32-10 blocks: ctr (n, 4) uint32, key (n, 2) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    _check(lib().wl_philox(ctr.shape[0], _p(ctr), _p(key), _p(out)), "wl_philox")
    return out


def wl_accept_threshold(ln_f_min: float, deterministic: int, r: np.ndarray) -> np.ndarray:
    """dmax of Eq. 3 for each random word: a move with ln g increase d (units of
    ln_f_min) is accepted iff d <= dmax."""
    r = np.ascontiguousarray(r, dtype=np.uint32).ravel()
    out = np.zeros(r.size, dtype=np.int64)
    _check(lib().wl_accept_threshold(ln_f_min, int(deterministic), r.size, _p(r), _p(out)),
           "wl_accept_threshold")
    return out


class wl_peaks(ctypes.Structure):
    _fields_ = [("smem_words_per_s", ctypes.c_double), ("l2_sectors_per_s", ctypes.c_double),
                ("hbm_sectors_per_s", ctypes.c_double), ("lop3_ops_per_s", ctypes.c_double),
                ("iadd3_ops_per_s", ctypes.c_double), ("imad_ops_per_s", ctypes.c_double),
                ("mulwide_ops_per_s", ctypes.c_double), ("sms", ctypes.c_int32)]


def wl_measure_peaks() -> dict:
    """Random-access and integer-issue rates of the current device (wl.h)."""
    p = wl_peaks()
    _check(lib().wl_measure_peaks(ctypes.byref(p)), "wl_measure_peaks")
    return {k: getattr(p, k) for k, _ in wl_peaks._fields_}


class Handle:
    """One lattice's set of micromagnetic-line walkers on the GPU."""

    def __init__(self, lattice, L: int, **options):
        if isinstance(lattice, str):
            lattice = LATTICES[lattice]
        self._h = ctypes.c_void_p()
        _check(lib().wl_create(lattice, L, ctypes.byref(self._h)), "wl_create")
        self.lattice, self.L = lattice, L
        self.N = self.get_option("N")
        self.NB = self.get_option("NB")
        self.lines = self.get_option("lines")
        for k, v in options.items():
            self.set_option(k, v)

    def close(self):
        if self._h:
            lib().wl_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, key: str, value: int):
        _check(lib().wl_set_option(self._h, key.encode(), int(value)), f"wl_set_option({key})")

    def get_option(self, key: str) -> int:
        v = ctypes.c_int64()
        _check(lib().wl_get_option(self._h, key.encode(), ctypes.byref(v)), f"wl_get_option({key})")
        return v.value

    def run(self, ln_f_min: float, flatness: float = 0.8, allow=(WL_OK, WL_ENOTCONVERGED)) -> int:
        """wl_run; returns the status (WL_OK or WL_ENOTCONVERGED by default)."""
        return _check(lib().wl_run(self._h, ln_f_min, flatness), "wl_run", ok=allow)

    def select_lines(self, ells):
        """Walk only these lines (wl_select_lines); an empty list restores all."""
        a = np.ascontiguousarray(list(ells), dtype=np.int32)
        _check(lib().wl_select_lines(self._h, _p(a) if a.size else None, int(a.size)),
               "wl_select_lines")

    def abort(self):
        _check(lib().wl_abort(self._h), "wl_abort")

    def reset(self):
        _check(lib().wl_reset(self._h), "wl_reset")

    def assemble(self):
        _check(lib().wl_assemble(self._h), "wl_assemble")

    def get_lng(self, ell: int) -> np.ndarray:
        n = ctypes.c_size_t()
        lib().wl_get_lng(self._h, ell, None, 0, None, None, ctypes.byref(n))
        out = np.empty(n.value, dtype=np.float64)
        _check(lib().wl_get_lng(self._h, ell, _p(out), out.size, None, None, None), "wl_get_lng")
        return out

    def get_surface(self, out: np.ndarray | None = None):
        """(ln g over all walked lines, ragged offsets)."""
        n = ctypes.c_size_t()
        lib().wl_get_surface(self._h, None, 0, None, 0, ctypes.byref(n))
        if out is None:
            out = np.empty(n.value, dtype=np.float64)
        lines = self.get_option("ell_max") - self.get_option("ell_min") + 1
        offs = np.empty(lines + 1, dtype=np.int64)
        _check(lib().wl_get_surface(self._h, _p(out), out.size, _p(offs), offs.size, None),
               "wl_get_surface")
        return out, offs

    def stats(self) -> dict:
        s = wl_stats()
        _check(lib().wl_get_stats(self._h, ctypes.byref(s)), "wl_get_stats")
        return s.as_dict()

    def line_state(self, ell: int) -> dict:
        nb = int(min(self.get_option("z") * min(ell, self.N - ell), self.NB)
                 // self.get_option("k_step") + 1)
        d = {"sc": np.zeros(8, dtype=np.int64), "perm": np.zeros(self.N, dtype=np.int32),
             "spins": np.zeros(self.N, dtype=np.uint8), "lng": np.zeros(nb, dtype=np.int64),
             "hist": np.zeros(nb, dtype=np.int64), "visited": np.zeros(nb, dtype=np.uint8)}
        _check(lib().wl_get_line_state(self._h, ell, _p(d["sc"]), _p(d["perm"]), _p(d["spins"]),
                                       _p(d["lng"]), _p(d["hist"]), _p(d["visited"])),
               "wl_get_line_state")
        return d

    def thermo(self, T, H) -> np.ndarray:
        """Eq. 2 thermodynamics per spin, shape (len(T), len(H), 6): ln Z/N, E/N,
        C/N, M/N, |M|/N, chi/N."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        H = np.ascontiguousarray(H, dtype=np.float64)
        out = np.zeros((T.size, H.size, 6), dtype=np.float64)
        _check(lib().wl_thermo(self._h, _p(T), T.size, _p(H), H.size, _p(out)), "wl_thermo")
        return out

    def exp_table(self):
        t = np.zeros(4096, dtype=np.uint64)
        q = ctypes.c_int()
        _check(lib().wl_get_exp_table(self._h, _p(t), ctypes.byref(q)), "wl_get_exp_table")
        return t, q.value


class wl_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("lattice", ctypes.c_int32),
                ("L", ctypes.c_int32), ("moves", ctypes.c_int64), ("bins", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Server:
    """Continuous-batching request loop (wl_server_*): submit lattices, wait for
    their assembled surfaces."""

    def __init__(self, hbm_budget: int = 0, max_active: int = 16):
        self._s = ctypes.c_void_p()
        _check(lib().wl_server_create(int(hbm_budget), int(max_active), ctypes.byref(self._s)),
               "wl_server_create")

    def submit(self, lattice, L: int, seed: int = 1, ln_f_min: float = 1e-6, flatness: float = 0.8,
               check_interval: int = 1000, move_budget: int = 2**62) -> int:
        if isinstance(lattice, str):
            lattice = LATTICES[lattice]
        rid = ctypes.c_int64()
        _check(lib().wl_server_submit(self._s, lattice, L, seed, ln_f_min, flatness, check_interval,
                                      move_budget, ctypes.byref(rid)), "wl_server_submit")
        return rid.value

    def info(self, rid: int) -> dict:
        i = wl_request_info()
        _check(lib().wl_server_info(self._s, rid, ctypes.byref(i)), "wl_server_info")
        return i.as_dict()

    def wait(self, rid: int, timeout_s: float = -1.0) -> int:
        return _check(lib().wl_server_wait(self._s, rid, timeout_s), "wl_server_wait",
                      ok=(WL_OK, WL_ENOTCONVERGED, WL_ETIMEOUT))

    def result(self, rid: int) -> np.ndarray:
        n = ctypes.c_size_t()
        lib().wl_server_result(self._s, rid, None, 0, ctypes.byref(n))
        out = np.empty(n.value, dtype=np.float64)
        _check(lib().wl_server_result(self._s, rid, _p(out), out.size, None), "wl_server_result")
        return out

    def release(self, rid: int):
        _check(lib().wl_server_release(self._s, rid), "wl_server_release")

    def close(self):
        if self._s:
            lib().wl_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
