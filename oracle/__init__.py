"""CPU oracle for the micromagnetic-ensemble Wang-Landau method (arXiv:1302.2320).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, independent
reference that the CUDA library is checked against.  Only ``tests/``, the
``smoke()`` check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the GPU library: the C
source ``wl_oracle.c`` is compiled on its own with gcc into
``oracle/_build/liboracle.so`` and loaded here through ctypes.

Every function cites the passage of the paper it follows; see the C source for
the arithmetic.  Lattice type codes: 0 square, 1 triangular, 2 simple cubic
(all periodic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wl_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

SQUARE, TRIANGULAR, CUBIC, SQUARE_OPEN = 0, 1, 2, 3
LATTICE_NAMES = {"square": SQUARE, "triangular": TRIANGULAR, "cubic": CUBIC,
                 "square_open": SQUARE_OPEN}

# scalar slots of a line state (same order as the C enum)
SC_K, SC_T, SC_F, SC_STAGE, SC_ACCEPTS, SC_TSTAGE, SC_STATUS, SC_CHECKS = range(8)
SC_COUNT = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP for the TM)."""
    with _lock:
        if (not force and os.path.exists(_OUT)
                and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        i32, i64, u32, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
        vp = ctypes.c_void_p
        L.or_lattice_info.argtypes = [i32, i32, vp, vp, vp]
        L.or_philox4x32_10.argtypes = [vp, vp, vp]
        L.or_philox4x32_10.restype = None
        L.or_exp_table_q.argtypes = [dbl]
        L.or_exp_table.argtypes = [dbl, vp, vp]
        L.or_threshold_of.argtypes = [dbl, i64]
        L.or_threshold_of.restype = ctypes.c_uint64
        L.or_lattice_kstep.argtypes = [i32]
        L.or_line_nbins.argtypes = [i32, i32, i32]
        L.or_line_nbins.restype = i64
        L.or_line_run.argtypes = [i32, i32, i32, u32, dbl, i64, i32, i64, i32, i32, i32,
                                  vp, vp, vp, vp, vp, vp]
        L.or_line_audit.argtypes = [i32, i32, i32, vp, vp, i64]
        L.or_flatness.argtypes = [vp, vp, i64, i32]
        L.or_assemble.argtypes = [i32, i32, i64, vp, vp, dbl, vp]
        L.or_assemble.restype = None
        L.or_brute_force.argtypes = [i32, i32, vp]
        L.or_tm_square.argtypes = [i32, i32, vp, i32]
        L.or_thermo.argtypes = [i32, i32, vp, vp, i32, vp, i32, vp, i32, vp]
        L.or_thermo.restype = None
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def lattice_info(lattice: int, L: int) -> dict:
    """N spins, N_B bonds and coordination z (Eq. 1 on the chosen lattice)."""
    n = (ctypes.c_int * 3)()
    if lib().or_lattice_info(lattice, L, ctypes.byref(n, 0), ctypes.byref(n, 4),
                             ctypes.byref(n, 8)):
        raise ValueError("bad lattice")
    return {"N": n[0], "NB": n[1], "z": n[2]}


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def exp_table(u: float):
    """The 4096-entry threshold table round(2^32 exp(-(i 2^q) u)) and its q."""
    t = np.zeros(4096, dtype=np.uint64)
    q = ctypes.c_int()
    if lib().or_exp_table(u, _p(t), ctypes.byref(q)):
        raise ValueError("u out of range")
    return t, q.value


def threshold(u: float, d: int) -> int:
    """Acceptance threshold T(d) of an uphill move of d units (d > 0)."""
    return int(lib().or_threshold_of(u, d))


def kstep(lattice: int) -> int:
    """Spacing of the reachable k: 2 on the periodic lattices, 1 with open boundaries."""
    return int(lib().or_lattice_kstep(lattice))


def line_nbins(lattice: int, L: int, ell: int) -> int:
    return int(lib().or_line_nbins(lattice, L, ell))


class LineState:
    """Full state of one micromagnetic line walker (text around Eq. 3)."""

    def __init__(self, lattice: int, L: int, ell: int):
        info = lattice_info(lattice, L)
        self.lattice, self.L, self.ell = lattice, L, ell
        self.N = info["N"]
        self.nbins = line_nbins(lattice, L, ell)
        self.perm = np.zeros(self.N, dtype=np.int32)
        self.spins = np.zeros(self.N, dtype=np.uint8)
        self.sc = np.zeros(SC_COUNT, dtype=np.int64)
        self.lng = np.zeros(self.nbins, dtype=np.int64)
        self.hist = np.zeros(self.nbins, dtype=np.int64)
        self.visited = np.zeros(self.nbins, dtype=np.uint8)

    def copy(self) -> "LineState":
        o = LineState.__new__(LineState)
        o.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                           for k, v in self.__dict__.items()})
        return o

    @property
    def k(self): return int(self.sc[SC_K])
    @property
    def t(self): return int(self.sc[SC_T])
    @property
    def F(self): return int(self.sc[SC_F])
    @property
    def stage(self): return int(self.sc[SC_STAGE])
    @property
    def converged(self): return bool(self.sc[SC_STATUS])


def run_line(lattice: int, L: int, ell: int, seed: int, u: float, C: int,
             flat_pm: int = 800, budget: int = 2**62, mode: int = 0,
             state: LineState | None = None, same_f_resets: int = 0) -> LineState:
    """Run (or continue) the walk on line ``ell`` until F == 0 or t == budget.

    mode 0 = deterministic (table acceptance), 1 = production (double exp).
    same_f_resets = R > 0 resets a histogram that is not flat at the first R
    checks of each stage, keeping f (the extra reset remarked after Eq. 4).
    """
    init = state is None
    if init:
        state = LineState(lattice, L, ell)
    rc = lib().or_line_run(lattice, L, ell, seed & 0xFFFFFFFF, u, C, flat_pm, budget, mode,
                           1 if init else 0, same_f_resets, _p(state.perm), _p(state.spins), _p(state.sc),
                           _p(state.lng), _p(state.hist), _p(state.visited))
    if rc:
        raise ValueError("or_line_run rejected its arguments")
    return state


def is_flat(hist, visited, flat_pm: int = 800) -> bool:
    """The flatness test of the WL recap (80%/80% at flat_pm = 800) on a
    histogram over a line's bins; only visited bins take part."""
    h = np.ascontiguousarray(hist, dtype=np.int64)
    v = np.ascontiguousarray(visited, dtype=np.uint8)
    assert h.shape == v.shape
    return bool(lib().or_flatness(_p(h), _p(v), h.size, flat_pm))


def audit(state: LineState) -> int:
    """0 when the lists, spins and k of a line state are consistent."""
    return int(lib().or_line_audit(state.lattice, state.L, state.ell, _p(state.perm),
                                   _p(state.spins), state.k))


def assemble(N: int, ell: int, lng: np.ndarray, visited: np.ndarray, u: float) -> np.ndarray:
    """ln g_kl over the line's bins: Eq. 4 normalisation to C(N, l), FP64."""
    lng = np.ascontiguousarray(lng, dtype=np.int64)
    vis = np.ascontiguousarray(visited, dtype=np.uint8)
    out = np.zeros(lng.shape[0], dtype=np.float64)
    lib().or_assemble(N, ell, lng.shape[0], _p(lng), _p(vis), u, _p(out))
    return out


def brute_force(lattice: int, L: int) -> np.ndarray:
    """Exact g_kl, shape (N_B+1, N+1), by enumerating all 2^N configurations."""
    info = lattice_info(lattice, L)
    g = np.zeros((info["NB"] + 1, info["N"] + 1), dtype=np.float64)
    if lib().or_brute_force(lattice, L, _p(g)):
        raise ValueError("brute force limited to N <= 30")
    return g


def tm_square(L: int, ell_max: int | None = None, nthreads: int | None = None) -> np.ndarray:
    """Exact g_kl of the periodic LxL square lattice, shape (2L^2+1, ell_max+1)."""
    N = L * L
    if ell_max is None:
        ell_max = N
    if nthreads is None:
        nthreads = max(1, min(os.cpu_count() or 1, 16))
    g = np.zeros((2 * N + 1, ell_max + 1), dtype=np.float64)
    if lib().or_tm_square(L, ell_max, _p(g), nthreads):
        raise ValueError("bad TM arguments")
    return g


THERMO_FIELDS = ("lnZ", "E", "C", "M", "absM", "chi")


def thermo(N: int, NB: int, offsets, lng, T, H, kstep: int = 2) -> np.ndarray:
    """Eq. 2 thermodynamics per spin over a (T, H) grid, shape (nT, nH, 6)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    lng = np.ascontiguousarray(lng, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    H = np.ascontiguousarray(H, dtype=np.float64)
    out = np.zeros((T.size, H.size, 6), dtype=np.float64)
    lib().or_thermo(N, NB, _p(offsets), _p(lng), kstep, _p(T), T.size, _p(H), H.size, _p(out))
    return out


def exact_surface(g: np.ndarray, step: int = 2):
    """Ragged ln g over lines l = 0..N/2 (bins k = 0, step, ... up to the line's
    largest k) from an exact table g[k, l]; -inf where g = 0."""
    N = g.shape[1] - 1
    offs, vals = [0], []
    for l in range(N // 2 + 1):
        col = g[:, l]
        nb = int(np.nonzero(col)[0].max()) // step + 1
        with np.errstate(divide="ignore"):
            vals.append(np.log(col[0:step * nb:step]))
        offs.append(offs[-1] + nb)
    return np.array(offs, dtype=np.int64), np.concatenate(vals)
