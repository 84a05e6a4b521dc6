"""wl_walk_noalloc, the walker entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc -- for example code running
while another framework owns the device memory pool, code that must not
trigger the synchronisation an allocation can imply, or hosts with a memory
plan fixed up front.  Such a caller owns every input and output buffer and
passes them in; the entry point's own scratch is a fixed array inside the
library.  Here the test plays that caller: it allocates the buffers itself
(with torch), calls the entry point twice in a row (initialise and walk, then
continue the same walk) and checks that the walker state after each call is
identical to what the handle API (wl_create / wl_run) produces on the same
inputs; it also walks a lattice to convergence over several of the entry
point's slices and fills the buffers of a full 64x64 surface.  Deterministic
mode, so identical means bit for bit, the tolerance of the other parity tests.
"""
import ctypes

import numpy as np
import pytest

import paper_1302_2320_gb300 as wl

pytestmark = pytest.mark.gpu

Z = {"square": 4, "triangular": 6, "cubic": 6}


def _fn():
    f = wl.lib().wl_walk_noalloc
    f.restype = ctypes.c_int
    i32, i64, u32, dbl, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
    f.argtypes = [i32, i32, i32, i32, u32, i32, dbl, dbl, i64, i64, i32, i32, vp, vp, vp, vp, vp, i64]
    return f


class Buffers:
    """Caller-owned device buffers in the layout the entry point documents."""

    def __init__(self, lattice, L, ell_first, nlines):
        import torch
        N = L * L if lattice != "cubic" else L ** 3
        z = Z[lattice]
        NB = N * z // 2
        isz = 2 if N <= 65536 else 4
        self.N, self.ell_first, self.nlines = N, ell_first, nlines
        self.P = ((N * isz + 15) // 16 * 16) // isz
        self.W = ((N + 31) // 32 * 4 + 15) // 16 * 4
        self.nbins = [min(z * min(l, N - l), NB) // 2 + 1
                      for l in range(ell_first, ell_first + nlines)]
        self.off = np.concatenate([[0], np.cumsum(self.nbins)])
        dev = torch.device("cuda", torch.cuda.current_device())
        self.perm = torch.zeros(nlines * self.P, dtype=torch.int16 if isz == 2 else torch.int32, device=dev)
        self.spins = torch.zeros(nlines * self.W, dtype=torch.int32, device=dev)
        self.lng = torch.zeros(int(self.off[-1]), dtype=torch.int64, device=dev)
        self.hist = torch.zeros(int(self.off[-1]), dtype=torch.int64, device=dev)
        self.state = torch.zeros(nlines * 9, dtype=torch.int64, device=dev)
        self.stream = torch.cuda.current_stream().cuda_stream

    def ptrs(self):
        return [ctypes.c_void_p(t.data_ptr()) for t in (self.perm, self.spins, self.lng, self.hist, self.state)]

    def line(self, i):
        """Line i of the buffers in the layout of Handle.line_state()."""
        N = self.N
        perm = self.perm.cpu().numpy().view(np.uint16 if self.perm.element_size() == 2 else np.uint32)
        words = self.spins.cpu().numpy().view(np.uint32)[i * self.W:(i + 1) * self.W]
        spins = ((words[np.arange(N) >> 5] >> (np.arange(N) & 31)) & 1).astype(np.uint8)
        h = self.hist.cpu().numpy().view(np.uint64)[self.off[i]:self.off[i + 1]]
        return {"sc": self.state.cpu().numpy()[i * 9:i * 9 + 8],
                "perm": perm[i * self.P:i * self.P + N].astype(np.int32),
                "spins": spins,
                "lng": self.lng.cpu().numpy()[self.off[i]:self.off[i + 1]],
                "hist": (h & np.uint64(0x7FFFFFFFFFFFFFFF)).astype(np.int64),
                "visited": (h >> np.uint64(63)).astype(np.uint8)}


@pytest.mark.parametrize("lattice,L,ell_first,nlines", [("square", 8, 0, 33), ("triangular", 6, 3, 8)])
def test_noalloc_two_calls_match_handle_api(lattice, L, ell_first, nlines):
    import torch
    f = _fn()
    seed, u, C, budgets = 3, 1e-6, 500, (20_000, 60_000)
    buf = Buffers(lattice, L, ell_first, nlines)
    lat = wl.LATTICES[lattice]
    h = wl.Handle(lattice, L, seed=seed, check_interval=C, mapping=8)
    h.set_option("ell_min", ell_first)
    h.set_option("ell_max", ell_first + nlines - 1)
    for call, budget in enumerate(budgets):
        rc = f(lat, L, ell_first, nlines, seed, 1, u, 0.8, C, budget, 8, 1 if call == 0 else 0,
               *buf.ptrs(), buf.stream)
        assert rc in (wl.WL_OK, wl.WL_ENOTCONVERGED), wl.wl_last_error()
        torch.cuda.synchronize()
        h.set_option("move_budget", budget)
        h.run(u, 0.8)
        for i in range(nlines):
            got, ref = buf.line(i), h.line_state(ell_first + i)
            for key in ref:
                assert np.array_equal(got[key], ref[key]), (call, ell_first + i, key)
    h.close()


def test_noalloc_walks_several_slices_to_convergence():
    """Checks every 2^18 moves: every 4x4 line needs 14 stages (ln f_min =
    1e-8), more than three of the entry point's 2^20-move slices, so its slice
    loop restarts the queue and re-reads the summary several times; the call
    returns WL_OK with the handle API's converged state, bit for bit."""
    import torch
    f = _fn()
    seed, u, C = 5, 1e-8, 1 << 18
    buf = Buffers("square", 4, 0, 9)
    rc = f(wl.WL_SQUARE, 4, 0, 9, seed, 1, u, 0.8, C, 2**62, 8, 1, *buf.ptrs(), buf.stream)
    assert rc == wl.WL_OK, wl.wl_last_error()
    torch.cuda.synchronize()
    h = wl.Handle("square", 4, seed=seed, check_interval=C, mapping=8)
    assert h.run(u, 0.8) == wl.WL_OK
    for i in range(9):
        got, ref = buf.line(i), h.line_state(i)
        assert i == 0 or got["sc"][1] > 3 << 20          # l = 0 has no move
        for key in ref:
            assert np.array_equal(got[key], ref[key]), (i, key)
    h.close()


def test_noalloc_full_64x64_surface_layout():
    """All 2049 lines of the 64x64 lattice in one call (near the 4096-line
    limit of the scratch), a short budget, then a continuation: sampled lines
    equal the handle API's, and a continuation with another ln_f_min is refused."""
    import torch
    f = _fn()
    seed, u, C = 2, 1e-6, 1024
    buf = Buffers("square", 64, 0, 2049)
    h = wl.Handle("square", 64, seed=seed, check_interval=C, mapping=8)
    for call, budget in enumerate((3000, 8192)):
        rc = f(wl.WL_SQUARE, 64, 0, 2049, seed, 1, u, 0.8, C, budget, 8, 1 if call == 0 else 0,
               *buf.ptrs(), buf.stream)
        assert rc == wl.WL_ENOTCONVERGED, wl.wl_last_error()
        torch.cuda.synchronize()
        h.set_option("move_budget", budget)
        h.run(u, 0.8)
        for i in (1, 2, 3, 100, 511, 1024, 1500, 2047, 2048):
            got, ref = buf.line(i), h.line_state(i)
            for key in ref:
                assert np.array_equal(got[key], ref[key]), (call, i, key)
    rc = f(wl.WL_SQUARE, 64, 0, 2049, seed, 1, 1e-7, 0.8, C, 9000, 8, 0, *buf.ptrs(), buf.stream)
    assert rc == wl.WL_EINVAL and "ln_f_min" in wl.wl_last_error()
    h.close()


def test_noalloc_rejects_more_lines_than_its_scratch_holds():
    f = _fn()
    rc = f(wl.WL_SQUARE, 128, 0, 4097, 1, 1, 1e-6, 0.8, 1000, 10, 8, 1,
           ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16),
           ctypes.c_void_p(16), 0)
    assert rc == 1                                   # WL_EINVAL, before any launch
    assert "scratch limit" in wl.wl_last_error()
