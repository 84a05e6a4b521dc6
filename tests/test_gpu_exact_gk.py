"""The check of Sec. 4 / Fig. 5 on the GPU: the whole 8x8 surface walked to
ln f_min by the CUDA library (deterministic, 10^6 moves between flatness
checks), assembled, summed over l and compared with the exact zero-field g_k
(Kaufman's partition function, oracle/exact_gk.py).  The deterministic chain
is the oracle's bit for bit (checked here on the middle line), so the bound is
the one the oracle meets in tests/test_exact_gk.py."""
import numpy as np
import pytest

import bench
import oracle
import paper_1302_2320_gb300 as wl
from oracle import exact_gk

pytestmark = pytest.mark.gpu


def test_summed_gpu_surface_L8_matches_exact_gk():
    L, N, NB, u, C = 8, 64, 128, 1e-6, 1_000_000
    wl.build()
    h = wl.Handle("square", L, seed=1, check_interval=C)
    h.run(u, 0.8)
    st = h.stats()
    assert st["lines_converged"] == N // 2 + 1
    ref_line = oracle.run_line(oracle.SQUARE, L, N // 2, 1, u, C, 800)
    got = h.line_state(N // 2)
    assert np.array_equal(got["sc"], ref_line.sc)
    assert np.array_equal(got["lng"], ref_line.lng)
    h.assemble()
    lines = [h.get_lng(ell) for ell in range(N // 2 + 1)]
    h.close()
    summed = bench.sum_over_lines(lines, N)
    ref = exact_gk.ln_gk(L)
    fin = np.isfinite(ref)
    assert summed.size == NB + 1 and np.array_equal(np.isfinite(summed), fin)
    d = np.abs(summed[fin] - ref[fin])
    assert d.max() / NB < 0.002
    assert d.max() < 0.1 and d.mean() < 0.02
