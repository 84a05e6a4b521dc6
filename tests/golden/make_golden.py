"""Writes the stored exact values used by the tests.  Calls only ``oracle/``.

    python tests/golden/make_golden.py [--threads N]

square_L{6,8,12}_exact.txt: exact ln g_kl of the periodic 6x6, 8x8 and 12x12
square Ising lattices (N_B = 2N) for l = 0..N/2, every k with g_kl > 0, from the
oracle's site-by-site transfer matrix (the exact surface that Eq. 2 sums over;
the paper cites transfer-matrix surfaces up to 12x12).  Columns: l, k, ln g_kl.
cubic_L3_exact.txt: exact g_kl of the periodic 3x3x3 simple cubic lattice by
enumeration of all 2^27 configurations.  Columns: l, k, g_kl.
square_L{16,32,64}_gk_exact.txt: exact zero-field ln g_k of the periodic L x L
square lattice from Kaufman's partition function (oracle/exact_gk.py), the
values the paper compares its summed surfaces with (Sec. 4, Fig. 5).  Columns:
k, ln g_k (k with g_k > 0 only).
"""
import argparse
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402


def write_square_tm(L, threads):
    t0 = time.time()
    N = L * L
    g = oracle.tm_square(L, ell_max=N // 2, nthreads=threads)
    path = os.path.join(HERE, f"square_L{L}_exact.txt")
    with open(path, "w") as f:
        f.write(f"# exact ln g_kl, periodic {L}x{L} square lattice, transfer matrix "
                "(tests/golden/make_golden.py)\n# l k ln_g\n")
        for ell in range(N // 2 + 1):
            for k in range(0, 2 * N + 1):
                if g[k, ell] > 0:
                    f.write(f"{ell} {k} {math.log(g[k, ell]):.17g}\n")
    print(f"square L={L}: {time.time() - t0:.1f} s -> {path}")


def write_cubic_l3():
    t0 = time.time()
    g = oracle.brute_force(oracle.CUBIC, 3)
    path = os.path.join(HERE, "cubic_L3_exact.txt")
    with open(path, "w") as f:
        f.write("# exact g_kl, periodic 3x3x3 simple cubic lattice, full enumeration "
                "(tests/golden/make_golden.py)\n# l k g\n")
        for ell in range(28):
            for k in range(82):
                if g[k, ell] > 0:
                    f.write(f"{ell} {k} {int(g[k, ell])}\n")
    print(f"cubic L=3: {time.time() - t0:.1f} s -> {path}")


def write_square_gk(L):
    from oracle import exact_gk
    t0 = time.time()
    lg = exact_gk.ln_gk(L)
    path = os.path.join(HERE, f"square_L{L}_gk_exact.txt")
    with open(path, "w") as f:
        f.write(f"# exact zero-field ln g_k, periodic {L}x{L} square lattice, Kaufman's "
                "partition function (tests/golden/make_golden.py)\n# k ln_g\n")
        for k in range(lg.size):
            if np.isfinite(lg[k]):
                f.write(f"{k} {lg[k]:.17g}\n")
    print(f"square g_k L={L}: {time.time() - t0:.1f} s -> {path}")


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", choices=["square", "square_small", "cubic", "gk"], default=None)
    a = ap.parse_args()
    if a.only in (None, "cubic"):
        write_cubic_l3()
    if a.only == "square_small":
        write_square_tm(6, a.threads)
        write_square_tm(8, a.threads)
    if a.only in (None, "square"):
        write_square_tm(6, a.threads)
        write_square_tm(8, a.threads)
        write_square_tm(12, a.threads)
    if a.only in (None, "gk"):
        for L in (16, 32, 64):
            write_square_gk(L)
