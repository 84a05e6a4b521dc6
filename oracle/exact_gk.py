"""Exact zero-field density of states g_k of the periodic L x L square Ising
lattice, k = number of unsatisfied bonds (E = -(N_B - 2k), N_B = 2L^2).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Sec. 4 (Fig. 5) checks the WL surface by summing g_kl over l and comparing the
sum with the exact zero-field g_k, which the paper takes from Beale's method:
Kaufman's closed form of the torus partition function expanded as a
polynomial in x = exp(-2K) by computer algebra.  Here the same polynomial

    P(x) = x^(N_B/2) Z(x) = sum_k g_k x^k

is evaluated in floating point at complex x, and its coefficients are taken
out by discrete Cauchy integrals (an FFT over M points of a circle |x| = rho).
One circle resolves the band of k around the energy that its rho weights most,
so rho is stepped from the ground state (k = 0) to the antiferromagnetic end
(k = N_B) and each k keeps the estimate from the circle that weights it most.
The result is ln g_k with a relative error near 1e-12 (checked against exact
enumeration and the transfer matrix by the tests), not the integers themselves.

Kaufman's form for an m x n torus (m = n = L, L even), with s = sinh 2K,
c_l = cosh(2K) coth(2K) - cos(pi l / n) and e^{g_l} a root of r + 1/r = 2 c_l:

    Z  = 1/2 (2s)^(mn/2) (Z1 + Z2 + Z3 + Z4)
    Z1 = prod_{l odd}  2 cosh(m g_l / 2)      Z2 = prod_{l odd}  2 sinh(m g_l / 2)
    Z3 = prod_{l even} 2 cosh(m g_l / 2)      Z4 = prod_{l even} 2 sinh(m g_l / 2)

over l = 1, 3, .., 2n-1 and l = 0, 2, .., 2n-2, where the two roots without a
partner carry a sign: e^{g_0} = e^{2K} tanh K and e^{g_n} = e^{2K} coth K.
Since c_{2n-l} = c_l the other terms pair up as

    (2 cosh(m g/2))^2 = r^m + 2 + r^-m,   (2 sinh(m g/2))^2 = r^m - 2 + r^-m,

which do not change under r -> 1/r.  Either root of r + 1/r = 2c serves, so
every factor is a single-valued function of x: there is no branch to choose.
Each factor takes s^m (a pair) or s^(m/2) (an unpaired root) of the prefactor,
and everything is summed in logarithms, so nothing overflows.
"""
from __future__ import annotations

import math

import numpy as np


def _log_terms(x: np.ndarray, L: int) -> np.ndarray:
    """log Z1..log Z4 (prefactor s^(mn/2) included), shape (4, x.size)."""
    m = n = L
    s = (1.0 / x - x) / 2.0                     # sinh 2K
    ch = (1.0 / x + x) / 2.0                    # cosh 2K
    log_s = np.log(s)
    c0 = ch * ch / s                            # cosh 2K coth 2K

    def pair_logs(ls):
        """log of s^m (r^m + 2 + r^-m) and s^m (r^m - 2 + r^-m) summed over l."""
        cosl = np.cos(np.pi * np.asarray(ls, dtype=np.float64) / n)[:, None]
        c = c0[None, :] - cosl
        r = c + np.sqrt(c * c - 1.0)
        r = np.where(np.abs(r) < 1.0, 1.0 / r, r)           # |r| >= 1 for stability
        rm = np.exp(-m * np.log(r))                         # r^-m, |r^-m| <= 1
        base = m * log_s[None, :] + m * np.log(r)
        la = base + 2.0 * np.log1p(rm)
        lb = base + 2.0 * np.log1p(-rm)
        return la.sum(axis=0), lb.sum(axis=0)

    def single_logs(rho):
        """log of s^(m/2) (rho^(m/2) + rho^-(m/2)) and of s^(m/2) (rho^(m/2) - rho^-(m/2))."""
        big = np.abs(rho) >= 1.0
        lr = np.log(rho)
        h = m // 2
        e = np.exp(-m * np.where(big, lr, -lr))             # rho^-m or rho^m, modulus <= 1
        lead = np.where(big, h * lr, -h * lr)
        lc = h * log_s + lead + np.log1p(e)
        # rho^h - rho^-h = rho^h (1 - rho^-m) = -rho^-h (1 - rho^m)
        ls_ = h * log_s + lead + np.log1p(-e) + np.where(big, 0.0, 1j * np.pi)
        return lc, ls_

    odd = list(range(1, n, 2))                  # partners 2n - l are the other odd l
    even = list(range(2, n - 1, 2))             # partners 2n - l; 0 and n stand alone
    a_odd, b_odd = pair_logs(odd)
    if even:
        a_even, b_even = pair_logs(even)
    else:
        a_even = b_even = np.zeros_like(x)
    t = (1.0 - x) / (1.0 + x)                   # tanh K
    r0c, r0s = single_logs(t / x)               # e^{g_0} = e^{2K} tanh K
    rnc, rns = single_logs(1.0 / (t * x))       # e^{g_n} = e^{2K} coth K
    return np.stack([a_odd, b_odd, r0c + rnc + a_even, r0s + rns + b_even])


def log_poly(x, L: int) -> np.ndarray:
    """log P(x) = log sum_k g_k x^k at complex points x (Kaufman's form)."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    m = n = L
    lt = _log_terms(x, L)
    top = lt.real.max(axis=0)
    total = np.exp(lt - top[None, :]).sum(axis=0)
    return (m * n / 2.0 - 1.0) * math.log(2.0) + m * n * np.log(x) + top + np.log(total)


def ln_gk(L: int, rel_floor: float = 1e-4) -> np.ndarray:
    """ln g_k for k = 0..2L^2 of the periodic L x L square lattice (L even,
    L >= 4); -inf where no circle resolved a coefficient (g_k = 0: odd k, and
    k = 2, N_B - 2)."""
    if L < 4 or L % 2:
        raise ValueError("Kaufman's form here needs an even L >= 4")
    N = L * L
    NB = 2 * N
    M = 1 << (NB + 1 - 1).bit_length()          # more points than coefficients
    j = np.arange(M)
    phase = np.exp(2j * np.pi * (j + 0.5) / M)  # half-step grid avoids x = +-1
    kk = np.arange(M)
    unshift = np.exp(-1j * np.pi * kk / M)
    best = np.full(NB + 1, -np.inf)
    best_w = np.zeros(NB + 1)
    lr = math.log(0.5 * (8.0 * N) ** -0.25)     # start where k = 0 dominates
    lr_end = -lr
    while True:
        rho = math.exp(lr)
        lp = log_poly(rho * phase, L)
        lam = lp.real.max()
        coef = (np.fft.fft(np.exp(lp - lam)) / M * unshift).real[: NB + 1]
        cmax = coef.max()
        good = coef > rel_floor * cmax
        est = np.log(np.where(good, coef, 1.0)) + lam - kk[: NB + 1] * lr
        better = good & (coef > best_w)
        best[better] = est[better]
        best_w[better] = coef[better]
        if lr >= lr_end:
            break
        w = np.where(coef > 0, coef, 0.0)
        w /= w.sum()
        mu = (w * kk[: NB + 1]).sum()
        sd = math.sqrt(max(((w * (kk[: NB + 1] - mu) ** 2).sum()), 1.0))
        lr = min(lr + 0.5 / sd, lr_end)
    return best
