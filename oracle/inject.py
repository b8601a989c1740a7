"""Oracle of the quantised-data injector (test infrastructure only), arXiv
2606.27262 Appendix B, written from its equations.

States: with L = 2^M levels, state k lies between mu + (k - L/2) l sigma and
mu + (k + 1 - L/2) l sigma (Appendix B: state n between mu + i l sigma and
mu + (i+1) l sigma with n - i = L/2 - 1), the first state extending to -inf
and the last to +inf.  The probability that a sample in state n moves to
state n + m when a signal S is added is the noise probability mass of state
n that lands in state n + m once shifted by S, over the mass of state n (the
general equation and its boundary equations; a negative overlap is no
overlap).  The sample moves to the most probable state, the lowest on exact
ties.  phi is the Gaussian CDF of the noise.
"""
from __future__ import annotations

import math

import numpy as np


def phi(x, mu, sigma):
    if x == math.inf:
        return 1.0
    if x == -math.inf:
        return 0.0
    return 0.5 * math.erfc(-(x - mu) / (sigma * math.sqrt(2.0)))


def state_bounds(k, M, mu, sigma, l):
    L = 2 ** M
    lo = -math.inf if k == 0 else mu + (k - L // 2) * l * sigma
    hi = math.inf if k == L - 1 else mu + (k + 1 - L // 2) * l * sigma
    return lo, hi


def prob(n, k, S, M, mu, sigma, l):
    """P(n -> k) for a signal S >= 0 (0 for k < n; 1 for the top state)."""
    L = 2 ** M
    if k < n:
        return 0.0
    if n == L - 1:
        return 1.0 if k == n else 0.0
    lo_n, hi_n = state_bounds(n, M, mu, sigma, l)
    lo_k, hi_k = state_bounds(k, M, mu, sigma, l)
    den = phi(hi_n, mu, sigma) - phi(lo_n, mu, sigma)
    if not den > 0:  # a state with no noise mass in double precision: the sample stays
        return 1.0 if k == n else 0.0
    num = phi(min(hi_k - S, hi_n), mu, sigma) - phi(max(lo_k - S, lo_n), mu, sigma)
    return max(num, 0.0) / den


def matrix(S, M, mu, sigma, l):
    L = 2 ** M
    return np.array([[prob(n, k, S, M, mu, sigma, l) for k in range(L)] for n in range(L)])


def new_state(n, S, M, mu, sigma, l):
    """Most probable state after injecting S into a sample of state n, and
    the gap to the runner-up (for near-tie handling in comparisons)."""
    L = 2 ** M
    if not S > 0 or n >= L - 1:
        return n, math.inf
    p = [prob(n, k, S, M, mu, sigma, l) for k in range(n, L)]
    order = np.argsort(-np.array(p), kind="stable")
    best = n + int(order[0])
    gap = p[order[0]] - (p[order[1]] if len(p) > 1 else 0.0)
    return best, gap


def inject(values, signal, M, mu, sigma, l):
    """Elementwise injection (pure Python; small arrays)."""
    out = np.array(values, dtype=np.int64).copy()
    gaps = np.full(out.shape, math.inf)
    flat_v, flat_s = out.reshape(-1), np.asarray(signal, np.float64).reshape(-1)
    flat_g = gaps.reshape(-1)
    for i in range(flat_v.size):
        flat_v[i], flat_g[i] = new_state(int(flat_v[i]), float(flat_s[i]), M, mu, sigma, l)
    return out, gaps
