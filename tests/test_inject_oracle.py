"""The quantised-injection oracle (arXiv 2606.27262, Appendix B) pinned to
the appendix's own closed forms and to invariants: every row of the
transition matrix sums to 1, S = 0 is the identity, the 1-bit and 2-bit
expressions (including the corrected P(2->3) and P(3->3)), the 8-bit
interior expression, and Monte-Carlo transition frequencies of a sampled
Gaussian quantised before and after adding S."""
import math

import numpy as np
import pytest

from oracle import inject as oi


def phi(x, mu, sig):
    return 0.5 * (1 + math.erf((x - mu) / (sig * math.sqrt(2))))


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_rows_sum_to_one_and_zero_signal_is_identity(M):
    rng = np.random.default_rng(M)
    for _ in range(5):
        mu, sig, l, S = rng.normal(), rng.uniform(0.5, 2), rng.uniform(0.2, 1.5), rng.uniform(0, 4)
        P = oi.matrix(S, M, mu, sig, l)
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
        assert (P >= 0).all() and np.allclose(np.tril(P, -1), 0)
        assert np.allclose(oi.matrix(0.0, M, mu, sig, l), np.eye(2 ** M), atol=1e-12)


def test_eight_bit_rows_sum_to_one():
    for n in (0, 1, 60, 127, 128, 200, 254, 255):
        for S in (0.0, 0.01, 0.5, 3.0):
            p = [oi.prob(n, k, S, 8, 0.0, 1.0, 0.030765) for k in range(256)]
            assert abs(sum(p) - 1) < 1e-10


def test_one_bit_closed_form():
    for mu, sig in ((0.0, 1.0), (2.0, 0.7)):
        for S in (0.0, 0.3, 1.0, 2.5):
            assert math.isclose(oi.prob(0, 1, S, 1, mu, sig, 1.0), 1 - 2 * phi(mu - S, mu, sig), abs_tol=1e-12)
            assert math.isclose(oi.prob(0, 0, S, 1, mu, sig, 1.0), 2 * phi(mu - S, mu, sig), abs_tol=1e-12)
            assert oi.prob(1, 0, S, 1, mu, sig, 1.0) == 0 and oi.prob(1, 1, S, 1, mu, sig, 1.0) == 1


def test_two_bit_closed_forms():
    """Appendix B's 2-bit expressions, retyped (a negative overlap is 0)."""
    mu, sig, l = 0.3, 1.2, 0.8
    ls = l * sig
    f = lambda x: phi(x, mu, sig)  # noqa: E731
    pos = lambda v: max(v, 0.0)  # noqa: E731
    for S in (0.0, 0.2, 0.5, 0.9, 1.5, 2.2, 4.0):
        want = {
            (0, 0): f(mu - ls - S) / f(mu - ls),
            (0, 1): pos(f(min(mu - S, mu - ls)) - f(mu - ls - S)) / f(mu - ls),
            (0, 2): pos(f(min(mu + ls - S, mu - ls)) - f(mu - S)) / f(mu - ls),
            (0, 3): pos(f(mu - ls) - f(mu + ls - S)) / f(mu - ls),
            (1, 1): pos(f(mu - S) - f(mu - ls)) / (0.5 - f(mu - ls)),
            (1, 2): pos(f(min(mu + ls - S, mu)) - f(max(mu - S, mu - ls))) / (0.5 - f(mu - ls)),
            (1, 3): pos(0.5 - f(max(mu + ls - S, mu - ls))) / (0.5 - f(mu - ls)),
            (2, 2): pos(f(mu + ls - S) - 0.5) / (f(mu + ls) - 0.5),
            (2, 3): pos(f(mu + ls) - f(max(mu + ls - S, mu))) / (f(mu + ls) - 0.5),
            (3, 3): 1.0,
        }
        for (n, k), v in want.items():
            assert math.isclose(oi.prob(n, k, S, 2, mu, sig, l), v, abs_tol=1e-12), (n, k, S)
        # the corrected row 2: P(2->2) + P(2->3) = 1 for every S
        assert math.isclose(want[(2, 2)] + want[(2, 3)], 1.0, abs_tol=1e-12)


def test_eight_bit_interior_closed_form():
    mu, sig, l = 0.0, 1.0, 0.030765
    f = lambda x: phi(x, mu, sig)  # noqa: E731
    for n, m, S in ((100, 0, 0.01), (100, 1, 0.02), (128, 3, 0.1), (60, 5, 0.16), (200, 2, 0.05)):
        num = f(min(mu + (n + m - 127) * l * sig - S, mu + (n - 127) * l * sig)) - \
            f(max(mu + (n + m - 128) * l * sig - S, mu + (n - 128) * l * sig))
        den = f(mu + (n - 127) * l * sig) - f(mu + (n - 128) * l * sig)
        assert math.isclose(oi.prob(n, n + m, S, 8, mu, sig, l), max(num, 0) / den, rel_tol=1e-9, abs_tol=1e-12)


def test_monte_carlo_transition_frequencies():
    rng = np.random.default_rng(7)
    M, mu, sig, l = 2, 0.0, 1.0, 0.9
    x = rng.normal(mu, sig, 400000)

    def state(v):
        return np.clip(np.floor((v - mu) / (l * sig)) + 2, 0, 3).astype(int)
    for S in (0.3, 1.1, 2.0):
        s0, s1 = state(x), state(x + S)
        P = oi.matrix(S, M, mu, sig, l)
        for n in range(4):
            sel = s0 == n
            freq = np.bincount(s1[sel], minlength=4) / sel.sum()
            err = np.sqrt(P[n] * (1 - P[n]) / sel.sum()) * 5 + 1e-4
            assert (np.abs(freq - P[n]) <= err).all(), (S, n, freq, P[n])


def test_most_probable_state():
    # interior 8-bit sample: the move follows S / (l sigma) to within a level
    mu, sig, l = 127.5, 16.0, 1 / 16
    for n in (40, 128, 200):
        for S in (0.4, 3.0, 17.2, 40.0):
            k, _ = oi.new_state(n, S, 8, mu, sig, l)
            assert abs(k - (n + S / (l * sig))) <= 1
    assert oi.new_state(255, 5.0, 8, mu, sig, l)[0] == 255
    assert oi.new_state(37, 0.0, 8, mu, sig, l)[0] == 37
