"""The kernels' modular arithmetic, restated on the host with Python integers
(mod 2^64 or 2^32 where the GPU words wrap) and checked against the exact
definitions (no GPU).  These pin the readings the kernels rest on:

  * the truncated high word of W' X (three of the four 32-bit partial
    products) falls short of floor(W' X / 2^64) by at most 2, so the Shoup
    remainder W X - Q q is the exact residue plus at most 3q: in [0, 4q) for
    q < 2^61, never wrapping (the reading of Section 2.2's Shoup quotient
    behind the lazy range [0, 8q) of the forward transform);
  * the Harvey butterflies keep X0, X1 in [0, 2m) (forward) and [0, m)
    (inverse) with m = 4q, with the right residues (Algorithms HF and HI);
  * the Barrett reduction of a 128-bit value below 2 q^2 (a product, or d1's
    sum of two) needs two conditional subtractions after its quotient
    estimate, not the one of Algorithm "Barrett Reduction" (the reading of
    Section 2.1 for q up to 2^61);
  * 32-bit words with beta = 2^32 keep the paper's ranges for q < 2^30."""
import random

import pytest

import workloads as W

M64, M32 = (1 << 64) - 1, (1 << 32) - 1


def mulhi64_trunc(a, b):
    a0, a1, b0, b1 = a & M32, a >> 32, b & M32, b >> 32
    return (a1 * b1 + ((a1 * b0) >> 32) + ((a0 * b1) >> 32)) & M64


def shoup_trunc(x, w, wp, q):
    """shoup_lazy64v<3>: W X - Q q mod 2^64 with the truncated Q."""
    return (w * x - mulhi64_trunc(wp, x) * q) & M64


def reduce_2q(x, m):
    d = (x - m) & M64
    return x if d >> 63 else d


def fwd(X0, X1, w, wp, q, m):
    x0 = reduce_2q(X0, m)
    t = shoup_trunc(X1, w, wp, q)
    return (x0 + t) & M64, (x0 - t + m) & M64


def inv(X0, X1, w, wp, q, m):
    y0 = reduce_2q((X0 + X1) & M64, m)
    t = (X0 - X1 + m) & M64
    return y0, shoup_trunc(t, w, wp, q)


def primes_below_2_61():
    two_n = W.MIXED_TWO_N
    big = (1 << 61) - ((1 << 61) % two_n) + 1
    while True:                      # the largest prime below 2^61 with q = 1 mod 2^18
        big -= two_n
        if pow(3, big - 1, big) == 1 and pow(5, big - 1, big) == 1:
            break
    return [W.ntt_primes(50, two_n, 1)[0], W.ntt_primes(60, two_n, 1)[0], big]


PRIMES = primes_below_2_61()
assert PRIMES[-1] < 1 << 61 and PRIMES[-1] % W.MIXED_TWO_N == 1


def operands(q, rng, hi, n):
    yield from (0, 1, hi - 1, hi - q, q - 1, q)
    for _ in range(n):
        yield rng.randrange(hi)


@pytest.mark.parametrize("q", PRIMES)
def test_truncated_quotient_and_shoup_range(q):
    rng = random.Random(q)
    for _ in range(300):
        w = rng.choice([1, q - 1, rng.randrange(q)])
        wp = (w << 64) // q
        for x in operands(q, rng, 1 << 64, 60):
            Q, Qt = (wp * x) >> 64, mulhi64_trunc(wp, x)
            assert 0 <= Q - Qt <= 2
            t = shoup_trunc(x, w, wp, q)
            assert t == w * x - Qt * q                  # no wrap
            assert t < 4 * q and t % q == w * x % q


@pytest.mark.parametrize("q", PRIMES)
def test_harvey_butterfly_ranges(q):
    rng = random.Random(q + 1)
    m = 4 * q
    for _ in range(2000):
        w = rng.randrange(q)
        wp = (w << 64) // q
        X0, X1 = rng.randrange(2 * m), rng.randrange(2 * m)
        if rng.random() < 0.1:
            X0, X1 = 2 * m - 1, 2 * m - 1
        Y0, Y1 = fwd(X0, X1, w, wp, q, m)
        assert Y0 < 2 * m and Y1 < 2 * m
        assert Y0 % q == (X0 + w * X1) % q and Y1 % q == (X0 - w * X1) % q
        Z0, Z1 = X0 % m, X1 % m
        V0, V1 = inv(Z0, Z1, w, wp, q, m)
        assert V0 < m and V1 < m
        assert V0 % q == (Z0 + Z1) % q and V1 % q == w * (Z0 - Z1) % q


def barrett128(d, q):
    """barrett_reduce128 with its corrections counted."""
    Qb = q.bit_length()
    k = (1 << (63 + Qb)) // q
    c1 = (d >> (Qb - 1)) & M64
    c3 = (c1 * k) >> 64
    c4 = ((d & M64) - c3 * q) & M64
    subs = 0
    while c4 >= q:
        c4 -= q
        subs += 1
    return c4, subs


@pytest.mark.parametrize("q", PRIMES + [(1 << 59) + 1, (1 << 60) - 93])
def test_barrett_needs_two_subtractions_at_most(q):
    rng = random.Random(q + 2)
    worst = 0
    for _ in range(20000):
        a, b = rng.randrange(q), rng.randrange(q)
        d = a * b + (rng.randrange(q) * rng.randrange(q) if rng.random() < 0.5 else 0)
        r, subs = barrett128(d, q)
        assert r == d % q and subs <= 2
        worst = max(worst, subs)
    d = 2 * (q - 1) ** 2                                # the largest d1
    r, subs = barrett128(d, q)
    assert r == d % q and subs <= 2
    assert worst >= 1


def test_barrett_can_need_the_second_subtraction():
    """A value below 2 q^2 (d1's range) whose quotient estimate falls short by
    2 -- found by a search over 61-bit q just above 2^60 with k's dropped
    fraction near 1 and d near 2 q^2 with a small remainder: one conditional
    subtraction, as the paper's algorithm has it, would leave d mod q + q."""
    q = 1210658930345534857
    d = 2909973386527182142091330259785225022
    assert q.bit_length() == 61 and d < 2 * q * q
    r, subs = barrett128(d, q)
    assert subs == 2 and r == d % q


def test_32_bit_words_keep_the_papers_ranges():
    q = W.ntt_primes(30, W.MIXED_TWO_N, 1)[0]
    assert q < 1 << 30
    rng = random.Random(7)
    for _ in range(20000):
        w = rng.randrange(q)
        wp = (w << 32) // q
        x = rng.randrange(1 << 32)
        Q = (wp * x) >> 32
        t = (w * x - Q * q) & M32
        assert t == w * x - Q * q and t < 2 * q and t % q == w * x % q
