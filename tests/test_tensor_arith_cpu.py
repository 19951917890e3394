"""The fused kernels' ciphertext-tensor arithmetic (tensor_r3 / tensor_rk in
the device code), restated on the host with Python integers that wrap where
the GPU words wrap, and checked against the definition of the step,
r_k = (d_k s + e_k) mod q with d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1
(no GPU).  The restatement follows the device code's order:

  * a' = a s mod q by a Shoup product on the raw operand (< 4q), exact or
    truncated quotient (64-bit words below 2^61) or 32-bit words (q < 2^30),
    then conditional subtractions to [0, q);
  * the three products a0' b0, a1' b1 and (a0' + a1')(b0 + b1), d1 exact as
    their difference (Karatsuba), each below 2^(63+Q) (2^(31+Q) on 32-bit
    words) as the Barrett reduction needs;
  * Barrett (L = 63 + Q; on 32-bit words L = 31 + Q with k' = k >> 32):
    c4 = d - c3 q below 3q with the exact quotient and below 5q with the
    truncated one, never wrapping;
  * r_k = the reduced value plus e_k, one subtraction.

Each bound is asserted where the device code relies on it."""
import random

import pytest

import workloads as W

M64, M32 = (1 << 64) - 1, (1 << 32) - 1


def mulhi_trunc(a, b):
    a0, a1, b0, b1 = a & M32, a >> 32, b & M32, b >> 32
    return (a1 * b1 + ((a1 * b0) >> 32) + ((a0 * b1) >> 32)) & M64


def consts(q, s):
    Q = q.bit_length()
    return dict(q=q, s=s, sp=(s << 64) // q, bk=(1 << (63 + Q)) // q, Qm1=Q - 1)


def scale64(a, c, tr):
    q = c["q"]
    assert a < 1 << 64
    Qt = mulhi_trunc(c["sp"], a) if tr else (c["sp"] * a) >> 64
    r = (c["s"] * a - Qt * q) & M64
    assert r < (4 if tr else 2) * q
    if tr:
        r = r - 2 * q if r >= 2 * q else r
    return r - q if r >= q else r


def barrett64(d, c, tr):
    q, Qm1 = c["q"], c["Qm1"]
    assert d < 1 << (64 + Qm1)                      # c1 fits 64 bits
    c1 = (d >> Qm1) & M64
    c3 = mulhi_trunc(c1, c["bk"]) if tr else (c1 * c["bk"]) >> 64
    c4 = ((d & M64) - c3 * q) & M64
    assert c4 < (5 if tr else 3) * q
    if tr:
        c4 = c4 - 4 * q if c4 >= 4 * q else c4
    c4 = c4 - 2 * q if c4 >= 2 * q else c4
    return c4 - q if c4 >= q else c4


def scale32(a, c):
    q, s = c["q"], c["s"]
    sp32 = c["sp"] >> 32
    assert sp32 == (s << 32) // q and a < 1 << 32
    r = (s * a - ((sp32 * a) >> 32) * q) & M32
    assert r < 2 * q
    return r - q if r >= q else r


def barrett32(d, c):
    q, Qm1 = c["q"], c["Qm1"]
    k32 = c["bk"] >> 32
    assert k32 == (1 << (31 + Qm1 + 1)) // q and k32 < 1 << 32
    assert d < 1 << 64 and (d >> Qm1) < 1 << 32
    c3 = (((d >> Qm1) & M32) * k32) >> 32
    c4 = ((d & M32) - c3 * q) & M32
    assert c4 < 3 * q
    c4 = c4 - 2 * q if c4 >= 2 * q else c4
    return c4 - q if c4 >= q else c4


def small_mod(x, q, mf):
    """small_mod_rt for input_mod_factor 1, 2, 4: subtract 2q, then q."""
    if mf >= 4:
        x = x - 2 * q if x >= 2 * q else x
    if mf >= 2:
        x = x - q if x >= q else x
    return x


def addq(x, e, q):
    t = x + e
    return t - q if t >= q else t


def tensor_r3(a0, a1, b0, b1, e, c, mf, wd):
    q = c["q"]
    b0, b1 = small_mod(b0, q, mf), small_mod(b1, q, mf)
    assert b0 < q and b1 < q
    if wd == 0:
        x0, x1 = scale32(a0, c), scale32(a1, c)
        p0, p2 = x0 * b0, x1 * b1
        assert (x0 + x1) < 1 << 32 and (b0 + b1) < 1 << 32
        p1 = ((x0 + x1) * (b0 + b1) - p0 - p2) & M64
        red = [barrett32(p, c) for p in (p0, p1, p2)]
    else:
        tr = wd == 1
        x0, x1 = scale64(a0, c, tr), scale64(a1, c, tr)
        assert x0 + x1 < 1 << 64 and b0 + b1 < 1 << 64
        p0, p2 = x0 * b0, x1 * b1
        kar = (x0 + x1) * (b0 + b1)
        assert kar < 1 << 128
        p1 = kar - p0 - p2
        red = [barrett64(p, c, tr) for p in (p0, p1, p2)]
    return [addq(r, ek, q) for r, ek in zip(red, e)]


def tensor_rk(k, a0, a1, b0, b1, ek, c, mf, wd):
    q = c["q"]
    a = a1 if k == 2 else a0
    b = small_mod(b0 if k == 0 else b1, q, mf)
    bs = small_mod(b0, q, mf)
    if wd == 0:
        d = scale32(a, c) * b
        if k == 1:
            d += scale32(a1, c) * bs
        return addq(barrett32(d, c), ek, q)
    tr = wd == 1
    d = scale64(a, c, tr) * b
    if k == 1:
        d += scale64(a1, c, tr) * bs
    assert d < 1 << 128
    return addq(barrett64(d, c, tr), ek, q)


def expected(a0, a1, b0, b1, e, s, q):
    a0, a1, b0, b1 = a0 % q, a1 % q, b0 % q, b1 % q
    d = (a0 * b0, a0 * b1 + a1 * b0, a1 * b1)
    return [(dk * s + ek) % q for dk, ek in zip(d, e)]


def prime_below(bound, step=2):
    q = bound - 1
    while True:
        if q % 2 and all(pow(b, q - 1, q) == 1 for b in (2, 3, 5, 7, 11, 13)):
            return q
        q -= step


TWO_N = W.MIXED_TWO_N
# (q, word class): 0 = 32-bit words, 1 = 64-bit truncated, 2 = 64-bit exact
CASES = [
    (12289, 0),
    (W.ntt_primes(30, TWO_N, 1)[0], 0),
    (prime_below(1 << 30), 0),
    (W.ntt_primes(50, TWO_N, 1)[0], 1),
    (W.ntt_primes(60, TWO_N, 1)[0], 1),
    (prime_below(1 << 61), 1),
    (prime_below((1 << 61) + (1 << 40)), 2),
    (prime_below(1 << 62), 2),
]


def test_cases_cover_each_word_class():
    for q, wd in CASES:
        assert wd == (0 if q < 1 << 30 else 1 if q < 1 << 61 else 2)


@pytest.mark.parametrize("q,wd", CASES)
@pytest.mark.parametrize("mf", [1, 2, 4])
def test_fused_tensor_step_equals_its_definition(q, wd, mf):
    rng = random.Random(q * 7 + mf)
    hi = mf * q
    edge = [0, 1, q - 1, q, hi - 1, hi - q]
    for it in range(1500):
        s = rng.choice([0, 1, q - 1, rng.randrange(q)])
        c = consts(q, s)
        pick = (lambda: rng.choice(edge)) if it % 3 == 0 else (lambda: rng.randrange(hi))
        a0, a1, b0, b1 = (min(max(pick(), 0), hi - 1) for _ in range(4))
        e = [rng.choice([0, q - 1, rng.randrange(q)]) for _ in range(3)]
        want = expected(a0, a1, b0, b1, e, s, q)
        assert tensor_r3(a0, a1, b0, b1, e, c, mf, wd) == want
        for k in range(3):
            assert tensor_rk(k, a0, a1, b0, b1, e[k], c, mf, wd) == want[k]


@pytest.mark.parametrize("q,wd", CASES)
def test_fused_tensor_step_at_the_largest_operands(q, wd):
    """Every operand at its largest (4q - 1 raw, q - 1 reduced) and s = q - 1:
    the products and d1 at their maxima."""
    c = consts(q, q - 1)
    e = [q - 1] * 3
    for a in (4 * q - 1, 2 * q - 1, q - 1):
        want = expected(a, a, a, a, e, q - 1, q)
        assert tensor_r3(a, a, a, a, e, c, 4, wd) == want
        for k in range(3):
            assert tensor_rk(k, a, a, a, a, e[k], c, 4, wd) == want[k]


def mulmod_fused(a, b, c, wd):
    """The fused polynomial multiply's dyadic product on reduced operands."""
    assert a < c["q"] and b < c["q"]
    return barrett32(a * b, c) if wd == 0 else barrett64(a * b, c, wd == 1)


@pytest.mark.parametrize("q,wd", CASES)
def test_fused_dyadic_product_equals_its_definition(q, wd):
    rng = random.Random(q + 11)
    c = consts(q, 1)
    edge = [0, 1, q - 1, q // 2, rng.randrange(q)]
    for _ in range(5000):
        a = rng.choice(edge) if rng.random() < 0.2 else rng.randrange(q)
        b = rng.choice(edge) if rng.random() < 0.2 else rng.randrange(q)
        assert mulmod_fused(a, b, c, wd) == a * b % q
    assert mulmod_fused(q - 1, q - 1, c, wd) == 1
