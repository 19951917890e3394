"""Pins for the CPU oracle: each check ties it to something other than itself
(closed forms, exhaustive search, Python big integers, sympy, invariants of
the transform), so that a dropped term, a wrong sign or index or a swapped
operand anywhere in the oracle fails at least one test.  CPU only."""
import itertools

import numpy as np
import pytest
import sympy
from sympy.ntheory.residue_ntheory import nthroot_mod

import oracle
import workloads as W
from oracle import bigint

# (N, q) pairs with q = 1 mod 2N, small enough for exhaustive Python checks
TINY = [(2, 5), (4, 17), (8, 17), (8, 97), (16, 97), (16, 193), (32, 193),
        (32, 257), (64, 257), (64, 7681), (128, 7681)]
BIG_Q = [562949953443841, 576460752308273153, 537133057, 4611686018427322369]


def _rand(n, q, seed):
    return W.uniform_mod(W.stream_key(seed, n, q % 1000003), n, q)


# ---------------------------------------------------------------- scalars
def test_mulmod_edges_against_python_ints():
    for q in BIG_Q + [2, 3, (1 << 63) - 25, (1 << 64) - 59]:
        vals = [0, 1, 2, q - 1, q - 2, q // 2, (1 << 63) % q, (1 << 64) - 1]
        for a, b in itertools.product(vals, vals):
            assert oracle.mulmod(a, b, q) == (a * b) % q
    rng = np.random.default_rng(1)
    for _ in range(2000):
        q = int(rng.integers(2, 1 << 62)) | 1
        a, b = (int(x) for x in rng.integers(0, 1 << 63, size=2, dtype=np.uint64))
        assert oracle.mulmod(a, b, q) == (a * b) % q
        assert oracle.powmod(a, b, q) == pow(a, b, q)


def test_addsub_mod_against_python_ints():
    L = oracle.lib()
    for q in BIG_Q + [(1 << 63) - 25]:
        for a, b in itertools.product([0, 1, q - 1, 2 * q - 1, (1 << 64) - 1], repeat=2):
            assert L.oracle_addmod(a, b, q) == (a + b) % q
            assert L.oracle_submod(a, b, q) == (a - b) % q


def test_is_prime_matches_sympy():
    cands = list(range(0, 3000)) + [561, 1105, 1729, 2047, 3215031751,
                                    3825123056546413051, 318665857834031151167461 % (1 << 64)]
    cands += list(W.ntt_primes(60, 1 << 18, 3)) + [q + 2 for q in BIG_Q]
    for n in cands:
        assert oracle.is_prime(n) == sympy.isprime(n), n


def test_workload_primes_are_the_smallest():
    # smallest primes = 1 mod 2N in [2^(b-1), 2^b), checked with sympy
    for bits, two_n, count in [(50, 2048, 1), (50, 32768, 4), (60, 32768, 4),
                               (30, 1 << 18, 11), (50, 1 << 18, 3), (60, 1 << 18, 3)]:
        got = W.ntt_primes(bits, two_n, count)
        exp, q = [], ((1 << (bits - 1)) // two_n) * two_n + 1
        while len(exp) < count:
            if q >= (1 << (bits - 1)) and sympy.isprime(q):
                exp.append(q)
            q += two_n
        assert list(got) == exp


# ---------------------------------------------------------------- psi
@pytest.mark.parametrize("N,q", TINY)
def test_min_root_exhaustive(N, q):
    roots = bigint.primitive_2n_roots(N, q)
    assert len(roots) == N
    assert oracle.min_primitive_root(N, q) == min(roots)


@pytest.mark.parametrize("N,q", [(1024, 562949953443841), (16384, 562949954142209),
                                 (16384, 576460752304439297), (65536, 537133057),
                                 (131072, 576460752315482113)])
def test_min_root_matches_sympy(N, q):
    roots = nthroot_mod(q - 1, N, q, all_roots=True)
    assert len(roots) == N
    assert oracle.min_primitive_root(N, q) == min(roots)


def test_min_root_rejects_bad_inputs():
    assert oracle.min_primitive_root(1000, 562949953443841) == 0
    assert oracle.min_primitive_root(1024, 562949953443841 + 2048) == 0 or \
        not sympy.isprime(562949953443841 + 2048)
    assert oracle.min_primitive_root(4096, 562949953443841) == 0   # q != 1 mod 8192


def test_bitrev_powers_table():
    N, q = 64, 7681
    psi = oracle.min_primitive_root(N, q)
    t = oracle.bitrev_powers(N, q, psi)
    assert t[0] == 1
    for k in range(1, N):
        assert int(t[k]) == pow(psi, bigint.bitrev(k, 6), q)


# ---------------------------------------------------------------- forward NTT
@pytest.mark.parametrize("N,q", TINY)
def test_forward_equals_closed_form_tiny(N, q):
    psi = oracle.min_primitive_root(N, q)
    for seed in range(3):
        a = _rand(N, q, seed)
        got = [int(x) for x in oracle.ntt_forward_1(a, q)]
        assert got == bigint.negacyclic_ntt_bitrev([int(x) for x in a], q, psi)


@pytest.mark.parametrize("q", BIG_Q[:3])
def test_forward_equals_closed_form_bigq(q):
    for N in (2, 8, 32):
        if (q - 1) % (2 * N):
            continue
        psi = oracle.min_primitive_root(N, q)
        a = _rand(N, q, 7)
        got = [int(x) for x in oracle.ntt_forward_1(a, q)]
        assert got == bigint.negacyclic_ntt_bitrev([int(x) for x in a], q, psi)


def test_closed_form_evaluator_matches_bigint():
    N, q = 32, 257
    psi = oracle.min_primitive_root(N, q)
    a = _rand(N, q, 3)
    got = oracle.ntt_forward_direct(a, q, psi, list(range(N)))
    assert [int(x) for x in got] == bigint.negacyclic_ntt_bitrev([int(x) for x in a], q, psi)


def test_forward_matches_closed_form_n1024_full():
    q = W.ntt_primes(50, 2048, 1)[0]
    N = 1024
    psi = oracle.min_primitive_root(N, q)
    a = _rand(N, q, 11)
    np.testing.assert_array_equal(oracle.ntt_forward_1(a, q),
                                  oracle.ntt_forward_direct(a, q, psi, np.arange(N)))


def test_forward_spot_checks_n65536():
    q = W.ntt_primes(60, 1 << 18, 1)[0]
    N = 1 << 16
    psi = oracle.min_primitive_root(N, q)
    a = _rand(N, q, 12)
    out = oracle.ntt_forward_1(a, q)
    idx = [0, 1, 2, 3, 255, 4096, 32767, 32768, 65534, 65535]
    np.testing.assert_array_equal(out[idx], oracle.ntt_forward_direct(a, q, psi, idx))


def test_forward_special_inputs():
    N, q = 256, 7681 * 0 + W.ntt_primes(50, 512, 1)[0]
    psi = oracle.min_primitive_root(N, q)
    delta = np.zeros(N, dtype=np.uint64); delta[0] = 1
    assert np.all(oracle.ntt_forward_1(delta, q) == 1)           # NTT(1) = 1
    c = 123456789
    assert np.all(oracle.ntt_forward_1(delta * np.uint64(c), q) == c)
    x = np.zeros(N, dtype=np.uint64); x[1] = 1                    # NTT(X)
    got = oracle.ntt_forward_1(x, q)
    exp = [pow(psi, 2 * bigint.bitrev(i, 8) + 1, q) for i in range(N)]
    assert [int(v) for v in got] == exp


def test_forward_linearity_and_lazy_inputs():
    N, q = 1024, W.ntt_primes(50, 2048, 1)[0]
    a, b = _rand(N, q, 21), _rand(N, q, 22)
    s = 987654321
    lhs = oracle.ntt_forward_1((a.astype(object) * s + b.astype(object)) % q, q)
    rhs = (oracle.ntt_forward_1(a, q).astype(object) * s
           + oracle.ntt_forward_1(b, q).astype(object)) % q
    assert [int(x) for x in lhs] == [int(x) for x in rhs]
    # inputs in [0, 4q) transform as their residues
    lifted = W.lazy_lift(5, a, q, 4)
    assert lifted.max() >= q
    np.testing.assert_array_equal(oracle.ntt_forward_1(lifted, q), oracle.ntt_forward_1(a, q))


# ---------------------------------------------------------------- inverse NTT
@pytest.mark.parametrize("N,q", TINY)
def test_inverse_is_inverse_tiny(N, q):
    a = _rand(N, q, 4)
    np.testing.assert_array_equal(oracle.ntt_inverse_1(oracle.ntt_forward_1(a, q), q), a)
    np.testing.assert_array_equal(oracle.ntt_forward_1(oracle.ntt_inverse_1(a, q), q), a)


@pytest.mark.parametrize("N,q", [(1024, 562949953443841), (16384, 576460752304439297),
                                 (65536, 537133057), (131072, 562949964955649)])
def test_inverse_is_inverse_large(N, q):
    a = _rand(N, q, 5)
    np.testing.assert_array_equal(oracle.ntt_inverse_1(oracle.ntt_forward_1(a, q), q), a)


def test_inverse_equals_cyclic_definition_tiny():
    # InvNTT of a bit-reversed spectrum = psi^-i * cyclic InvNTT (Section 2.2)
    for N, q in TINY:
        psi = oracle.min_primitive_root(N, q)
        logn = N.bit_length() - 1
        A = [int(x) for x in _rand(N, q, 6)]
        spectrum = [0] * N
        for i in range(N):
            spectrum[bigint.bitrev(i, logn)] = A[i]
        c = bigint.cyclic_intt(spectrum, q, psi * psi % q)
        psi_inv = pow(psi, -1, q)
        exp = [c[i] * pow(psi_inv, i, q) % q for i in range(N)]
        got = [int(x) for x in oracle.ntt_inverse_1(np.array(A, dtype=np.uint64), q)]
        assert got == exp


# ---------------------------------------------------------------- products
@pytest.mark.parametrize("N,q", TINY)
def test_polymul_equals_schoolbook_tiny(N, q):
    a, b = _rand(N, q, 8), _rand(N, q, 9)
    exp = bigint.negacyclic_product([int(x) for x in a], [int(x) for x in b], q)
    got = oracle.poly_mul(a[None, None], b[None, None], [q])[0, 0]
    assert [int(x) for x in got] == exp
    psi = oracle.min_primitive_root(N, q)
    assert bigint.negacyclic_product_via_twist([int(x) for x in a], [int(x) for x in b],
                                               q, psi) == exp


def test_schoolbook_c_matches_bigint():
    N, q = 64, 7681
    a, b = _rand(N, q, 10), _rand(N, q, 11)
    assert [int(x) for x in oracle.negacyclic_schoolbook(a, b, q)] == \
        bigint.negacyclic_product([int(x) for x in a], [int(x) for x in b], q)


@pytest.mark.parametrize("N,q", [(1024, 562949953443841), (4096, 576460752308273153)])
def test_polymul_equals_schoolbook_full(N, q):
    a, b = _rand(N, q, 12), _rand(N, q, 13)
    got = oracle.poly_mul(a[None, None], b[None, None], [q])[0, 0]
    np.testing.assert_array_equal(got, oracle.negacyclic_schoolbook(a, b, q))


def test_polymul_by_monomial_is_negacyclic_shift():
    N, q = 1024, 562949953443841
    a = _rand(N, q, 14)
    for k in (1, 5, 1023):
        xk = np.zeros(N, dtype=np.uint64); xk[k] = 1
        got = oracle.poly_mul(a[None, None], xk[None, None], [q])[0, 0]
        exp = np.empty(N, dtype=object)
        for i in range(N):
            j = i - k
            exp[i] = int(a[j]) if j >= 0 else (q - int(a[j + N])) % q
        assert [int(x) for x in got] == list(exp)


# ---------------------------------------------------------------- eltwise
def test_eltwise_against_python_ints():
    for q in BIG_Q[:3] + [(1 << 61) - 1]:
        n = 257
        a, b = _rand(n, q, 15), _rand(n, q, 16)
        a4 = W.lazy_lift(1, a, q, 4)
        s = 1234567 % q
        ai, bi, a4i = ([int(x) for x in v] for v in (a, b, a4))
        assert [int(x) for x in oracle.eltwise_add_mod_1(a, b, q)] == [(x + y) % q for x, y in zip(ai, bi)]
        assert [int(x) for x in oracle.eltwise_sub_mod_1(a, b, q)] == [(x - y) % q for x, y in zip(ai, bi)]
        assert [int(x) for x in oracle.eltwise_mult_mod_1(a4, b, q)] == [(x * y) % q for x, y in zip(a4i, bi)]
        assert [int(x) for x in oracle.eltwise_fma_mod_1(a4, s, b, q)] == [(x * s + y) % q for x, y in zip(a4i, bi)]
        assert [int(x) for x in oracle.eltwise_fma_mod_1(a4, s, None, q)] == [(x * s) % q for x in a4i]


def test_ciphertext_tensor_equals_schoolbook_products():
    N, moduli = 64, [7681, 12289, W.ntt_primes(50, 1 << 18, 1)[0]]
    seed = 33
    a0, a1, b0, b1, e0, e1, e2 = (W.poly_batch(seed, t, 1, moduli, N) for t in range(7))
    s = W.scalars(seed, 99, moduli)
    r0, r1, r2 = oracle.ciphertext_tensor(a0, a1, b0, b1, s, e0, e1, e2, moduli)
    for l, q in enumerate(moduli):
        P = lambda x, y: np.array(bigint.negacyclic_product(
            [int(v) for v in x[0, l]], [int(v) for v in y[0, l]], q), dtype=object)
        E = lambda e: np.array([int(v) for v in oracle.ntt_inverse_1(e[0, l], q)], dtype=object)
        sl = int(s[l])
        exp0 = (P(a0, b0) * sl + E(e0)) % q
        exp1 = ((P(a0, b1) + P(a1, b0)) * sl + E(e1)) % q
        exp2 = (P(a1, b1) * sl + E(e2)) % q
        assert [int(x) for x in r0[0, l]] == list(exp0)
        assert [int(x) for x in r1[0, l]] == list(exp1)
        assert [int(x) for x in r2[0, l]] == list(exp2)


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes():
    """Corrupt the oracle's own tables (a wrong twiddle, swapped entries, the
    non-inverse root) and check that the pins above would fail."""
    N, q = 32, 257
    psi = oracle.min_primitive_root(N, q)
    T = oracle.tables(N, q)
    a = [int(x) for x in _rand(N, q, 17)]
    ref = bigint.negacyclic_ntt_bitrev(a, q, psi)
    arr = np.array(a, dtype=np.uint64)
    bad = T.psi_rev.copy(); bad[5] = (int(bad[5]) + 1) % q                 # wrong twiddle
    assert [int(x) for x in oracle.ntt_forward_1(arr, q, psi_rev=bad)] != ref
    bad = T.psi_rev.copy(); bad[[3, 4]] = bad[[4, 3]]                      # index swap
    assert [int(x) for x in oracle.ntt_forward_1(arr, q, psi_rev=bad)] != ref
    fwd = oracle.ntt_forward_1(arr, q)
    wrong_inv = oracle.ntt_inverse_1(fwd, q, psiinv_rev=T.psi_rev)        # psi for psi^-1
    assert not np.array_equal(wrong_inv, arr)
    bad = T.psi_rev.copy(); bad[1:] = T.psi_rev[::-1][:-1]                 # reversed table
    assert [int(x) for x in oracle.ntt_forward_1(arr, q, psi_rev=bad)] != ref


# ---------------------------------------------------------------- negation
def test_negate_against_definition_and_invariants():
    """(q - a) mod q: 0 stays 0; a + (-a) = 0 and -(-a) = a through the
    oracle's own addition; values match Python integers."""
    for q in BIG_Q + [3, 97]:
        a = np.concatenate([np.array([0, 1, q - 1, q // 2], dtype=np.uint64),
                            _rand(500, q, 41)])
        na = oracle.eltwise_negate_mod_1(a, q)
        assert [int(x) for x in na] == [(q - int(x)) % q for x in a]
        assert int(na[0]) == 0 and int(na[2]) == 1
        assert not oracle.eltwise_add_mod_1(a, na, q).any()
        np.testing.assert_array_equal(oracle.eltwise_negate_mod_1(na, q), a)


# ---------------------------------------------------------------- cyclic NTT
CYC = [(2, 3), (4, 5), (8, 17), (16, 97), (32, 97), (64, 193), (128, 257), (256, 7681)]


@pytest.mark.parametrize("N,q", CYC)
def test_min_nth_root_exhaustive(N, q):
    """Against a brute-force search over Z_q for elements of order exactly N."""
    order_n = [x for x in range(1, q) if pow(x, N, q) == 1 and
               all(pow(x, d, q) != 1 for d in sympy.divisors(N) if d < N)]
    assert oracle.min_primitive_nth_root(N, q) == min(order_n)


def test_min_nth_root_rejects_bad_inputs():
    assert oracle.min_primitive_nth_root(16, 96) == 0      # not prime
    assert oracle.min_primitive_nth_root(16, 23) == 0      # 16 does not divide 22
    assert oracle.min_primitive_nth_root(12, 13) == 0      # N not a power of two


@pytest.mark.parametrize("N,q", CYC[2:])
def test_cyclic_special_inputs(N, q):
    """NTT(delta_0) = all ones, NTT(all ones) = N delta_0 (the geometric sums
    of a primitive N-th root vanish), NTT(X) = (omega^i)_i."""
    w = oracle.min_primitive_nth_root(N, q)
    delta = np.zeros(N, dtype=np.uint64); delta[0] = 1
    assert (oracle.cyclic_ntt_1(delta, q, w) == 1).all()
    ones = np.ones(N, dtype=np.uint64)
    got = oracle.cyclic_ntt_1(ones, q, w)
    assert int(got[0]) == N % q and not got[1:].any()
    x = np.zeros(N, dtype=np.uint64); x[1] = 1
    assert [int(v) for v in oracle.cyclic_ntt_1(x, q, w)] == [pow(w, i, q) for i in range(N)]


@pytest.mark.parametrize("N,q", [(64, 193), (256, 7681), (1024, 562949953443841),
                                 (512, 576460752308273153)])
def test_cyclic_inverse_and_convolution_theorem(N, q):
    """InvNTT(NTT(a)) = a, and InvNTT(NTT(a) . NTT(b)) is the product in
    Z_q[X] / (X^N - 1) (Section 2.2), against the cyclic schoolbook."""
    w = oracle.min_primitive_nth_root(N, q)
    a, b = _rand(N, q, 51), _rand(N, q, 52)
    fa, fb = oracle.cyclic_ntt_1(a, q, w), oracle.cyclic_ntt_1(b, q, w)
    np.testing.assert_array_equal(oracle.cyclic_intt_1(fa, q, w), a)
    prod = oracle.cyclic_intt_1(oracle.eltwise_mult_mod_1(fa, fb, q), q, w)
    np.testing.assert_array_equal(prod, oracle.cyclic_schoolbook(a, b, q))


def test_cyclic_schoolbook_monomial_is_rotation():
    """a * X^k in Z_q[X] / (X^N - 1) rotates the coefficients, with no sign
    change (unlike the negacyclic ring)."""
    N, q = 128, 7681
    a = _rand(N, q, 53)
    for k in (0, 1, 5, 127):
        x = np.zeros(N, dtype=np.uint64); x[k] = 1
        np.testing.assert_array_equal(oracle.cyclic_schoolbook(a, x, q), np.roll(a, k))


@pytest.mark.parametrize("N,q", [(16, 97), (256, 7681), (1024, 562949953443841)])
def test_cyclic_is_the_untwisted_negacyclic(N, q):
    """With psi a primitive 2N-th root and omega = psi^2, the cyclic NTT of a
    read in bit-reversed order equals the (separately pinned) negacyclic NTT
    of the twisted input a_j psi^-j."""
    psi = oracle.min_primitive_root(N, q)
    w = psi * psi % q
    a = _rand(N, q, 54)
    pinv = oracle.invmod(psi, q)
    tw = np.array([int(a[j]) * pow(pinv, j, q) % q for j in range(N)], dtype=np.uint64)
    neg = oracle.ntt_forward_1(tw, q, psi)
    cyc = oracle.cyclic_ntt_1(a, q, w)
    logn = N.bit_length() - 1
    brv = [int(format(i, f"0{logn}b")[::-1], 2) for i in range(N)]
    np.testing.assert_array_equal(neg, cyc[brv])
    # planted mistakes: the inverse root, or a root of order N/2, break it
    assert not np.array_equal(neg, oracle.cyclic_ntt_1(a, q, oracle.invmod(w, q))[brv])
    assert not np.array_equal(neg, oracle.cyclic_ntt_1(a, q, w * w % q)[brv])
