"""Pure-Python big-integer definitions for tiny N (test infrastructure only).

Written from the definitions of Section 2 alone, with no transform
algorithm, so that they pin the C oracle independently:
  * ``negacyclic_product``: the vector-vector multiplication formula
    c_i = sum_{j<=i} a_j b_{i-j} - sum_{j>i} a_j b_{N+i-j} (Section 2).
  * ``cyclic_ntt`` / ``cyclic_intt``: the cyclic NTT and its inverse with the
    1/N factor (Section 2.2).
  * ``negacyclic_ntt_bitrev``: cyclic NTT (omega = psi^2) of the psi-twisted
    input, read at bit-reversed positions (Section 2.2, negative wrapped
    convolution and bit-reversed output order).
  * ``primitive_2n_roots``: every x in Z_q whose multiplicative order is 2N,
    by exhaustive search (tiny q only).
"""
from __future__ import annotations

from typing import List, Sequence


def bitrev(i: int, logn: int) -> int:
    return int(format(i, f"0{logn}b")[::-1], 2) if logn else 0


def negacyclic_product(a: Sequence[int], b: Sequence[int], q: int) -> List[int]:
    N = len(a)
    out = []
    for i in range(N):
        pos = sum(a[j] * b[i - j] for j in range(i + 1))
        neg = sum(a[j] * b[N + i - j] for j in range(i + 1, N))
        out.append((pos - neg) % q)
    return out


def cyclic_ntt(a: Sequence[int], q: int, omega: int) -> List[int]:
    N = len(a)
    return [sum(a[j] * pow(omega, i * j, q) for j in range(N)) % q for i in range(N)]


def cyclic_intt(a: Sequence[int], q: int, omega: int) -> List[int]:
    N = len(a)
    n_inv = pow(N, -1, q)
    w_inv = pow(omega, -1, q)
    return [n_inv * sum(a[j] * pow(w_inv, i * j, q) for j in range(N)) % q
            for i in range(N)]


def negacyclic_ntt_bitrev(a: Sequence[int], q: int, psi: int) -> List[int]:
    """NTT(a_hat) with a_hat_j = psi^j a_j and omega = psi^2, output index i
    holding the transform at position brv(i)."""
    N = len(a)
    logn = N.bit_length() - 1
    twisted = [a[j] * pow(psi, j, q) % q for j in range(N)]
    spectrum = cyclic_ntt(twisted, q, psi * psi % q)
    return [spectrum[bitrev(i, logn)] for i in range(N)]


def negacyclic_product_via_twist(a, b, q, psi):
    """c = psi^-i * InvNTT(NTT(a_hat) . NTT(b_hat)) (Section 2.2)."""
    N = len(a)
    omega = psi * psi % q
    ah = [a[j] * pow(psi, j, q) % q for j in range(N)]
    bh = [b[j] * pow(psi, j, q) % q for j in range(N)]
    A, B = cyclic_ntt(ah, q, omega), cyclic_ntt(bh, q, omega)
    c = cyclic_intt([x * y % q for x, y in zip(A, B)], q, omega)
    psi_inv = pow(psi, -1, q)
    return [c[i] * pow(psi_inv, i, q) % q for i in range(N)]


def multiplicative_order(x: int, q: int) -> int:
    k, y = 1, x % q
    while y != 1:
        y = y * x % q
        k += 1
    return k


def primitive_2n_roots(N: int, q: int) -> List[int]:
    return [x for x in range(1, q) if multiplicative_order(x, q) == 2 * N]
