"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds no arithmetic of the NTT method itself: it draws uniform
residues, picks NTT-friendly primes for the workloads and describes the five
workload shapes.  Both the CPU oracle and the CUDA library receive its output
as plain arrays and moduli; neither imports the other.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter form: the i-th
output of the stream keyed by ``k`` is ``mix(k + (i + 1) * GAMMA)``.  Values
uniform in [0, q) are drawn by mask-and-reject (mask to the bit length of q,
discard candidates >= q), so every accepted value is exactly uniform.

Moduli: primes q in [2^(b-1), 2^b) with q = 1 mod 2N, the smallest first
(Section 2 of the paper requires q prime and q = 1 mod 2N).  Primality uses
deterministic Miller-Rabin with the first twelve prime bases, exact for every
n < 3.3e24, so for every 64-bit n.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import lru_cache
from typing import List, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

#: seed of workload k is SEED_BASE + k
SEED_BASE = 0x5EED0000


# --------------------------------------------------------------------------
# SplitMix64, counter form
# --------------------------------------------------------------------------
def splitmix64_scalar(key: int, i: int) -> int:
    """i-th output (i >= 0) of the SplitMix64 stream whose state starts at key."""
    z = (key + (i + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def splitmix64_block(key: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the stream keyed by key (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = np.uint64(key & MASK64) + idx * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, *tags: int) -> int:
    """Derive an independent stream key from a seed and integer tags
    (e.g. polynomial and limb index) by chaining SplitMix64 outputs."""
    k = seed & MASK64
    for t in tags:
        k = splitmix64_scalar(k ^ (t & MASK64), 0)
    return k


def uniform_mod(key: int, n: int, q: int) -> np.ndarray:
    """n values uniform in [0, q) from the stream ``key`` (mask-and-reject)."""
    assert q >= 2
    mask = (1 << (q - 1).bit_length()) - 1
    out = np.empty(n, dtype=np.uint64)
    filled, pos = 0, 0
    while filled < n:
        want = max(64, (n - filled) * 2 + 64)
        cand = splitmix64_block(key, pos, want) & np.uint64(mask)
        pos += want
        ok = cand[cand < np.uint64(q)]
        take = min(len(ok), n - filled)
        out[filled:filled + take] = ok[:take]
        filled += take
    return out


def lazy_lift(key: int, x: np.ndarray, q: int, factor: int) -> np.ndarray:
    """Return x + k*q with k uniform in [0, factor), so that values in
    [0, factor*q) really occur (inputs for input_mod_factor > 1)."""
    if factor == 1:
        return x.copy()
    k = splitmix64_block(key, 0, len(x)) % np.uint64(factor)
    with np.errstate(over="ignore"):
        return x + k * np.uint64(q)


# --------------------------------------------------------------------------
# NTT-friendly primes
# --------------------------------------------------------------------------
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


@lru_cache(maxsize=None)
def ntt_primes(bits: int, two_n: int, count: int) -> Tuple[int, ...]:
    """The ``count`` smallest primes q in [2^(bits-1), 2^bits) with q = 1 mod two_n."""
    lo = 1 << (bits - 1)
    q = lo - (lo % two_n) + 1
    if q < lo:
        q += two_n
    out = []
    while len(out) < count:
        if q >= (1 << bits):
            raise ValueError(f"fewer than {count} {bits}-bit primes = 1 mod {two_n}")
        if is_prime(q):
            out.append(q)
        q += two_n
    return tuple(out)


#: one prime set serves every N <= 2^17 when q = 1 mod 2^18
MIXED_TWO_N = 1 << 18
WIDTHS = (30, 50, 60)


def mixed_width_primes(n_limbs: int, two_n: int = MIXED_TWO_N,
                       widths: Sequence[int] = WIDTHS) -> List[int]:
    """Limb l gets width widths[l % 3] and the (l // 3)-th smallest prime of
    that width (the mixed 30/50/60-bit RNS basis of the ciphertext workload)."""
    per = {w: ntt_primes(w, two_n, (n_limbs + len(widths) - 1) // len(widths) + 1)
           for w in widths}
    return [per[widths[l % len(widths)]][l // len(widths)] for l in range(n_limbs)]


# --------------------------------------------------------------------------
# Polynomial batches in the [poly][limb][N] layout
# --------------------------------------------------------------------------
def poly_batch(seed: int, tag: int, n_polys: int, moduli: Sequence[int], N: int,
               in_mf: int = 1) -> np.ndarray:
    """uint64 array [n_polys, n_limbs, N]; limb l uniform in [0, in_mf*q_l)."""
    L = len(moduli)
    out = np.empty((n_polys, L, N), dtype=np.uint64)
    for p in range(n_polys):
        for l, q in enumerate(moduli):
            key = stream_key(seed, tag, p, l)
            x = uniform_mod(key, N, q)
            if in_mf > 1:
                x = lazy_lift(stream_key(key, 0x11F7), x, q, in_mf)
            out[p, l] = x
    return out


def scalars(seed: int, tag: int, moduli: Sequence[int]) -> np.ndarray:
    """One uniform scalar in [0, q_l) per limb."""
    return np.array([int(uniform_mod(stream_key(seed, tag, l), 1, q)[0])
                     for l, q in enumerate(moduli)], dtype=np.uint64)


# --------------------------------------------------------------------------
# The five workload shapes
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    seed: int
    N: int
    moduli: List[int]
    n_polys: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def n_limbs(self) -> int:
        return len(self.moduli)


def single_ntt_1024() -> Workload:
    """N=1024, one 50-bit prime (the smallest = 1 mod 2048)."""
    return Workload("single_ntt_n1024_q50", SEED_BASE + 1, 1024,
                    list(ntt_primes(50, 2048, 1)), n_polys=2)


def rns_polymul_16384() -> Workload:
    """N=16384, 8 limbs: four 50-bit and four 60-bit primes = 1 mod 32768."""
    q = list(ntt_primes(50, 32768, 4)) + list(ntt_primes(60, 32768, 4))
    return Workload("rns_polymul_n16384_l8", SEED_BASE + 2, 16384, q, n_polys=2)


def ciphertext_tensor(N: int = 65536, n_limbs: int = 32) -> Workload:
    """Two ciphertexts of two polynomials each, 32 mixed 30/50/60-bit limbs."""
    return Workload(f"ciphertext_tensor_n{N}_l{n_limbs}", SEED_BASE + 3, N,
                    mixed_width_primes(n_limbs), n_polys=4)


def ragged_batch(n_polys: int = 512, seed: int = SEED_BASE + 4,
                 log_n_range=(10, 17), max_limbs: int = 32):
    """Ragged list of (N, moduli) entries: N uniform over 2^10..2^17, limb
    count uniform in 1..32, each limb's width uniform over {30, 50, 60}."""
    key = stream_key(seed, 0xBA7C)
    draws = splitmix64_block(key, 0, 3 * n_polys + 64 * n_polys)
    pool = {w: ntt_primes(w, MIXED_TWO_N, max_limbs) for w in WIDTHS}
    items = []
    d = 0
    for p in range(n_polys):
        lo, hi = log_n_range
        logn = lo + int(draws[d] % np.uint64(hi - lo + 1)); d += 1
        nl = 1 + int(draws[d] % np.uint64(max_limbs)); d += 1
        used = {w: 0 for w in WIDTHS}
        qs = []
        for _ in range(nl):
            w = WIDTHS[int(draws[d] % np.uint64(3))]; d += 1
            qs.append(pool[w][used[w]])
            used[w] += 1
        items.append((1 << logn, qs))
    return items
