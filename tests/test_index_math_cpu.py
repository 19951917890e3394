"""The NTT pass kernels' index arithmetic, restated on the host and checked
against the definitions (no GPU).

A pass over stages [s0, s0 + K) cuts the transform into tiles of
2^logGb x 2^K x 2^logGc elements; a block of TE / 2^logR threads runs the K
stages as register rounds (`Sched`), each thread holding 2^logR elements.
The restatement follows the kernel's own formulas -- the group bits of a
thread (bl | e_hi | e_lo | cl), its tile-local base `lbase`, the local to
global map `tile_gidx`, the register strides `sshift`/`gshift`, the padded
shared-memory position `pad`, the twiddle index `hp << k` and the staged
twiddle layout -- and the tests check what the kernel relies on:
  * every tile covers its elements once and the tiles cover [0, N) once;
  * in every round each local element sits in exactly one (thread, register);
  * a register's global address is the thread's base address plus
    v << gshift, and its shared-memory slot pad(base) + pad_off(v, sshift)
    equals pad(local index) (the compile-time offsets the kernel uses);
  * every butterfly pairs x with x + N / 2^(s+1) at stage s and reads
    twiddle 2^s + floor(x / (N / 2^s)) -- Algorithm CT's loop (and Algorithm
    GS's, which visits the same pairs in reverse stage order);
  * twiddle indices fit the kernel's 32-bit arithmetic;
  * the staged-twiddle copy fills distinct in-range slots and every staged
    read returns the twiddle the butterfly needs;
and, end to end, a transform computed with exactly these maps (plain
modular arithmetic) equals the oracle's."""
import numpy as np
import pytest

import oracle
import workloads as W


def sched(K, logR):
    """Sched<K, LOG_R>: ceil(K / logR) rounds of near-equal size."""
    nr = (K + logR - 1) // logR
    size = [K // nr + (1 if i < K % nr else 0) for i in range(nr)]
    off = [sum(size[:i]) for i in range(nr)]
    return size, off


def pad(l):
    return l + (l >> 4)


def pad_off(v, s):
    return (v << s) + ((v << s) >> 4)


class Pass:
    def __init__(self, L, s0, K, logGb, logGc, logR):
        self.L, self.s0, self.K, self.logGb, self.logGc, self.logR = L, s0, K, logGb, logGc, logR
        self.w = L - s0 - K
        self.column = logGc > 0
        self.row = not self.column             # the kernel's ROW template argument
        self.logTE = logGb + K + logGc
        self.T = 1 << (self.logTE - logR)
        self.log_tiles_c = self.w - logGc

    def tiles(self):
        for tile in range(1 << (self.L - self.logTE)):
            tile_c = tile & ((1 << self.log_tiles_c) - 1)
            tile_b = tile >> self.log_tiles_c
            yield tile_b << self.logGb, tile_c << self.logGc

    def gidx(self, l, b_base, c_base):
        """tile_gidx<K, ROW>."""
        if self.row or self.w == 0:
            return (b_base << self.K) + l
        cl = l & ((1 << self.logGc) - 1)
        rho = l >> self.logGc
        e = rho & ((1 << self.K) - 1)
        bl = rho >> self.K
        return ((b_base + bl) << (self.L - self.s0)) + (e << self.w) + c_base + cl

    def rounds(self):
        size, off = sched(self.K, self.logR)
        return list(zip(off, size))

    def groups(self, P, R, b_base):
        """Per (u, thread): lbase, hp, hiu as the round computes them."""
        U, ELO = 1 << (self.logR - R), self.K - P - R
        for u in range(U):
            for tid in range(self.T):
                g = u * self.T + tid
                cl = g & ((1 << self.logGc) - 1)
                t1 = g >> self.logGc
                elo = t1 & ((1 << ELO) - 1)
                t2 = t1 >> ELO
                ehi = t2 & ((1 << P) - 1)
                bl = t2 >> P
                lbase = ((bl << (self.K + self.logGc)) | (ehi << (self.K - P + self.logGc))
                         | (elo << self.logGc) | cl)
                hp = (1 << (self.s0 + P)) | (((b_base + bl) << P) & 0xffffffff) | ehi
                hiu = (bl << P) | ehi
                yield u, tid, lbase, hp, hiu

    def shifts(self, P, R):
        ELO = self.K - P - R
        return (ELO, ELO) if self.row else (ELO + self.logGc, ELO + self.w)


def shapes(Ls=(10, 12, 14, 16, 17)):
    """Pass shapes of one- and two-pass schedules within the kernels' limits
    (32 to 1024 threads a block)."""
    out = []
    for L in Ls:
        cands = []
        if L <= 13:
            cands += [(0, L, 0, 0, r) for r in (2, 3, 4)]
        for K1 in range(6, 10):
            K2 = L - K1
            if not 6 <= K2 <= 13:
                continue
            cands += [(0, K1, 0, g, r) for g in (2, 3, 4, 5) for r in (3, 4) if g <= K2]
            cands += [(K1, K2, b, 0, r) for b in range(0, 6) for r in (3, 4) if b <= K1]
        for s0, K, b, g, r in cands:
            p = Pass(L, s0, K, b, g, r)
            if 32 <= p.T <= 1024 and max(sched(K, r)[0]) <= r:
                out.append(p)
    return out


SHAPES = shapes()
SAMPLE = SHAPES[::7]          # every shape is checked by the cheap tests, a sample by the rest


@pytest.mark.parametrize("p", SAMPLE, ids=lambda p: f"L{p.L}s{p.s0}K{p.K}b{p.logGb}c{p.logGc}r{p.logR}")
def test_tiles_cover_the_transform_once(p):
    seen = np.zeros(1 << p.L, np.int32)
    TE = 1 << p.logTE
    for b_base, c_base in p.tiles():
        g = [p.gidx(l, b_base, c_base) for l in range(TE)]
        assert len(set(g)) == TE
        seen[g] += 1
    assert (seen == 1).all()


@pytest.mark.parametrize("p", SAMPLE, ids=lambda p: f"L{p.L}s{p.s0}K{p.K}b{p.logGb}c{p.logGc}r{p.logR}")
def test_rounds_registers_butterflies_and_twiddles(p):
    N, L = 1 << p.L, p.L
    TE = 1 << p.logTE
    tiles = list(p.tiles())
    for b_base, c_base in (tiles[0], tiles[-1], tiles[len(tiles) // 2]):
        for P, R in p.rounds():
            sshift, gshift = p.shifts(P, R)
            owner = np.zeros(TE, np.int32)
            for u, tid, lbase, hp, hiu in p.groups(P, R, b_base):
                assert hp < 1 << 32 and (hp << (R - 1)) < 1 << 32
                g0 = p.gidx(lbase, b_base, c_base)
                for v in range(1 << R):
                    l = lbase + (v << sshift)
                    owner[l] += 1
                    assert p.gidx(l, b_base, c_base) == g0 + (v << gshift)
                    assert pad(lbase) + pad_off(v, sshift) == pad(l)
                for k in range(R):
                    s = p.s0 + P + k
                    t = N >> (s + 1)
                    for v in range(1 << R):
                        if v & (1 << (R - 1 - k)):
                            continue
                        x = p.gidx(lbase + (v << sshift), b_base, c_base)
                        y = p.gidx(lbase + ((v | (1 << (R - 1 - k))) << sshift), b_base, c_base)
                        assert y - x == t
                        tw = ((hp << k) & 0xffffffff) + (v >> (R - k))
                        assert tw == (1 << s) + (x >> (L - s))
            assert (owner == 1).all()


@pytest.mark.parametrize("p", SAMPLE, ids=lambda p: f"L{p.L}s{p.s0}K{p.K}b{p.logGb}c{p.logGc}r{p.logR}")
def test_staged_twiddles_layout(p):
    """stage_twiddles' copy and the staged reads of the rounds."""
    size, off = sched(p.K, p.logR)
    lgb = p.logGb
    tiles = list(p.tiles())
    for b_base, _ in (tiles[0], tiles[-1]):
        slot = {}
        cap = ((1 << p.K) - 1) << lgb
        for q in range(p.K):
            P = max(o for o in off if q >= o)
            k = q - P
            src = (1 << (p.s0 + q)) + (b_base << q)
            dst = ((1 << q) - 1) << lgb
            for i in range(1 << (lgb + q)):
                pos = dst + ((i & ((1 << k) - 1)) << (lgb + P)) + (i >> k)
                assert 0 <= pos < cap and pos not in slot
                slot[pos] = src + i
        for P, R in p.rounds():
            for u, tid, lbase, hp, hiu in p.groups(P, R, b_base):
                for k in range(R):
                    base = (((1 << (P + k)) - 1) << lgb) + hiu
                    for v in range(0, 1 << R, 1 << (R - k)):
                        j = v >> (R - k)
                        assert slot[base + (j << (lgb + P))] == ((hp << k) & 0xffffffff) + j


def test_every_shape_keeps_its_invariants_on_one_tile():
    """The cheap invariants on the first tile of every shape."""
    for p in SHAPES:
        b_base, c_base = next(p.tiles())
        for P, R in p.rounds():
            sshift, gshift = p.shifts(P, R)
            for u, tid, lbase, hp, hiu in p.groups(P, R, b_base):
                g0 = p.gidx(lbase, b_base, c_base)
                for v in range(1 << R):
                    l = lbase + (v << sshift)
                    assert p.gidx(l, b_base, c_base) == g0 + (v << gshift)
                    assert pad(lbase) + pad_off(v, sshift) == pad(l)
    assert len(SHAPES) > 100


@pytest.mark.parametrize("L,split", [(10, None), (12, (7, 4, 0, 3, 3)), (12, (6, 3, 1, 0, 4))])
def test_transform_with_these_maps_equals_the_oracle(L, split):
    """Runs the forward transform pass by pass, round by round, register by
    register through the maps above (exact modular arithmetic) and compares
    with the oracle."""
    N, q = 1 << L, W.ntt_primes(50, 1 << (L + 1), 1)[0]
    psi = oracle.min_primitive_root(N, q)
    rev = [int(format(i, f"0{L}b")[::-1], 2) for i in range(N)]
    W_ = [pow(psi, rev[i], q) for i in range(N)]
    x = [int(v) for v in W.poly_batch(W.SEED_BASE + 990, 0, 1, [q], N)[0, 0]]
    if split is None:
        passes = [Pass(L, 0, L, 0, 0, 3)]
    else:
        K1, logGc, logGb, _, logR = split
        passes = [Pass(L, 0, K1, 0, logGc, 4), Pass(L, K1, L - K1, logGb, 0, logR)]
    for p in passes:
        for b_base, c_base in p.tiles():
            for P, R in p.rounds():
                sshift, _ = p.shifts(P, R)
                for u, tid, lbase, hp, hiu in p.groups(P, R, b_base):
                    for k in range(R):
                        for v in range(1 << R):
                            if v & (1 << (R - 1 - k)):
                                continue
                            xi = p.gidx(lbase + (v << sshift), b_base, c_base)
                            yi = p.gidx(lbase + ((v | (1 << (R - 1 - k))) << sshift),
                                        b_base, c_base)
                            w = W_[((hp << k) & 0xffffffff) + (v >> (R - k))]
                            a, b = x[xi], x[yi] * w % q
                            x[xi], x[yi] = (a + b) % q, (a - b) % q
    exp = oracle.ntt_forward_1(W.poly_batch(W.SEED_BASE + 990, 0, 1, [q], N)[0, 0], q)
    np.testing.assert_array_equal(np.array(x, dtype=np.uint64), exp)


# The ragged kernels' fixed menu (2048-element tiles; 1024 for N = 2^10):
# log2 N -> (first pass K, column?), (second pass K) as rag_kinds() picks them.
RAG_KINDS = {10: ((10, False), None), 11: ((11, False), None), 12: ((5, True), 7),
             13: ((6, True), 7), 14: ((7, True), 7), 15: ((7, True), 8), 16: ((8, True), 8),
             17: ((8, True), 9)}


def rag_pass(L, K, column):
    """rag_tile's geometry for a menu entry (S10 runs 4 elements a thread)."""
    s0 = 0 if column or K >= L else L - K
    logGc = 11 - K if column else 0
    logGb = 0 if column else (0 if K >= L else 11 - K)
    return Pass(L, s0, K, logGb, logGc, 2 if K == 10 else 3)


@pytest.mark.parametrize("L", range(10, 18))
def test_ragged_menu_passes(L):
    (K1, column), K2 = RAG_KINDS[L]
    passes = [rag_pass(L, K1, column)] + ([rag_pass(L, K2, False)] if K2 else [])
    assert sum(p.K for p in passes) == L
    for p in passes:
        assert p.logTE == min(L, 11) and p.T == 256     # 256 threads, 2048 elements (1024 at 2^10)
        test_tiles_cover_the_transform_once(p)
        test_rounds_registers_butterflies_and_twiddles(p)


@pytest.mark.parametrize("logTE", range(8, 13))
@pytest.mark.parametrize("tiles", [2, 4])
def test_step_kernels_element_wise_step_covers_each_tile_once(logTE, tiles):
    """The step kernels' element-wise step (the tensor, or the product): with
    8 elements a thread and TE >> 3 threads, thread t at step it handles
    positions 2i and 2i + 1, i = t + it * threads, it < 4, reading and
    writing tile k at k * padded(TE) + pad(2i) (+ 1): every position of every
    tile exactly once, inside its own tile, with the pair in one 16-word row
    (pad(2i) + 1 = pad(2i + 1))."""
    TE = 1 << logTE
    threads = TE >> 3
    padded = TE + TE // 16
    seen = [set() for _ in range(tiles)]
    for t in range(threads):
        for it in range(4):
            i = t + it * threads
            l = pad(2 * i)
            assert l + 1 == pad(2 * i + 1) and l + 1 < padded
            for k in range(tiles):
                for h in (0, 1):
                    off = k * padded + l + h
                    assert k * padded <= off < (k + 1) * padded
                    assert 2 * i + h not in seen[k]
                    seen[k].add(2 * i + h)
    assert all(s == set(range(TE)) for s in seen)
