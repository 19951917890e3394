"""The cluster-fused transform's index arithmetic (ntt_cluster.cuh), restated
on the host and checked against the definitions (no GPU).

A cluster of C = 2^logC CTAs transforms one limb of N = 2^K1 x 2^K2 points:
CTA k holds, in its column phase, the column-pass tile with c_base =
k 2^logGc (logGc = K2 - logC) and, in its row phase, the row-pass tile with
b_base = k 2^logGb (logGb = K1 - logC); both are N / C elements in a padded
shared-memory array.  The exchange round reads element l of its new tile
from CTA `owner` at padded position pad(rl) (exchange_load).  Checked here:
  * the grid: cluster c = blockIdx.x >> logC covers polynomial c, rank =
    blockIdx.x mod C, and the C CTAs' tiles cover [0, N) once in each phase;
  * every exchange read stays in the cluster (owner < C) and inside the
    owner's tile (pad(rl) < padded(N / C)), and fetches exactly the element
    the owner's other phase left there (same global index);
  * the staged row tiles (16-byte copies in and out) stay in [0, N);
and, end to end, the forward and the inverse transform run CTA by CTA,
round by round, through per-CTA shared-memory arrays and the exchange map
(exact modular arithmetic, Algorithm CT / Algorithm GS order) equal the
oracle's."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_index_math_cpu import Pass, pad, sched

# the (K1, K2) pairs the library instantiates (HX_CLUSTER_MENU)
MENU = [(6, 8), (7, 7), (8, 6), (6, 9), (7, 8), (8, 7), (9, 6), (7, 9), (8, 8), (9, 7), (8, 9),
        (9, 8)]


def padded(te):
    return te + (te >> 4)


def shapes():
    """Every (K1, K2, logC, logR) the host accepts (cluster_shape)."""
    out = []
    for K1, K2 in MENU:
        L = K1 + K2
        for logC in range(1, 5):
            logGc, logGb = K2 - logC, K1 - logC
            if logGc < 2 or logGb < 0:
                continue
            for logR in (3, 4):
                logT = L - logC - logR
                if 5 <= logT <= 10 and 8 * padded(1 << (L - logC)) <= 200 * 1024:
                    out.append((K1, K2, logC, logR))
    return out


SHAPES = shapes()


def phases(K1, K2, logC, logR, rank):
    L = K1 + K2
    col = Pass(L, 0, K1, 0, K2 - logC, logR)
    row = Pass(L, K1, K2, K1 - logC, 0, logR)
    return col, (0, rank << (K2 - logC)), row, (rank << (K1 - logC), 0)


def exchange(K1, K2, logC, rank, l, from_column):
    """exchange_load's (owner, rl) for element l of CTA `rank`'s new tile."""
    logGc, logGb = K2 - logC, K1 - logC
    if from_column:                               # forward: l in the row tile
        row = (rank << logGb) + (l >> K2)
        col = l & ((1 << K2) - 1)
        return col >> logGc, (row << logGc) | (col & ((1 << logGc) - 1))
    row = l >> logGc                              # inverse: l in the column tile
    return row >> logGb, (((row & ((1 << logGb) - 1)) << K2)
                          | ((rank << logGc) + (l & ((1 << logGc) - 1))))


def test_menu_shapes_exist():
    assert len(SHAPES) >= 24
    assert (8, 8, 3, 4) in SHAPES and (8, 8, 2, 4) in SHAPES


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "K%d_%d_c%d_r%d" % s)
def test_tiles_and_exchange(shape):
    K1, K2, logC, logR = shape
    L, C = K1 + K2, 1 << logC
    E = 1 << (L - logC)
    T = E >> logR
    assert 32 <= T <= 1024
    # grid: blockIdx.x = (poly << logC) | rank, clusters of C consecutive blocks
    for bx in range(3 * C):
        assert (bx >> logC, bx & (C - 1)) == (bx // C, bx % C)
    seen_col = np.zeros(1 << L, np.int32)
    seen_row = np.zeros(1 << L, np.int32)
    gcol = {}
    grow = {}
    for rank in range(C):
        col, (cb, cc), row, (rb, rc) = phases(K1, K2, logC, logR, rank)
        assert col.logTE == L - logC and row.logTE == L - logC
        for l in range(E):
            g = col.gidx(l, cb, cc)
            seen_col[g] += 1
            gcol[(rank, l)] = g
            h = row.gidx(l, rb, rc)
            seen_row[h] += 1
            grow[(rank, l)] = h
        # staged copies of the row tile: 16-byte pairs from (b_base << K2)
        assert (rb << K2) + E <= 1 << L
    assert (seen_col == 1).all() and (seen_row == 1).all()
    for rank in range(C):
        for l in range(E):
            o, rl = exchange(K1, K2, logC, rank, l, True)
            assert 0 <= o < C and pad(rl) < padded(E)
            assert gcol[(o, rl)] == grow[(rank, l)]
            o, rl = exchange(K1, K2, logC, rank, l, False)
            assert 0 <= o < C and pad(rl) < padded(E)
            assert grow[(o, rl)] == gcol[(rank, l)]


def _run_phase(p, base, sm, x_of, tw, q, fwd, ninv=None):
    """One phase of one CTA: the rounds in execution order on the CTA's
    shared-memory array `sm` (indexed by pad(local)); x_of(l) supplies the
    first round's elements (HBM or the exchange)."""
    b_base, c_base = base
    size, off = sched(p.K, p.logR)
    order = range(len(size)) if fwd else reversed(range(len(size)))
    first = True
    for i in order:
        P, R = off[i], size[i]
        sshift, _ = p.shifts(P, R)
        regs = {}
        for u, tid, lbase, hp, hiu in p.groups(P, R, b_base):
            xs = [x_of(lbase + (v << sshift)) if first else sm[pad(lbase + (v << sshift))]
                  for v in range(1 << R)]
            ks = range(R) if fwd else reversed(range(R))
            for k in ks:
                for v in range(1 << R):
                    if v & (1 << (R - 1 - k)):
                        continue
                    v1 = v | (1 << (R - 1 - k))
                    if not fwd and ninv is not None and p.s0 + P + k == 0:
                        a, b = xs[v], xs[v1]
                        xs[v], xs[v1] = (a + b) * ninv % q, (a - b) * ninv % q * tw[1] % q
                        continue
                    w = tw[((hp << k) & 0xffffffff) + (v >> (R - k))]
                    a, b = xs[v], xs[v1]
                    if fwd:
                        b = b * w % q
                        xs[v], xs[v1] = (a + b) % q, (a - b) % q
                    else:
                        xs[v], xs[v1] = (a + b) % q, (a - b) * w % q
            for v in range(1 << R):
                regs[lbase + (v << sshift)] = xs[v]
        for l, val in regs.items():        # stores after every read of the round
            sm[pad(l)] = val
        first = False


@pytest.mark.parametrize("shape", [(7, 7, 2, 4), (8, 6, 3, 3), (6, 8, 1, 4)],
                         ids=lambda s: "K%d_%d_c%d_r%d" % s)
def test_forward_and_inverse_through_the_maps_equal_the_oracle(shape):
    K1, K2, logC, logR = shape
    L, C = K1 + K2, 1 << logC
    N, E = 1 << L, 1 << (L - logC)
    q = W.ntt_primes(50, 1 << (L + 1), 1)[0]
    psi = oracle.min_primitive_root(N, q)
    rev = [int(format(i, f"0{L}b")[::-1], 2) for i in range(N)]
    fw = [pow(psi, rev[i], q) for i in range(N)]
    iv = [pow(psi, (2 * N - rev[i]) % (2 * N), q) for i in range(N)]
    a = W.poly_batch(W.SEED_BASE + 991, 0, 1, [q], N)[0, 0]
    xin = [int(v) for v in a]

    # forward: column phase from HBM, exchange, row phase, out via smem
    sm = [[0] * padded(E) for _ in range(C)]
    for r in range(C):
        col, cbase, _, _ = phases(K1, K2, logC, logR, r)
        _run_phase(col, cbase, sm[r], lambda l, col=col, cbase=cbase: xin[col.gidx(l, *cbase)],
                   fw, q, True)
    sm2 = [[0] * padded(E) for _ in range(C)]
    for r in range(C):
        _, _, row, rbase = phases(K1, K2, logC, logR, r)
        _run_phase(row, rbase, sm2[r],
                   lambda l, r=r: sm[exchange(K1, K2, logC, r, l, True)[0]][
                       pad(exchange(K1, K2, logC, r, l, True)[1])], fw, q, True)
    out = [0] * N
    for r in range(C):
        _, _, row, rbase = phases(K1, K2, logC, logR, r)
        for l in range(E):
            out[row.gidx(l, *rbase)] = sm2[r][pad(l)]
    exp = oracle.ntt_forward_1(a, q)
    np.testing.assert_array_equal(np.array(out, dtype=np.uint64), exp)

    # inverse: row tile staged in, row phase, exchange, column phase to HBM
    ninv = pow(N, q - 2, q)
    sm = [[0] * padded(E) for _ in range(C)]
    for r in range(C):
        _, _, row, rbase = phases(K1, K2, logC, logR, r)
        for l in range(E):
            sm[r][pad(l)] = int(exp[row.gidx(l, *rbase)])
        _run_phase(row, rbase, sm[r], lambda l, s=sm[r]: s[pad(l)], iv, q, False)
    back = [0] * N
    for r in range(C):
        col, cbase, _, _ = phases(K1, K2, logC, logR, r)
        scratch = [0] * padded(E)
        _run_phase(col, cbase, scratch,
                   lambda l, r=r: sm[exchange(K1, K2, logC, r, l, False)[0]][
                       pad(exchange(K1, K2, logC, r, l, False)[1])], iv, q, False, ninv)
        for l in range(E):
            back[col.gidx(l, *cbase)] = scratch[pad(l)]
    np.testing.assert_array_equal(np.array(back, dtype=np.uint64), a)
