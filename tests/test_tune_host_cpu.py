"""The autotuner's host logic (no GPU): every candidate schedule runs the
stages 0 .. log2 N - 1 exactly once, in order, as one pass (N <= 2^13) or a
column pass then a row pass of 6 to 13 stages each, or a cluster-fused
pair of 6 to 9 stages each with one cluster size; cache keys tell apart
the GPU, N, the width mix and the batch; the cache survives a round trip."""
import pytest

import workloads as W
from paper_2103_16400_gb300 import tune


@pytest.mark.parametrize("logN", range(10, 18))
def test_candidates_cover_every_stage_once(logN):
    cands = tune.candidates(logN)
    assert cands
    for sched in cands:
        s0 = 0
        for p in sched:
            assert p[0] == s0                          # passes follow each other
            s0 += p[1]
            assert (p[4], p[5], p[6]) in tune.VARIANTS or p[5] == 3
        assert s0 == logN
        if sched[0][5] == 3:                           # cluster-fused: both passes one launch
            col, row = sched
            assert row[5] == 3 and col[4] == row[4] and col[4] in tune.CLUSTER_LOGR
            c = row[1] - col[3]
            assert 1 <= c <= 4 and col[1] - row[2] == c    # same cluster size both ways
            assert 6 <= col[1] <= 9 and 6 <= row[1] <= 9
            continue
        if len(sched) == 1:
            assert logN <= 13 and sched[0][2] == sched[0][3] == 0
        else:
            col, row = sched
            assert col[2] == 0 and col[3] in (2, 3, 4, 5)   # column tiles
            assert row[3] == 0 and 0 <= row[2] <= 5         # row tiles
            assert 6 <= col[1] <= 13 and 6 <= row[1] <= 13
    assert any(len(s) == 1 for s in cands) == (logN <= 13)
    assert any(s[0][5] == 3 for s in cands) == (12 <= logN <= 18)


def test_cache_keys_tell_workloads_apart():
    mixed = W.mixed_width_primes(32)
    k = tune._key(1 << 16, mixed, 4, "GB300")
    assert tune.width_class(mixed) == "11n21w"
    assert len({k, tune._key(1 << 15, mixed, 4, "GB300"), tune._key(1 << 16, mixed[:31], 4, "GB300"),
                tune._key(1 << 16, mixed, 3, "GB300"), tune._key(1 << 16, mixed, 4, "B200")}) == 5
    # the same width mix in another order shares the entry
    assert tune._key(1 << 16, mixed[::-1], 4, "GB300") == k


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "sub" / "cache.json"))
    assert tune.load_cache() == {}
    entry = {"forward": [[0, 7, 0, 4, 4, 0, 1], [7, 9, 0, 0, 3, 0, 1]], "us": 91.5}
    tune.save_cache({"k": entry})
    assert tune.load_cache() == {"k": entry}
    (tmp_path / "sub" / "cache.json").write_text("{not json")
    assert tune.load_cache() == {}                   # a damaged cache is ignored


def test_ragged_split_menu_and_keys():
    """The ragged kernels' splits: a column pass of 5..9 stages and a row
    pass of 6..11 on 2048-element tiles, for N = 2^12..2^17 only; cache keys
    tell apart GPU, N, width mix and transform count (rounded down to a power
    of two)."""
    assert tune.ragged_splits(11) == [] and tune.ragged_splits(18) == []
    for L in range(12, 18):
        ks = tune.ragged_splits(L)
        assert ks == [k for k in range(5, 10) if 6 <= L - k <= 11] and ks
        assert all(2 <= 11 - k <= 6 and 0 <= 11 - (L - k) <= k for k in ks)   # tile shapes
    assert sum(len(tune.ragged_splits(L)) for L in range(12, 18)) == 23
    mixed = W.mixed_width_primes(8)
    k = tune._ragged_key(16, mixed, 100, "GB300")
    assert k == tune._ragged_key(16, mixed[::-1], 127, "GB300")      # same mix, same bucket
    assert len({k, tune._ragged_key(15, mixed, 100, "GB300"),
                tune._ragged_key(16, mixed[:7], 100, "GB300"),
                tune._ragged_key(16, mixed, 128, "GB300"),
                tune._ragged_key(16, mixed, 100, "B200")}) == 5


def test_cluster_options_fit_the_menu():
    """Cluster schedules: both phases 6..9 stages, cluster of 2..16 CTAs,
    8 or 16 elements a thread; every (K1, K2) the library instantiates."""
    menu = {(6, 8), (7, 7), (8, 6), (6, 9), (7, 8), (8, 7), (9, 6), (7, 9), (8, 8), (9, 7),
            (8, 9), (9, 8)}
    for L in range(14, 18):
        opts = tune.cluster_options(L)
        assert {(a[1], b[1]) for a, b in opts} == {p for p in menu if sum(p) == L}
        for a, b in opts:
            c = b[1] - a[3]
            assert a[5] == b[5] == 3 and 1 <= c <= 4 and a[1] - b[2] == c


def test_step_candidates_share_their_row_passes():
    """Every (forward, inverse) pair offered for hx_ciphertext_step: both
    two-pass, row passes over the same stages (6..9) in the same row tiles
    with 8 elements a thread and 32..512 threads, four padded tiles within
    192 KB; none at N where no row pass can have 6..9 stages."""
    for logN in (14, 15, 16, 17):
        cands = tune.step_candidates(logN)
        assert cands
        for f, i in cands:
            assert len(f) == len(i) == 2
            assert f[0][0] == i[0][0] == 0 and f[0][1] == i[0][1]
            fr, ir = f[1], i[1]
            assert fr[:5] == ir[:5] and fr[3] == 0 and fr[4] == 3
            assert fr[0] + fr[1] == logN and 6 <= fr[1] <= 9
            assert 5 <= fr[2] + fr[1] - 3 <= 9
            te = 1 << (fr[2] + fr[1])
            assert 32 * (te + te // 16) <= 192 * 1024
            assert ir[6] == 2 and fr[6] == 1
    assert tune.step_candidates(10) == []
    assert len({(tuple(f), tuple(i)) for f, i in tune.step_candidates(16)}) == \
        len(tune.step_candidates(16))
