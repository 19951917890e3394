"""The continuous-batching server: every product is the same bits served
alone, served in a mix with concurrent arrivals, and computed by the
unbatched baseline, and equals the oracle on sampled requests; the HBM budget
bounds what is in flight; oversized requests are refused."""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import serve

pytestmark = pytest.mark.gpu


def make_requests(n, seed, max_limbs=6):
    pool = W.mixed_width_primes(max_limbs)
    draws = W.splitmix64_block(W.stream_key(seed, 77), 0, 2 * n)
    reqs = []
    for i in range(n):
        N = (1 << 12, 1 << 14, 1 << 16)[int(draws[2 * i] % np.uint64(3))]
        L = 1 + int(draws[2 * i + 1] % np.uint64(max_limbs))
        qs = tuple(pool[:L])
        a = W.poly_batch(seed, 2 * i, 1, qs, N)[0]
        b = W.poly_batch(seed, 2 * i + 1, 1, qs, N)[0]
        reqs.append(serve.Request(N, qs, a, b))
    return reqs


def clone(reqs):
    return [serve.Request(r.N, r.moduli, r.a, r.b, op=r.op) for r in reqs]


def test_results_identical_alone_and_in_the_mix(hexlib):
    reqs = make_requests(48, W.SEED_BASE + 5)
    # in the mix: submit in three waves while earlier ones are on the GPU
    mixed = clone(reqs)
    with serve.Server(hbm_budget=8 << 30, streams=3) as srv:
        futs = []
        for w in range(3):
            futs += [srv.submit(r) for r in mixed[w * 16:(w + 1) * 16]]
            time.sleep(0.002)
        got_mix = [f.result(timeout=120) for f in futs]
        assert srv.stats["requests"] == 48 and srv.stats["batches"] >= 2
    # alone: one request at a time through a fresh server
    alone = clone(reqs)
    with serve.Server(hbm_budget=8 << 30, streams=1) as srv:
        got_alone = [srv.submit(r).result(timeout=120) for r in alone]
    # the unbatched baseline
    base = clone(reqs)
    serve.serve_one_by_one(base)
    for r, m, a, b in zip(reqs, got_mix, got_alone, base):
        np.testing.assert_array_equal(m, a)
        np.testing.assert_array_equal(m, b.result)
    # oracle on a sample
    for k in (0, 7, 19, 33, 47):
        r = reqs[k]
        exp = oracle.poly_mul(r.a[None], r.b[None], r.moduli)[0]
        np.testing.assert_array_equal(got_mix[k], exp)
    r = next(r for r in reqs if r.N == 1 << 12)
    k = reqs.index(r)
    idx = [0, 1, 2047, 4095]
    np.testing.assert_array_equal(got_mix[k][0, idx],
                                  oracle.negacyclic_schoolbook(r.a[0], r.b[0], r.moduli[0], idx))


def test_budget_admission_bounds_inflight_bytes(hexlib):
    reqs = make_requests(12, W.SEED_BASE + 6, max_limbs=3)
    biggest = max(r.device_bytes for r in reqs)
    budget = 2 * biggest
    with serve.Server(hbm_budget=budget, streams=3) as srv:
        futs = [srv.submit(r) for r in reqs]
        peak = 0
        while not all(f.done() for f in futs):
            peak = max(peak, srv.in_use)
            time.sleep(0.0002)
        assert peak <= budget
        assert srv.in_use == 0
    for r, f in zip(reqs, futs):
        np.testing.assert_array_equal(f.result(), oracle.poly_mul(r.a[None], r.b[None], r.moduli)[0])


def test_hbm_resident_operands(hexlib):
    """Operands already in HBM: the results stay on the device and equal the
    host-operand results and the oracle."""
    import torch
    from paper_2103_16400_gb300.tensors import to_device, to_host
    reqs = make_requests(24, W.SEED_BASE + 9)
    res = [serve.Request(r.N, r.moduli, to_device(r.a), to_device(r.b)) for r in reqs]
    torch.cuda.synchronize()
    with serve.Server(hbm_budget=8 << 30, streams=2) as srv:
        futs = [srv.submit(r) for r in res]
        got = [f.result(timeout=120) for f in futs]
    host = clone(reqs)
    with serve.Server(hbm_budget=8 << 30, streams=2) as srv:
        exp = [srv.submit(r).result(timeout=120) for r in host]
    for g, e, r in zip(got, exp, reqs):
        assert g.is_cuda
        np.testing.assert_array_equal(to_host(g), e)
    r = reqs[3]
    np.testing.assert_array_equal(to_host(got[3]), oracle.poly_mul(r.a[None], r.b[None], r.moduli)[0])


def test_oversized_request_is_refused(hexlib):
    r = make_requests(1, W.SEED_BASE + 8, max_limbs=2)[0]
    srv = serve.Server(hbm_budget=r.device_bytes - 1, streams=1)
    with pytest.raises(serve.BudgetError):
        srv.submit(r)


def test_servers_share_given_streams_and_stamp_given_arrivals(hexlib):
    """Two servers in turn on the same two caller-made streams give the same
    bits; a submission stamped with an earlier arrival counts its latency
    from that time."""
    import torch
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    reqs = make_requests(12, W.SEED_BASE + 11)
    got = []
    for _ in range(2):
        with serve.Server(hbm_budget=8 << 30, streams=streams) as srv:
            assert srv.streams == streams
            t = time.perf_counter() - 0.25
            rs = clone(reqs)
            got.append([srv.submit(r, arrival=t).result(timeout=120) for r in rs])
            assert all(r.arrival == t and r.latency >= 0.25 for r in rs)
    for a, b in zip(*got):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(ValueError):
        serve.Server(streams=[])


def test_launch_failure_fails_its_requests_and_stops_the_server(hexlib, monkeypatch):
    """A batch whose launch raises (an error injected on the host, before any
    kernel runs): its requests and the waiting ones get the error, later
    submissions are refused, and stop() re-raises it."""
    from paper_2103_16400_gb300 import capi

    def broken(*args, **kwargs):
        raise capi.HexError("hx_polymul_ragged", -7, "injected")

    monkeypatch.setattr(capi, "hx_polymul_ragged", broken)
    reqs = make_requests(6, W.SEED_BASE + 13)
    srv = serve.Server(hbm_budget=8 << 30, streams=1, fast_path=False).start()
    futs = [srv.submit(r) for r in reqs]
    for f in futs:
        with pytest.raises(capi.HexError):
            f.result(timeout=60)
    with pytest.raises(RuntimeError):
        srv.submit(clone(reqs)[0])
    with pytest.raises(capi.HexError):
        srv.stop()
    assert srv.in_use == 0 and srv.n_inflight == 0
    # an idle server launches on the submitting thread: the failure comes
    # back through that request's future, and later submissions are refused
    srv = serve.Server(hbm_budget=8 << 30, streams=1).start()
    f = srv.submit(clone(reqs)[0])
    with pytest.raises(capi.HexError):
        f.result(timeout=60)
    with pytest.raises(RuntimeError):
        srv.submit(clone(reqs)[1])
    with pytest.raises(capi.HexError):
        srv.stop()
    assert srv.in_use == 0 and srv.n_inflight == 0


def test_products_and_transforms_in_one_stream_of_requests(hexlib):
    """Forward and inverse NTT requests mixed with products, host and
    HBM-resident operands: every result equals the one-by-one baseline's
    and the oracle's."""
    from paper_2103_16400_gb300.tensors import to_device, to_host
    reqs = make_requests(24, W.SEED_BASE + 17)
    for k, r in enumerate(reqs):
        r.op = ("mul", "fwd", "inv")[k % 3]
    resident = [serve.Request(r.N, r.moduli, to_device(r.a), op=op)
                for r, op in zip(reqs[:4], ("fwd", "inv", "fwd", "inv"))]
    with serve.Server(hbm_budget=8 << 30, streams=3) as srv:
        futs = [srv.submit(r) for r in clone(reqs) + resident]
        got = [f.result(timeout=120) for f in futs]
    base = clone(reqs)
    serve.serve_one_by_one(base)
    for r, g, b in zip(reqs, got, base):
        np.testing.assert_array_equal(g, b.result)
        if r.op == "fwd":
            exp = oracle.ntt_forward(r.a[None], r.moduli)[0]
        elif r.op == "inv":
            exp = oracle.ntt_inverse(r.a[None], r.moduli)[0]
        else:
            exp = oracle.poly_mul(r.a[None], r.b[None], r.moduli)[0]
        np.testing.assert_array_equal(g, exp)
    for r, g, src in zip(resident, got[len(reqs):], reqs[:4]):
        f = oracle.ntt_forward if r.op == "fwd" else oracle.ntt_inverse
        np.testing.assert_array_equal(to_host(g), f(src.a[None], src.moduli)[0])


def test_idle_server_serves_resident_requests_with_per_request_calls(hexlib):
    """Requests submitted one at a time to an idle server go out on the
    submitting thread through the per-request calls (forward transforms into
    the stream's workspace, hx_dyadic_inverse): same bits as the one-by-one
    baseline and the oracle, for products and both transforms."""
    from paper_2103_16400_gb300.tensors import to_device, to_host
    reqs = make_requests(9, W.SEED_BASE + 19)
    for k, r in enumerate(reqs):
        r.op = ("mul", "fwd", "inv")[k % 3]
    res = [serve.Request(r.N, r.moduli, to_device(r.a), to_device(r.b), op=r.op) for r in reqs]
    with serve.Server(hbm_budget=8 << 30, streams=2) as srv:
        got = [to_host(srv.submit(r).result(timeout=120)) for r in res]
        assert srv.stats["fast_path"] == len(reqs)
    base = clone(reqs)
    serve.serve_one_by_one(base)
    for r, g, b in zip(reqs, got, base):
        np.testing.assert_array_equal(g, b.result)
        if r.op == "mul":
            np.testing.assert_array_equal(g, oracle.poly_mul(r.a[None], r.b[None], r.moduli)[0])
