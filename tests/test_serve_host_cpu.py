"""The server's scheduling on the host, without a GPU: a server whose launch
step is replaced by a fake (no kernels, no streams, no device) must admit
requests in FIFO order, batch the ones that arrive while a batch is in
flight (continuous batching), keep the bytes in flight within the HBM
budget and the batches in flight within the stream slots, hand every
request its own slice of its batch's result, launch on the submitting thread
when idle, and fail cleanly when a launch fails."""
import contextlib
import threading
import time

import numpy as np
import pytest
import torch

from paper_2103_16400_gb300 import capi, serve


class _Done:
    """Stands in for a batch's end event: fires when the test releases it."""

    def __init__(self, gate):
        self.gate = gate

    def synchronize(self):
        if not self.gate.wait(timeout=30):
            raise TimeoutError("batch never released")

    def query(self):
        return self.gate.is_set()


class FakeServer(serve.Server):
    def __init__(self, budget, n_streams, hold_first=False, fail=False, fast_path=True):
        super().__init__(hbm_budget=budget, streams=list(range(n_streams)), fast_path=fast_path)
        self.batches = []
        self.max_in_use = 0
        self.max_inflight = 0
        self.gates = []
        self.hold_first = hold_first
        self.fail = fail

    def _bind_device(self):
        pass

    def _device_scope(self):
        return contextlib.nullcontext()

    def _launch(self, reqs, sid, need):
        if self.fail:
            raise capi.HexError("hx_polymul_ragged", -7, "injected")
        with self._lock:
            self.max_in_use = max(self.max_in_use, self.in_use)
            self.max_inflight = max(self.max_inflight, self.n_inflight)
        self.batches.append([r.tag for r in reqs])
        sizes = np.array([r.limbs * r.N for r in reqs], np.int64)
        res = torch.empty(int(sizes.sum()), dtype=torch.int64)
        out = torch.cat([torch.full((int(n),), r.tag, dtype=torch.int64)
                         for r, n in zip(reqs, sizes)])
        gate = threading.Event()
        if not (self.hold_first and len(self.batches) == 1):
            gate.set()
        self.gates.append(gate)
        return {"reqs": reqs, "work": (res, sizes, out, None, None, None),
                "event": _Done(gate), "sid": sid, "bytes": need}


def request(tag, N=1 << 10, limbs=2):
    a = np.zeros((limbs, N), np.uint64)
    r = serve.Request(N, tuple(range(limbs)), a, a)
    r.tag = tag
    return r


def test_fifo_continuous_batching_and_own_results():
    srv = FakeServer(budget=1 << 30, n_streams=1, hold_first=True).start()
    first = [srv.submit(request(t)) for t in range(3)]
    deadline = time.time() + 10
    while not srv.batches and time.time() < deadline:
        time.sleep(0.001)
    later = [srv.submit(request(t)) for t in range(3, 10)]   # arrive while batch 1 runs
    time.sleep(0.05)
    assert len(srv.batches) == 1                  # one stream: batch 2 waits for it
    srv.gates[0].set()
    for t, f in enumerate(first + later):
        got = f.result(timeout=10)
        assert got.shape == (2, 1 << 10) and (got == t).all()
    srv.stop()
    order = [t for b in srv.batches for t in b]
    assert order == list(range(10))               # FIFO
    # everything that arrived while the first batch held the only stream
    # went out as one second batch
    assert len(srv.batches) == 2 and srv.batches[1][-1] == 9
    assert srv.max_inflight == 1


def test_budget_bounds_bytes_in_flight():
    one = request(0).device_bytes
    srv = FakeServer(budget=3 * one, n_streams=4).start()
    futs = [srv.submit(request(t)) for t in range(40)]
    for f in futs:
        f.result(timeout=10)
    srv.stop()
    assert srv.max_in_use <= 3 * one
    assert all(len(b) <= 3 for b in srv.batches)
    assert [t for b in srv.batches for t in b] == list(range(40))
    assert srv.in_use == 0 and srv.n_inflight == 0 and sorted(srv.free_streams) == [0, 1, 2, 3]


def test_oversized_request_is_refused():
    srv = FakeServer(budget=request(0).device_bytes - 1, n_streams=1)
    with pytest.raises(serve.BudgetError):
        srv.submit(request(0))


def test_failed_launch_fails_requests_and_stops():
    srv = FakeServer(budget=1 << 30, n_streams=2, fail=True, fast_path=False).start()
    futs = [srv.submit(request(t)) for t in range(5)]
    for f in futs:
        with pytest.raises(capi.HexError):
            f.result(timeout=10)
    with pytest.raises(RuntimeError):
        srv.submit(request(9))
    with pytest.raises(capi.HexError):
        srv.stop()
    assert srv.in_use == 0 and srv.n_inflight == 0


def test_transform_requests_are_checked_and_sized():
    srv = FakeServer(budget=1 << 30, n_streams=1)
    a = np.zeros((2, 1 << 10), np.uint64)
    with pytest.raises(ValueError):
        srv.submit(serve.Request(1 << 10, (1, 2), a, a, op="square"))
    with pytest.raises(ValueError):
        srv.submit(serve.Request(1 << 10, (1, 2), a, op="mul"))      # no second operand
    fwd = serve.Request(1 << 10, (1, 2), a, op="fwd")
    mul = serve.Request(1 << 10, (1, 2), a, a)
    # a transform holds its result and its staged operand; a product two
    # spectra, its result and two staged operands
    assert fwd.device_bytes < mul.device_bytes / 2


def test_mixed_ops_keep_fifo_order():
    srv = FakeServer(budget=1 << 30, n_streams=2).start()
    reqs = [request(t) for t in range(12)]
    for r, op in zip(reqs, ["mul", "fwd", "inv"] * 4):
        r.op = op
    futs = [srv.submit(r) for r in reqs]
    for t, f in enumerate(futs):
        assert (f.result(timeout=10) == t).all()
    srv.stop()
    assert [t for b in srv.batches for t in b] == list(range(12))


def test_idle_server_launches_on_the_submitting_thread():
    """Idle (nothing waiting, a stream free): submit() launches the request
    itself, so its batch exists when submit returns; while that batch holds
    the only stream, later requests go through the engine as one batch."""
    srv = FakeServer(budget=1 << 30, n_streams=1, hold_first=True).start()
    f0 = srv.submit(request(0))
    assert srv.batches == [[0]] and srv.stats["fast_path"] == 1
    later = [srv.submit(request(t)) for t in range(1, 5)]
    time.sleep(0.05)
    assert srv.batches == [[0]]                   # the stream is busy: they wait
    srv.gates[0].set()
    for t, f in enumerate([f0] + later):
        assert (f.result(timeout=10) == t).all()
    srv.stop()
    assert srv.batches == [[0], [1, 2, 3, 4]] and srv.stats["fast_path"] == 1
    assert srv.in_use == 0 and srv.n_inflight == 0


def test_failed_fast_path_launch_fails_its_request_and_stops():
    srv = FakeServer(budget=1 << 30, n_streams=2, fail=True).start()
    f = srv.submit(request(0))                    # idle: launched here, and fails
    with pytest.raises(capi.HexError):
        f.result(timeout=10)
    with pytest.raises(RuntimeError):             # later submissions are refused
        srv.submit(request(1))
    with pytest.raises(capi.HexError):
        srv.stop()
    assert srv.in_use == 0 and srv.n_inflight == 0
