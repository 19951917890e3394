"""Continuous-batching server for negacyclic polynomial products and NTTs.

A request is one product c = a * b in R_q = Z_q[X]/(X^N + 1) over an RNS
basis (a, b: uint64 [limbs][N] residues), computed as in the paper's
Listing 4: forward NTT of both operands with outputs left in [0, 4q),
EltwiseMultMod with input_mod_factor 4, inverse NTT to [0, q) -- or one
forward or inverse NTT of a (Algorithms CT and GS, outputs in [0, q)).

The paper's polynomial layer is single-threaded and per call (Section 3);
its integration section notes that one call is too small to offload to an
accelerator (Section 4).  The server answers that by batching, with two
threads and no polling:
  * the engine thread sleeps on the request queue; woken by a submission
    (or by a finished batch), it moves every newly submitted request to a
    FIFO wait list and admits waiting requests in order while their device
    memory (operands, one result per request, in HBM) fits the HBM budget
    and a stream slot is free -- requests that arrive while earlier batches
    are still on the GPU join the next batch (continuous batching) -- and
    launches each admitted batch on its own CUDA stream as one ragged call
    per kind of request (hx_polymul_ragged: four kernels for all the batch's
    products, whatever their mix of N and moduli; hx_ntt_ragged: two for
    its forward and two for its inverse transforms) into workspaces taken
    from the torch allocator, with one upload and one download for host
    operands;
  * the completer thread waits on each launched batch's end event in turn
    (spinning in the driver, or sleeping there with blocking_wait; either
    wait releases the interpreter lock), completes its requests,
    stamping their latency, returns their budget and stream, and wakes the
    engine for any requests that were waiting for them.
When the server is idle -- nothing in flight, waiting or queued, and the
request within the budget -- submit() launches an HBM-resident request on
the calling thread at once, through the per-request calls on that thread's
current stream (what a direct call would do), so a request alone on an idle
GPU is answered about as fast as the direct calls would answer it.  Small
batches of HBM-resident requests (up to DIRECT_MAX) go out through the same
per-request calls on their stream: the ragged call's descriptor lists cost
more host time than they save until a batch grows.  Under load, requests
queue and go out in ragged batches as above.
Batches on different streams overlap on the GPU.  Plans (and so the twiddle
tables) are created once per (N, moduli) and stay resident.

All arithmetic runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import collections
import contextlib
import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import capi


OPS = ("mul", "fwd", "inv")


@dataclass
class Request:
    """One request on an RNS polynomial, uint64 [limbs][N] residues in [0, q):
    op "mul" -- the product a * b in R_q (Listing 4); "fwd" -- the forward
    NTT of a (Algorithm CT, bit-reversed order, output in [0, q)); "inv" --
    the inverse NTT of a (Algorithm GS with N^-1, bit-reversed input).  a, b
    are numpy arrays on the host (the result comes back as a numpy array) or
    int64-typed CUDA tensors resident in HBM (the result is a CUDA tensor
    view, nothing leaves the device); b is only read by "mul".

    A resident result is a view of its batch's result tensor, allocated on
    the stream that ran the batch (a server stream, or the submitting
    thread's current stream when an idle server launched it there) and
    complete when the future resolves.  A caller that reads it on another stream should call
    result.record_stream(that_stream) first, so the caching allocator does
    not hand the memory out again while that stream still reads it.  The
    HBM budget covers work in flight: a result is no longer counted once its
    request completes, however long the caller keeps it."""
    N: int
    moduli: Tuple[int, ...]
    a: object
    b: object = None
    op: str = "mul"
    arrival: float = 0.0             # perf_counter() at submission
    done: float = 0.0
    path: str = ""                   # how it went out: "idle", "direct" or "ragged"
    result: object = None
    future: Future = field(default_factory=Future)

    @property
    def limbs(self) -> int:
        return len(self.moduli)

    @property
    def resident(self) -> bool:
        return not isinstance(self.a, np.ndarray)

    @property
    def device_bytes(self) -> int:
        """HBM the request holds while in flight: for a product two spectra
        in the batch workspace and the result, for a transform the result,
        plus the staged operands when they come from the host and the tile
        lists (32 bytes per tile of 2048 coefficients per pass)."""
        words = self.limbs * self.N
        if self.op == "mul":
            return (3 + (0 if self.resident else 2)) * words * 8 + (3 * words // 2048 + 4) * 64
        return (1 + (0 if self.resident else 1)) * words * 8 + (2 * words // 2048 + 2) * 32

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class BudgetError(ValueError):
    pass


_WAKE = object()   # queue token: re-check admission, nothing submitted


class Server:
    """Engine and completer threads + streams; `submit()` is thread-safe and
    returns a Future that resolves to the request's result (the product or
    the transform, uint64 [limbs][N])."""

    def __init__(self, hbm_budget: int = 64 << 30, streams=3,
                 max_batch: int = 256, device: int = 0, blocking_wait: bool = False,
                 fast_path: bool = True, poll_us: float = 0.0):
        """streams: how many CUDA streams to create, or the streams to use
        (servers that share streams also share the caching allocator's blocks,
        which the allocator keeps per stream).  blocking_wait: the completer
        sleeps in the driver until a batch's end event fires (a blocking-sync
        event) instead of spinning a host core on it (the default: the spin
        answers tens of microseconds sooner; either wait releases the
        interpreter lock) -- after first polling the event for up to poll_us
        microseconds (0: no polling).  fast_path:
        an idle server launches a submitted request on the submitting thread
        (an HBM-resident one through the per-request calls)."""
        import torch
        self.torch = torch
        self.device = device
        self.budget = int(hbm_budget)
        self.max_batch = max_batch
        self.blocking_wait = blocking_wait
        self.fast_path = fast_path
        self.poll_s = max(0.0, poll_us) * 1e-6
        self._bind_device()
        capi.load()
        if isinstance(streams, int):
            streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.streams = list(streams)
        if not self.streams:
            raise ValueError("a server needs at least one stream")
        self.free_streams = list(range(len(self.streams)))
        self.in_use = 0
        self.n_inflight = 0
        self.plans: Dict[Tuple[int, Tuple[int, ...]], capi.Plan] = {}
        self.inbox: "queue.Queue" = queue.Queue()
        self.done_q: "queue.Queue" = queue.Queue()
        self.waiting: "collections.deque[Request]" = collections.deque()
        # launch_ms_max: the longest host time spent launching one batch
        # (marshalling, allocation, the ragged call); complete_ms_max: the
        # longest spent handing one finished batch's results to its futures
        self.stats = {"batches": 0, "requests": 0, "max_batch": 0, "launches": 0,
                      "launch_ms_max": 0.0, "complete_ms_max": 0.0, "fast_path": 0,
                      "direct_batches": 0, "completed_by_polling": 0}
        self._lock = threading.Lock()   # in_use, free_streams, n_inflight, stats; _error vs submit
        self._stop = threading.Event()
        self._threads: List[threading.Thread] = []
        self._error: Optional[BaseException] = None
        self._queued = 0                         # requests in the inbox
        self._direct_ws: Dict[object, object] = {}   # per stream (and the idle path): spectra
        self._idle_ev = None                     # the idle path's end event
        self._batch_ws: Dict[Tuple[int, str], object] = {}   # per (stream, kind) workspace

    def _bind_device(self):
        """Makes the server's device current in the calling thread."""
        self.torch.cuda.set_device(self.device)

    def _device_scope(self):
        """The server's device made current for a launch from a client thread
        (restored afterwards)."""
        return self.torch.cuda.device(self.device)

    # ------------------------------------------------------------ client side
    def plan(self, N: int, moduli: Sequence[int]) -> "capi.Plan":
        key = (N, tuple(int(q) for q in moduli))
        p = self.plans.get(key)
        if p is None:
            p = self.plans[key] = capi.Plan(N, key[1])
        return p

    def submit(self, req: Request, arrival: Optional[float] = None) -> Future:
        """Queue a request; its latency counts from `arrival` (a perf_counter()
        time, e.g. when a load generator scheduled it) or from now."""
        if req.op not in OPS:
            raise ValueError(f"unknown op {req.op!r}; expected one of {OPS}")
        if req.op == "mul" and req.b is None:
            raise ValueError("a product needs both operands")
        if req.device_bytes > self.budget:
            raise BudgetError(f"request needs {req.device_bytes} bytes, budget {self.budget}")
        if type(req.moduli) is not tuple:
            req.moduli = tuple(int(q) for q in req.moduli)   # the plan table's key form
        req.arrival = time.perf_counter() if arrival is None else arrival
        sid = None
        with self._lock:
            if self._error is not None:
                raise RuntimeError("the server stopped after an error") from self._error
            if (self.fast_path and self._threads and not self._stop.is_set()
                    and self.n_inflight == 0 and self._queued == 0 and not self.waiting
                    and self.free_streams and self.in_use + req.device_bytes <= self.budget):
                # idle: this request is the next batch; launch it here (an
                # HBM-resident one on the caller's own stream).  Under load
                # the engine's batches do better: per-request launches from
                # the submitting thread, with the completer and the engine
                # also wanting the interpreter lock, capped at ~6 k
                # requests/s where batching carries ~31 k.
                idle = True
                need = req.device_bytes
                self.in_use += need
                self.n_inflight += 1
                sid = self.free_streams.pop()
                self.stats["fast_path"] += 1
            else:
                self._queued += 1
                self.inbox.put(req)
        if sid is not None:
            self._launch_batch([req], sid, need, on_device=True, idle=idle)
        return req.future

    #: batches of at most this many HBM-resident requests go out through the
    #: per-request calls (about 15 us of host time a request) rather than
    #: one ragged call (about 95 us of host time whatever the batch)
    DIRECT_MAX = 4

    def _launch_direct(self, reqs: List["Request"], sid: int, need: int,
                       on_caller_stream: bool = False) -> dict:
        """HBM-resident requests through the per-request calls, one after
        another on one stream (no descriptor lists): a product is one
        hx_poly_product call (a and b kept; their spectra in a workspace kept
        per stream, which requests on one stream reuse in order); a transform
        writes its result directly.  on_caller_stream: the idle path -- the submitting
        thread's current stream (as a direct call would run; the server is
        idle, so the idle path's workspace and event are free), waited on by
        spinning in the driver; else server stream `sid`."""
        torch = self.torch
        dev_name = f"cuda:{self.device}"
        stream = torch.cuda.current_stream(self.device) if on_caller_stream else self.streams[sid]
        key = "idle" if on_caller_stream else sid
        sh = stream.cuda_stream
        n = len(reqs)
        sizes = np.fromiter((r.limbs * r.N for r in reqs), np.int64, n)
        need_ws = 2 * int(sizes.max())
        with torch.cuda.stream(stream) if not on_caller_stream else contextlib.nullcontext():
            res = torch.empty(int(sizes.sum()), dtype=torch.int64, device=dev_name)
            ws = self._direct_ws.get(key)
            if ws is None or ws.numel() < need_ws:
                ws = self._direct_ws[key] = torch.empty(need_ws, dtype=torch.int64,
                                                        device=dev_name)
            wa = ws.data_ptr()
            out = res.data_ptr()
            launches = 0
            for r, words in zip(reqs, sizes.tolist()):
                plan = self.plans.get((r.N, r.moduli))
                if plan is None:
                    plan = self.plan(r.N, r.moduli)
                if r.op == "mul":
                    # both spectra in the workspace, the product inside the
                    # inverse (four launches where the plan's schedules
                    # share their row passes)
                    capi.hx_poly_product(plan, out, r.a, r.b, wa, 1, sh)
                    launches += 1
                else:
                    (capi.hx_ntt_forward if r.op == "fwd" else capi.hx_ntt_inverse)(
                        plan, out, r.a, 1, 1, 1, sh)
                    launches += 1
                out += 8 * words
            if on_caller_stream:
                ev = self._idle_ev
                if ev is None:
                    ev = self._idle_ev = torch.cuda.Event()
            else:
                ev = torch.cuda.Event(blocking=self.blocking_wait)
            ev.record(stream)
        with self._lock:
            self.stats["batches"] += 1
            self.stats["requests"] += n
            self.stats["max_batch"] = max(self.stats["max_batch"], n)
            self.stats["launches"] += launches
            self.stats["direct_batches"] += 1
        return {"reqs": reqs, "work": (res, sizes, None, None, None, None),
                "event": ev, "sid": sid, "bytes": need}

    def start(self) -> "Server":
        self._threads = [threading.Thread(target=self._run, name="hexgpu-serve", daemon=True),
                         threading.Thread(target=self._complete, name="hexgpu-complete",
                                          daemon=True)]
        for t in self._threads:
            t.start()
        return self

    def stop(self, drain: bool = True):
        if drain:
            while self._error is None:
                with self._lock:
                    busy = self.n_inflight > 0
                if not (busy or self.waiting or not self.inbox.empty()):
                    break
                time.sleep(0.0005)
        self._stop.set()
        self.inbox.put(_WAKE)
        self.done_q.put(None)
        for t in self._threads:
            t.join()
        if self._error is not None:
            raise self._error

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop(drain=exc[0] is None)

    # ------------------------------------------------------------ engine
    def _fail(self, e: BaseException):
        with self._lock:                  # no submission slips in after the drain
            self._error = e
            self._drain_inbox()
        for r in list(self.waiting):
            if not r.future.done():
                r.future.set_exception(e)
        self.waiting.clear()

    def _run(self):
        self._bind_device()
        try:
            while not self._stop.is_set():
                try:
                    item = self.inbox.get(timeout=0.05)
                except queue.Empty:
                    continue
                if item is not _WAKE:
                    self._take(item)
                if self._error is not None:       # a launch on a client thread failed
                    self._fail(self._error)
                    return
                self._drain_inbox()
                while self._admit_and_launch():
                    self._drain_inbox()
        except BaseException as e:              # surface engine errors to the client
            self._fail(e)

    def _take(self, req: "Request"):
        """A submitted request moves from the inbox to the FIFO wait list."""
        with self._lock:
            self._queued -= 1
        self.waiting.append(req)

    def _drain_inbox(self):
        while True:
            try:
                item = self.inbox.get_nowait()
            except queue.Empty:
                return
            if item is not _WAKE:
                self._take(item)

    def _admit_and_launch(self) -> bool:
        if not self.waiting:
            return False
        with self._lock:
            if not self.free_streams:
                return False
            batch, need = [], 0
            while self.waiting and len(batch) < self.max_batch:
                r = self.waiting[0]
                if self.in_use + need + r.device_bytes > self.budget:
                    break
                batch.append(self.waiting.popleft())
                need += r.device_bytes
            if not batch:
                return False
            self.in_use += need
            self.n_inflight += 1
            sid = self.free_streams.pop()
        self._launch_batch(batch, sid, need)
        return True

    def _launch_batch(self, batch: List[Request], sid: int, need: int, on_device=False,
                      idle=False):
        """Launches an admitted batch (stream `sid` and `need` bytes already
        reserved) and hands it to the completer.  on_device: called from a
        client thread, which may have another device current; idle: nothing
        else in flight (the client thread's own stream may then run it)."""
        t = time.perf_counter()
        try:
            direct = len(batch) <= self.DIRECT_MAX and all(r.resident for r in batch)
            for r in batch:
                r.path = ("idle" if on_device else "direct") if direct else "ragged"
            if on_device:
                with self._device_scope():
                    if direct:
                        b = self._launch_direct(batch, sid, need, on_caller_stream=idle)
                    else:
                        b = self._launch(batch, sid, need)
            elif direct:
                b = self._launch_direct(batch, sid, need)
            else:
                b = self._launch(batch, sid, need)
        except BaseException as e:
            # the batch never reached the GPU: fail its requests, give back
            # its budget and stream, then stop the server (the engine fails
            # the rest; a client thread re-raises to its caller)
            for r in batch:
                if not r.future.done():
                    r.future.set_exception(e)
            with self._lock:
                self.in_use -= need
                self.n_inflight -= 1
                self.free_streams.append(sid)
                if on_device and self._error is None:
                    self._error = e       # later submissions are refused
            if not on_device:
                raise
            self.inbox.put(_WAKE)         # the engine fails what is queued and stops
            return
        t = (time.perf_counter() - t) * 1e3
        with self._lock:
            self.stats["launch_ms_max"] = max(self.stats["launch_ms_max"], t)
        self.done_q.put(b)

    def _launch(self, reqs: List[Request], sid: int, need: int) -> dict:
        torch = self.torch
        stream = self.streams[sid]
        dev_name = f"cuda:{self.device}"
        n = len(reqs)
        sizes = np.fromiter((r.limbs * r.N for r in reqs), np.int64, n)
        res_off = np.zeros(n + 1, np.int64)
        np.cumsum(sizes, out=res_off[1:])
        host_reqs = [k for k, r in enumerate(reqs) if not r.resident]
        with torch.cuda.stream(stream):
            res = torch.empty(int(res_off[-1]), dtype=torch.int64, device=dev_name)
            res_ptr = res.data_ptr() + 8 * res_off[:-1]
            staged = pinned = None
            a_ptr = [0] * n
            b_ptr = [0] * n
            if host_reqs:
                # all host operands through one pinned buffer and one upload
                n_ops = [2 if reqs[k].op == "mul" else 1 for k in host_reqs]
                total = int(sum(int(sizes[k]) * m for k, m in zip(host_reqs, n_ops)))
                pinned = torch.empty(total, dtype=torch.int64, pin_memory=True)
                pv = pinned.numpy().view(np.uint64)
                staged = torch.empty(total, dtype=torch.int64, device=dev_name)
                base = staged.data_ptr()
                o = 0
                for k, m in zip(host_reqs, n_ops):
                    r, sz = reqs[k], int(sizes[k])
                    pv[o:o + sz] = r.a.reshape(-1)
                    a_ptr[k] = base + 8 * o
                    if m == 2:
                        pv[o + sz:o + 2 * sz] = r.b.reshape(-1)
                        b_ptr[k] = base + 8 * (o + sz)
                    o += m * sz
                staged.copy_(pinned, non_blocking=True)
            plans = self.plans
            handles = []
            for k, r in enumerate(reqs):
                p = plans.get((r.N, r.moduli))
                handles.append((p if p is not None else self.plan(r.N, r.moduli)).handle)
                if r.resident:
                    a_ptr[k] = r.a.data_ptr()
                    if r.op == "mul":
                        b_ptr[k] = r.b.data_ptr()
            # one ragged call per kind of request, each into its own workspace;
            # results back to back in `res`, operands read in place
            workspaces = []
            for op in OPS:
                idx = [k for k, r in enumerate(reqs) if r.op == op]
                if not idx:
                    continue
                h = [handles[k] for k in idx]
                if op == "mul":
                    arr = capi.polymul_items_array(h, [a_ptr[k] for k in idx],
                                                   [b_ptr[k] for k in idx], res_ptr[idx])
                    wsb = capi.hx_polymul_ragged_workspace(arr)
                    ws = self._workspace(sid, op, wsb, dev_name)
                    capi.hx_polymul_ragged(arr, ws, wsb, stream.cuda_stream)
                    self._count_launches(4)
                else:
                    arr = capi.ragged_items_array(h, [a_ptr[k] for k in idx], res_ptr[idx])
                    wsb = capi.hx_ntt_ragged_workspace(arr)
                    ws = self._workspace(sid, op, wsb, dev_name)
                    capi.hx_ntt_ragged(arr, ws, wsb, 1 if op == "fwd" else 2, 1, 1,
                                       stream.cuda_stream)
                    self._count_launches(2)
                workspaces.append(ws)
            out_host = None
            if host_reqs:
                out_host = torch.empty(int(res_off[-1]), dtype=torch.int64, pin_memory=True)
                out_host.copy_(res, non_blocking=True)
            ev = torch.cuda.Event(blocking=self.blocking_wait)
            ev.record(stream)
        with self._lock:
            self.stats["batches"] += 1
            self.stats["requests"] += n
            self.stats["max_batch"] = max(self.stats["max_batch"], n)
        work = (res, sizes, out_host, staged, pinned, workspaces)
        return {"reqs": reqs, "work": work, "event": ev, "sid": sid, "bytes": need}

    def _workspace(self, sid: int, op: str, nbytes: int, dev_name: str):
        """The workspace of a batch's ragged call of kind `op` on stream
        `sid`, kept per (stream, kind) and grown on demand: batches on one
        stream run in order, so the next one may reuse it; a replaced one
        goes back to the caching allocator's pool of that stream, whose
        later work runs after the batches that used it."""
        ws = self._batch_ws.get((sid, op))
        if ws is None or ws.numel() < nbytes:
            ws = self._batch_ws[(sid, op)] = self.torch.empty(
                max(nbytes, 1 << 20), dtype=self.torch.uint8, device=dev_name)
        return ws

    def _count_launches(self, k: int):
        with self._lock:
            self.stats["launches"] += k

    # ------------------------------------------------------------ completer
    def _complete(self):
        self._bind_device()
        while True:
            b = self.done_q.get()
            if b is None:
                return
            try:
                ev = b["event"]
                polled = False
                if self.poll_s > 0:
                    # a short batch is often done within a few hundred
                    # microseconds: poll (yielding the interpreter lock between
                    # queries) before the blocking wait's sleep-and-wake
                    deadline = time.perf_counter() + self.poll_s
                    while not (polled := ev.query()) and time.perf_counter() < deadline:
                        time.sleep(0)
                if not polled:
                    ev.synchronize()
                now = time.perf_counter()
                res, sizes, out_host, _, _, _ = b["work"]
                parts = res.split(sizes.tolist())        # one view per request
                hv = out_host.numpy().view(np.uint64) if out_host is not None else None
                lo = 0
                for r, part in zip(b["reqs"], parts):
                    hi = lo + part.numel()
                    if r.resident:
                        r.result = part.view(r.limbs, r.N)
                    else:
                        r.result = hv[lo:hi].reshape(r.limbs, r.N).copy()
                    lo = hi
                    r.done = now
                # the batch's budget and stream are free before its futures
                # resolve: a client that submits as soon as it has its result
                # finds the server idle
                self._release(b)
                for r in b["reqs"]:
                    r.future.set_result(r.result)
                t = (time.perf_counter() - now) * 1e3
                with self._lock:
                    self.stats["complete_ms_max"] = max(self.stats["complete_ms_max"], t)
                    self.stats["completed_by_polling"] += polled
            except BaseException as e:
                self._error = e
                self._release(b)
                for r in b["reqs"]:
                    if not r.future.done():
                        r.future.set_exception(e)
            # the engine needs waking only for requests that wait for the
            # budget or a stream this batch gave back (a later submission
            # wakes it on its own)
            if self.waiting or self._queued or self._error is not None:
                self.inbox.put(_WAKE)

    def _release(self, b: dict):
        with self._lock:
            if b.get("released"):
                return
            b["released"] = True
            self.in_use -= b["bytes"]
            self.free_streams.append(b["sid"])
            self.n_inflight -= 1


def serve_one_by_one(reqs: Sequence[Request], arrivals: Optional[Sequence[float]] = None,
                     plans: Optional[dict] = None, device: int = 0) -> None:
    """The unbatched baseline: each request alone, in arrival order, with the
    plain per-request calls (upload, hx_poly_mul or hx_ntt_forward /
    hx_ntt_inverse, download, wait).  When
    `arrivals` (offsets in seconds) are given, a request does not start
    before its arrival time; latency counts from arrival."""
    import torch
    plans = {} if plans is None else plans
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        if arrivals is not None:
            wait = arrivals[i] - (time.perf_counter() - t0)
            if wait > 1e-4:                       # sleep (not spin) until the arrival
                time.sleep(wait - 5e-5)
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            r.arrival = t0 + arrivals[i]
        else:
            r.arrival = time.perf_counter()
        key = (r.N, tuple(r.moduli))
        if key not in plans:
            plans[key] = capi.Plan(r.N, key[1])
        dev = f"cuda:{device}"
        if r.op == "mul":
            if r.resident:
                a, b = r.a.clone(), r.b.clone()     # hx_poly_mul overwrites its operands
            else:
                a = torch.from_numpy(r.a.view(np.int64)).to(dev, non_blocking=True)
                b = torch.from_numpy(r.b.view(np.int64)).to(dev, non_blocking=True)
            capi.hx_poly_mul(plans[key], a, a, b, 1, stream.cuda_stream)
        else:
            x = r.a if r.resident else torch.from_numpy(r.a.view(np.int64)).to(
                dev, non_blocking=True)
            a = torch.empty_like(x)
            (capi.hx_ntt_forward if r.op == "fwd" else capi.hx_ntt_inverse)(
                plans[key], a, x, 1, 1, 1, stream.cuda_stream)
        if r.resident:
            stream.synchronize()
            r.result = a
        else:
            r.result = a.cpu().numpy().view(np.uint64)
        r.done = time.perf_counter()
