"""Throughput of the negacyclic NTT hot path on GB300, one JSON line.

Workload (one step): the ciphertext-shaped product at N = 65536 with 32 RNS
limbs of mixed 30/50/60-bit primes -- two ciphertexts of two polynomials
each.  Forward NTT of the four input polynomials (output range [0, 4q)),
the fused tensor product d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 with the
scaled accumulation r_k = d_k s + e_k (EltwiseFMAMod), inverse NTT of r_0..2:
7 x 32 = 224 limb-transforms per step.  Inputs are seeded synthetic uniform
residues already resident in HBM; three input sets rotate so the working set
(3 x 112 MiB of inputs plus 112 MiB of intermediates) exceeds the 129 MB L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hexgpu|reference]

Multi-GPU (torchrun, one rank per GPU): each rank runs the same per-GPU
workload on its own GPU (limbs and polynomials are independent; no data-path
collective), timing is the max over ranks, value is the whole-job total.

--impl reference times the CPU oracle (plain C, one thread) on a bounded
sample of the same workload: the pipeline on three limbs (one per width).
"""
from __future__ import annotations

import argparse
import ctypes
import gc
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_2103_16400_gb300 import shard  # noqa: E402

METRIC = "NTT limb-transforms/s at N=2^16 (% of int-mul/HBM roofline); served p99 latency"
UNIT = "limb-transforms/s"
N_DEFAULT = 1 << 16
LIMBS_DEFAULT = 32


# ------------------------------------------------------------------ workload
def workload_arrays(N, n_limbs, n_sets, rank=0):
    """n_sets input sets, each (ins, es): ins = [a0, a1, b0, b1], es = [e0, e1,
    e2], every one a [1][n_limbs][N] uint64 array of uniform residues.  Under
    weak scaling each rank draws its own independent sets (same shapes)."""
    wl = W.ciphertext_tensor(N=N, n_limbs=n_limbs)
    seed = shard.rank_seed(wl.seed, rank)
    sets = []
    for k in range(n_sets):
        ins = [W.poly_batch(seed + 1000 * k, t, 1, wl.moduli, N) for t in range(4)]
        es = [W.poly_batch(seed + 1000 * k, 10 + t, 1, wl.moduli, N) for t in range(3)]
        sets.append((ins, es))
    s = W.scalars(wl.seed, 20, wl.moduli)
    return wl, sets, s


def device_sets(sets):
    """Each set as two device tensors: the four inputs back to back [4][L][N]
    and the three addends [3][L][N]."""
    from paper_2103_16400_gb300.tensors import to_device
    return [(to_device(np.concatenate(ins)), to_device(np.concatenate(es))) for ins, es in sets]


#: IMAD-pipe issue slots of one Shoup butterfly as the kernels compute it, in
#: units of one 32-bit mad.lo (the probes measure mad.hi at half that rate
#: and mad.wide at under half): a full 32x32-bit product counts 1 + 2.
#: 64-bit words, q < 2^61 (truncated quotient) -- high word of W'X from three
#: partial products (two high halves, one full product: 2*2 + 3 = 7), plus
#: the remainder W X - Q q mod 2^64 from two full low products and four low
#: halves (2*3 + 4 = 10): 17.  64-bit words, q >= 2^61 (exact quotient) --
#: high word from four partial products (2 + 3*3 = 11) plus the remainder:
#: 21.  32-bit words -- one high half and two low halves (2 + 1 + 1 = 4).
SLOTS_WIDE_TRUNC, SLOTS_WIDE, SLOTS_NARROW = 17, 21, 4


def slots_per_butterfly(q):
    if q < (1 << 30):
        return SLOTS_NARROW
    return SLOTS_WIDE_TRUNC if q < (1 << 61) else SLOTS_WIDE


#: IMAD slots of the ciphertext tensor's element-wise step per coefficient
#: position (three outputs), in the same units, as the fused kernels compute
#: it (tensor_r3): two Shoup products a' = a s (a butterfly's multiply each:
#: 17, or 21 with the exact quotient), three 128-bit products (four full
#: 32x32 products each, 12; d1 by Karatsuba) and three Barrett reductions
#: (the high word of c1 k -- truncated 7, exact 11 -- and the low word of
#: c3 q, 5).  64-bit words below 2^61: 2 * 17 + 3 * 12 + 3 * (7 + 5) = 106;
#: at or above 2^61: 2 * 21 + 3 * 12 + 3 * (11 + 5) = 126.  32-bit words: a
#: Shoup product 4, a product one full 32x32 (3), a reduction one high half
#: and one low half (2 + 1): 2 * 4 + 3 * 3 + 3 * 3 = 26.
SLOTS_TENSOR_WIDE_TRUNC, SLOTS_TENSOR_WIDE, SLOTS_TENSOR_NARROW = 106, 126, 26


def slots_per_tensor_position(q):
    if q < (1 << 30):
        return SLOTS_TENSOR_NARROW
    return SLOTS_TENSOR_WIDE_TRUNC if q < (1 << 61) else SLOTS_TENSOR_WIDE


def kernel_source_hash():
    """Short hash of the library's sources (kernels and host launch code): a
    DRAM-traffic figure captured with ncu is reported only while the sources
    it was captured from are the ones running."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_16400_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(f.encode())
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


#: DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) at N = 65536 x 32
#: mixed limbs from ncu captures, keyed by (kernel name or "forward_call",
#: schedule JSON -- the inverse schedule for the fused tensor pass and the
#: step kernel --, kernel_source_hash() of the captured build).  A key whose
#: hash is not the running build's gives no figure (the field is null), so a
#: changed kernel never reports stale traffic.  profiles/ records the
#: capture commands.
TRAFFIC_BYTES = {
    ("forward_call", "[[0, 7, 0, 4, 4, 0, 1], [7, 9, 0, 0, 3, 0, 1]]",
     "4117db26c6aea96b"): 67256064 + 16780800 + 100656128 + 13868288,
    ("forward_call", "[[0, 8, 0, 3, 4, 0, 1], [8, 8, 1, 0, 3, 0, 1]]",
     "4117db26c6aea96b"): 67320064 + 22699776 + 100587776 + 13716992,
    ("forward_call", "[[0, 8, 0, 3, 4, 0, 1], [8, 8, 2, 0, 3, 0, 1]]",
     "4117db26c6aea96b"): 67319808 + 22932992 + 100590080 + 13775616,
    ("forward_call", "[[0, 7, 0, 3, 4, 0, 1], [7, 9, 0, 0, 3, 0, 1]]",
     "4117db26c6aea96b"): 67253760 + 23036160 + 100656640 + 13927680,
    ("ntt_tensor_inv_kernel<3, 9, 0, 3>", "[[0, 7, 0, 3, 4, 0, 1], [7, 9, 0, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 151037696 + 20775680,
    ("ntt_tensor_inv_kernel<3, 9, 0, 3>", "[[0, 7, 0, 4, 4, 0, 1], [7, 9, 0, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 151021568 + 20788224,
    ("ntt_tensor_inv_kernel<3, 9, 0, 3>", "[[0, 7, 0, 4, 4, 2, 1], [7, 9, 0, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 151013632 + 20402688,
    ("ntt_ct_row_kernel<3, 9>", "[[0, 7, 0, 4, 4, 0, 1], [7, 9, 1, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 184727552 + 26205696,
    ("ntt_ct_row_kernel<3, 8>", "[[0, 8, 0, 3, 4, 0, 1], [8, 8, 1, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 184367360 + 26626304,
    ("ntt_ct_row_kernel<3, 9>", "[[0, 7, 0, 4, 4, 0, 1], [7, 9, 0, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 184738304 + 26228992,
    ("ntt_ct_row_kernel<3, 9>", "[[0, 7, 0, 4, 4, 2, 1], [7, 9, 1, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 184725248 + 26214400,
    ("ntt_ct_row_kernel<3, 9>", "[[0, 7, 0, 3, 4, 0, 1], [7, 9, 1, 0, 3, 0, 2]]",
     "4117db26c6aea96b"): 184711936 + 26242304,
}


def traffic_for(what, sched):
    if sched is None:
        return None
    return TRAFFIC_BYTES.get((what, json.dumps([list(p) for p in sched]), kernel_source_hash()))


#: The roofline's plain operation count: a Shoup butterfly on 64-bit words is
#: 10 IMAD-class operations (the high word of W'X from four 32x32-bit partial
#: products, the low words of W X and Q q from three each), on 32-bit words 3,
#: each counted at the mad.lo issue rate; the memory side is one HBM read and
#: one write of every coefficient (operands read, results written) at the
#: measured copy bandwidth; the bound is the slower of the two.
OPS_WIDE, OPS_NARROW = 10, 3


def ops_per_butterfly(q):
    return OPS_NARROW if q < (1 << 30) else OPS_WIDE


def _kernel_shape(kid, N):
    """(kind, forward, stages, ends the inverse, tensor-fused) of a kernel id."""
    kind, fwd, column, K = kid & 3, (kid >> 2) & 1, (kid >> 3) & 1, (kid >> 7) & 31
    if kind == 3:                                   # cluster-fused: K1 + K2 stages
        K += (kid >> 15) & 31
        return kind, fwd, K, not fwd, bool((kid >> 12) & 1)
    return kind, fwd, K, (not fwd) and (column or K == N.bit_length() - 1), kind == 2


def kernel_slots(kid, N, moduli, n_ct=1, per_butterfly=None):
    """Algorithmic IMAD work of one launch of a timed kernel in the step: a
    pass over its K stages (four polynomials forward, three inverse), a
    cluster-fused launch over all stages, a fused pass (the element-wise
    tensor step plus its inverse stages on three polynomials per ciphertext
    pair), or the step kernel (the same plus the forward's K row stages on
    the four operands).  An inverse launch that ends the transform also scales by N^-1
    (Algorithm GS's final loop): folded into its last stage, that is one
    more Shoup product per butterfly there.  In IMAD slots by default; with
    per_butterfly=ops_per_butterfly, the plain operation count (butterflies
    and N^-1 products only)."""
    kind, fwd, K, ends_inv, tensor = _kernel_shape(kid, N)
    per = per_butterfly or slots_per_butterfly
    bfly = sum(N // 2 * K * per(q) for q in moduli)
    if ends_inv:
        bfly += sum(N // 2 * per(q) for q in moduli)
    if tensor:
        extra = 0 if per_butterfly else sum(N * slots_per_tensor_position(q) for q in moduli)
        if (kid >> 17) & 1:
            # the product's step kernel: the forward's row stages on a and b,
            # the inverse's on their product (the dyadic product not counted)
            return n_ct * 3 * bfly
        if (kid >> 16) & 1:
            # the step kernel: the forward's row stages on four polynomials
            # as well, as many stages as the inverse's
            return n_ct * (7 * bfly + extra)
        return n_ct * (3 * bfly + extra)
    return (4 if fwd else 3) * n_ct * bfly


def kernel_bytes(kid, N, n_limbs, n_ct=1):
    """Algorithmic HBM bytes of one launch: a pass or a transform reads and
    writes each coefficient once (four polynomials forward, three inverse);
    the tensor-fused launch and the step kernel read the seven operands
    (A0, A1, B0, B1 -- spectra, or the forward's column pass output -- and
    e0, e1, e2) and write their three outputs."""
    kind, fwd, K, ends_inv, tensor = _kernel_shape(kid, N)
    if tensor and (kid >> 17) & 1:
        return 3 * 8 * N * n_limbs * n_ct        # the product's: a, b in, a b out
    if tensor:
        return 10 * 8 * N * n_limbs * n_ct
    return 2 * (4 if fwd else 3) * 8 * N * n_limbs * n_ct


def op_roofline(ops, nbytes, us, imad_rate, hbm_gbs):
    """The roofline of `ops` integer operations and `nbytes` of HBM traffic
    done in `us` microseconds: the slower side is the bound; achieved and
    peak are that side's rate."""
    t_int = ops / imad_rate * 1e6
    t_hbm = nbytes / (hbm_gbs * 1e9) * 1e6
    if t_int >= t_hbm:
        return {"bound": "alu", "achieved": ops / (us * 1e-6) / 1e12, "peak": imad_rate / 1e12,
                "unit": "T IMAD-op/s", "frac": t_int / us, "int_us": t_int, "hbm_us": t_hbm}
    return {"bound": "hbm", "achieved": nbytes / (us * 1e-6) / 1e9, "peak": hbm_gbs,
            "unit": "GB/s", "frac": t_hbm / us, "int_us": t_int, "hbm_us": t_hbm}


def step_work(N, moduli):
    """Algorithmic work of one timed step (forward call over four
    polynomials; tensor step and inverse over three with N^-1): (operations
    of the operation count, IMAD slots of the slot model, HBM bytes: the
    forward reads 4 and writes 4 polynomials, the tensor + inverse call reads
    the 4 spectra and 3 addends and writes 3 results)."""
    logn = N.bit_length() - 1
    nl = len(moduli)
    ops = (4 * logn + 3 * (logn + 1)) * sum(N // 2 * ops_per_butterfly(q) for q in moduli)
    slots = ((4 * logn + 3 * (logn + 1)) * sum(N // 2 * slots_per_butterfly(q) for q in moduli)
             + sum(N * slots_per_tensor_position(q) for q in moduli))
    nbytes = (8 + 10) * 8 * N * nl
    return ops, slots, nbytes


def imad_slots_per_transform(N, moduli):
    """Algorithmic IMAD-pipe slots of one limb-transform: N/2 log2 N Harvey
    butterflies, each one Shoup product."""
    logn = N.bit_length() - 1
    bf = N // 2 * logn
    return [bf * slots_per_butterfly(q) for q in moduli]


#: CUDA streams the timed steps alternate over: consecutive steps are
#: independent batches, so step i + 1's kernels fill the SMs (and the last
#: waves) that step i's latency-bound kernels leave idle -- measured on GB300
#: at N = 2^16 x 32 limbs: 192.4 us a step on one stream, 164.3 us on two,
#: 178.7 us on three.
STEP_STREAMS = 2


class HexStep:
    """The timed step, through the C ABI, with autotuned schedules: the
    ciphertext product of four inputs into three results.  It runs as
    hx_ciphertext_step (three launches: the forward's column pass, one kernel
    for the forward's row stages, the tensor step and the inverse's row
    stages, the inverse's column pass) on a plan tuned for that call, unless
    the composition -- one forward call over the four inputs, then the
    tensor/FMA step fused into the inverse of the three outputs, on a plan
    tuned for those two calls -- times faster.  Step i runs on stream
    i mod `n_streams` with that stream's own preallocated buffers (A: the
    four spectra or the forward column pass's output, R: the three results),
    so steps on different streams overlap and every step does its whole work
    on its own batch."""

    def __init__(self, N, moduli, s, dev_sets, torch, tune=True, n_streams=STEP_STREAMS,
                 path=None):
        from paper_2103_16400_gb300 import capi, tune as hx_tune
        from paper_2103_16400_gb300.tensors import empty
        self.capi, self.torch = capi, torch
        self.N, self.moduli, self.s = N, moduli, s
        self.plan = capi.Plan(N, moduli)          # the composition's two calls
        self.step_plan = capi.Plan(N, moduli)     # hx_ciphertext_step (tables shared)
        self.tuned = {}
        if tune:
            self.tuned = {"forward": hx_tune.tune(self.plan, 4, direction=capi.Plan.FORWARD),
                          "inverse": hx_tune.tune_tensor(self.plan, 1, s),
                          "step": hx_tune.tune_step(self.step_plan, 1, s, iters=8,
                                                    streams=n_streams)}
        self.dev_sets = dev_sets
        L = len(moduli)
        self.stream = torch.cuda.current_stream()
        self.streams = [self.stream] + [torch.cuda.Stream() for _ in range(n_streams - 1)]
        self.bufs = [(empty((4, L, N)), empty((3, L, N))) for _ in range(n_streams)]
        self.A, self.R = self.bufs[0]
        self.fwd_events = []
        self.inv_events = []
        self.step_events = []
        if path is None:
            times = {p: self.time_path(p) for p in ("step", "composed")}
            path = min(times, key=times.get)
            self.path_us = times
        self.path = path

    def time_path(self, path, n=100):
        """Mean device time of one step by one path, the steps alternating
        over the step streams as the timed region runs them."""
        torch = self.torch
        for i in range(4):
            self.run(i, path=path)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        self.begin(e0)
        for i in range(n):
            self.run(i, path=path)
        self.join()
        e1.record(self.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / n

    def begin(self, ev):
        """Every step stream waits for `ev` (recorded on the first stream)."""
        for st in self.streams[1:]:
            st.wait_event(ev)

    def join(self):
        """The first stream waits for every other step stream's work."""
        for st in self.streams[1:]:
            e = self.torch.cuda.Event()
            e.record(st)
            self.stream.wait_event(e)

    def run(self, i, record=False, one_stream=False, path=None):
        """Step i: on stream i mod n_streams (on the first stream alone with
        one_stream, or when recording per-call events), by `path` ("step" or
        "composed"; the chosen one by default).  With record, the composed
        path records its two calls' events, the step path its call's."""
        c, N = self.capi, self.N
        path = path or self.path
        k = 0 if (one_stream or record) else i % len(self.streams)
        st = self.streams[k]
        self.A, self.R = self.bufs[k]
        ins, es = self.dev_sets[i % len(self.dev_sets)]
        A, R = self.A, self.R
        if path == "step":
            if record:
                e0 = self.torch.cuda.Event(enable_timing=True)
                e1 = self.torch.cuda.Event(enable_timing=True)
                e0.record(st)
            c.hx_ciphertext_step(self.step_plan, R, ins, A, self.s, es, 1, st)
            if record:
                e1.record(st)
                self.step_events.append((e0, e1))
            return [R[0:1], R[1:2], R[2:3]]
        if record:
            e0 = self.torch.cuda.Event(enable_timing=True)
            e1 = self.torch.cuda.Event(enable_timing=True)
            e0.record(st)
        c.hx_ntt_forward(self.plan, A, ins, 4, 1, 4, st)
        if record:
            e1.record(st)
            self.fwd_events.append((e0, e1))
        # tensor, FMA and inverse NTT: the element-wise step runs inside the
        # inverse's first pass (operands back to back)
        c.hx_tensor_fma_inverse(self.plan, R[0], R[1], R[2], A[0], A[1], A[2], A[3], self.s,
                                es[0], es[1], es[2], 1, 4, st)
        if record:
            e2 = self.torch.cuda.Event(enable_timing=True)
            e2.record(st)
            self.inv_events.append((e1, e2))
        return [R[0:1], R[1:2], R[2:3]]

    def kernel_plan(self):
        """The plan whose schedules the timed step's kernels run."""
        return self.step_plan if self.path == "step" else self.plan


# ------------------------------------------------------------------ ragged batch
#: the ragged kernels' column-pass stages per log2 N before any tuning
RAGGED_DEFAULT_SPLITS = {12: 5, 13: 6, 14: 7, 15: 7, 16: 8, 17: 8}


def ragged_report(torch, imad_rate=None, hbm_gbs=None, n_polys=512, reps=5):
    """The ragged workload (N ~ U{2^10..2^17}, 1-32 limbs of 30/50/60 bits):
    forward NTT of every polynomial as one graph replay of the persistent
    ragged kernels -- with the default pass shapes and with the shapes the
    ragged autotuner picks per N -- against one plain launch per
    (polynomial, limb) and one call per polynomial; outputs of all are
    compared on the device.  The tuned batch's roofline fraction is the
    operation count's (N/2 log2 N butterflies per transform, 10 or 3
    operations each, against 16 bytes of HBM per coefficient)."""
    from paper_2103_16400_gb300 import capi, tune as hx_tune
    from paper_2103_16400_gb300.tensors import empty, to_device
    entries = W.ragged_batch(n_polys)
    plans, dins, douts, dref, dref2 = [], [], [], [], []
    for k, (N, qs) in enumerate(entries):
        x = W.poly_batch(W.SEED_BASE + 4, k, 1, qs, N)
        plans.append(capi.Plan(N, qs))
        dins.append(to_device(x))
        douts.append(empty(x.shape))
        dref.append(empty(x.shape))
        dref2.append(empty(x.shape))
    items = [(p, i, o, 1) for p, i, o in zip(plans, dins, douts)]
    for L, k1 in RAGGED_DEFAULT_SPLITS.items():
        capi.hx_ragged_set_split(L, k1)
    dfixed = [empty(o.shape) for o in douts]
    fixed = capi.Batch([(p, i, o, 1) for p, i, o in zip(plans, dins, dfixed)], 1, 1, 1)
    tuned_splits = hx_tune.tune_ragged(items)    # applied process-wide from here on
    batch = capi.Batch(items, 1, 1, 1)
    info = batch.info()
    one_limb = {}
    for (N, qs) in entries:
        for q in qs:
            if (N, q) not in one_limb:
                one_limb[(N, q)] = capi.Plan(N, [q])
    st = torch.cuda.current_stream()

    def per_limb():
        for (N, qs), i, o in zip(entries, dins, dref):
            for l, q in enumerate(qs):
                capi.hx_ntt_forward(one_limb[(N, q)], o[0, l], i[0, l], 1, 1, 1, st)

    def per_poly():
        for p, i, o in zip(plans, dins, dref2):
            capi.hx_ntt_forward(p, o, i, 1, 1, 1, st)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_fixed = timed(lambda: fixed.run(st))
    t_batch = timed(lambda: batch.run(st))
    t_limb = timed(per_limb)
    t_poly = timed(per_poly)
    same = all(torch.equal(a, b) and torch.equal(a, c) and torch.equal(a, d)
               for a, b, c, d in zip(douts, dref, dref2, dfixed))
    lt = info["limb_transforms"]
    ops = sum(N // 2 * (N.bit_length() - 1) * ops_per_butterfly(q) for N, qs in entries
              for q in qs)
    nbytes = sum(16 * N * len(qs) for N, qs in entries)
    roof = (op_roofline(ops, nbytes, t_batch * 1e3, imad_rate, hbm_gbs)
            if imad_rate and hbm_gbs else None)
    return {"workload": f"ragged_{n_polys}_polys_N2^10..2^17_1-32_limbs",
            "limb_transforms": lt, "tiles": info["tiles"], "launches_per_replay": info["launches"],
            "batch_ms": t_batch, "batch_limb_transforms_per_s": lt / (t_batch * 1e-3),
            "fixed_menu_ms": t_fixed, "tuned_over_fixed_speedup": t_fixed / t_batch,
            "splits": {"tuned": {L: r["k1"] for L, r in tuned_splits.items()},
                       "fixed": RAGGED_DEFAULT_SPLITS},
            "roofline": roof,
            "per_limb_launch_ms": t_limb, "per_limb_limb_transforms_per_s": lt / (t_limb * 1e-3),
            "per_poly_call_ms": t_poly, "per_poly_limb_transforms_per_s": lt / (t_poly * 1e-3),
            "speedup_vs_per_limb": t_limb / t_batch, "bit_exact_equal": bool(same)}


# ------------------------------------------------------------------ element-wise
def hbm_peak_gbs():
    """Measured copy bandwidth (read + write bytes) of this machine's GPUs, from
    the peaks file at the repository root, else the profiling fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def ntt_rates_report(torch, step, dev_sets, imad_rate, hbm_gbs, iters=200):
    """The plain transforms of the step's plan timed on their own: the forward
    call (four polynomials, the step's inputs rotating over the input sets)
    and the inverse call (three polynomials from the addend sets, rotating --
    values in [0, q)), CUDA events on the launching stream; their
    limb-transform rates, forward + inverse, and the forward + inverse
    roofline fraction (the inverse's slots include the N^-1 scaling).  Then
    the same step with L2 warm: one input set, no rotation."""
    from paper_2103_16400_gb300 import capi
    from paper_2103_16400_gb300.tensors import empty
    N, moduli, st = step.N, step.moduli, step.stream
    nl = len(moduli)
    R = empty((3, nl, N))
    out = empty((4, nl, N))

    def timed(fn):
        for i in range(3):
            fn(i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for i in range(iters):
            fn(i)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / iters * 1e3          # us per call

    fwd_us = timed(lambda i: capi.hx_ntt_forward(step.plan, out, dev_sets[i % len(dev_sets)][0],
                                                 4, 1, 1, st))
    inv_us = timed(lambda i: capi.hx_ntt_inverse(step.plan, R, dev_sets[i % len(dev_sets)][1],
                                                 3, 1, 1, st))
    warm_ms = timed(lambda i: step.run(0, one_stream=True)) / 1e3
    # forward + inverse pairs alternating over the step streams (pair i on
    # stream i mod n, each stream with its own output buffers): throughput
    # of independent pairs, as the timed step runs
    bufs = [(empty((4, nl, N)), empty((3, nl, N))) for _ in step.streams]

    def pair(i):
        k = i % len(step.streams)
        s_k = step.streams[k]
        o4, o3 = bufs[k]
        capi.hx_ntt_forward(step.plan, o4, dev_sets[i % len(dev_sets)][0], 4, 1, 1, s_k)
        capi.hx_ntt_inverse(step.plan, o3, dev_sets[i % len(dev_sets)][1], 3, 1, 1, s_k)

    for i in range(3):
        pair(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    step.begin(e0)
    for i in range(iters):
        pair(i)
    step.join()
    e1.record(st)
    torch.cuda.synchronize()
    pair_us = e0.elapsed_time(e1) / iters * 1e3
    out = fwd_inv_figures(N, moduli, fwd_us, inv_us, imad_rate, hbm_gbs)
    two = fwd_inv_figures(N, moduli, pair_us * fwd_us / (fwd_us + inv_us),
                          pair_us * inv_us / (fwd_us + inv_us), imad_rate, hbm_gbs)
    out["two_streams"] = {"pair_us": pair_us,
                          "fwd_plus_inv_frac": two["fwd_plus_inv_frac"],
                          "fwd_plus_inv_frac_slots": two["fwd_plus_inv_frac_slots"],
                          "limb_transforms_per_s": 7 * nl / (pair_us * 1e-6),
                          "how": f"a forward call (4 polynomials) and an inverse call (3) per "
                                 f"pair, pairs alternating over {len(step.streams)} streams "
                                 f"with their own buffers, {iters} pairs"}
    out.update({"schedules": {"forward": step.plan.schedule(step.plan.FORWARD),
                              "inverse": step.plan.schedule(step.plan.INVERSE)},
                "l2_warm_step": {"ms_per_step": warm_ms,
                                 "limb_transforms_per_s": 7 * nl / (warm_ms * 1e-3),
                                 "how": "the step on one input set, no rotation, one stream"},
                "how": f"{iters} calls each, CUDA events, inputs rotating over "
                       f"{len(dev_sets)} sets (> L2); *_frac: operation-count roofline, "
                       f"*_frac_slots: IMAD-slot model"})
    return out


def fwd_inv_figures(N, moduli, fwd_us, inv_us, imad_rate, hbm_gbs):
    """Rates and roofline fractions of a forward call over four polynomials
    (fwd_us) and an inverse call over three (inv_us, with the N^-1 scaling)
    on all limbs: the operation-count roofline of each call (the slower of
    its integer and HBM sides) and of the two together, and the IMAD-slot
    model's fraction of the two together."""
    nl = len(moduli)
    slots_f = sum(imad_slots_per_transform(N, moduli))        # one polynomial, all limbs
    slots_i = slots_f + sum(N // 2 * slots_per_butterfly(q) for q in moduli)
    t_f, t_i = fwd_us / (4 * nl), inv_us / (3 * nl)           # us per limb-transform
    logn = N.bit_length() - 1
    ops_f = sum(N // 2 * logn * ops_per_butterfly(q) for q in moduli)
    ops_i = ops_f + sum(N // 2 * ops_per_butterfly(q) for q in moduli)
    rf = op_roofline(4 * ops_f, 4 * 16 * N * nl, fwd_us, imad_rate, hbm_gbs)
    ri = op_roofline(3 * ops_i, 3 * 16 * N * nl, inv_us, imad_rate, hbm_gbs)
    bound_us = max(rf["int_us"], rf["hbm_us"]) + max(ri["int_us"], ri["hbm_us"])
    return {"forward_us": fwd_us, "inverse_us": inv_us,
            "forward_limb_transforms_per_s": 1e6 / t_f,
            "inverse_limb_transforms_per_s": 1e6 / t_i,
            "fwd_plus_inv_pairs_per_s": 1e6 / (t_f + t_i),
            "fwd_plus_inv_frac": bound_us / (fwd_us + inv_us),
            "fwd_plus_inv_frac_slots":
                (4 * slots_f + 3 * slots_i) / ((fwd_us + inv_us) * 1e-6) / imad_rate,
            "forward_frac": rf["frac"], "forward_bound": rf["bound"],
            "inverse_frac": ri["frac"], "inverse_bound": ri["bound"]}


def eltwise_report(torch, N=1 << 16, nl=32, P=4, reps=20):
    """The element-wise kernels on 4 polynomials x 32 limbs x 65536 (64 MiB
    an operand; two rotating operand sets exceed L2): algorithmic HBM bytes
    (8 B per operand element read or written) per second against the
    measured copy bandwidth."""
    from paper_2103_16400_gb300 import capi
    from paper_2103_16400_gb300.tensors import empty, to_device
    wl = W.ciphertext_tensor(N=N, n_limbs=nl)
    mods = wl.moduli
    sets = [(to_device(W.poly_batch(wl.seed + 40 + k, 0, P, mods, N)),
             to_device(W.poly_batch(wl.seed + 40 + k, 1, P, mods, N)),
             to_device(W.poly_batch(wl.seed + 40 + k, 2, P, mods, N))) for k in range(2)]
    outs = [empty((P, nl, N)) for _ in range(2)]
    s = W.scalars(wl.seed, 21, mods)
    st = torch.cuda.current_stream()
    peak, src = hbm_peak_gbs()
    ops = {
        "add": (3, lambda a, b, d, r: capi.hx_eltwise_add_mod(r, a, b, N, mods, P, st)),
        "sub": (3, lambda a, b, d, r: capi.hx_eltwise_sub_mod(r, a, b, N, mods, P, st)),
        "negate": (2, lambda a, b, d, r: capi.hx_eltwise_negate_mod(r, a, N, mods, P, st)),
        "mult": (3, lambda a, b, d, r: capi.hx_eltwise_mult_mod(r, a, b, N, mods, P, 1, st)),
        "fma": (3, lambda a, b, d, r: capi.hx_eltwise_fma_mod(r, a, s, d, N, mods, P, 1, st)),
        "fma_no_addend": (2, lambda a, b, d, r: capi.hx_eltwise_fma_mod(r, a, s, None, N, mods,
                                                                        P, 1, st)),
    }
    out = {"workload": f"{P} polys x {nl} limbs x {N}, mixed 30/50/60-bit",
           "peak_gbs": peak, "peak_source": f"{src} copy bandwidth (read + write bytes)"}
    for name, (operands, fn) in ops.items():
        for k in range(2):
            fn(*sets[k], outs[k])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(reps):
            fn(*sets[i % 2], outs[i % 2])
        e1.record(st)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        gbs = operands * 8 * P * nl * N / (us * 1e-6) / 1e9
        out[name] = {"us": us, "alg_gbs": gbs, "frac": gbs / peak}
    return out


# ------------------------------------------------------------------ serving
def cgroup_cpu():
    """The container's CPU quota and throttling counters (cgroup v2, else v1),
    or None: a quota that runs out stalls every thread of the process until
    the next period, which shows in tail latency."""
    for d in ("/sys/fs/cgroup", "/sys/fs/cgroup/cpu,cpuacct", "/sys/fs/cgroup/cpu"):
        try:
            with open(os.path.join(d, "cpu.stat")) as f:
                st = dict(line.split() for line in f if len(line.split()) == 2)
        except OSError:
            continue
        out = {"nr_throttled": int(st.get("nr_throttled", 0)),
               "throttled_usec": int(st.get("throttled_usec", int(st.get("throttled_time", 0)) // 1000))}
        try:
            with open(os.path.join(d, "cpu.max")) as f:
                quota, period = f.read().split()
            out["quota_cpus"] = None if quota == "max" else int(quota) / int(period)
        except (OSError, ValueError):
            try:
                with open(os.path.join(d, "cpu.cfs_quota_us")) as f:
                    quota = int(f.read())
                with open(os.path.join(d, "cpu.cfs_period_us")) as f:
                    period = int(f.read())
                out["quota_cpus"] = None if quota < 0 else quota / period
            except (OSError, ValueError):
                out["quota_cpus"] = None
        return out
    return None


def _throttled_since(before):
    now = cgroup_cpu()
    if before is None or now is None:
        return None
    return {"periods": now["nr_throttled"] - before["nr_throttled"],
            "usec": now["throttled_usec"] - before["throttled_usec"]}


def precise_sleep():
    """Sets this thread's timer slack to 1 ns (Linux prctl, a setting of the
    calling thread alone), so that its sleeps end when asked instead of up
    to 50 us later: the load generators then submit on schedule."""
    try:
        libc = ctypes.CDLL(None)
        libc.prctl(29, 1, 0, 0, 0)            # PR_SET_TIMERSLACK
    except (OSError, AttributeError):
        pass


def serving_report(torch, rates=(2000, 8000, 32000), n_req=2000, budget=64 << 30,
                   blocking_wait=False):
    """Poisson arrivals of polynomial-multiply requests (N uniform over
    {2^12, 2^14, 2^16}, 4-32 limbs of the mixed 30/50/60-bit basis, operands
    uniform mod q and resident in HBM) at each rate: the continuous-batching
    server against the same requests served one by one with plain calls.
    Reports throughput and p50/p99 latency and checks every result is the
    same bits both ways."""
    from paper_2103_16400_gb300 import serve
    from paper_2103_16400_gb300.tensors import to_device
    precise_sleep()
    moduli = W.mixed_width_primes(32)
    Ns = (1 << 12, 1 << 14, 1 << 16)
    pool = {N: [(to_device(W.poly_batch(W.SEED_BASE + 5, 10 * k, 1, moduli, N)[0]),
                 to_device(W.poly_batch(W.SEED_BASE + 5, 10 * k + 1, 1, moduli, N)[0]))
                for k in range(4)] for N in Ns}
    draws = W.splitmix64_block(W.stream_key(W.SEED_BASE + 5, 1), 0, 4 * n_req)
    spec = [(Ns[int(draws[3 * i] % np.uint64(3))], 4 + int(draws[3 * i + 1] % np.uint64(29)),
             int(draws[3 * i + 2] % np.uint64(4))) for i in range(n_req)]
    u = (W.splitmix64_block(W.stream_key(W.SEED_BASE + 5, 2), 0, n_req) >> np.uint64(11)) \
        .astype(np.float64) / float(1 << 53)

    def requests():
        return [serve.Request(N, tuple(moduli[:L]), pool[N][k][0][:L], pool[N][k][1][:L])
                for N, L, k in spec]

    streams = [torch.cuda.Stream() for _ in range(3)]   # shared by every server below
    srv = serve.Server(hbm_budget=budget, streams=streams, blocking_wait=blocking_wait)
    for N in Ns:                                   # plans (twiddles) resident up front
        for L in range(4, 33):
            srv.plan(N, moduli[:L])
    plans = dict(srv.plans)
    # warm both paths (kernels, and the allocator's blocks on the servers'
    # streams: every request at once, so batches reach their largest sizes)
    with srv:
        for f in [srv.submit(r) for r in requests()]:
            f.result()
    serve.serve_one_by_one(requests()[:64], plans=plans)
    torch.cuda.synchronize()
    gc.collect()
    gc.freeze()        # the long-lived heap leaves the collector's scans

    lt_per_req = [3 * L for _, L, _ in spec]
    out = []
    for rate in rates:
        arrivals = np.cumsum(-np.log1p(-u) / rate)
        served = requests()
        srv = serve.Server(hbm_budget=budget, streams=streams, blocking_wait=blocking_wait)
        srv.plans = plans
        cg = cgroup_cpu()
        srv.start()
        t0 = time.perf_counter()
        futs = []
        for r, t in zip(served, arrivals):
            # sleep until the arrival (the interpreter lock stays free for the
            # server's threads; the thread's timer slack is 1 ns, so the sleep
            # ends on time, as the one-by-one baseline's sleep does);
            # requests already due go in at once, each stamped with its
            # scheduled arrival, so lateness here counts as latency in both
            wait = t - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            futs.append(srv.submit(r, arrival=t0 + t))
        for f in futs:
            f.result(timeout=600)
        srv.stop()
        thr_served = _throttled_since(cg)
        base = requests()
        cg = cgroup_cpu()
        serve.serve_one_by_one(base, arrivals, plans=plans)
        thr_base = _throttled_since(cg)
        same = all(torch.equal(a.result, b.result) for a, b in zip(served, base))

        def summary(rs):
            lat = np.array([r.latency for r in rs]) * 1e3
            span = max(r.done for r in rs) - min(r.arrival for r in rs)
            out = {"requests_per_s": len(rs) / span,
                   "limb_transforms_per_s": sum(lt_per_req) / span,
                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "mean_ms": float(lat.mean())}
            paths = {}
            for r, x in zip(rs, lat):
                if r.path:
                    paths.setdefault(r.path, []).append(x)
            if paths:                  # the server: latency by the path a request took
                out["by_path"] = {k: {"requests": len(v), "p50_ms": float(np.percentile(v, 50)),
                                      "p99_ms": float(np.percentile(v, 99))}
                                  for k, v in sorted(paths.items())}
            return out
        out.append({"offered_rate_per_s": rate, "requests": n_req, "served": summary(served),
                    "one_by_one": summary(base), "batches": srv.stats["batches"],
                    "max_batch": srv.stats["max_batch"],
                    "launch_ms_max": srv.stats["launch_ms_max"],
                    "complete_ms_max": srv.stats["complete_ms_max"],
                    "bit_exact_equal": bool(same),
                    "cpu_throttled": {"served": thr_served, "one_by_one": thr_base}})
    gc.unfreeze()
    return {"workload": "poly-multiply requests, N in {2^12,2^14,2^16}, 4-32 limbs, "
                        "operands HBM-resident, Poisson arrivals", "hbm_budget_bytes": budget,
            "streams": 3, "completer_wait": "blocking" if blocking_wait else "spin",
            "cpu_quota": cgroup_cpu(), "rates": out}


# ------------------------------------------------------------------ clocks
_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class ClockSampler:
    """Samples SM clock and clock-event reasons during the timed region, by
    NVML through ctypes (read-only queries), else by nvidia-smi."""

    def __init__(self, device_index=0, period=0.004):
        self.period, self.samples, self.reasons = period, [], set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._nvml = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                bus = os.environ.get("HX_PCI_BUS_ID")
                ok = -1
                if bus:
                    ok = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h))
                if ok != 0:
                    ok = nv.nvmlDeviceGetHandleByIndex_v2(device_index, ctypes.byref(h))
                if ok == 0:
                    self._nvml, self._h = nv, h
                    mx = ctypes.c_uint()
                    if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                        self.max_mhz = mx.value
        except OSError:
            self._nvml = None

    def _poll_nvml(self):
        nv, h = self._nvml, self._h
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                self.samples.append(clk.value)
            if fn(h, ctypes.byref(rs)) == 0:
                for bit, name in _REASONS.items():
                    if rs.value & bit:
                        self.reasons.add(name)
            time.sleep(self.period)

    def _poll_smi(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                      "-i", "0"], capture_output=True, text=True, timeout=5).stdout
                f = [x.strip() for x in out.strip().split(",")]
                self.samples.append(float(f[0]))
                self.max_mhz = float(f[1])
                for name, v in zip(names, f[2:]):
                    if v.lower().startswith("active"):
                        self.reasons.add(name)
            except Exception:
                pass
            time.sleep(0.2)

    def __enter__(self):
        target = self._poll_nvml if self._nvml else self._poll_smi
        self._t = threading.Thread(target=target, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        med = float(np.median(self.samples)) if self.samples else None
        return {"sm_mhz": med, "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons),
                "samples": len(self.samples)}


# ------------------------------------------------------------------ oracle timing
def host_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_sample(N, moduli, s, sets, threads=1):
    """One bounded oracle run of the same pipeline: with one thread on the
    first 30-, 50- and 60-bit limbs in turn; with T > 1 threads on the first T
    limbs (mixed widths), one limb per thread (the oracle's C calls release
    the interpreter lock).  Returns (limb-transforms, wall seconds)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    pick = [0, 1, 2] if threads == 1 else list(range(min(threads, len(moduli))))
    ins, es = sets[0]
    oracle.lib()
    for l in pick:
        oracle.tables(N, int(moduli[l]))        # root and tables, outside the timing

    def one(ls):
        qs = [moduli[l] for l in ls]
        oracle.ciphertext_tensor(*[x[:, ls] for x in ins],
                                 np.array([s[l] for l in ls], dtype=np.uint64),
                                 *[x[:, ls] for x in es], qs)

    t0 = time.perf_counter()
    if threads == 1:
        one(pick)
    else:
        with ThreadPoolExecutor(len(pick)) as ex:
            list(ex.map(lambda l: one([l]), pick))
    return 7 * len(pick), time.perf_counter() - t0


def timed_oracle(N, moduli, s, sets, threads, min_seconds):
    units, secs, reps = 0, 0.0, 0
    while secs < min_seconds:
        u, t = oracle_sample(N, moduli, s, sets, threads)
        units += u
        secs += t
        reps += 1
    return units, secs, reps


def cpu_baseline(N, moduli, s, sets, min_seconds=6.0):
    T = host_threads()
    u1, s1, r1 = timed_oracle(N, moduli, s, sets, 1, min_seconds)
    uT, sT, rT = timed_oracle(N, moduli, s, sets, T, min_seconds) if T > 1 else (u1, s1, r1)
    return {"value": uT / sT, "unit": UNIT, "cores": T, "kind": "oracle",
            "sample": f"{rT} x ciphertext-tensor pipeline at N={N} on {min(T, len(moduli))} "
                      f"limbs, one limb per thread: {uT} limb-transforms in {sT:.2f} s "
                      f"({T} threads)",
            "single_thread": {"value": u1 / s1, "cores": 1,
                              "sample": f"{r1} x the pipeline on 3 limbs (30/50/60-bit): "
                                        f"{u1} limb-transforms in {s1:.2f} s"},
            "cpu": platform.processor() or platform.machine()}


# ------------------------------------------------------------------ main
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    N, nl = args.N, args.limbs
    wl, sets, s = workload_arrays(N, nl, 1)
    T = host_threads()
    for _ in range(args.warmup):
        oracle_sample(N, wl.moduli, s, sets, T)
    units, secs = 0, 0.0
    for _ in range(args.steps):
        u, t = oracle_sample(N, wl.moduli, s, sets, T)
        units += u
        secs += t
    value = units / secs
    per_step = units // max(args.steps, 1)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"ciphertext_tensor_n{N}_l{nl} (oracle sample: "
                                   f"{per_step // 7} limbs, one per thread)",
                       "N": N, "limbs": nl},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": T, "kind": "oracle",
                             "sample": f"per step: the pipeline on {per_step // 7} limbs, "
                                       f"{per_step} limb-transforms, {T} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_case(args):
    """One kernel family alone, for profiling and tuning (not the contract line)."""
    import torch
    from paper_2103_16400_gb300 import build as hbuild, capi
    from paper_2103_16400_gb300.tensors import empty, to_device
    hbuild.build()
    N, nl = args.N, args.limbs
    out = {"case": args.case, "N": N, "limbs": nl}
    if args.case == "serving":
        print(json.dumps({"case": "serving", "serving": serving_report(torch)}))
        return 0
    if args.case == "probes":
        for kind in capi.PROBE_KINDS:
            r, ms = capi.hx_probe_int_mul_rate(kind, 8192)
            out[f"int_mul_{kind}_Tops"] = r / 1e12
        for w in W.WIDTHS:
            q = W.ntt_primes(w, W.MIXED_TWO_N, 1)[0]
            for v in (0, 1, 2, 3):
                for inv in (False, True):
                    if w == 30 and v > 0:
                        continue
                    r, ms = capi.hx_probe_butterfly_rate(q, v, inv, 8192)
                    out[f"bfly_{w}bit_v{v}_{'inv' if inv else 'fwd'}_T_per_s"] = r / 1e12
        print(json.dumps(out))
        return 0
    wl = W.ciphertext_tensor(N=N, n_limbs=nl)
    P = args.polys
    if args.case == "tensor_inv":
        return run_tensor_inv(args, wl, torch)
    if args.case == "ct_step":
        return run_ct_step(args, wl, torch)
    n_sets = 2
    xs = [to_device(W.poly_batch(wl.seed + k, 0, P, wl.moduli, N)) for k in range(n_sets)]
    ys = [empty(x.shape) for x in xs]
    plan = capi.Plan(N, wl.moduli)
    if args.schedule and args.case in ("fwd", "inv"):
        sched = [tuple(p) for p in json.loads(args.schedule)]
        plan.set_schedule(sched, plan.FORWARD if args.case == "fwd" else plan.INVERSE)
        out["schedule"] = [list(p) for p in sched]
    elif args.tuned and args.case in ("fwd", "inv"):
        from paper_2103_16400_gb300 import tune as hx_tune
        t = hx_tune.tune(plan, P, direction=plan.FORWARD if args.case == "fwd" else plan.INVERSE,
                         verbose=bool(os.environ.get("HX_TUNE_VERBOSE")))
        out["schedule"] = t["forward" if args.case == "fwd" else "inverse"]
    s = W.scalars(wl.seed, 20, wl.moduli)
    st = torch.cuda.current_stream()

    def once(i):
        x, y = xs[i % n_sets], ys[i % n_sets]
        if args.case == "fwd":
            capi.hx_ntt_forward(plan, y, x, P, 1, 4, st)
        elif args.case == "inv":
            capi.hx_ntt_inverse(plan, y, x, P, 1, 1, st)
        else:
            # P/4 ciphertext pairs: A0..B1 are the four quarters of x, the
            # addends the first three quarters of the other set, outputs in y
            Q, o = P // 4, xs[(i + 1) % n_sets]
            capi.hx_dyadic_tensor_fma(y[:Q], y[Q:2 * Q], y[2 * Q:3 * Q], x[:Q], x[Q:2 * Q],
                                      x[2 * Q:3 * Q], x[3 * Q:], s, o[:Q], o[Q:2 * Q],
                                      o[2 * Q:3 * Q], N, wl.moduli, Q, 4, st)

    for i in range(max(args.warmup, 1)):
        once(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(args.steps):
        once(i)
    e1.record(st)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / args.steps
    out.update({"polys": P, "us_per_call": us})
    if args.case in ("fwd", "inv"):
        out["limb_transforms_per_s"] = P * nl / (us * 1e-6)
        ops = sum(imad_slots_per_transform(N, wl.moduli)) * P
        out["imad_slot_T_per_s"] = ops / (us * 1e-6) / 1e12
        out["hbm_alg_GBs"] = 16 * N * nl * P / (us * 1e-6) / 1e9
    print(json.dumps(out))
    return 0


def run_tensor_inv(args, wl, torch):
    """hx_tensor_fma_inverse on one ciphertext pair: its tuned schedule, the
    fused call's time, and the composed path (element-wise kernel, then the
    inverse transform) on the same schedule (diagnostic line)."""
    from paper_2103_16400_gb300 import capi, tune as hx_tune
    from paper_2103_16400_gb300.tensors import empty, to_device
    N, nl = args.N, args.limbs
    plan = capi.Plan(N, wl.moduli)
    s = W.scalars(wl.seed, 20, wl.moduli)
    if args.schedule:
        sched = [tuple(p) for p in json.loads(args.schedule)]
        plan.set_schedule(sched, plan.INVERSE)
        t = {"inverse": [list(p) for p in sched]}
    else:
        t = hx_tune.tune_tensor(plan, 1, s, verbose=bool(os.environ.get("HX_TUNE_VERBOSE")))
    A = to_device(np.stack([W.poly_batch(wl.seed, k, 1, wl.moduli, N) for k in range(4)]))
    E = to_device(np.stack([W.poly_batch(wl.seed, 10 + k, 1, wl.moduli, N) for k in range(3)]))
    R = empty((3, 1, nl, N))
    st = torch.cuda.current_stream()

    def fused():
        capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], A[0], A[1], A[2], A[3], s, E[0],
                                   E[1], E[2], 1, 4, st)

    def composed():
        capi.hx_dyadic_tensor_fma(R[0], R[1], R[2], A[0], A[1], A[2], A[3], s, E[0], E[1], E[2],
                                  N, wl.moduli, 1, 4, st)
        capi.hx_ntt_inverse(plan, R, R, 3, 1, 1, st)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / args.steps

    print(json.dumps({"case": "tensor_inv", "N": N, "limbs": nl, "schedule": t["inverse"],
                      "fused_us": timed(fused), "composed_us": timed(composed)}))
    return 0


def run_ct_step(args, wl, torch):
    """hx_ciphertext_step on one ciphertext pair with the (forward, inverse)
    schedule pair given as --schedule '[forward, inverse]' (else the step
    tuner's): the call's time, and the composition (forward call, then the
    fused tensor + inverse call) on the same plan (diagnostic line)."""
    from paper_2103_16400_gb300 import capi, tune as hx_tune
    from paper_2103_16400_gb300.tensors import empty, to_device
    N, nl = args.N, args.limbs
    plan = capi.Plan(N, wl.moduli)
    s = W.scalars(wl.seed, 20, wl.moduli)
    if args.schedule:
        f, i = ([tuple(p) for p in sch] for sch in json.loads(args.schedule))
        plan.set_schedule(f, plan.FORWARD)
        plan.set_schedule(i, plan.INVERSE)
    else:
        hx_tune.tune_step(plan, 1, s, verbose=bool(os.environ.get("HX_TUNE_VERBOSE")))
    X = to_device(np.stack([W.poly_batch(wl.seed, k, 1, wl.moduli, N) for k in range(4)]))
    E = to_device(np.stack([W.poly_batch(wl.seed, 10 + k, 1, wl.moduli, N) for k in range(3)]))
    Wk, R = empty((4, 1, nl, N)), empty((3, 1, nl, N))
    st = torch.cuda.current_stream()

    def step():
        capi.hx_ciphertext_step(plan, R, X, Wk, s, E, 1, st)

    def composed():
        capi.hx_ntt_forward(plan, Wk, X, 4, 1, 4, st)
        capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], Wk[0], Wk[1], Wk[2], Wk[3], s,
                                   E[0], E[1], E[2], 1, 4, st)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / args.steps

    print(json.dumps({"case": "ct_step", "N": N, "limbs": nl,
                      "schedule": {"forward": [list(p) for p in plan.schedule(plan.FORWARD)],
                                   "inverse": [list(p) for p in plan.schedule(plan.INVERSE)]},
                      "step_us": timed(step), "composed_us": timed(composed)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hexgpu", choices=["hexgpu", "reference"])
    ap.add_argument("--N", type=int, default=N_DEFAULT)
    ap.add_argument("--limbs", type=int, default=LIMBS_DEFAULT)
    ap.add_argument("--sets", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ragged", action="store_true",
                    help="skip the ragged-batch report (512 polynomials, mixed N)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving report (Poisson arrivals, p50/p99 latency)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--case", default="pipeline",
                    choices=["pipeline", "fwd", "inv", "tensor", "tensor_inv", "ct_step", "probes",
                             "serving"],
                    help="pipeline: the contract line; others: one kernel family alone "
                         "(diagnostic line, used for profiling)")
    ap.add_argument("--polys", type=int, default=8, help="polynomials per call for --case fwd/inv")
    ap.add_argument("--tuned", action="store_true",
                    help="--case fwd/inv: apply the autotuned schedule (cached) instead of the default")
    ap.add_argument("--schedule", default=None,
                    help="--case fwd/inv/tensor_inv: JSON list of passes to apply instead "
                         "(profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case != "pipeline":
        return run_case(args)
    args.warmup = max(args.warmup, 3)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2103_16400_gb300 import build as hbuild, capi
    from paper_2103_16400_gb300.tensors import pinned_from
    hbuild.build()

    N, nl = args.N, args.limbs
    wl, sets, s = workload_arrays(N, nl, args.sets, rank)
    dev_sets = device_sets(sets)
    step = HexStep(N, wl.moduli, s, dev_sets, torch)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    for i in range(args.warmup):
        step.run(i)
    barrier()
    stream = step.stream
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    launches0 = capi.hx_launch_count()
    with ClockSampler(local) as clocks:
        t0.record(stream)
        step.begin(t0)
        for i in range(args.steps):
            step.run(i)
        step.join()
        t1.record(stream)
        torch.cuda.synchronize()
    launches = capi.hx_launch_count() - launches0
    total_ms = t0.elapsed_time(t1)
    total_ms = shard.max_over_ranks(total_ms, device="cuda")
    barrier()

    # the two calls of the step timed apart (CUDA events between them), in
    # a region of their own after the contract's timed region
    calls_steps = min(args.steps, 200)
    step.fwd_events.clear()
    step.inv_events.clear()
    step.step_events.clear()
    for i in range(calls_steps):
        step.run(i, record=True, path="composed")
        if step.path == "step":
            step.run(i, record=True, path="step")
    torch.cuda.synchronize()
    fwd_ms = [a.elapsed_time(b) for a, b in step.fwd_events]
    inv_ms = [a.elapsed_time(b) for a, b in step.inv_events]
    step_call_ms = [a.elapsed_time(b) for a, b in step.step_events]

    # kernel-timing region: the same steps again with the library's events
    # around every launch (each pair adds a start-up bubble of a microsecond
    # or two, so it stays out of the region that gives `value`)
    kt_steps = min(args.steps, 500)
    capi.hx_timing_read(64)                    # nothing left over
    capi.hx_timing_enable(True, 4 * kt_steps + 64)
    for i in range(kt_steps):
        step.run(i, one_stream=True)           # launches one after another
    torch.cuda.synchronize()
    capi.hx_timing_enable(False)
    timed = capi.hx_timing_read(4 * kt_steps + 64)
    barrier()

    per_step_units = 7 * nl
    value = per_step_units * args.steps * ws / (total_ms / 1e3)

    # Rooflines.  Primary figure: the operation count (10 IMAD operations per
    # 64-bit-word butterfly, 3 per 32-bit-word one, at the live mad.lo rate)
    # against one HBM read + write per coefficient (measured copy
    # bandwidth), the slower side being the bound.  Second figure
    # (`slots`): the IMAD-slot model, which weighs each multiply form by its
    # measured issue cost (mad.hi and mad.wide issue at half the mad.lo rate
    # or less).
    imad_rate, _ = capi.hx_probe_int_mul_rate("mad.lo", 8192)
    hbm_gbs, hbm_src = hbm_peak_gbs()
    peak_source = (f"IMAD: hx_probe_int_mul_rate mad.lo.u32, measured live; HBM: "
                   f"{hbm_gbs:.0f} GB/s copy bandwidth ({hbm_src}, MEASURED_PEAKS.json)")
    logn = N.bit_length() - 1
    fwd_call_ms = float(np.mean(fwd_ms))
    inv_call_ms = float(np.mean(inv_ms))
    fwd_ops = 4 * sum(N // 2 * logn * ops_per_butterfly(q) for q in wl.moduli)
    fwd_bytes = 4 * 16 * N * nl
    alg_slots = 4 * sum(imad_slots_per_transform(N, wl.moduli))
    fwd_sched = step.plan.schedule(step.plan.FORWARD)
    inv_sched = step.plan.schedule(step.plan.INVERSE)
    traffic = traffic_for("forward_call", fwd_sched) if (N, nl) == (1 << 16, 32) else None
    roofline_forward_call = dict(
        op_roofline(fwd_ops, fwd_bytes, fwd_call_ms * 1e3, imad_rate, hbm_gbs),
        traffic=traffic,
        traffic_unit="DRAM bytes per forward call (ncu, this build's sources), else null",
        kernel="hx_ntt_forward, 4 polys x 32 limbs",
        fwd_call_us=fwd_call_ms * 1e3, alg_ops_per_call=fwd_ops, alg_bytes_per_call=fwd_bytes,
        slots={"frac": alg_slots / (fwd_call_ms * 1e-3) / imad_rate,
               "achieved": alg_slots / (fwd_call_ms * 1e-3) / 1e12, "peak": imad_rate / 1e12,
               "unit": "T IMAD-slot/s", "alg_slots_per_call": alg_slots},
        dram_gbs_measured=(traffic / (fwd_call_ms * 1e-3) / 1e9) if traffic else None,
        peak_source=peak_source,
        schedules={"forward": [list(p) for p in fwd_sched],
                   "inverse": [list(p) for p in inv_sched]})

    # every kernel of the step timed live (library events around each launch
    # in the kernel-timing region); the roofline object is the dominant kernel's
    kernels = {}
    for kid, ms in timed:
        k = kernels.setdefault(kid, {"kernel": capi.hx_kernel_name(kid), "launches": 0,
                                     "total_ms": 0.0})
        k["launches"] += 1
        k["total_ms"] += ms
    timed_total = sum(k["total_ms"] for k in kernels.values()) or 1.0
    for kid, k in kernels.items():
        k["avg_us"] = k["total_ms"] / k["launches"] * 1e3
        k["share"] = k["total_ms"] / timed_total
        k["alg_ops_per_launch"] = kernel_slots(kid, N, wl.moduli, per_butterfly=ops_per_butterfly)
        k["alg_bytes_per_launch"] = kernel_bytes(kid, N, nl)
        r = op_roofline(k["alg_ops_per_launch"], k["alg_bytes_per_launch"], k["avg_us"],
                        imad_rate, hbm_gbs)
        k["bound"], k["frac"] = r["bound"], r["frac"]
        k["alg_slots_per_launch"] = kernel_slots(kid, N, wl.moduli)
        k["frac_slots"] = k["alg_slots_per_launch"] / (k["avg_us"] * 1e-6) / imad_rate
    # the whole step at the timed rate (two streams): its algorithmic work
    # against the step time, both models
    s_ops, s_slots, s_bytes = step_work(N, wl.moduli)
    step_us = total_ms / args.steps * 1e3
    step_roof = dict(op_roofline(s_ops, s_bytes, step_us, imad_rate, hbm_gbs),
                     frac_slots=s_slots / (step_us * 1e-6) / imad_rate, step_us=step_us,
                     alg_ops=s_ops, alg_slots=s_slots, alg_bytes=s_bytes)
    roofline = roofline_forward_call
    if kernels:
        dom_id = max(kernels, key=lambda i: kernels[i]["total_ms"])
        dom = kernels[dom_id]
        r = op_roofline(dom["alg_ops_per_launch"], dom["alg_bytes_per_launch"], dom["avg_us"],
                        imad_rate, hbm_gbs)
        kp = step.kernel_plan()
        dom_traffic = traffic_for(dom["kernel"], kp.schedule(kp.INVERSE) if not (dom_id >> 2) & 1
                                  else kp.schedule(kp.FORWARD)) if (N, nl) == (1 << 16, 32) else None
        roofline = dict(
            r, traffic=dom_traffic,
            traffic_unit="DRAM bytes per launch (ncu, this build's sources), else null",
            kernel=dom["kernel"], launches=dom["launches"], avg_launch_us=dom["avg_us"],
            share_of_timed_kernels=dom["share"], alg_ops_per_launch=dom["alg_ops_per_launch"],
            alg_bytes_per_launch=dom["alg_bytes_per_launch"],
            slots={"frac": dom["frac_slots"],
                   "achieved": dom["alg_slots_per_launch"] / (dom["avg_us"] * 1e-6) / 1e12,
                   "peak": imad_rate / 1e12, "unit": "T IMAD-slot/s",
                   "alg_slots_per_launch": dom["alg_slots_per_launch"]},
            dram_gbs_measured=(dom_traffic / (dom["avg_us"] * 1e-6) / 1e9
                               if dom_traffic else None),
            peak_source=peak_source,
            timing=f"CUDA events recorded by the library around every launch, on the "
                   f"launching stream, over {kt_steps} steps after the timed region (same "
                   f"inputs, stream and schedules); each duration includes its launch's "
                   f"start-up",
            forward_call={"frac": roofline_forward_call["frac"],
                          "bound": roofline_forward_call["bound"],
                          "frac_slots": roofline_forward_call["slots"]["frac"],
                          "us": fwd_call_ms * 1e3},
            step=step_roof,
            schedules=dict(roofline_forward_call["schedules"],
                           step={"forward": [list(p) for p in
                                             step.step_plan.schedule(step.step_plan.FORWARD)],
                                 "inverse": [list(p) for p in
                                             step.step_plan.schedule(step.step_plan.INVERSE)]},
                           path=step.path))

    # the plain forward and inverse calls on their own: the goal's forward +
    # inverse figure, carried inside the roofline object as well
    rates = None
    if rank == 0:
        try:
            rates = ntt_rates_report(torch, step, dev_sets, imad_rate, hbm_gbs)
            roofline["fwd_inv"] = {k: rates[k] for k in (
                "forward_us", "inverse_us", "fwd_plus_inv_pairs_per_s", "fwd_plus_inv_frac",
                "fwd_plus_inv_frac_slots", "forward_frac", "inverse_frac", "two_streams")}
        except Exception as e:               # noqa: BLE001 -- reported, not hidden
            rates = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.synchronize()

    # end to end through the public API with host buffers: every step uploads
    # its inputs from pinned host memory and downloads its three results; the
    # pipeline (three streams, two device buffer sets) overlaps the transforms
    # of step i with the copies of steps i-1 and i+1
    from paper_2103_16400_gb300.pipeline import TensorPipeline
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 200))
    host_in = [(pinned_from(np.concatenate(ins)).view(4, 1, nl, N),
                pinned_from(np.concatenate(es)).view(3, 1, nl, N)) for ins, es in sets]
    host_out = [torch.empty((3, 1, nl, N), dtype=torch.int64).pin_memory() for _ in range(2)]
    h2d = sum(x.numel() * 8 for x in host_in[0])
    d2h = host_out[0].numel() * 8
    pipe = TensorPipeline(step.kernel_plan(), s, 1, depth=2)
    for i in range(3):
        pipe.submit(*host_in[i % len(host_in)], host_out[i % 2])
    pipe.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(pipe.s_up)
    for i in range(e2e_steps):
        pipe.submit(*host_in[i % len(host_in)], host_out[i % 2])
    e1.record(pipe.s_down)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = shard.max_over_ranks(e2e_ms, device="cuda")
    e2e_value = per_step_units * e2e_steps * ws / (e2e_ms / 1e3)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"ciphertext_tensor_n{N}_l{nl}", "N": N, "limbs": nl,
                       "widths": "30/50/60-bit, limb l -> (30,50,60)[l%3]",
                       "polys_per_step": "4 in (fwd), 3 out (inv)",
                       "limb_transforms_per_step": per_step_units,
                       "l2": f"{args.sets} rotating input sets, "
                             f"{args.sets * 7 * nl * N * 8 / 2**20:.0f} MiB of inputs > 129 MB L2",
                       "streams": f"{len(step.streams)}: step i on stream i mod "
                                  f"{len(step.streams)}, each with its own buffers",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roofline,
            "roofline_forward_call": roofline_forward_call,
            "kernels": sorted(kernels.values(), key=lambda k: -k["total_ms"]),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "ms_per_step": e2e_ms / e2e_steps,
                    "how": "pinned host -> device -> pinned host every step; upload, "
                           "compute and download on three streams, two buffer sets"},
            "calls": {"forward_us": fwd_call_ms * 1e3,
                      "forward_limb_transforms_per_s": 4 * nl / (fwd_call_ms * 1e-3),
                      "tensor_inverse_us": float(np.mean(inv_ms)) * 1e3,
                      "tensor_inverse_limb_transforms_per_s":
                          3 * nl / (float(np.mean(inv_ms)) * 1e-3),
                      "step_path": step.path,
                      "step_us": (float(np.mean(step_call_ms)) * 1e3 if step_call_ms
                                  else (fwd_call_ms + inv_call_ms) * 1e3),
                      "path_us": getattr(step, "path_us", None),
                      "how": f"CUDA events around each call, {calls_steps} steps in a "
                             f"region after the timed one; step_us: the step's own call(s) "
                             f"(hx_ciphertext_step on the path 'step', the forward call plus "
                             f"the tensor + inverse call on 'composed'); path_us: both paths "
                             f"timed as the timed region runs them, the faster one taken"},
            "gpu_launches": launches,
            "clocks": clocks.summary()}
    # the secondary reports run on rank 0 only; the other ranks wait.  A
    # report that fails records its error instead of taking the line with it
    def report(key, fn):
        try:
            line[key] = fn(torch)
        except Exception as e:               # noqa: BLE001 -- reported, not hidden
            line[key] = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line["ntt_rates"] = rates
        report("eltwise", eltwise_report)
    if rank == 0 and not args.no_ragged:
        report("batched", lambda t: ragged_report(t, imad_rate, hbm_gbs))
    if rank == 0 and not args.no_serving:
        report("serving", serving_report)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(N, wl.moduli, s, sets)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
