"""Autotuner for the NTT kernel schedule.

The paper leaves the choice between its kernel variants to fixed CPUID rules
and names choosing "via a small number of trials" as future work (Section
3.2).  Here the trials are the schedule: how the log2 N stages split into
passes, the tile shape of each pass, elements per thread, and which kernel
a pass runs (per-tile, persistent double-buffered, or per-tile with staged
twiddles) -- or whether both passes run as one cluster-fused launch, and
with how many CTAs a cluster.  Every schedule computes the same result; `tune()` times
candidates of the forward and of the inverse transform on the caller's plan
and batch size with CUDA events and keeps the fastest of each: every
single-pass schedule, and per split of the stages a coordinate search over
the first pass, then the second (the passes are separate launches, so their
times add).
Winners are cached in a JSON file keyed by GPU name, N, limb-width mix and
batch size.
"""
from __future__ import annotations

import json
import os
import sys
import threading
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

from . import capi

Pass = Tuple[int, int, int, int, int, int, int]   # s0, K, logGb, logGc, logR, pipe, np
CACHE_PATH = os.environ.get("HX_TUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                         "_build", "tune_cache.json"))
_lock = threading.Lock()


#: per-pass kernel variants: (logR, pipe, np) -- 16 or 8 elements per thread;
#: per-tile kernel with twiddles read through the read-only cache (pipe 0),
#: persistent double-buffered kernel (1), per-tile kernel with the tile's
#: twiddles staged in shared memory (2); one or two polynomials per thread
VARIANTS = ((3, 0, 1), (4, 0, 1), (3, 1, 1), (4, 1, 1), (3, 0, 2), (3, 2, 1), (4, 2, 1),
            (3, 2, 2))


def single_pass(logN: int, variants=VARIANTS) -> List[List[Pass]]:
    return [[(0, logN, 0, 0) + v] for v in variants] if logN <= 13 else []


def splits(logN: int) -> List[int]:
    """First-pass stage counts K1 of the two-pass schedules (both passes 6..13 stages)."""
    return [K1 for K1 in range(6, 10) if 6 <= logN - K1 <= 13]


def pass_options(logN: int, K1: int, variants=VARIANTS) -> Tuple[List[Pass], List[Pass]]:
    """(first-pass options, second-pass options) of the split at K1: column
    passes over stages [0, K1) in 2^logGc-column tiles, row passes over the
    rest in 2^logGb-row tiles, each with every kernel variant."""
    firsts = [(0, K1, 0, logGc) + v for logGc in (2, 3, 4, 5) for v in variants]
    seconds = [(K1, logN - K1, logGb, 0) + v for logGb in range(0, 6) for v in variants]
    return firsts, seconds


#: elements per thread of the cluster-fused kernels
CLUSTER_LOGR = (4, 3)


def cluster_options(logN: int) -> List[List[Pass]]:
    """Cluster-fused schedules (pipe 3 on both passes): one launch of
    clusters of 2^c CTAs per limb-transform, CTA k holding columns
    [k 2^(K2-c), (k+1) 2^(K2-c)) in the column phase and rows
    [k 2^(K1-c), (k+1) 2^(K1-c)) in the row phase, exchanging through
    distributed shared memory."""
    out = []
    for K1 in range(6, 10):
        K2 = logN - K1
        if not 6 <= K2 <= 9:
            continue
        for c in (1, 2, 3, 4):
            for r in CLUSTER_LOGR:
                out.append([(0, K1, 0, K2 - c, r, 3, 1), (K1, K2, K1 - c, 0, r, 3, 1)])
    return out


def candidates(logN: int, variants=VARIANTS) -> List[List[Pass]]:
    """Every schedule worth trying for log2 N (validity is checked by the library)."""
    out = single_pass(logN, variants)
    for K1 in splits(logN):
        firsts, seconds = pass_options(logN, K1, variants)
        out += [[a, b] for a in firsts for b in seconds]
    return out + cluster_options(logN)


def valid(plan: "capi.Plan", sched: List[Pass]) -> bool:
    """Whether the library can run `sched` on this plan; the plan's own
    schedules are left as they were."""
    keep = (plan.schedule(plan.FORWARD), plan.schedule(plan.INVERSE))
    try:
        plan.set_schedule(sched)
        return True
    except capi.HexError:
        return False
    finally:
        plan.set_schedule(keep[0], plan.FORWARD)
        plan.set_schedule(keep[1], plan.INVERSE)


def width_class(moduli: Sequence[int]) -> str:
    nar = sum(1 for q in moduli if q < (1 << 30))
    return f"{nar}n{len(moduli) - nar}w"


def _key(N: int, moduli: Sequence[int], n_polys: int, device_name: str) -> str:
    return f"{device_name}|N={N}|{width_class(moduli)}|P={n_polys}"


def load_cache() -> Dict[str, dict]:
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
    tmp = CACHE_PATH + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE_PATH)


def _valid_pair(plan, firsts: List[Pass], seconds: List[Pass]):
    """One valid (first pass, second pass) pair, or None.  Validity is a
    property of each pass on its own, so a pass that is valid with one
    partner is valid with every valid partner."""
    for b in seconds:
        for a in firsts:
            if valid(plan, [a, b]):
                return a, b
    return None


def covering(plan: "capi.Plan", variants=VARIANTS) -> List[List[Pass]]:
    """Valid schedules that between them use every valid pass configuration:
    the single-pass ones, and per split each valid first pass with one valid
    second pass and each valid second pass with one valid first pass."""
    logN = plan.N.bit_length() - 1
    out = [s for s in single_pass(logN, variants) if valid(plan, s)]
    out += [s for s in cluster_options(logN) if valid(plan, s)]
    for K1 in splits(logN):
        firsts, seconds = pass_options(logN, K1, variants)
        pair = _valid_pair(plan, firsts, seconds)
        if pair is None:
            continue
        a0, b0 = pair
        out += [[a, b0] for a in firsts if valid(plan, [a, b0])]
        out += [[a0, b] for b in seconds if b != b0 and valid(plan, [a0, b])]
    return out


def time_schedule(plan, sched, x, y, n_polys: int, iters: int = 5,
                  direction: int = 3) -> Tuple[float, float]:
    """(forward us, inverse us) per call for one schedule, averaged over
    iters; a direction not asked for is reported as inf."""
    import torch
    plan.set_schedule(sched, plan.BOTH)
    st = torch.cuda.current_stream()
    if direction & 1:
        capi.hx_ntt_forward(plan, y, x, n_polys, 1, 4, st)
    if direction & 2:
        capi.hx_ntt_inverse(plan, y, x, n_polys, 1, 1, st)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(st)
    for _ in range(iters if direction & 1 else 0):
        capi.hx_ntt_forward(plan, y, x, n_polys, 1, 4, st)
    ev[1].record(st)
    for _ in range(iters if direction & 2 else 0):
        capi.hx_ntt_inverse(plan, y, x, n_polys, 1, 1, st)
    ev[2].record(st)
    torch.cuda.synchronize()
    f = ev[0].elapsed_time(ev[1]) * 1e3 / iters if direction & 1 else float("inf")
    i = ev[1].elapsed_time(ev[2]) * 1e3 / iters if direction & 2 else float("inf")
    return f, i


def _search(plan, timer, label: str, verbose: bool):
    """Fastest schedule by `timer(schedule) -> us`: every single-pass
    schedule, and per split a coordinate search -- the best first pass
    against a fixed valid second pass, then the best second pass against that
    first pass.  The passes are separate launches, so a schedule's time is the
    sum of its passes' and the search finds the best pair.  Returns (us,
    schedule, schedules timed)."""
    logN = plan.N.bit_length() - 1
    best, tried = (float("inf"), None), 0

    def run(s):
        nonlocal best, tried
        t = timer(s)
        tried += 1
        if verbose:
            print(f"{label} {t:9.1f}  {s}", file=sys.stderr)
        if t < best[0]:
            best = (t, s)
        return t

    timed = []

    def run_keep(s):
        t = run(s)
        timed.append((t, s))
        return t

    for s in single_pass(logN) + cluster_options(logN):
        if valid(plan, s):
            run_keep(s)
    for K1 in splits(logN):
        firsts, seconds = pass_options(logN, K1)
        pair = _valid_pair(plan, firsts, seconds)
        if pair is None:
            continue
        b0 = pair[1]
        a_best = min((a for a in firsts if valid(plan, [a, b0])), key=lambda a: run_keep([a, b0]))
        for b in seconds:
            if b != b0 and valid(plan, [a_best, b]):
                run_keep([a_best, b])
    # the leaders are often within timing noise of each other: time the three
    # best again, four times as long, and keep the fastest of that
    finalists = [s for _, s in sorted(timed, key=lambda r: r[0])[:3]]
    if len(finalists) > 1:
        best = min(((sum(timer(s) for _ in range(4)) / 4, s) for s in finalists),
                   key=lambda r: r[0])
    return best[0], best[1], tried


def tune(plan: "capi.Plan", n_polys: int, scheds: Optional[Iterable[List[Pass]]] = None,
         iters: int = 5, use_cache: bool = True, verbose: bool = False,
         direction: int = 3) -> dict:
    """Pick the fastest forward and the fastest inverse schedule for this plan
    and batch size, apply them to the plan (only the forward one for
    direction 1, only the inverse one for 2) and return {"forward",
    "inverse", "fwd_us", "inv_us", "tried"}.  Without `scheds` the search of
    _search runs; with it, exactly those schedules are timed.  Inputs are
    uniform synthetic residues."""
    import torch
    from .tensors import to_device, empty
    import numpy as np

    name = torch.cuda.get_device_name()
    key = _key(plan.N, plan.moduli, n_polys, name) + f"|d={direction}"
    keep = (plan.schedule(plan.FORWARD), plan.schedule(plan.INVERSE))

    def apply(f, i):
        plan.set_schedule(f if direction & 1 else keep[0], plan.FORWARD)
        plan.set_schedule(i if direction & 2 else keep[1], plan.INVERSE)

    if use_cache and scheds is None:
        with _lock:
            hit = load_cache().get(key)
        if hit:
            f = [tuple(p) for p in hit["forward"]]
            i = [tuple(p) for p in hit["inverse"]]
            if valid(plan, f) and valid(plan, i):
                apply(f, i)
                return dict(hit, cached=True)
    rng = np.random.default_rng(1)
    host = np.empty((n_polys, plan.n_limbs, plan.N), dtype=np.uint64)
    for l, q in enumerate(plan.moduli):
        host[:, l] = rng.integers(0, q, size=(n_polys, plan.N), dtype=np.uint64)
    x, y = to_device(host), empty(host.shape)
    if scheds is None:
        fu = iu = float("inf")
        fs = is_ = None
        nf = ni = 0
        if direction & 1:
            fu, fs, nf = _search(plan, lambda sc: time_schedule(plan, sc, x, y, n_polys, iters,
                                                                1)[0], "fwd", verbose)
        if direction & 2:
            iu, is_, ni = _search(plan, lambda sc: time_schedule(plan, sc, x, y, n_polys, iters,
                                                                 2)[1], "inv", verbose)
        fs = fs or keep[0]
        is_ = is_ or keep[1]
        tried = nf + ni
    else:
        results = []
        for sched in scheds:
            if not valid(plan, sched):
                continue
            f, i = time_schedule(plan, sched, x, y, n_polys, iters)
            results.append((f, i, sched))
            if verbose:
                print(f"{f:9.1f} {i:9.1f}  {sched}", file=sys.stderr)
        if not results:
            raise RuntimeError("no valid schedule")
        fu, fs = min((r[0], r[2]) for r in results)
        iu, is_ = min((r[1], r[2]) for r in results)
        tried = len(results)
    if fs is None or is_ is None:
        raise RuntimeError("no valid schedule")
    apply(fs, is_)
    out = {"forward": [list(p) for p in fs], "inverse": [list(p) for p in is_],
           "fwd_us": fu, "inv_us": iu, "tried": tried}
    if use_cache:
        with _lock:
            cache = load_cache()
            cache[key] = out
            save_cache(cache)
    return out


def tune_tensor(plan: "capi.Plan", n_ct: int, scalars, iters: int = 5, use_cache: bool = True,
                verbose: bool = False) -> dict:
    """Pick the inverse schedule for hx_tensor_fma_inverse on n_ct ciphertext
    pairs (operands back to back, so the element-wise step can run inside
    the inverse's first pass) by timing that call itself, apply it to the
    plan and return {"inverse", "us", "tried"}.  Cached like tune()."""
    import torch
    from .tensors import to_device, empty
    import numpy as np

    name = torch.cuda.get_device_name()
    key = _key(plan.N, plan.moduli, n_ct, name) + "|tensor_inverse"
    if use_cache:
        with _lock:
            hit = load_cache().get(key)
        if hit:
            sch = [tuple(p) for p in hit["inverse"]]
            if valid(plan, sch):
                plan.set_schedule(sch, plan.INVERSE)
                return dict(hit, cached=True)
    keep_f = plan.schedule(plan.FORWARD)
    rng = np.random.default_rng(2)
    shape = (n_ct, plan.n_limbs, plan.N)

    def operand(k, bound_mf):
        h = np.empty((k,) + shape, dtype=np.uint64)
        for l, q in enumerate(plan.moduli):
            h[:, :, l] = rng.integers(0, bound_mf * q, size=(k, n_ct, plan.N), dtype=np.uint64)
        return to_device(h)

    A, E, R = operand(4, 4), operand(3, 1), empty((3,) + shape)
    st = torch.cuda.current_stream()

    def timer(sched):
        plan.set_schedule(sched, plan.BOTH)
        capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], A[0], A[1], A[2], A[3], scalars,
                                   E[0], E[1], E[2], n_ct, 4, st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(iters):
            capi.hx_tensor_fma_inverse(plan, R[0], R[1], R[2], A[0], A[1], A[2], A[3], scalars,
                                       E[0], E[1], E[2], n_ct, 4, st)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / iters

    us, sch, tried = _search(plan, timer, "tensor_inv", verbose)
    if sch is None:
        raise RuntimeError("no valid schedule")
    plan.set_schedule(keep_f, plan.FORWARD)
    plan.set_schedule(sch, plan.INVERSE)
    out = {"inverse": [list(p) for p in sch], "us": us, "tried": tried}
    if use_cache:
        with _lock:
            cache = load_cache()
            cache[key] = out
            save_cache(cache)
    return out


# ---------------------------------------------------------------- the ciphertext step
def step_candidates(logN: int) -> List[Tuple[List[Pass], List[Pass]]]:
    """(forward, inverse) schedule pairs under which hx_ciphertext_step runs
    as three launches: both two-pass, the row passes over the same stages
    K1 .. logN-1 (6..9 of them) in the same 2^logGb-row tiles with 8
    elements a thread (32..512 threads, four padded tiles within 192 KB of
    shared memory); the column passes' tile widths and the inverse column
    pass's twiddle staging vary."""
    out = []
    for K1 in splits(logN):
        K2 = logN - K1
        if not 6 <= K2 <= 9:
            continue
        for logGb in range(0, 4):
            te = 1 << (logGb + K2)
            if not 5 <= logGb + K2 - 3 <= 9 or 8 * 4 * (te + te // 16) > 192 * 1024:
                continue
            for fc in (3, 4):
                for ic in (3, 4):
                    for ipipe in (0, 2):
                        out.append(([(0, K1, 0, fc, 4, 0, 1), (K1, K2, logGb, 0, 3, 0, 1)],
                                    [(0, K1, 0, ic, 4, ipipe, 1), (K1, K2, logGb, 0, 3, 0, 2)]))
    return out


def tune_step(plan: "capi.Plan", n_ct: int, scalars, iters: int = 5, use_cache: bool = True,
              verbose: bool = False, streams: int = 1) -> Optional[dict]:
    """Pick the (forward, inverse) schedule pair for hx_ciphertext_step on
    n_ct ciphertext pairs by timing the call itself over step_candidates
    (the three best re-timed four times as long), apply it to the plan and
    return {"forward", "inverse", "us", "tried"}; None when log2 N has no
    candidate (the call then runs as the composition).  With streams > 1
    consecutive calls alternate over that many CUDA streams, each with its
    own output and scratch buffers (independent products overlapping, a
    throughput setting).  Cached like tune()."""
    import torch
    from .tensors import to_device, empty
    import numpy as np

    cands = [c for c in step_candidates(plan.N.bit_length() - 1)
             if valid(plan, c[0]) and valid(plan, c[1])]
    if not cands:
        return None
    name = torch.cuda.get_device_name()
    key = _key(plan.N, plan.moduli, n_ct, name) + f"|ciphertext_step|S={streams}"
    if use_cache:
        with _lock:
            hit = load_cache().get(key)
        if hit:
            f = [tuple(p) for p in hit["forward"]]
            i = [tuple(p) for p in hit["inverse"]]
            if valid(plan, f) and valid(plan, i):
                plan.set_schedule(f, plan.FORWARD)
                plan.set_schedule(i, plan.INVERSE)
                return dict(hit, cached=True)
    rng = np.random.default_rng(3)
    shape = (n_ct, plan.n_limbs, plan.N)

    def operand(k):
        h = np.empty((k,) + shape, dtype=np.uint64)
        for l, q in enumerate(plan.moduli):
            h[:, :, l] = rng.integers(0, q, size=(k, n_ct, plan.N), dtype=np.uint64)
        return to_device(h)

    X, E = operand(4), operand(3)
    st = torch.cuda.current_stream()
    sts = [st] + [torch.cuda.Stream() for _ in range(streams - 1)]
    bufs = [(empty((4,) + shape), empty((3,) + shape)) for _ in sts]

    def timer(pair, n):
        plan.set_schedule(pair[0], plan.FORWARD)
        plan.set_schedule(pair[1], plan.INVERSE)
        for k, s in enumerate(sts):
            capi.hx_ciphertext_step(plan, bufs[k][1], X, bufs[k][0], scalars, E, n_ct, s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for s in sts[1:]:
            s.wait_event(e0)
        for j in range(n):
            k = j % len(sts)
            capi.hx_ciphertext_step(plan, bufs[k][1], X, bufs[k][0], scalars, E, n_ct, sts[k])
        for s in sts[1:]:
            ev = torch.cuda.Event()
            ev.record(s)
            st.wait_event(ev)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / n

    first = sorted((timer(c, iters), k) for k, c in enumerate(cands))
    final = sorted((timer(cands[k], 4 * iters), k) for _, k in first[:3])
    us, k = final[0]
    f, i = cands[k]
    plan.set_schedule(f, plan.FORWARD)
    plan.set_schedule(i, plan.INVERSE)
    if verbose:
        print(f"ciphertext step: {us:.1f} us, forward {f}, inverse {i}")
    out = {"forward": [list(p) for p in f], "inverse": [list(p) for p in i], "us": us,
           "tried": len(cands)}
    if use_cache:
        with _lock:
            cache = load_cache()
            cache[key] = out
            save_cache(cache)
    return out


# ---------------------------------------------------------------- ragged batches
def ragged_splits(log2_n: int) -> List[int]:
    """Column-pass stage counts the ragged kernels can run at N = 2^log2_n
    (2048-element tiles: column passes of 5..9 stages, row passes of 6..11)."""
    if not 12 <= log2_n <= 17:
        return []
    return [k1 for k1 in range(5, 10) if 6 <= log2_n - k1 <= 11]


def _ragged_key(log2_n: int, moduli: Sequence[int], transforms: int, device_name: str) -> str:
    # transforms rounded to a power of two: a batch's time depends on how many
    # tiles it has, not on the exact count
    bucket = 1 << max(0, int(transforms).bit_length() - 1)
    return f"{device_name}|ragged|L={log2_n}|{width_class(moduli)}|T={bucket}"


def tune_ragged(items, reps: int = 3, use_cache: bool = True, verbose: bool = False) -> dict:
    """Pick the column/row split of the ragged kernels per log2 N for a set
    of ragged items (plan, d_in, d_out, n_polys) -- every N from 2^12 up
    present among them: for each such N, a forward and an inverse ragged call
    (hx_ntt_ragged, out of place, in a workspace) over that N's items alone,
    timed under every split of the menu; the fastest sum wins, is applied
    (hx_ragged_set_split, process-wide) and cached per (GPU, N, width mix,
    transform count).  Returns {log2 N: {"k1", "us", "tried"}}.  The item
    buffers are overwritten (d_out with spectra)."""
    import torch
    name = torch.cuda.get_device_name()
    by_n: Dict[int, list] = {}
    for it in items:
        plan = it[0]
        by_n.setdefault(plan.N.bit_length() - 1, []).append(it)
    st = torch.cuda.current_stream()
    out = {}
    for L, its in sorted(by_n.items()):
        cands = ragged_splits(L)
        if not cands:
            continue
        moduli = [q for it in its for q in it[0].moduli]
        transforms = sum(it[0].n_limbs * it[3] for it in its)
        key = _ragged_key(L, moduli, transforms, name)
        if use_cache:
            with _lock:
                hit = load_cache().get(key)
            if hit and hit.get("k1") in cands:
                capi.hx_ragged_set_split(L, hit["k1"])
                out[L] = dict(hit, cached=True)
                continue
        h = [it[0].handle for it in its]
        din = [capi.ptr(it[1]) for it in its]
        dout = [capi.ptr(it[2]) for it in its]
        npol = [it[3] for it in its]
        arr = capi.ragged_items_array(h, din, dout, npol)
        back = capi.ragged_items_array(h, dout, dout, npol)
        keep = capi.hx_ragged_get_split(L)
        best = None
        for k1 in cands:
            capi.hx_ragged_set_split(L, k1)
            wsb = max(capi.hx_ntt_ragged_workspace(arr), capi.hx_ntt_ragged_workspace(back))
            ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")

            def run():
                capi.hx_ntt_ragged(arr, ws, wsb, 1, 1, 1, st)
                capi.hx_ntt_ragged(back, ws, wsb, 2, 1, 1, st)

            run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                run()
            e1.record(st)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / reps
            if verbose:
                print(f"ragged L={L} k1={k1} {us:9.1f} us", file=sys.stderr)
            if best is None or us < best[0]:
                best = (us, k1)
        capi.hx_ragged_set_split(L, best[1] if best else keep)
        res = {"k1": best[1], "us": best[0], "tried": len(cands)}
        out[L] = res
        if use_cache:
            with _lock:
                cache = load_cache()
                cache[key] = res
                save_cache(cache)
    return out
