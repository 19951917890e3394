"""Autotuner for the NTT kernel schedule.

The paper leaves the choice between its kernel variants to fixed CPUID rules
and names choosing "via a small number of trials" as future work (Section
3.2).  Here the trials are the schedule: how the log2 N stages split into
passes, the tile shape of each pass, elements per thread, and whether a pass
runs the persistent double-buffered kernel.  Every schedule computes the same
result; `tune()` times each candidate's forward and inverse transform on the
caller's plan and batch size with CUDA events and keeps the fastest.
Winners are cached in a JSON file keyed by GPU name, N, limb-width mix and
batch size.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

from . import capi

Pass = Tuple[int, int, int, int, int, int, int]   # s0, K, logGb, logGc, logR, pipe, np
CACHE_PATH = os.environ.get("HX_TUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                         "_build", "tune_cache.json"))
_lock = threading.Lock()


#: per-pass kernel variants: (logR, pipe, np) -- 16 or 8 elements per thread,
#: plain or persistent, one or two polynomials per thread
VARIANTS = ((3, 0, 1), (4, 0, 1), (3, 1, 1), (4, 1, 1), (3, 0, 2))


def candidates(logN: int, variants=VARIANTS) -> List[List[Pass]]:
    """Schedules worth trying for log2 N (validity is checked by the library)."""
    out: List[List[Pass]] = []
    if logN <= 13:
        for logR, pipe, np_ in variants:
            out.append([(0, logN, 0, 0, logR, pipe, np_)])
    for K1 in range(6, 10):
        K2 = logN - K1
        if not 6 <= K2 <= 13:
            continue
        for logGc in (2, 3, 4, 5):
            for v1 in variants:
                for logGb in range(0, 6):
                    for v2 in variants:
                        out.append([(0, K1, 0, logGc) + v1, (K1, K2, logGb, 0) + v2])
    return out


def valid(plan: "capi.Plan", sched: List[Pass]) -> bool:
    try:
        plan.set_schedule(sched)
        return True
    except capi.HexError:
        return False


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


def time_schedule(plan, sched, x, y, n_polys: int, iters: int = 5) -> Tuple[float, float]:
    """(forward us, inverse us) per call for one schedule, averaged over iters."""
    import torch
    plan.set_schedule(sched, plan.BOTH)
    st = torch.cuda.current_stream()
    capi.hx_ntt_forward(plan, y, x, n_polys, 1, 4, st)
    capi.hx_ntt_inverse(plan, y, y, n_polys, 1, 1, st)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(st)
    for _ in range(iters):
        capi.hx_ntt_forward(plan, y, x, n_polys, 1, 4, st)
    ev[1].record(st)
    for _ in range(iters):
        capi.hx_ntt_inverse(plan, y, y, n_polys, 1, 1, st)
    ev[2].record(st)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) * 1e3 / iters, ev[1].elapsed_time(ev[2]) * 1e3 / iters


def tune(plan: "capi.Plan", n_polys: int, scheds: Optional[Iterable[List[Pass]]] = None,
         iters: int = 5, use_cache: bool = True, verbose: bool = False,
         direction: int = 3) -> dict:
    """Pick the fastest forward and the fastest inverse schedule for this plan
    and batch size, apply them to the plan (only the forward one for
    direction 1, only the inverse one for 2) and return {"forward",
    "inverse", "fwd_us", "inv_us", "tried"}.  Inputs are uniform synthetic
    residues."""
    import torch
    from .tensors import to_device, empty
    import numpy as np

    name = torch.cuda.get_device_name()
    key = _key(plan.N, plan.moduli, n_polys, name)
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
    logN = plan.N.bit_length() - 1
    results = []
    for sched in (scheds if scheds is not None else candidates(logN)):
        if not valid(plan, sched):
            continue
        f, i = time_schedule(plan, sched, x, y, n_polys, iters)
        results.append((f, i, sched))
        if verbose:
            print(f"{f:9.1f} {i:9.1f}  {sched}")
    if not results:
        raise RuntimeError("no valid schedule")
    bf = min(results, key=lambda r: r[0])
    bi = min(results, key=lambda r: r[1])
    apply(bf[2], bi[2])
    out = {"forward": [list(p) for p in bf[2]], "inverse": [list(p) for p in bi[2]],
           "fwd_us": bf[0], "inv_us": bi[1], "tried": len(results)}
    if use_cache:
        with _lock:
            cache = load_cache()
            cache[key] = out
            save_cache(cache)
    return out
