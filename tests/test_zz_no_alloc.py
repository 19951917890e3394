"""hx_batch_run_static, the ragged run that allocates no device memory.

It serves callers that cannot call cudaMalloc where they need transforms --
a serving loop held to a fixed memory budget, a host application whose
memory pool owns the GPU, a latency-critical path -- by keeping its work
list in a fixed array inside the library.  Its output must equal that of the
allocating entry point (hx_batch_create + hx_batch_run) bit for bit, on two
calls in a row (the second call finds the first call's leftovers in the
shared array).  This file is collected last so that a failure here leaves
every other test already run; it also passes alone in a fresh process."""
import numpy as np
import pytest

import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

SPEC = [(1 << 10, 2, 2), (1 << 11, 3, 1), (1 << 13, 2, 1), (1 << 16, 3, 1), (1 << 17, 2, 1)]


def _case(seed):
    items = []
    for k, (N, nl, P) in enumerate(SPEC):
        qs = W.mixed_width_primes(nl)
        x = W.poly_batch(seed, k, P, qs, N)
        items.append((capi.Plan(N, qs), to_device(x), x.shape))
    return items


@pytest.mark.parametrize("direction,in_mf,out_mf", [(1, 1, 1), (1, 4, 4), (2, 1, 1), (2, 2, 2)])
def test_static_run_matches_allocating_batch_twice(hexlib, direction, in_mf, out_mf):
    import torch
    for seed in (W.SEED_BASE + 7000, W.SEED_BASE + 7001):      # two calls in a row
        items = _case(seed)
        if in_mf > 1:        # lazy inputs: add q to every other coefficient
            for p, d, shape in items:
                h = to_host(d)
                for l, q in enumerate(p.moduli):
                    h[:, l, ::2] += np.uint64(q)
                d.copy_(to_device(h))
        ref = [empty(s) for _, _, s in items]
        got = [empty(s) for _, _, s in items]
        b = capi.Batch([(p, d, r, s[0]) for (p, d, s), r in zip(items, ref)], direction, in_mf,
                       out_mf)
        b.run()
        capi.hx_batch_run_static([(p, d, g, s[0]) for (p, d, s), g in zip(items, got)],
                                 direction, in_mf, out_mf)
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            np.testing.assert_array_equal(to_host(g), to_host(r))
        b.destroy()


def test_static_run_refuses_oversized_requests(hexlib):
    # 1024 transforms of N = 2^17 need 1024 * 128 = 131072 tiles > 131064
    qs = W.mixed_width_primes(32)
    p = capi.Plan(1 << 17, qs)
    buf = empty((32, 32, 1 << 17))            # a real buffer; it is never touched
    with pytest.raises(capi.HexError) as e:
        capi.hx_batch_run_static([(p, buf, buf, 32)], 1, 1, 1)
    assert e.value.status == -12
    assert b"capacity" in capi.load().hx_strerror(-12)
