"""TensorPipeline (host-resident ciphertext products streamed through three
CUDA streams with double-buffered device sets) against the oracle's
ciphertext pipeline: several batches in flight, both buffer sets reused,
one and two ciphertext pairs per batch, every result compared bit for bit."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.pipeline import TensorPipeline

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_ct,depth", [(1, 2), (2, 3)])
def test_pipeline_matches_oracle(hexlib, n_ct, depth):
    import torch
    N, moduli = 1 << 12, W.mixed_width_primes(3)
    L = len(moduli)
    plan = capi.Plan(N, moduli)
    s = W.scalars(W.SEED_BASE + 990, 20, moduli)
    pipe = TensorPipeline(plan, s, n_ct, depth)
    batches, outs = [], []
    for b in range(5):
        ins = [W.poly_batch(W.SEED_BASE + 991 + b, t, n_ct, moduli, N) for t in range(4)]
        es = [W.poly_batch(W.SEED_BASE + 991 + b, 10 + t, n_ct, moduli, N) for t in range(3)]
        h_in = torch.from_numpy(np.stack(ins).view(np.int64)).pin_memory()
        h_add = torch.from_numpy(np.stack(es).view(np.int64)).pin_memory()
        h_out = torch.empty((3, n_ct, L, N), dtype=torch.int64).pin_memory()
        pipe.submit(h_in, h_add, h_out)
        batches.append((ins, es, h_in, h_add))    # host buffers stay alive until the end
        outs.append(h_out)
    pipe.synchronize()
    for (ins, es, _, _), h_out in zip(batches, outs):
        exp = oracle.ciphertext_tensor(*ins, s, *es, moduli)
        got = h_out.numpy().view(np.uint64)
        for k in range(3):
            np.testing.assert_array_equal(got[k], exp[k])
