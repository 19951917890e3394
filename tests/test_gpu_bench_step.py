"""The benchmark's own timed step (bench.HexStep: autotuned schedules, one
forward call over the four inputs, then the tensor/FMA step fused into the
inverse transform of the three outputs) at its full size -- N = 65536, 32
mixed limbs -- compared element by element with the oracle's ciphertext
pipeline."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_bench_step_full_size_parity(hexlib):
    import torch

    import bench
    from paper_2103_16400_gb300.tensors import to_host
    N, nl = 1 << 16, 32
    wl, sets, s = bench.workload_arrays(N, nl, 2)
    step = bench.HexStep(N, wl.moduli, s, bench.device_sets(sets), torch)
    for i in (1, 0):                                  # second set first, then the first
        R = [to_host(r) for r in step.run(i)]
        torch.cuda.synchronize()
        ins, es = sets[i]
        exp = oracle.ciphertext_tensor(*ins, s, *es, wl.moduli)
        for got, e in zip(R, exp):
            np.testing.assert_array_equal(got, e)
