"""The benchmark's own timed step (bench.HexStep: autotuned schedules; the
ciphertext product as hx_ciphertext_step's three launches, or as the
composition of one forward call over the four inputs and the tensor/FMA step
fused into the inverse transform of the three outputs) at its full size --
N = 65536, 32 mixed limbs -- compared element by element with the oracle's
ciphertext pipeline, on both paths: steps run one after another on one
stream, and consecutive steps alternating over the step streams (each with
its own buffers), as the timed region runs them."""
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
    assert len(step.streams) == bench.STEP_STREAMS >= 2
    assert step.path in ("step", "composed")
    exp = [oracle.ciphertext_tensor(*ins, s, *es, wl.moduli) for ins, es in sets]
    for path in ("step", "composed"):
        step.path = path
        for i in (1, 0):                              # second set first, then the first
            R = [to_host(r) for r in step.run(i, one_stream=True)]
            torch.cuda.synchronize()
            for got, e in zip(R, exp[i]):
                np.testing.assert_array_equal(got, e)
        # four steps in a row over the step streams: step i on stream i mod 2
        # with that stream's buffers and input set i mod 2; the last two are
        # checked
        ev = torch.cuda.Event()
        ev.record(step.stream)
        step.begin(ev)
        outs = [step.run(i) for i in range(4)]
        step.join()
        torch.cuda.synchronize()
        for i in (2, 3):
            for got, e in zip(outs[i], exp[i % 2]):
                np.testing.assert_array_equal(to_host(got), e)
