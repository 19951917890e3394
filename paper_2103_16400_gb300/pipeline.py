"""Host-resident ciphertext products streamed through the GPU.

One batch is the ciphertext product of hx_ciphertext_tensor on operands that
live in pinned host memory: upload the four input polynomials (a0, a1, b0,
b1) and the three addends (e0, e1, e2), run hx_ciphertext_step on them in
place (forward NTT, tensor, FMA and inverse NTT: three launches when the
plan's schedules share their row passes, else the forward call and the
fused inverse), download the three results.

The host link is slower than the transforms (about 0.2 TB/s each way against
several TB/s of HBM), so batches overlap: three CUDA streams -- upload,
compute, download -- and `depth` device buffer sets let the upload of batch
i+1 and the download of batch i-1 run while batch i computes.  Events order
the reuse of each buffer set: an upload waits until the compute that last
read its set is done; a compute waits for its upload and for the download
that last read its result buffer.

All arithmetic runs in the CUDA library; this module only moves memory and
orders streams (PyTorch supplies the pinned and device buffers and the
streams).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

from . import capi


class TensorPipeline:
    """Streams ciphertext products of one plan (N, moduli) with n_ct pairs per
    batch.  Host buffers: inputs [4][n_ct][L][N] and addends [3][n_ct][L][N]
    (pinned uint64 stored as int64), results [3][n_ct][L][N] (pinned).

        pipe = TensorPipeline(plan, scalars, n_ct=1)
        for h_in, h_add, h_out in batches:
            pipe.submit(h_in, h_add, h_out)      # returns at once
        pipe.synchronize()                        # every h_out is filled

    A host result buffer may be reused once the event returned by submit()
    for it has completed (or after synchronize())."""

    def __init__(self, plan: "capi.Plan", scalars: Sequence[int], n_ct: int = 1,
                 depth: int = 2):
        import torch
        from .tensors import empty
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.torch = torch
        self.plan, self.scalars, self.n_ct, self.depth = plan, scalars, n_ct, depth
        L, N = plan.n_limbs, plan.N
        self.A = [empty((4, n_ct, L, N)) for _ in range(depth)]
        self.E = [empty((3, n_ct, L, N)) for _ in range(depth)]
        self.R = [empty((3, n_ct, L, N)) for _ in range(depth)]
        self.s_up, self.s_comp, self.s_down = (torch.cuda.Stream() for _ in range(3))
        self.up_done = [torch.cuda.Event() for _ in range(depth)]
        self.comp_done = [torch.cuda.Event() for _ in range(depth)]
        self.down_done = [torch.cuda.Event() for _ in range(depth)]
        self.used: List[bool] = [False] * depth
        self.n = 0

    def submit(self, h_in, h_add, h_out):
        """Enqueue one batch; returns the event that fires when h_out holds
        its results."""
        torch = self.torch
        k = self.n % self.depth
        A, E, R = self.A[k], self.E[k], self.R[k]
        with torch.cuda.stream(self.s_up):
            if self.used[k]:
                self.s_up.wait_event(self.comp_done[k])
            A.copy_(h_in, non_blocking=True)
            E.copy_(h_add, non_blocking=True)
            self.up_done[k].record(self.s_up)
        s = self.s_comp
        s.wait_event(self.up_done[k])
        if self.used[k]:
            s.wait_event(self.down_done[k])
        # the whole product in place on A: three launches when the plan's
        # schedules allow (hx_ciphertext_step), else forward + fused inverse
        capi.hx_ciphertext_step(self.plan, R, A, A, self.scalars, E, self.n_ct, s)
        self.comp_done[k].record(s)
        with torch.cuda.stream(self.s_down):
            self.s_down.wait_event(self.comp_done[k])
            h_out.copy_(R, non_blocking=True)
            self.down_done[k].record(self.s_down)
        self.used[k] = True
        self.n += 1
        return self.down_done[k]

    def streams(self):
        return self.s_up, self.s_comp, self.s_down

    def synchronize(self):
        for s in self.streams():
            s.synchronize()
