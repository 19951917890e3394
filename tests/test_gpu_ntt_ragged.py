"""hx_ntt_ragged (a ragged set of transforms in a caller-owned workspace, the
serving primitive for NTT requests) against the oracle: items of every pass
shape (single-pass N = 2^10, 2^11; two-pass 2^12 .. 2^16), several limbs and
polynomials, forward and inverse, lazy output range, in place and out of
place, two calls overlapping on two streams with their own workspaces, and a
workspace one step too small refused."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_2103_16400_gb300 import capi
from paper_2103_16400_gb300.tensors import empty, to_device, to_host

pytestmark = pytest.mark.gpu

SPEC = [(10, 2, 1), (11, 3, 2), (12, 1, 1), (14, 4, 2), (16, 2, 1)]   # log2 N, limbs, polys


def workload(seed):
    pool = W.mixed_width_primes(4)
    out = []
    for k, (logN, L, P) in enumerate(SPEC):
        qs = pool[:L]
        out.append((1 << logN, qs, W.poly_batch(seed, k, P, qs, 1 << logN)))
    return out


def test_forward_and_inverse_vs_oracle(hexlib):
    sets = workload(W.SEED_BASE + 980)
    plans = [capi.Plan(N, qs) for N, qs, _ in sets]
    dx = [to_device(x) for _, _, x in sets]
    dy = [empty(x.shape) for _, _, x in sets]
    items = [(p, a, b, x.shape[0]) for p, a, b, (_, _, x) in zip(plans, dx, dy, sets)]
    wsb = capi.hx_ntt_ragged_workspace(items)
    ws = empty((wsb // 8,))
    capi.hx_ntt_ragged(items, ws, wsb, 1, 1, 1)
    spectra = [oracle.ntt_forward(x, qs) for _, qs, x in sets]
    for y, exp in zip(dy, spectra):
        np.testing.assert_array_equal(to_host(y), exp)
    # lazy output range: [0, 4q) and the same residues
    capi.hx_ntt_ragged(items, ws, wsb, 1, 1, 4)
    for y, exp, (_, qs, _) in zip(dy, spectra, sets):
        got = to_host(y)
        for l, q in enumerate(qs):
            assert (got[:, l] < np.uint64(4 * q)).all()
            np.testing.assert_array_equal(got[:, l] % np.uint64(q), exp[:, l])
    # inverse in place, from the lazy spectra (input_mod_factor 2 covers [0, 2q) only,
    # so first bring them back to [0, q) with a plain forward)
    capi.hx_ntt_ragged(items, ws, wsb, 1, 1, 1)
    inv_items = [(p, b, b, x.shape[0]) for p, b, (_, _, x) in zip(plans, dy, sets)]
    capi.hx_ntt_ragged(inv_items, ws, wsb, 2, 1, 1)
    for y, (_, _, x) in zip(dy, sets):
        np.testing.assert_array_equal(to_host(y), x)
    with pytest.raises(capi.HexError):
        capi.hx_ntt_ragged(items, ws, wsb - 256, 1, 1, 1)


def test_two_streams_two_workspaces(hexlib):
    sets = workload(W.SEED_BASE + 981)
    plans = [capi.Plan(N, qs) for N, qs, _ in sets]
    dx = [to_device(x) for _, _, x in sets]
    dy = [empty(x.shape) for _, _, x in sets]
    dz = [empty(x.shape) for _, _, x in sets]
    a_items = [(p, a, b, x.shape[0]) for p, a, b, (_, _, x) in zip(plans, dx, dy, sets)]
    b_items = [(p, a, c, x.shape[0]) for p, a, c, (_, _, x) in zip(plans, dx, dz, sets)]
    wsb = capi.hx_ntt_ragged_workspace(a_items)
    ws1, ws2 = empty((wsb // 8,)), empty((wsb // 8,))
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    capi.hx_ntt_ragged(a_items, ws1, wsb, 1, 1, 1, s1)     # forward on one stream
    capi.hx_ntt_ragged(b_items, ws2, wsb, 2, 1, 1, s2)     # inverse on the other
    torch.cuda.synchronize()
    for y, z, (_, qs, x) in zip(dy, dz, sets):
        np.testing.assert_array_equal(to_host(y), oracle.ntt_forward(x, qs))
        np.testing.assert_array_equal(to_host(z), oracle.ntt_inverse(x, qs))
