"""Golden fixtures (written by tests/golden/make_golden.py from the oracle),
re-checked here against sympy and Python big integers so that the stored
values are pinned independently of the oracle that wrote them."""
import os

from sympy.ntheory.residue_ntheory import nthroot_mod

from oracle import bigint

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_params_fixture_independent():
    rows = _rows("params.txt")
    assert len(rows) >= 9
    for N, q, psi, psi_inv, n_inv in ([int(x) for x in r] for r in rows):
        assert (q - 1) % (2 * N) == 0
        assert min(nthroot_mod(q - 1, N, q, all_roots=True)) == psi   # psi^N = -1, smallest
        assert psi * psi_inv % q == 1
        assert N * n_inv % q == 1


def test_ntt16_fixture_against_closed_form():
    a, out = ([int(x) for x in r] for r in _rows("ntt_n16_q97.txt"))
    psi = min(bigint.primitive_2n_roots(16, 97))
    assert bigint.negacyclic_ntt_bitrev(a, 97, psi) == out
