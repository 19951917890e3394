"""Writes the fixtures in this folder.  Calls only the CPU oracle (and the
seeded input generator); nothing here touches the CUDA library.

  python tests/golden/make_golden.py

Fixtures:
  params.txt   -- per workload modulus: N, q, the smallest primitive 2N-th
                  root psi (the reading taken where the paper leaves psi
                  open, Section 3 NTT class API), psi^-1 and N^-1 mod q.
  ntt_n16_q97.txt -- a seeded length-16 vector mod 97 and its forward
                  negacyclic NTT (bit-reversed output, Section 2.2).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    rows = []
    cases = [(1024, q) for q in W.ntt_primes(50, 2048, 1)]
    cases += [(16384, q) for q in W.ntt_primes(50, 32768, 4) + W.ntt_primes(60, 32768, 4)]
    cases += [(65536, q) for q in W.mixed_width_primes(6)]
    for N, q in cases:
        psi = oracle.min_primitive_root(N, q)
        rows.append(f"{N} {q} {psi} {oracle.invmod(psi, q)} {oracle.invmod(N, q)}")
    with open(os.path.join(HERE, "params.txt"), "w") as f:
        f.write("# N q psi psi_inv N_inv   (written by make_golden.py from the oracle)\n")
        f.write("\n".join(rows) + "\n")
    q, N = 97, 16
    a = W.uniform_mod(W.stream_key(W.SEED_BASE, 97), N, q)
    out = oracle.ntt_forward_1(a, q)
    with open(os.path.join(HERE, "ntt_n16_q97.txt"), "w") as f:
        f.write("# q=97 N=16 psi=min root; line 1 input, line 2 forward NTT (bit-reversed)\n")
        f.write(" ".join(str(int(x)) for x in a) + "\n")
        f.write(" ".join(str(int(x)) for x in out) + "\n")


if __name__ == "__main__":
    main()
