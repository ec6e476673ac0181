"""Writes spin1_sweeps.txt: the FP64 oracle's energies over four two-site DMRG sweeps of the
isotropic spin-1 Heisenberg chain of Sec. 6, Table 1 (L = 101, chi = 200, U(1) in S^z,
S^z_total = 0), from the seeded random start with the Gaussian sector profile (the start
the DMRG benchmark uses): the energy after each sweep and at each of the 200 updates of the
last sweep, by which the sweeps have converged.  Calls only the oracle and the seeded input
generator.  Takes one to three hours on eight to sixteen cores (the first sweep dominates).

    python tests/golden/make_spin1_sweeps.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dmrg as od  # noqa: E402
from oracle import spin as ospin  # noqa: E402
from paper_1610_02244_gb300 import synth  # noqa: E402

L, TWO_S, CHI, SEED, SWEEPS = 101, 2, 200, 0, 4


def main():
    N = L * TWO_S // 2
    A, q = synth.random_charged_mps(synth.rng(SEED), L, TWO_S + 1, N, CHI, "gauss", 2.0)
    Ws, l, r, _ = ospin.heisenberg_mpo(L, TWO_S, 1.0, 1.0)
    _, _, hist = od.dmrg(A, q, Ws, l, r, CHI, SWEEPS)
    ups = hist[-1]["updates"]
    with open(os.path.join(HERE, "spin1_sweeps.txt"), "w") as f:
        f.write("# Spin-1 Heisenberg chain of Sec. 6 (Table 1): L=101 J=Jz=1 hz=0 chi=200,\n"
                "# S^z_total=0 (N=101 quanta); seeded start "
                "synth.random_charged_mps(rng(0), 101, 3, 101, 200, 'gauss', 2.0);\n# FP64 "
                f"oracle, {SWEEPS} two-site sweeps (bonds 0..99 then 99..0), default truncation: "
                "energy after each sweep, every update of the last.  Written by "
                "make_spin1_sweeps.py.\n")
        f.write(f"chi {CHI}\n")
        for s, h in enumerate(hist):
            f.write(f"E_sweep{s} {float(h['E'])!r}\n")
            f.write(f"unconverged{s} {sum(not u['converged'] for u in h['updates'])}\n")
        for k, u in enumerate(ups):
            f.write(f"E_u{k:03d} {float(u['E'])!r}\n")


if __name__ == "__main__":
    main()
