"""Writes e1_trap_sweep0.txt: the FP64 oracle's energies in the first two-site DMRG sweep
of the first example of Sec. 5 (Fig. 4: L = 100, N = 100, n_max = 3, U/J = 5, trap
V/J = 0.01 about the chain centre, chi = 100), from the seeded random start with the
Gaussian sector profile: after the sweep and at each of its 198 updates.  Calls only the
oracle and the seeded input generator.  Takes about a quarter of an hour on eight cores.

    python tests/golden/make_e1_sweep0.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import bose_hubbard as bh  # noqa: E402
from oracle import dmrg as od  # noqa: E402
from paper_1610_02244_gb300 import synth  # noqa: E402

L, N, N_MAX, J, U, V, CHI, SEED = 100, 100, 3, 1.0, 5.0, 0.01, 100, 4


def main():
    j_c = (L + 1) / 2.0
    A, q = synth.random_charged_mps(synth.rng(SEED), L, N_MAX + 1, N, CHI, "gauss", 2.0)
    Ws, l, r = bh.bh_mpo(L, N_MAX, J, U, 0.0, V, j_c)
    _, _, hist = od.dmrg(A, q, Ws, l, r, CHI, 1)
    ups = hist[0]["updates"]
    with open(os.path.join(HERE, "e1_trap_sweep0.txt"), "w") as f:
        f.write("# First example of Sec. 5 (Fig. 4): L=100 N=100 n_max=3 J=1 U=5 V=0.01 "
                "j_c=50.5 chi=100,\n# seeded start synth.random_charged_mps(rng(4), 100, 4, "
                "100, 100, 'gauss', 2.0); FP64 oracle,\n# one two-site sweep (bonds 0..98 "
                "then 98..0), default truncation.  Written by make_e1_sweep0.py.\n")
        f.write(f"E_sweep0 {float(hist[0]['E'])!r}\n")
        f.write(f"unconverged {sum(not u['converged'] for u in ups)}\n")
        f.write(f"matvecs {sum(u['matvecs'] for u in ups)}\n")
        for k, u in enumerate(ups):  # every update, in sweep order
            f.write(f"E_u{k:03d} {float(u['E'])!r}\n")


if __name__ == "__main__":
    main()
