"""Writes tebd_mott64_step50.txt: the FP64 oracle's state after 50 second-order Trotter
steps of the quench from the Mott state |1...1> of the 64-site Bose-Hubbard chain (Eq. 2
with n_max = 4, J = 1, U = 2; dt = 0.01, chi_max = 512, truncation error 1e-10 in the
2-norm of Eq. 3, no renormalisation): <psi|psi>, <H>/<psi|psi>, the summed truncation
errors and discarded weights, the largest bond dimension, and <n_j> for every site.
Calls only the oracle.  Takes a few minutes on eight cores.

    python tests/golden/make_tebd_mott64.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import bose_hubbard as bh  # noqa: E402
from oracle import contract as oc  # noqa: E402
from oracle import tebd as ot  # noqa: E402
from oracle.svd import TruncParams  # noqa: E402

L, N_MAX, J, U, DT, CHI, EPS, STEPS = 64, 4, 1.0, 2.0, 0.01, 512, 1e-10, 50


def main():
    A, q = ot.product_state([1] * L, N_MAX)
    tb = ot.Tebd(A, q, N_MAX, J, U, DT, TruncParams(chi_max=CHI, err_tol=EPS, rel_tol=1e-16,
                                                     abs_tol=-1.0))
    for _ in range(STEPS):
        tb.step()
    Ws, l, r = bh.bh_mpo(L, N_MAX, J, U)
    norm2 = oc.mps_overlap(tb.A, tb.A).real
    E = oc.mps_expect_mpo(tb.A, Ws, l, r).real / norm2
    # <n_j> as the expectation of an MPO of bond dimension one (identity on every site but
    # j, the number operator on j): environments instead of a transfer sweep per site
    d = N_MAX + 1
    eye = np.eye(d, dtype=np.complex128).reshape(1, 1, d, d)
    num = np.diag(np.arange(d, dtype=np.float64)).astype(np.complex128).reshape(1, 1, d, d)
    one = np.ones(1, dtype=np.complex128)
    n = [oc.mps_expect_mpo(tb.A, [num if k == j else eye for k in range(L)], one, one).real / norm2
         for j in range(L)]
    with open(os.path.join(HERE, "tebd_mott64_step50.txt"), "w") as f:
        f.write("# Quench from |1...1>, Bose-Hubbard L=64 n_max=4 J=1 U=2 (Eq. 2), second-order "
                "Trotter dt=0.01,\n# chi_max=512, 2-norm truncation error 1e-10, no "
                "renormalisation: FP64 oracle after 50 steps.\n# Written by "
                "make_tebd_mott64.py.\n")
        f.write(f"norm2 {float(norm2)!r}\n")
        f.write(f"E {float(E)!r}\n")
        f.write(f"eps_sum {float(tb.eps_sum)!r}\n")
        f.write(f"disc_sum {float(tb.disc_sum)!r}\n")
        f.write(f"max_chi {max(a.shape[2] for a in tb.A)}\n")
        for j in range(L):
            f.write(f"n_{j:02d} {float(n[j])!r}\n")


if __name__ == "__main__":
    main()
