"""Second-order Trotter TEBD, FP64 (Sec. 3 Trotterised update, Sec. 5 time evolution).

The paper names the Trotterised update and runs it (Sec. 5: quench from a product state,
accumulated truncation error and 1 - <psi|psi> tracked over time) but prints no scheme;
the scheme used here is the symmetric second-order split

  U(dt) = exp(-i H_odd dt/2) exp(-i H_even dt) exp(-i H_odd dt/2)

with odd bonds (1,2), (3,4), ... and even bonds (2,3), (4,5), ... (1-based), hbar = 1.
Each gate acts on one bond: theta = A_i A_{i+1}, theta' = G theta, truncated SVD
(App. B.1.2).  Before each gate the orthogonality centre is moved onto site i or i+1 by
exact SVD moves, so every truncation happens at the centre.  The state is not
renormalised after truncation, so 1 - <psi|psi> accumulates the discarded weight.
The gates of a layer commute; the layers alternate direction (ascending, descending,
ascending, then descending first in the next step): an ascending gate leaves
A_i <- U, A_{i+1} <- S V^H (centre on i+1), a descending one A_i <- U S, A_{i+1} <- V^H
(centre on i).
"""
from __future__ import annotations

import numpy as np

from .bose_hubbard import bond_hamiltonian, bond_weights, gate
from .contract import gate_apply, theta_form
from .dmrg import EXACT, site_charges, theta_charges
from .svd import TruncParams, svd_truncate


def product_state(occupations, n_max: int):
    """MPS of the Fock state |n_1, ..., n_L> with bond labels (bosons to the left)."""
    d = n_max + 1
    A, q = [], [np.zeros(1, dtype=np.int64)]
    tot = 0
    for n in occupations:
        t = np.zeros((1, d, 1), dtype=np.complex128)
        t[0, int(n), 0] = 1.0
        A.append(t)
        tot += int(n)
        q.append(np.array([tot], dtype=np.int64))
    return A, q


class Tebd:
    def __init__(self, A, q, n_max: int, J: float, U: float, dt: float,
                 trunc: TruncParams, mu: float = 0.0):
        self.A = [t.copy() for t in A]
        self.q = [c.copy() for c in q]
        self.d = n_max + 1
        self.trunc = trunc
        self.centre = 0
        L = len(A)
        self.L = L
        self.gates = {}
        for tau_key, tau in (("half", dt / 2), ("full", dt)):
            for i in range(L - 1):
                c1, c2 = bond_weights(L, i + 1)
                h = bond_hamiltonian(n_max, J, U, c1, c2, mu)
                self.gates[(tau_key, i)] = gate(h, tau)
        self.eps_sum = 0.0     # sum of per-gate truncation errors (Eq. 3)
        self.disc_sum = 0.0    # sum of discarded weights
        self.up = True         # direction of the next layer

    @classmethod
    def from_bond_hamiltonians(cls, A, q, bond_hs, dt: float, trunc: TruncParams):
        """The same scheme for any nearest-neighbour Hamiltonian: bond_hs[i] is the d^2 x
        d^2 term of bond (i, i+1) (0-based), on-site parts already split between bonds."""
        d = A[0].shape[1]
        self = cls(A, q, d - 1, 0.0, 0.0, dt, trunc)
        for i, h in enumerate(bond_hs):
            self.gates[("half", i)] = gate(h, dt / 2)
            self.gates[("full", i)] = gate(h, dt)
        return self

    def _move_right(self):
        j, d = self.centre, self.d
        chl, _, chr_ = self.A[j].shape
        rows, _ = site_charges(self.q[j], self.q[j + 1], d)
        U, S, Vh, bq, _ = svd_truncate(self.A[j].reshape(chl * d, chr_), rows,
                                       self.q[j + 1], EXACT)
        self.A[j] = U.reshape(chl, d, -1)
        self.A[j + 1] = np.einsum("km,msb->ksb", S[:, None] * Vh, self.A[j + 1])
        self.q[j + 1] = bq
        self.centre += 1

    def _move_left(self):
        j, d = self.centre, self.d
        chl, _, chr_ = self.A[j].shape
        _, cols = site_charges(self.q[j], self.q[j + 1], d)
        U, S, Vh, bq, _ = svd_truncate(self.A[j].reshape(chl, d * chr_), self.q[j], cols,
                                       EXACT)
        self.A[j] = Vh.reshape(-1, d, chr_)
        self.A[j - 1] = np.einsum("asm,mk->ask", self.A[j - 1], U * S[None, :])
        self.q[j] = bq
        self.centre -= 1

    def apply_gate(self, i: int, G: np.ndarray, ascending: bool = True):
        while self.centre < i:
            self._move_right()
        while self.centre > i + 1:
            self._move_left()
        d = self.d
        theta = gate_apply(G, theta_form(self.A[i], self.A[i + 1]))
        chl, _, _, chr_ = theta.shape
        rows, cols = theta_charges(self.q[i], self.q[i + 2], d)
        U, S, Vh, bq, info = svd_truncate(theta.reshape(chl * d, d * chr_), rows, cols,
                                          self.trunc)
        k = len(S)
        if ascending:
            self.A[i] = U.reshape(chl, d, k)
            self.A[i + 1] = (S[:, None] * Vh).reshape(k, d, chr_)
            self.centre = i + 1
        else:
            self.A[i] = (U * S[None, :]).reshape(chl, d, k)
            self.A[i + 1] = Vh.reshape(k, d, chr_)
            self.centre = i
        self.q[i + 1] = bq
        self.eps_sum += info["err"]
        self.disc_sum += info["disc"]

    def step(self):
        odd = range(0, self.L - 1, 2)
        even = range(1, self.L - 1, 2)
        for layer, key in ((odd, "half"), (even, "full"), (odd, "half")):
            order = layer if self.up else reversed(layer)
            for i in order:
                self.apply_gate(i, self.gates[(key, i)], self.up)
            self.up = not self.up
