"""Spin-S Heisenberg chain, FP64: the model of the paper's performance runs (Sec. 6,
Tables 1 and 2: the isotropic spin-1 chain, d = 3).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU leg use it.

    H = sum_{j<L} [J (Sx_j Sx_{j+1} + Sy_j Sy_{j+1}) + Jz Sz_j Sz_{j+1}] - hz sum_j Sz_j

Basis |s>, s = 0..2S, magnetisation m = s - S: s counts quanta like a boson number, so the
U(1) labels of the Bose-Hubbard chain (sum of s to the left of a bond) apply unchanged and
the sector Sz_total = 0 holds N = L S quanta.  Operators O[s', s] = <s'|O|s>.

The exact diagonalisation here builds H from Sx and Sy (not from the ladder operators the
MPO uses) on the full product space, then restricts it to a magnetisation sector.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def spin_ops(two_s: int):
    """(S+, S-, Sz, Sx, Sy, I) for spin S = two_s / 2 in the basis s = m + S."""
    S = two_s / 2.0
    d = two_s + 1
    m = np.arange(d) - S
    sp_ = np.zeros((d, d), dtype=np.complex128)
    for s in range(d - 1):
        sp_[s + 1, s] = np.sqrt(S * (S + 1) - m[s] * (m[s] + 1))
    sm = sp_.conj().T.copy()
    sz = np.diag(m).astype(np.complex128)
    sx = 0.5 * (sp_ + sm)
    sy = -0.5j * (sp_ - sm)
    return sp_, sm, sz, sx, sy, np.eye(d, dtype=np.complex128)


def heisenberg_mpo(L: int, two_s: int, J: float, Jz: float, hz: float = 0.0):
    """MPO of H with bond dimension 5 (Sec. 4.3: MPOs built by hand), lower-triangular:

        row 0: I
        row 1: S-
        row 2: S+
        row 3: Sz
        row 4: -hz Sz   J/2 S+   J/2 S-   Jz Sz   I

    A string enters channel 4 at the left boundary and leaves through channel 0 at the
    right: 4 -> 1 -> 0 places J/2 S+_j S-_{j+1}, 4 -> 2 -> 0 places J/2 S-_j S+_{j+1},
    4 -> 3 -> 0 places Jz Sz_j Sz_{j+1} (J (Sx Sx + Sy Sy) = J/2 (S+ S- + S- S+)).
    Returns (W list [5, 5, d, d], left boundary, right boundary, wq) with wq the U(1)
    charges of the MPO bond index: channel 1 follows an S+ (the bra has one quantum more),
    channel 2 an S-.
    """
    sp_, sm, sz, _, _, ident = spin_ops(two_s)
    d = two_s + 1
    Ws = []
    for _ in range(L):
        W = np.zeros((5, 5, d, d), dtype=np.complex128)
        W[0, 0] = ident
        W[1, 0] = sm
        W[2, 0] = sp_
        W[3, 0] = sz
        W[4, 0] = -hz * sz
        W[4, 1] = 0.5 * J * sp_
        W[4, 2] = 0.5 * J * sm
        W[4, 3] = Jz * sz
        W[4, 4] = ident
        Ws.append(W)
    left = np.zeros(5, dtype=np.complex128)
    left[4] = 1.0
    right = np.zeros(5, dtype=np.complex128)
    right[0] = 1.0
    return Ws, left, right, np.array([0, 1, -1, 0, 0])


def bond_hamiltonian(two_s: int, J: float, Jz: float, hz: float, c1: float,
                     c2: float) -> np.ndarray:
    """Two-site term of bond (j, j+1) for the Trotter gates, d^2 x d^2, rows (s1', s2'),
    columns (s1, s2); the field is split between the bonds touching a site with weights
    c1, c2 (1 on an end site, 1/2 inside, as for the Bose-Hubbard on-site term)."""
    _, _, sz, sx, sy, ident = spin_ops(two_s)
    h = J * (np.kron(sx, sx) + np.kron(sy, sy)) + Jz * np.kron(sz, sz)
    return h - hz * (c1 * np.kron(sz, ident) + c2 * np.kron(ident, sz))


def full_hamiltonian(L: int, two_s: int, J: float, Jz: float, hz: float = 0.0) -> sp.csr_matrix:
    """Sparse H on the full d^L product space (site 1 most significant), from Sx, Sy, Sz
    Kronecker products."""
    _, _, sz, sx, sy, _ = spin_ops(two_s)
    d = two_s + 1

    def embed(ops_at):  # ops_at: {site: op}
        M = sp.identity(1, dtype=np.complex128, format="csr")
        for j in range(L):
            o = ops_at.get(j)
            M = sp.kron(M, sp.csr_matrix(o) if o is not None else sp.identity(d, format="csr"),
                        format="csr")
        return M

    H = sp.csr_matrix((d ** L, d ** L), dtype=np.complex128)
    for j in range(L - 1):
        H = H + J * (embed({j: sx, j + 1: sx}) + embed({j: sy, j + 1: sy}))
        H = H + Jz * embed({j: sz, j + 1: sz})
    for j in range(L):
        H = H - hz * embed({j: sz})
    return H.tocsr()


def sector_indices(L: int, two_s: int, N: int) -> np.ndarray:
    """Full-space indices of the product states with sum_j s_j = N."""
    d = two_s + 1
    idx = np.arange(d ** L)
    tot = np.zeros(d ** L, dtype=np.int64)
    rem = idx.copy()
    for _ in range(L):
        tot += rem % d
        rem //= d
    return np.nonzero(tot == N)[0]


def ground_state(L: int, two_s: int, J: float, Jz: float, hz: float, N: int):
    """Lowest eigenpair of H in the sector sum s = N: (E0, full-space vector)."""
    H = full_hamiltonian(L, two_s, J, Jz, hz)
    ix = sector_indices(L, two_s, N)
    Hs = H[ix][:, ix]
    if Hs.shape[0] <= 400:
        lam, V = np.linalg.eigh(Hs.toarray())
        e, v = lam[0], V[:, 0]
    else:
        lam, V = spla.eigsh(Hs, k=1, which="SA", tol=1e-14)
        e, v = lam[0], V[:, 0]
    full = np.zeros((two_s + 1) ** L, dtype=np.complex128)
    full[ix] = v
    return float(e), full
