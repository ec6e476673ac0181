"""Bose-Hubbard model pieces (Sec. 5, Eq. 2), FP64.

H = -J sum_{j<L} (b+_j b_{j+1} + h.c.) + U/2 sum_j n_j (n_j - 1) + V sum_j (j - j_c)^2 n_j
    - mu sum_j n_j

The chemical potential term is not in Eq. 2; it is added with mu = 0 by default, which
leaves Eq. 2 unchanged.  Sites are numbered j = 1..L as in Eq. 2.

Operator convention: an operator O is a d x d matrix O[s', s] = <s'|O|s> (s' out/bra,
s in/ket), basis |n>, n = 0..n_max.  The MPO tensor is W[w, w', s', s].
"""
from __future__ import annotations

import numpy as np


def local_ops(n_max: int):
    """Annihilator b, creator b+, number n and identity on the truncated Fock space."""
    d = n_max + 1
    b = np.zeros((d, d), dtype=np.complex128)
    for n in range(1, d):
        b[n - 1, n] = np.sqrt(n)  # b|n> = sqrt(n)|n-1>
    bd = b.conj().T.copy()
    num = np.diag(np.arange(d, dtype=np.float64)).astype(np.complex128)
    ident = np.eye(d, dtype=np.complex128)
    return b, bd, num, ident


def site_term(n_max: int, U: float, mu: float = 0.0, V: float = 0.0, j: int = 1,
              j_c: float = 0.0) -> np.ndarray:
    """On-site operator U/2 n(n-1) + V (j-j_c)^2 n - mu n of Eq. 2 (plus -mu n)."""
    _, _, num, ident = local_ops(n_max)
    return 0.5 * U * num @ (num - ident) + (V * (j - j_c) ** 2 - mu) * num


def bh_mpo(L: int, n_max: int, J: float, U: float, mu: float = 0.0, V: float = 0.0,
           j_c: float = 0.0):
    """Matrix product operator of Eq. 2 with MPO bond dimension D = 4.

    The paper builds its MPOs by hand (Sec. 4.3, figure of <psi|O|psi>); this is the
    standard lower-triangular hand construction, entries W[w, w'] (operators on one site):

        row 0: I       0       0       0
        row 1: b       0       0       0
        row 2: b+      0       0       0
        row 3: h_j   -J b+   -J b      I

    A string starts in channel 3 at the left boundary and ends in channel 0 at the right
    boundary: 3 -> 3 ... (I), then 3 -> 0 places h_j, and 3 -> 1 -> 0 places
    -J b+_j b_{j+1}, 3 -> 2 -> 0 places -J b_j b+_{j+1}.
    Returns (W list over sites 1..L, each [4, 4, d, d], left boundary vector, right
    boundary vector).
    """
    b, bd, _, ident = local_ops(n_max)
    d = n_max + 1
    Ws = []
    for j in range(1, L + 1):
        W = np.zeros((4, 4, d, d), dtype=np.complex128)
        W[0, 0] = ident
        W[1, 0] = b
        W[2, 0] = bd
        W[3, 0] = site_term(n_max, U, mu, V, j, j_c)
        W[3, 1] = -J * bd
        W[3, 2] = -J * b
        W[3, 3] = ident
        Ws.append(W)
    left = np.zeros(4, dtype=np.complex128)
    left[3] = 1.0
    right = np.zeros(4, dtype=np.complex128)
    right[0] = 1.0
    return Ws, left, right


def mpo_to_matrix(Ws, left, right) -> np.ndarray:
    """Dense d^L x d^L matrix of an MPO (tiny L only); site 1 is the most significant digit."""
    d = Ws[0].shape[2]
    # M[w] is the operator accumulated so far with open right MPO index w
    M = np.einsum("w,wvts->vts", left, Ws[0])  # [w', s', s]
    for W in Ws[1:]:
        # combine: new[w'', (s'_old s'), (s_old s)] = sum_w M[w, s'_old, s_old] W[w, w'', s', s]
        M = np.einsum("wab,wvts->vatbs", M, W)
        D, a, t, bb, s = M.shape
        M = M.reshape(D, a * t, bb * s)
    return np.einsum("vab,v->ab", M, right)


def bond_hamiltonian(n_max: int, J: float, U: float, c1: float, c2: float,
                     mu: float = 0.0) -> np.ndarray:
    """Two-site term h_{j,j+1} used by the Trotter gates, as a d^2 x d^2 matrix.

    h = -J (b+ (x) b + b (x) b+) + c1 [U/2 n(n-1) - mu n] (x) I + c2 I (x) [U/2 n(n-1) - mu n]
    The on-site part of Eq. 2 is shared between the two bonds touching a site: c = 1/2 in
    the interior and c = 1 for the end sites 1 and L (each touches one bond).
    Index order: row (s1', s2'), column (s1, s2), s1 the left site, most significant.
    """
    b, bd, _, ident = local_ops(n_max)
    hs = site_term(n_max, U, mu)
    h = -J * (np.kron(bd, b) + np.kron(b, bd))
    h = h + c1 * np.kron(hs, ident) + c2 * np.kron(ident, hs)
    return h


def bond_weights(L: int, j: int):
    """(c1, c2) of bond (j, j+1), j = 1..L-1."""
    c1 = 1.0 if j == 1 else 0.5
    c2 = 1.0 if j + 1 == L else 0.5
    return c1, c2


def gate(h: np.ndarray, tau: float) -> np.ndarray:
    """G = exp(-i tau h) of a Hermitian h through its eigendecomposition (App. A.1.2:
    a functional node exponentiating a sum of operators)."""
    lam, Q = np.linalg.eigh(h)
    return (Q * np.exp(-1j * tau * lam)[None, :]) @ Q.conj().T
