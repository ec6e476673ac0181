"""Exact diagonalisation of Eq. 2 (Sec. 5) in a fixed boson-number sector, FP64.

Built directly from the Fock basis (occupation strings), independent of the MPO: this is
the pin the MPO, the MPS contractions, DMRG and TEBD are checked against.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def fock_basis(L: int, N: int, n_max: int):
    """All occupation tuples (n_1..n_L), 0 <= n_j <= n_max, sum = N, in lexicographic
    order (site 1 most significant), with a lookup dict."""
    basis = [c for c in itertools.product(range(n_max + 1), repeat=L) if sum(c) == N]
    index = {c: i for i, c in enumerate(basis)}
    return basis, index


def hamiltonian(L: int, N: int, n_max: int, J: float, U: float, mu: float = 0.0,
                V: float = 0.0, j_c: float = 0.0) -> sp.csr_matrix:
    """Sparse H of Eq. 2 (plus -mu N) on the sector with N bosons."""
    basis, index = fock_basis(L, N, n_max)
    rows, cols, vals = [], [], []
    for i, c in enumerate(basis):
        diag = 0.0
        for j in range(L):  # j = 0..L-1 is site j+1
            n = c[j]
            diag += 0.5 * U * n * (n - 1) + (V * ((j + 1) - j_c) ** 2 - mu) * n
        rows.append(i)
        cols.append(i)
        vals.append(diag)
        for j in range(L - 1):
            # b+_j b_{j+1}: move a boson from site j+1 to site j
            if c[j + 1] > 0 and c[j] < n_max:
                t = list(c)
                amp = np.sqrt((t[j] + 1) * t[j + 1])
                t[j] += 1
                t[j + 1] -= 1
                k = index[tuple(t)]
                rows.append(k)
                cols.append(i)
                vals.append(-J * amp)
                # its Hermitian conjugate b_j b+_{j+1}
                rows.append(i)
                cols.append(k)
                vals.append(-J * amp)
    n = len(basis)
    return sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(n, n))


def lowest(H: sp.csr_matrix, k: int = 1):
    """The k lowest eigenpairs (dense eigh below 2000 states, else Lanczos by ARPACK)."""
    n = H.shape[0]
    if n <= 2000:
        w, v = np.linalg.eigh(H.toarray())
        return w[:k], v[:, :k]
    w, v = spla.eigsh(H, k=k, which="SA", tol=1e-14, maxiter=100000)
    o = np.argsort(w)
    return w[o], v[:, o]


def embed(vec: np.ndarray, L: int, N: int, n_max: int) -> np.ndarray:
    """Sector vector -> full d^L vector (site 1 most significant digit)."""
    d = n_max + 1
    basis, _ = fock_basis(L, N, n_max)
    full = np.zeros(d ** L, dtype=np.complex128)
    for amp, c in zip(vec, basis):
        idx = 0
        for n in c:
            idx = idx * d + n
        full[idx] = amp
    return full


def number_operator_full(L: int, n_max: int, j: int) -> np.ndarray:
    """Diagonal of n_j (j = 1..L) on the full d^L space."""
    d = n_max + 1
    idx = np.arange(d ** L)
    return ((idx // d ** (L - j)) % d).astype(np.float64)
