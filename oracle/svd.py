"""Truncated singular value decomposition of the two-site tensor, FP64 (App. B.1.2).

The tensor theta[a,s1,s2,b] is read as the matrix M[(a s1), (s2 b)] (row legs a, s1 go
to U, column legs s2, b to V^dagger).  With U(1) boson-number labels the matrix is block
diagonal: row (a, s1) carries q_a + s1, column (s2, b) carries q_b - s2, and only
equal-charge rows and columns couple (App. A.1.1: an element is kept only when the
charges flowing in and out balance).  Each block is decomposed with numpy.linalg.svd;
with all labels equal this is one dense SVD.

Truncation (App. B.1.2): four rules, the one giving the smallest bond dimension wins:
  1. keep at most chi_max values;
  2. discard lambda_i < a           (absolute tolerance; a <= 0 switches it off);
  3. discard lambda_i / lambda_0 < r (relative tolerance);
  4. discard the largest number of values whose truncation error stays below eps_tol,
     the error being (Eq. 3) sqrt(sum_{i>chi} lambda_i^2) ("2norm"), or the sum of
     squares ("sumsq"), or the 1-norm ("1norm") of the discarded values.
Rule 4 measures the discarded values after normalising them so that sum lambda^2 = 1.
At least one value is always kept.  Global order of the values: lambda descending, then
block charge ascending, then position inside the block.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TRUNC_2NORM, TRUNC_SUMSQ, TRUNC_1NORM = 0, 1, 2


@dataclass
class TruncParams:
    chi_max: int = 1 << 30
    abs_tol: float = -1.0        # App. A.3 defaults: absolute tolerance -1 (off)
    rel_tol: float = 1e-16       # relative tolerance 1e-16
    err_tol: float = 1e-8        # truncation error tolerance 1e-8
    err_type: int = TRUNC_2NORM  # truncation type 2norm


def trunc_error(discarded: np.ndarray, err_type: int) -> float:
    """Eq. 3 and its two alternatives, on already-normalised discarded values."""
    if err_type == TRUNC_2NORM:
        return float(np.sqrt(np.sum(discarded ** 2)))
    if err_type == TRUNC_SUMSQ:
        return float(np.sum(discarded ** 2))
    if err_type == TRUNC_1NORM:
        return float(np.sum(np.abs(discarded)))
    raise ValueError(err_type)


def choose_chi(sig_desc: np.ndarray, p: TruncParams) -> int:
    """Number of values kept from a descending list under the four rules."""
    n = len(sig_desc)
    if n == 0:
        return 0
    chi1 = min(n, p.chi_max)
    chi2 = int(np.sum(sig_desc >= p.abs_tol)) if p.abs_tol > 0 else n
    s0 = sig_desc[0]
    chi3 = int(np.sum(sig_desc / s0 >= p.rel_tol)) if s0 > 0 else n
    norm = np.sqrt(np.sum(sig_desc ** 2))
    shat = sig_desc / norm if norm > 0 else sig_desc
    chi4 = n
    for keep in range(n - 1, -1, -1):  # try discarding one more value each time
        if trunc_error(shat[keep:], p.err_type) < p.err_tol:
            chi4 = keep
        else:
            break
    return max(1, min(chi1, chi2, chi3, chi4))


def svd_truncate(M: np.ndarray, row_q: np.ndarray, col_q: np.ndarray, p: TruncParams):
    """Block-wise truncated SVD of M with charge labels on rows and columns.

    Returns (U, S, Vh, bond_q, info): U[m, k], S[k] (descending within equal charge),
    Vh[k, n], the charge of each kept index (ascending), and a dict with the truncation
    error `err` (type p.err_type, normalised values), the discarded weight `disc`
    (sum of raw discarded lambda^2) and the full descending spectrum `spectrum`.
    """
    m, n = M.shape
    charges = sorted(set(row_q.tolist()) & set(col_q.tolist()))
    entries = []   # (sigma, charge, index-in-block)
    blocks = {}
    for q in charges:
        r = np.nonzero(row_q == q)[0]
        c = np.nonzero(col_q == q)[0]
        u, s, vh = np.linalg.svd(M[np.ix_(r, c)], full_matrices=False)
        blocks[q] = (r, c, u, s, vh)
        for i, sv in enumerate(s):
            entries.append((sv, q, i))
    entries.sort(key=lambda e: (-e[0], e[1], e[2]))
    sig = np.array([e[0] for e in entries])
    chi = choose_chi(sig, p)
    kept = entries[:chi]
    disc = sig[chi:]
    norm = np.sqrt(np.sum(sig ** 2))
    err = trunc_error(disc / norm if norm > 0 else disc, p.err_type)
    # kept bond indices ordered by charge, then by value descending
    kept.sort(key=lambda e: (e[1], -e[0], e[2]))
    U = np.zeros((m, chi), dtype=np.complex128)
    Vh = np.zeros((chi, n), dtype=np.complex128)
    S = np.zeros(chi)
    bond_q = np.zeros(chi, dtype=np.int64)
    for k, (sv, q, i) in enumerate(kept):
        r, c, u, s, vh = blocks[q]
        U[r, k] = u[:, i]
        Vh[k, c] = vh[i, :]
        S[k] = sv
        bond_q[k] = q
    info = {"err": err, "disc": float(np.sum(disc ** 2)), "spectrum": sig, "chi": chi}
    return U, S, Vh, bond_q, info


def autoblock(M: np.ndarray, tol: float):
    """Automatic blocking (Sec. 6, figure of the blocked array): entries with |M_ij| <= tol
    are set to zero, and rows and columns are grouped into the connected components of the
    remaining non-zero pattern (row i and column j are joined by a non-zero M_ij).  Returns
    (the zeroed matrix, row labels, column labels); a component is numbered by the order of
    its first row, components holding columns only come after, in column order."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    m, n = M.shape
    Mz = np.where(np.abs(M) > tol, M, 0.0)
    rows, cols = np.nonzero(Mz)
    adj = sp.coo_matrix((np.ones(len(rows)), (rows, m + cols)), shape=(m + n, m + n))
    _, comp = connected_components(adj, directed=False)
    order = {}
    for v in range(m + n):
        order.setdefault(comp[v], len(order))
    lab = np.array([order[comp[v]] for v in range(m + n)], dtype=np.int64)
    return Mz, lab[:m], lab[m:]


def svd_truncate_auto(M: np.ndarray, tol: float, p: TruncParams):
    """Truncated SVD of M over its automatic blocks (autoblock, then svd_truncate)."""
    Mz, rq, cq = autoblock(M, tol)
    return svd_truncate(Mz, rq, cq, p)
