"""Two-site DMRG ground-state sweeps, FP64 (Sec. 3, Sec. 4.3 Listing 2, Sec. 5).

The library's sweep (Listing 2) walks the chain, prepares the effective Hamiltonian
network around the current site, hands it to the eigensolver with the current tensor as
the starting vector and writes the result back before moving on.  This is the two-site
form of that loop, on bonds (i, i+1), with the truncated SVD of App. B.1.2 splitting the
optimised two-site tensor back into two sites:

  initial state: right-canonical form (exact SVD moves from the right end), unit norm
  one sweep:     bonds 0..L-2 left to right, then L-2..0 right to left (2(L-1) updates)
  left to right: theta = A_i A_{i+1};  Lanczos;  theta = U S V^H (truncated);
                 A_i <- U, A_{i+1} <- S V^H with S rescaled to sum S^2 = 1;
                 L_{i+1} <- grow L_i by site i
  right to left: ... A_{i+1} <- V^H, A_i <- U S (rescaled); R_{i+1} <- grow R_{i+2}

Sites are 0-based here.  Lenv[i] holds sites 0..i-1, Renv[i] sites i..L-1.  U(1) labels
ride along as integer arrays so each SVD is block-wise (dense storage, charge mask).
"""
from __future__ import annotations

import numpy as np

from .contract import (boundary_left, boundary_right, env_left, env_right, heff_apply,
                       theta_form)
from .lanczos import lanczos_ground
from .svd import TruncParams, svd_truncate

EXACT = TruncParams(chi_max=1 << 30, abs_tol=-1.0, rel_tol=1e-16, err_tol=0.0)


def theta_charges(ql: np.ndarray, qr: np.ndarray, d: int):
    """Row labels q_a + s1 of (a, s1) and column labels q_b - s2 of (s2, b)."""
    s = np.arange(d)
    rows = (ql[:, None] + s[None, :]).reshape(-1)
    cols = (qr[None, :] - s[:, None]).reshape(-1)
    return rows, cols


def site_charges(ql: np.ndarray, qr: np.ndarray, d: int):
    """Labels for splitting one site tensor A[a, s, b] as M[a, (s b)] (right move) or
    M[(a s), b] (left move)."""
    s = np.arange(d)
    right_cols = (qr[None, :] - s[:, None]).reshape(-1)  # (s, b) -> q_b - s
    left_rows = (ql[:, None] + s[None, :]).reshape(-1)   # (a, s) -> q_a + s
    return left_rows, right_cols


def right_canonicalize(A, q):
    """Exact right-to-left SVD moves: A_j <- V^H for j = L-1..1, push U S into A_{j-1};
    finally divide A_0 by the state norm."""
    L = len(A)
    d = A[0].shape[1]
    for j in range(L - 1, 0, -1):
        chl, _, chr_ = A[j].shape
        _, cols = site_charges(q[j], q[j + 1], d)
        M = A[j].reshape(chl, d * chr_)
        U, S, Vh, bq, _ = svd_truncate(M, q[j], cols, EXACT)
        A[j] = Vh.reshape(-1, d, chr_)
        A[j - 1] = np.einsum("asm,mk->ask", A[j - 1], U * S[None, :])
        q[j] = bq
    A[0] = A[0] / np.linalg.norm(A[0])
    return A, q


def build_right_envs(A, Ws, right):
    L = len(A)
    Renv = [None] * (L + 1)
    Renv[L] = boundary_right(right)
    for j in range(L - 1, 0, -1):
        Renv[j] = env_right(Renv[j + 1], Ws[j], A[j])
    return Renv


def two_site_update(A, q, Ws, Lenv, Renv, i, direction, trunc: TruncParams, lz: dict):
    """One bond update (a1, a3-a8 of the two-site step).  Returns stats."""
    d = A[i].shape[1]
    theta = theta_form(A[i], A[i + 1])
    W1, W2, Le, Re = Ws[i], Ws[i + 1], Lenv[i], Renv[i + 2]
    E, theta, nmv, resid, conv = lanczos_ground(
        lambda x: heff_apply(Le, W1, W2, Re, x), theta, **lz)
    chl, _, _, chr_ = theta.shape
    rows, cols = theta_charges(q[i], q[i + 2], d)
    M = theta.reshape(chl * d, d * chr_)
    U, S, Vh, bq, info = svd_truncate(M, rows, cols, trunc)
    S = S / np.linalg.norm(S)
    k = len(S)
    if direction > 0:
        A[i] = U.reshape(chl, d, k)
        A[i + 1] = (S[:, None] * Vh).reshape(k, d, chr_)
    else:
        A[i] = (U * S[None, :]).reshape(chl, d, k)
        A[i + 1] = Vh.reshape(k, d, chr_)
    q[i + 1] = bq
    return {"E": E, "matvecs": nmv, "resid": resid, "converged": conv, "chi": k,
            "err": info["err"], "disc": info["disc"], "S": S}


def dmrg(tensors, charges, Ws, left, right, chi_max: int, n_sweeps: int,
         trunc: TruncParams | None = None, lanczos: dict | None = None):
    """Run n_sweeps two-site sweeps.  Returns (A, q, history) with one dict per sweep
    (energy after the sweep, largest truncation error, per-update stats)."""
    trunc = trunc or TruncParams()
    trunc = TruncParams(chi_max=chi_max, abs_tol=trunc.abs_tol, rel_tol=trunc.rel_tol,
                        err_tol=trunc.err_tol, err_type=trunc.err_type)
    lz = {"tol": 1e-12, "krylov_cap": 32, "max_matvec": 300}
    lz.update(lanczos or {})
    A = [t.astype(np.complex128).copy() for t in tensors]
    q = [c.copy() for c in charges]
    L = len(A)
    right_canonicalize(A, q)
    Renv = build_right_envs(A, Ws, right)
    Lenv = [None] * (L + 1)
    Lenv[0] = boundary_left(left)
    history = []
    for _ in range(n_sweeps):
        ups = []
        for i in range(0, L - 1):
            st = two_site_update(A, q, Ws, Lenv, Renv, i, +1, trunc, lz)
            Lenv[i + 1] = env_left(Lenv[i], Ws[i], A[i])
            ups.append(st)
        for i in range(L - 2, -1, -1):
            st = two_site_update(A, q, Ws, Lenv, Renv, i, -1, trunc, lz)
            Renv[i + 1] = env_right(Renv[i + 2], Ws[i + 1], A[i + 1])
            ups.append(st)
        history.append({"E": ups[-1]["E"], "max_err": max(u["err"] for u in ups),
                        "updates": ups})
    return A, q, history
