"""Single-site DMRG with subspace expansion by direct sums, FP64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU leg use it.

The sweep of Sec. 4.3 (Listing 2: prepare the effective Hamiltonian around the current
site, eigensolve, write back, move on) on one site at a time.  A one-site update cannot
enlarge the bond it hands over, so the optimised centre tensor M is first enlarged by a
direct sum along the bond it leaves through (App. B node algebra, the direct sum that
expands the basis on one leg), and the neighbour it hands the weight to gets the matching
zero block (the direct sum that expands a leg with zeros inserted):

  left to right at site i (centre M = A_i, sites > i right-canonical):
    M            <- lowest eigenvector of L_i . W_i . R_{i+1}
    P[a',s',(w',b)] = alpha sum_{w,a,s} L_i[a',w,a] W_i[w,w',s',s] M[a,s,b]
    M~ = M (+)_right P          (chl x d x (chr + D chr))
    B~ = B_{i+1} (+)_left 0     ((chr + D chr) x d x chr')
    M~[(a s), :] = U S V^H (truncated, S rescaled to unit weight)
    A_i <- U,  A_{i+1} <- S V^H B~,  L_{i+1} <- grow L_i by A_i
  right to left at site i: the mirror image, P[(w,a),s',b'] = alpha sum W_i R_{i+1} M,
    M~ = M (+)_left P, A~_{i-1} = A_{i-1} (+)_right 0, A_i <- V^H, A_{i-1} <- A~ U S.

Since M~ B~ = M B (the zero block meets the expansion), the state before the truncation
is unchanged; the expansion only offers the SVD new directions.  U(1) labels of the new
indices follow from the charge rules: the index (w', b) of P carries q_b + wq[w'] and the
index (w, a) carries q_a + wq[w].  alpha shrinks from sweep to sweep (alpha_0 10^-s) and is
zero in the last sweeps, where the energy is the variational energy of the kept state.
One sweep: sites 0..L-2 left to right, then L-1..1 right to left.
"""
from __future__ import annotations

import numpy as np

from .contract import boundary_left, boundary_right, contract2, env_left, env_right
from .dmrg import build_right_envs, right_canonicalize
from .lanczos import lanczos_ground
from .svd import TruncParams, svd_truncate


def heff1_apply(L: np.ndarray, W: np.ndarray, R: np.ndarray, M: np.ndarray) -> np.ndarray:
    """y[a',s',b'] = sum L[a',w,a] W[w,w',s',s] R[b',w',b] M[a,s,b] (the one-site form of
    the contractor of Listing 1)."""
    T1 = contract2("pwa,asb->pwsb", L, M)        # [a', w, s, b]
    T2 = contract2("pwsb,wvts->ptvb", T1, W)     # [a', s', w', b]
    return contract2("ptvb,qvb->ptq", T2, R)     # [a', s', b']


def direct_sum_right(M: np.ndarray, P: np.ndarray) -> np.ndarray:
    """[M | P] along the last leg (the other legs identical)."""
    return np.concatenate([M, P], axis=2)


def direct_sum_left(M: np.ndarray, P: np.ndarray) -> np.ndarray:
    """[M ; P] along the first leg."""
    return np.concatenate([M, P], axis=0)


def expansion_right(L, W, M, alpha):
    """P[a', s', (w', b)] = alpha sum L[a',w,a] W[w,w',s',s] M[a,s,b]."""
    T = contract2("pwa,asb->pwsb", L, M)
    T = contract2("pwsb,wvts->ptvb", T, W)       # [a', s', w', b]
    a, d, D, b = T.shape
    return alpha * T.reshape(a, d, D * b)


def expansion_left(W, R, M, alpha):
    """P[(w, a), s', b'] = alpha sum W[w,w',s',s] R[b',w',b] M[a,s,b]."""
    T = contract2("asb,qvb->asqv", M, R)         # [a, s, b', w']
    T = contract2("asqv,wvts->watq", T, W)       # [w, a, s', b']
    D, a, d, q = T.shape
    return alpha * T.reshape(D * a, d, q)


def dmrg1(tensors, charges, Ws, left, right, wq, chi_max: int, n_sweeps: int,
          alpha0: float = 1e-3, zero_alpha_sweeps: int = 2, trunc: TruncParams | None = None,
          lanczos: dict | None = None):
    """n_sweeps single-site sweeps with subspace expansion; alpha = alpha0 10^-s in sweep s,
    zero in the last zero_alpha_sweeps.  wq: U(1) charges of the MPO bond index.
    Returns (A, q, history)."""
    trunc = trunc or TruncParams()
    trunc = TruncParams(chi_max=chi_max, abs_tol=trunc.abs_tol, rel_tol=trunc.rel_tol,
                        err_tol=trunc.err_tol, err_type=trunc.err_type)
    lz = {"tol": 1e-12, "krylov_cap": 32, "max_matvec": 300}
    lz.update(lanczos or {})
    wq = np.asarray(wq, dtype=np.int64)
    A = [t.astype(np.complex128).copy() for t in tensors]
    q = [c.copy() for c in charges]
    L = len(A)
    d = A[0].shape[1]
    D = Ws[0].shape[0]
    right_canonicalize(A, q)
    Renv = build_right_envs(A, Ws, right)
    Lenv = [None] * (L + 1)
    Lenv[0] = boundary_left(left)
    Renv[L] = boundary_right(right)
    history = []
    s_idx = np.arange(d)
    for sweep in range(n_sweeps):
        alpha = 0.0 if sweep >= n_sweeps - zero_alpha_sweeps else alpha0 * 10.0 ** (-sweep)
        ups = []
        for i in range(0, L - 1):  # left to right
            M = A[i]
            E, M, nmv, resid, conv = lanczos_ground(
                lambda x: heff1_apply(Lenv[i], Ws[i], Renv[i + 1], x), M, **lz)
            chl, _, chr_ = M.shape
            qr_new = q[i + 1]
            Mt, Bt = M, A[i + 1]
            if alpha > 0:
                P = expansion_right(Lenv[i], Ws[i], M, alpha)
                qP = (q[i + 1][None, :] + wq[:, None]).reshape(-1)   # (w', b)
                Mt = direct_sum_right(M, P)
                Bt = direct_sum_left(A[i + 1], np.zeros((len(qP),) + A[i + 1].shape[1:],
                                                        dtype=np.complex128))
                qr_new = np.concatenate([q[i + 1], qP])
            rows = (q[i][:, None] + s_idx[None, :]).reshape(-1)
            U, S, Vh, bq, info = svd_truncate(Mt.reshape(chl * d, -1), rows, qr_new, trunc)
            S = S / np.linalg.norm(S)
            k = len(S)
            A[i] = U.reshape(chl, d, k)
            A[i + 1] = contract2("km,msb->ksb", S[:, None] * Vh, Bt)
            q[i + 1] = bq
            Lenv[i + 1] = env_left(Lenv[i], Ws[i], A[i])
            ups.append({"E": E, "matvecs": nmv, "converged": conv, "chi": k, "err": info["err"]})
        for i in range(L - 1, 0, -1):  # right to left
            M = A[i]
            E, M, nmv, resid, conv = lanczos_ground(
                lambda x: heff1_apply(Lenv[i], Ws[i], Renv[i + 1], x), M, **lz)
            chl, _, chr_ = M.shape
            ql_new = q[i]
            Mt, At = M, A[i - 1]
            if alpha > 0:
                P = expansion_left(Ws[i], Renv[i + 1], M, alpha)
                qP = (q[i][None, :] + wq[:, None]).reshape(-1)       # (w, a)
                Mt = direct_sum_left(M, P)
                At = direct_sum_right(A[i - 1], np.zeros(A[i - 1].shape[:2] + (len(qP),),
                                                         dtype=np.complex128))
                ql_new = np.concatenate([q[i], qP])
            cols = (q[i + 1][None, :] - s_idx[:, None]).reshape(-1)
            U, S, Vh, bq, info = svd_truncate(Mt.reshape(Mt.shape[0], d * chr_), ql_new, cols,
                                              trunc)
            S = S / np.linalg.norm(S)
            k = len(S)
            A[i] = Vh.reshape(k, d, chr_)
            A[i - 1] = contract2("asm,mk->ask", At, U * S[None, :])
            q[i] = bq
            Renv[i] = env_right(Renv[i + 1], Ws[i], A[i])
            ups.append({"E": E, "matvecs": nmv, "converged": conv, "chi": k, "err": info["err"]})
        history.append({"E": ups[-1]["E"], "alpha": alpha, "updates": ups,
                        "max_chi": max(u["chi"] for u in ups)})
    return A, q, history
