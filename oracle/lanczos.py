"""Lanczos ground-state solver with full re-orthogonalisation, FP64.

The library hands H_eff.theta to an external iterative sparse eigensolver as a callback
and uses the current tensor as the starting vector (Sec. 4.3, Listing 2 with the
contractor of Listing 1); the eigensolver stops after at most 300 iterations by default
(App. A.3, Listing 5).  This is a plain Lanczos iteration standing in for that solver:

  v_0 = x / |x|
  for k = 0, 1, ...:
      w      = H v_k
      alpha_k = <v_k|w>
      w     -= alpha_k v_k + beta_{k-1} v_{k-1}
      w     -= V (V^H w)              (classical Gram-Schmidt, done twice)
      beta_k = |w|
      (theta_k, y) = lowest eigenpair of the (k+1)x(k+1) tridiagonal T_k
      stop if |theta_k - theta_{k-1}| <= tol |theta_k| and beta_k |y_k| <= max(tol, c u)|theta_k|
      v_{k+1} = w / beta_k
  restart from the Ritz vector sum_i y_i v_i when k reaches the Krylov cap.

The eigenpair of T_k uses numpy.linalg.eigh (a library primitive).
"""
from __future__ import annotations

import numpy as np


def tridiag_lowest(alphas, betas):
    """Lowest eigenpair of the symmetric tridiagonal matrix with diagonal `alphas` and
    off-diagonal `betas` (len(betas) = len(alphas) - 1)."""
    k = len(alphas)
    T = np.zeros((k, k))
    T[np.arange(k), np.arange(k)] = alphas
    if k > 1:
        T[np.arange(k - 1), np.arange(1, k)] = betas
        T[np.arange(1, k), np.arange(k - 1)] = betas
    w, v = np.linalg.eigh(T)
    return w[0], v[:, 0]


def lanczos_ground(matvec, x0: np.ndarray, tol: float = 1e-12, krylov_cap: int = 32,
                   max_matvec: int = 300, unit_roundoff: float = 2.0 ** -52,
                   c: float = 10.0):
    """Lowest eigenpair of the Hermitian operator `matvec` from the start vector x0.

    Returns (E, x, n_matvec, resid, converged) with x the unit-norm Ritz vector and
    resid = beta_k |y_k| the Lanczos residual estimate |H x - E x|.
    """
    shape = x0.shape
    v = x0.reshape(-1).astype(np.complex128)
    v = v / np.linalg.norm(v)
    total = 0
    E_prev = None
    rtol = max(tol, c * unit_roundoff)
    while True:
        V = [v]
        alphas, betas = [], []
        E = None
        y = None
        resid = np.inf
        stop = False
        converged = False
        for k in range(krylov_cap):
            w = matvec(V[k].reshape(shape)).reshape(-1)
            total += 1
            alpha = np.vdot(V[k], w).real
            w = w - alpha * V[k]
            if k > 0:
                w = w - betas[k - 1] * V[k - 1]
            for _ in range(2):
                coef = np.array([np.vdot(Vi, w) for Vi in V])
                for ci, Vi in zip(coef, V):
                    w = w - ci * Vi
            beta = np.linalg.norm(w)
            alphas.append(alpha)
            E, y = tridiag_lowest(alphas, betas)
            resid = beta * abs(y[-1])
            if E_prev is not None and abs(E - E_prev) <= tol * abs(E) \
                    and resid <= rtol * abs(E):
                converged = True
            if beta <= rtol * abs(E) * 1e-3:
                converged = True  # invariant subspace: T_k is exact
            E_prev = E
            if converged or total >= max_matvec:
                stop = True
                break
            betas.append(beta)
            V.append(w / beta)
        x = np.zeros_like(v)
        for yi, Vi in zip(y, V):
            x = x + yi * Vi
        x = x / np.linalg.norm(x)
        if stop:
            return E, x.reshape(shape), total, resid, converged
        v = x
