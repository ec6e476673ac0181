"""Tensor contractions of the two-site update, FP64 (Sec. 3, Sec. 4.2, App. B.1.1).

A contraction sums over a shared index (Sec. 3: C_pbk = sum_c A_cb B_pck); the library
does it by reordering indices and one matrix product (App. B.1.1).  Here each step is
one numpy.einsum over named indices, in the order the docstrings state.

Leg conventions
  A[a, s, b]          MPS site tensor (left bond, physical, right bond)
  theta[a, s1, s2, b] two-site tensor
  W[w, w', s', s]     MPO tensor, s' out (bra), s in (ket)
  L[a', w, a]         left environment (a' bra side, a ket side)
  R[b', w, b]         right environment
"""
from __future__ import annotations

import numpy as np


def contract2(spec: str, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """One pairwise contraction, evaluated as a matrix product (BLAS) by numpy.einsum."""
    return np.einsum(spec, a, b, optimize=True)


def theta_form(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """theta[a,s1,s2,b] = sum_m A[a,s1,m] B[m,s2,b]: the two-site object, contracted over
    the shared bond (Sec. 3 contraction; App. B.1.1)."""
    return contract2("asm,mtb->astb", A, B)


def gate_apply(G: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """theta'[a,s1',s2',b] = sum_{s1,s2} G[(s1' s2'), (s1 s2)] theta[a,s1,s2,b] (TEBD gate;
    Sec. 3 Trotterised update, Sec. 5 time evolution example)."""
    d = theta.shape[1]
    G4 = G.reshape(d, d, d, d)  # [s1', s2', s1, s2]
    return contract2("xyst,astb->axyb", G4, theta)


def heff_apply(L: np.ndarray, W1: np.ndarray, W2: np.ndarray, R: np.ndarray,
               theta: np.ndarray) -> np.ndarray:
    """y = L . W1 . W2 . R . theta, the two-site effective Hamiltonian applied to theta.

    y[a',s1',s2',b'] = sum L[a',w,a] W1[w,w1,s1',s1] W2[w1,w2,s2',s2] R[b',w2,b] theta[a,s1,s2,b]

    This is the two-site analogue of the HeffA_contract contractor of Listing 1, contracted
    in the order that costs least (App. B.1.1 picks the cheapest order for 3-4 nodes):
      T1 = L . theta   (sum over a)
      T2 = T1 . W1     (sum over w, s1)
      T3 = T2 . W2     (sum over w1, s2)
      y  = T3 . R      (sum over w2, b)
    """
    T1 = contract2("pwa,astb->pwstb", L, theta)          # [a', w, s1, s2, b]
    T2 = contract2("pwstb,wvxs->pxvtb", T1, W1)          # [a', s1', w1, s2, b]
    T3 = contract2("pxvtb,vuyt->pxyub", T2, W2)          # [a', s1', s2', w2, b]
    return contract2("pxyub,qub->pxyq", T3, R)           # [a', s1', s2', b']


def heff_dense(L, W1, W2, R) -> np.ndarray:
    """Explicit H_eff matrix (rows y index, columns theta index) for tiny shapes."""
    H = np.einsum("pwa,wvxs,vuyt,qub->pxyqastb", L, W1, W2, R)
    n = L.shape[0] * W1.shape[2] * W2.shape[2] * R.shape[0]
    return H.reshape(n, -1)


def env_left(Lenv: np.ndarray, W: np.ndarray, A: np.ndarray) -> np.ndarray:
    """L_next[m',w',m] = sum conj(A[a',s',m']) L[a',w,a] W[w,w',s',s] A[a,s,m].

    Grows <psi|H|psi> by one site from the left: the environment H_prepare builds for the
    next site (Listing 2; Sec. 4.3 network of <psi|O|psi>).
    """
    X = contract2("pwa,asm->pwsm", Lenv, A)              # ket side
    Y = contract2("pwsm,wvts->ptvm", X, W)               # MPO
    return contract2("ptn,ptvm->nvm", A.conj(), Y)       # bra side


def env_right(Renv: np.ndarray, W: np.ndarray, B: np.ndarray) -> np.ndarray:
    """R_next[a',w,a] = sum conj(B[a',s',b']) R[b',w',b] W[w,w',s',s] B[a,s,b] (mirror of
    env_left)."""
    X = contract2("asb,qvb->asqv", B, Renv)              # ket side
    Y = contract2("asqv,wvts->awtq", X, W)               # MPO
    return contract2("ptq,awtq->pwa", B.conj(), Y)       # bra side


def boundary_left(vec: np.ndarray) -> np.ndarray:
    """L_0[0, w, 0] = left boundary vector of the MPO."""
    return vec.reshape(1, -1, 1).astype(np.complex128)


def boundary_right(vec: np.ndarray) -> np.ndarray:
    return vec.reshape(1, -1, 1).astype(np.complex128)


def mps_to_state(tensors) -> np.ndarray:
    """Full d^L amplitude vector of an open-boundary MPS (site 1 most significant):
    psi_j = tTr[ (x)_nu T^(nu) ] of Sec. 3, Eq. 1 for a chain."""
    psi = tensors[0]  # [1, s, b]
    for A in tensors[1:]:
        psi = contract2("xsm,mtb->xstb", psi, A)
        psi = psi.reshape(psi.shape[0], -1, psi.shape[-1])
    return psi.reshape(-1)


def mps_overlap(bra, ket) -> complex:
    """<bra|ket> by a transfer-matrix sweep."""
    E = np.ones((1, 1), dtype=np.complex128)
    for A, B in zip(bra, ket):
        E = np.einsum("pa,psq,asb->qb", E, A.conj(), B)
    return complex(E[0, 0])


def mps_expect_mpo(tensors, Ws, left, right) -> complex:
    """<psi|O|psi> for an MPO O, by growing the left environment over the chain."""
    E = boundary_left(left)
    for A, W in zip(tensors, Ws):
        E = env_left(E, W, A)
    return complex(np.einsum("pwa,w->", E, right))


def density(tensors, n_max: int) -> np.ndarray:
    """<n_j> for every site of a (not necessarily normalised) MPS, divided by <psi|psi>."""
    d = n_max + 1
    num = np.diag(np.arange(d, dtype=np.float64)).astype(np.complex128)
    L = len(tensors)
    norm = mps_overlap(tensors, tensors).real
    out = np.zeros(L)
    for j in range(L):
        E = np.ones((1, 1), dtype=np.complex128)
        for k, A in enumerate(tensors):
            if k == j:
                E = np.einsum("pa,psq,st,atb->qb", E, A.conj(), num, A)
            else:
                E = np.einsum("pa,psq,asb->qb", E, A.conj(), A)
        out[j] = E[0, 0].real / norm
    return out


def bdagb(tensors, n_max: int) -> np.ndarray:
    """Single-particle density matrix rho_ij = <b+_i b_j> / <psi|psi> (Sec. 5 examples):
    b+ placed at site i and b at site j in one transfer-matrix sweep (b+ b at i = j)."""
    d = n_max + 1
    b = np.diag(np.sqrt(np.arange(1, d, dtype=np.float64)), k=1).astype(np.complex128)
    bd = b.conj().T
    L = len(tensors)
    norm = mps_overlap(tensors, tensors).real
    rho = np.zeros((L, L), dtype=np.complex128)
    for i in range(L):
        for j in range(L):
            E = np.ones((1, 1), dtype=np.complex128)
            for k, A in enumerate(tensors):
                op = None
                if k == i and k == j:
                    op = bd @ b
                elif k == i:
                    op = bd
                elif k == j:
                    op = b
                if op is None:
                    E = np.einsum("pa,psq,asb->qb", E, A.conj(), A)
                else:
                    E = np.einsum("pa,psq,st,atb->qb", E, A.conj(), op, A)
            rho[i, j] = E[0, 0] / norm
    return rho
