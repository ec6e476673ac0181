"""Seeded synthetic inputs for the two-site update.

This module is shared by both sides of every parity test: the CUDA path (through the
binding) and the FP64 CPU oracle receive the very same arrays from here.  It holds random
draws and integer structure only (shapes, U(1) charge labels and the sizes of charge
sectors); none of the method's arithmetic (no contraction, decomposition, Hamiltonian or
gauge fixing) lives here.

Conventions (shared with the C-ABI):
  * complex tensors are numpy complex128, C order;
  * an MPS site tensor is A[a, s, b] (left bond, physical, right bond);
  * an environment is E[a', w, a] (bra bond, MPO bond, ket bond);
  * theta is theta[a, s1, s2, b].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "complex_gaussian",
    "hermitian_env",
    "sector_counts",
    "bond_charges",
    "random_charged_mps",
    "mott_occupations",
    "charge_mask",
    "gaussian_sector_labels",
    "env_mask",
    "theta_mask",
    "BH_WQ",
]

# charges of the Bose-Hubbard MPO bond index w = 0..3 (left boundary 3, right boundary 0):
# an environment channel w relates bra and ket bond labels by q' = q + BH_WQ[w]
BH_WQ = (0, 1, -1, 0)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def complex_gaussian(g: np.random.Generator, shape) -> np.ndarray:
    """i.i.d. complex Gaussian entries, re and im ~ N(0, 1/2) (so E|z|^2 = 1)."""
    s = np.sqrt(0.5)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) * s


def hermitian_env(g: np.random.Generator, chi: int, D: int = 4, pair=(1, 2)) -> np.ndarray:
    """Random environment E[a', w, a] whose MPO channels respect the Hermitian pairing.

    Channels w outside `pair` are Hermitian matrices (a' x a); the two channels in `pair`
    are conjugate transposes of each other.  With the Bose-Hubbard MPO (whose operator
    entries obey W[w,w']^H = W[pi w, pi w'] for pi swapping the b and b^dagger channels)
    this makes the two-site effective Hamiltonian Hermitian, as it is for environments
    built from a real state, while every free entry is still an i.i.d. complex Gaussian.
    """
    G = complex_gaussian(g, (D, chi, chi))
    E = np.empty((chi, D, chi), dtype=np.complex128)
    p, q = pair
    for w in range(D):
        if w in (p, q):
            continue
        H = (G[w] + G[w].conj().T) * np.sqrt(0.5)
        E[:, w, :] = H
    E[:, p, :] = G[p]
    E[:, q, :] = G[p].conj().T
    return np.ascontiguousarray(E)


def sector_counts(k: int, n_max: int) -> np.ndarray:
    """cnt[q] = number of occupation strings of k sites (0..n_max each) summing to q."""
    cnt = np.zeros(k * n_max + 1, dtype=np.int64)
    cnt[0] = 1
    for _ in range(k):
        new = np.zeros_like(cnt)
        for n in range(n_max + 1):
            new[n:] += cnt[: len(cnt) - n]
        cnt = new
    return cnt


def bond_charges(L: int, d: int, N: int, chi_max: int) -> list[np.ndarray]:
    """Charge label (bosons to the left of the bond) of every index of bonds 0..L.

    Bond k separates sites 1..k from k+1..L.  Every charge q reachable from both sides is
    a sector; sector sizes are capped by the exact Schmidt bound min(#left, #right) and
    filled one index at a time, round robin over sectors in ascending q, until the bond
    holds min(chi_max, exact bound) indices.  Labels are returned sorted ascending.
    """
    n_max = d - 1
    out = []
    for k in range(L + 1):
        left = sector_counts(k, n_max)
        right = sector_counts(L - k, n_max)
        qs, caps = [], []
        for q in range(0, N + 1):
            if q < len(left) and 0 <= N - q < len(right):
                c = min(int(left[q]), int(right[N - q]))
                if c > 0:
                    qs.append(q)
                    caps.append(c)
        total = min(chi_max, sum(caps))
        sizes = [0] * len(qs)
        filled = 0
        while filled < total:
            for i in range(len(qs)):
                if filled < total and sizes[i] < caps[i]:
                    sizes[i] += 1
                    filled += 1
        lab = np.concatenate([np.full(s, q, dtype=np.int64) for q, s in zip(qs, sizes)])
        out.append(lab)
    return out


def charge_mask(ql: np.ndarray, d: int, qr: np.ndarray) -> np.ndarray:
    """Boolean mask of allowed A[a, s, b]: qr[b] == ql[a] + s (boson number conserved)."""
    s = np.arange(d)
    return (ql[:, None, None] + s[None, :, None]) == qr[None, None, :]


def random_charged_mps(g: np.random.Generator, L: int, d: int, N: int, chi_max: int):
    """Random-normal MPS in the fixed-N sector: Gaussian entries inside allowed blocks.

    Returns (tensors, charges): tensors[j] is A_j[a, s, b] (complex128) for sites
    j = 0..L-1 and charges[k] the labels of bond k = 0..L.  No normalisation or gauge is
    applied: both sides bring the state to canonical form themselves.
    """
    charges = bond_charges(L, d, N, chi_max)
    tensors = []
    for j in range(L):
        ql, qr = charges[j], charges[j + 1]
        A = complex_gaussian(g, (len(ql), d, len(qr)))
        A = np.where(charge_mask(ql, d, qr), A, 0.0)
        tensors.append(np.ascontiguousarray(A.astype(np.complex128)))
    return tensors, charges


def mott_occupations(L: int, filling: int = 1) -> np.ndarray:
    return np.full(L, filling, dtype=np.int32)


def gaussian_sector_labels(chi: int, n_sectors: int, sigma: float, q_center: int) -> np.ndarray:
    """Sorted labels of one bond with n_sectors consecutive charges around q_center whose
    sizes follow exp(-(q - q_center)^2 / (2 sigma^2)), at least 1 each, summing to chi
    (the uneven sector profile of a U(1) bond at large chi)."""
    qs = np.arange(n_sectors) - n_sectors // 2 + q_center
    w = np.exp(-((qs - q_center) ** 2) / (2.0 * sigma ** 2))
    sizes = np.maximum(1, np.floor(w / w.sum() * chi).astype(np.int64))
    i = 0
    order = np.argsort(-w, kind="stable")
    while sizes.sum() < chi:
        sizes[order[i % n_sectors]] += 1
        i += 1
    while sizes.sum() > chi:
        j = order[i % n_sectors]
        if sizes[j] > 1:
            sizes[j] -= 1
        i += 1
    return np.concatenate([np.full(int(n), int(q), dtype=np.int64) for q, n in zip(qs, sizes)])


def env_mask(q_bra: np.ndarray, q_ket: np.ndarray, wq=BH_WQ) -> np.ndarray:
    """Boolean mask of allowed E[a', w, a]: q_bra[a'] == q_ket[a] + wq[w]."""
    wq = np.asarray(wq)
    return q_bra[:, None, None] == (q_ket[None, None, :] + wq[None, :, None])


def theta_mask(qa: np.ndarray, d: int, qb: np.ndarray) -> np.ndarray:
    """Boolean mask of allowed theta[a, s1, s2, b]: qb[b] == qa[a] + s1 + s2."""
    s = np.arange(d)
    return (qa[:, None, None, None] + s[None, :, None, None] + s[None, None, :, None]) == qb[None, None, None, :]
