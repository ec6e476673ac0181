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
    "block_env",
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


def block_env(g: np.random.Generator, chi: int, side: str, gap: float = 1.0,
              width: float = 10.0, coupling: float = 1.0, D: int = 4) -> np.ndarray:
    """Environment E[a', w, a] with the channel structure a DMRG environment of the
    lower-triangular Bose-Hubbard MPO has (left boundary channel 3, right boundary
    channel 0), in the eigenbasis of its block Hamiltonian:

      identity channel (3 on the left, 0 on the right): the unit matrix (a canonical block);
      Hamiltonian channel (0 on the left, 3 on the right): diag(lam), lam_0 = 0 and the
        other chi - 1 levels drawn uniformly in [gap, gap + width] (a gapped block spectrum);
      channels 1 and 2: a boundary operator B with i.i.d. complex Gaussian entries of
        variance coupling^2 / chi, and B^H (the Hermitian pairing of hermitian_env).

    The two-site effective Hamiltonian built from a left and a right such environment is
    Hermitian and has an isolated lowest level, as H_eff of a DMRG state does, so a
    Lanczos solve converges (about 150 matvecs to 1e-12 at gap 1, width 10, chi 64..256)
    where the i.i.d. Gaussian environments of hermitian_env give a dense low spectrum."""
    if side not in ("left", "right"):
        raise ValueError("side must be 'left' or 'right'")
    ident, ham = (3, 0) if side == "left" else (0, 3)
    E = np.zeros((chi, D, chi), dtype=np.complex128)
    E[:, ident, :] = np.eye(chi)
    lam = np.concatenate(([0.0], gap + width * np.sort(g.random(chi - 1))))
    E[:, ham, :] = np.diag(lam)
    B = complex_gaussian(g, (chi, chi)) * (coupling / np.sqrt(chi))
    E[:, 1, :] = B
    E[:, 2, :] = B.conj().T
    return E


COUNT_CAP = 1 << 40  # sector counts saturate here (3^101 does not fit in int64)


def sector_counts(k: int, n_max: int) -> np.ndarray:
    """cnt[q] = number of occupation strings of k sites (0..n_max each) summing to q,
    saturated at COUNT_CAP (only ever compared with bond dimensions)."""
    cnt = np.zeros(k * n_max + 1, dtype=np.int64)
    cnt[0] = 1
    for _ in range(k):
        new = np.zeros_like(cnt)
        for n in range(n_max + 1):
            new[n:] += cnt[: len(cnt) - n]
        cnt = np.minimum(new, COUNT_CAP)
    return cnt


def _gauss_sizes(qs, caps, total, centre, sigma):
    """Sector sizes proportional to exp(-(q - centre)^2 / 2 sigma^2), each within its cap,
    summing to total (largest remainders first, spilling to the next-heaviest sectors)."""
    qs, caps = np.asarray(qs, dtype=np.float64), np.asarray(caps, dtype=np.int64)
    w = np.exp(-0.5 * ((qs - centre) / sigma) ** 2)
    sizes = np.zeros(len(qs), dtype=np.int64)
    left = total
    while left > 0:
        free = sizes < caps
        ww = np.where(free, w, 0.0)
        if ww.sum() <= 0:  # far tails underflow: fill by distance from the centre
            ww = np.where(free, 1.0 / (1.0 + np.abs(qs - centre)), 0.0)
        target = left * ww / ww.sum()
        add = np.minimum(np.floor(target).astype(np.int64), caps - sizes)
        if add.sum() == 0:  # hand out single indices by remainder
            order = np.argsort(-(target - np.floor(target)) - 1e-9 * np.arange(len(qs)))
            for i in order:
                if left == 0:
                    break
                if sizes[i] < caps[i]:
                    sizes[i] += 1
                    left -= 1
            continue
        sizes += add
        left -= int(add.sum())
    return sizes


def bond_charges(L: int, d: int, N: int, chi_max: int, profile: str = "even",
                 sigma: float = 2.0) -> list[np.ndarray]:
    """Charge label (bosons to the left of the bond) of every index of bonds 0..L.

    Bond k separates sites 1..k from k+1..L.  Every charge q reachable from both sides is
    a sector, its size capped by the exact Schmidt bound min(#left, #right); the bond holds
    min(chi_max, exact bound) indices.  profile "even": filled one index at a time, round
    robin over sectors in ascending q.  profile "gauss": sizes proportional to a Gaussian
    of width sigma around the mean filling N k / L (the sector profile of a ground state or
    of a state evolved from one).  Labels are returned sorted ascending.
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
        total = int(min(chi_max, sum(caps)))
        if profile == "gauss":
            sizes = [int(x) for x in _gauss_sizes(qs, caps, total, N * k / L, sigma)]
        else:
            sizes = [0] * len(qs)
            filled = 0
            while filled < total:
                for i in range(len(qs)):
                    if filled < total and sizes[i] < caps[i]:
                        sizes[i] += 1
                        filled += 1
        lab = np.concatenate([np.full(s, q, dtype=np.int64) for q, s in zip(qs, sizes) if s > 0])
        out.append(lab)
    return out


def charge_mask(ql: np.ndarray, d: int, qr: np.ndarray) -> np.ndarray:
    """Boolean mask of allowed A[a, s, b]: qr[b] == ql[a] + s (boson number conserved)."""
    s = np.arange(d)
    return (ql[:, None, None] + s[None, :, None]) == qr[None, None, :]


def random_charged_mps(g: np.random.Generator, L: int, d: int, N: int, chi_max: int,
                       profile: str = "even", sigma: float = 2.0):
    """Random-normal MPS in the fixed-N sector: Gaussian entries inside allowed blocks,
    bond sectors as bond_charges(profile, sigma), each site scaled to |A_j|_F^2 = chi_{j+1}
    (the left transfer map then keeps the identity at about unit size, so the norm of a
    long chain stays near one instead of growing like prod_j |A_j|; the scale of a site
    does not change the normalised state).

    Returns (tensors, charges): tensors[j] is A_j[a, s, b] (complex128) for sites
    j = 0..L-1 and charges[k] the labels of bond k = 0..L.  No gauge is applied: both
    sides bring the state to canonical form themselves.
    """
    charges = bond_charges(L, d, N, chi_max, profile, sigma)
    tensors = []
    for j in range(L):
        ql, qr = charges[j], charges[j + 1]
        A = complex_gaussian(g, (len(ql), d, len(qr)))
        A = np.where(charge_mask(ql, d, qr), A, 0.0)
        nrm = np.linalg.norm(A)
        if nrm > 0:
            A = A * (np.sqrt(len(qr)) / nrm)
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
