"""Pins of the oracle's model layer: exact diagonalisation, the MPO and the Trotter terms
against closed forms, combinatorics and each other (independent constructions)."""
import itertools
from math import comb

import numpy as np
import pytest
import scipy.linalg

from oracle import bose_hubbard as bh
from oracle import ed

pytestmark = pytest.mark.cpu


def sector_dim_formula(L, N, n_max):
    """Inclusion-exclusion count of compositions of N into L parts of size <= n_max."""
    return sum((-1) ** k * comb(L, k) * comb(N - k * (n_max + 1) + L - 1, L - 1)
               for k in range(L + 1) if N - k * (n_max + 1) >= 0)


@pytest.mark.parametrize("L,N,n_max", [(8, 8, 3), (5, 4, 2), (6, 3, 1), (7, 7, 4)])
def test_sector_dimension(L, N, n_max):
    basis, _ = ed.fock_basis(L, N, n_max)
    assert len(basis) == sector_dim_formula(L, N, n_max)
    assert len(set(basis)) == len(basis)


def test_cfg1_sector_dimension_is_3823():
    assert len(ed.fock_basis(8, 8, 3)[0]) == 3823


@pytest.mark.parametrize("L,N,n_max,J", [(8, 3, 3, 1.0), (7, 2, 2, 0.7), (6, 4, 4, 1.3)])
def test_free_bosons_closed_form(L, N, n_max, J):
    """U = 0 and N <= n_max: every boson sits in the lowest hopping mode,
    E0 = -2 J N cos(pi / (L + 1))."""
    E, _ = ed.lowest(ed.hamiltonian(L, N, n_max, J, 0.0))
    assert abs(E[0] - (-2 * J * N * np.cos(np.pi / (L + 1)))) < 1e-12


@pytest.mark.parametrize("L,N,J", [(8, 4, 1.0), (7, 3, 0.8), (9, 2, 1.0)])
def test_hard_core_free_fermion_closed_form(L, N, J):
    """n_max = 1 on an open chain maps to free fermions: E0 = -2J sum_{k<=N} cos(k pi/(L+1))."""
    E, _ = ed.lowest(ed.hamiltonian(L, N, 1, J, 5.0))
    exact = -2 * J * sum(np.cos(k * np.pi / (L + 1)) for k in range(1, N + 1))
    assert abs(E[0] - exact) < 1e-12


def test_atomic_limit_brute_force():
    """J = 0: H is diagonal; the ground energy is the minimum over occupation strings of
    U/2 sum n(n-1) + V sum (j - j_c)^2 n - mu N, found by brute force."""
    L, N, n_max, U, V, jc, mu = 5, 4, 3, 1.1, 0.37, 2.5, 0.2
    best = min(sum(0.5 * U * n * (n - 1) + (V * (j + 1 - jc) ** 2 - mu) * n
                   for j, n in enumerate(c))
               for c in itertools.product(range(n_max + 1), repeat=L) if sum(c) == N)
    E, _ = ed.lowest(ed.hamiltonian(L, N, n_max, 0.0, U, mu, V, jc))
    assert abs(E[0] - best) < 1e-13


def test_hermitian_and_number_conserving():
    H = ed.hamiltonian(6, 5, 2, 0.9, 1.7, 0.3, 0.05, 3.0).toarray()
    assert np.abs(H - H.conj().T).max() == 0.0


def full_ed_matrix(L, n_max, J, U, mu, V, jc):
    """Block-diagonal assembly over all N sectors in the full d^L basis."""
    d = n_max + 1
    Hf = np.zeros((d ** L, d ** L), dtype=np.complex128)
    for N in range(L * n_max + 1):
        basis, _ = ed.fock_basis(L, N, n_max)
        idx = [int("".join(map(str, c)), d) if d <= 10 else None for c in basis]
        Hs = ed.hamiltonian(L, N, n_max, J, U, mu, V, jc).toarray()
        Hf[np.ix_(idx, idx)] = Hs
    return Hf


@pytest.mark.parametrize("L,n_max", [(4, 2), (5, 1), (3, 3)])
def test_mpo_equals_ed(L, n_max):
    """The hand-built MPO (Sec. 4.3) contracts to exactly the Fock-space H of Eq. 2."""
    J, U, mu, V, jc = 0.83, 1.9, 0.31, 0.07, 2.2
    Ws, l, r = bh.bh_mpo(L, n_max, J, U, mu, V, jc)
    Hm = bh.mpo_to_matrix(Ws, l, r)
    Hf = full_ed_matrix(L, n_max, J, U, mu, V, jc)
    assert np.abs(Hm - Hf).max() < 1e-13


@pytest.mark.parametrize("L,n_max", [(4, 2), (5, 2), (2, 3)])
def test_bond_terms_sum_to_hamiltonian(L, n_max):
    """sum over bonds of the weighted Trotter terms h_{j,j+1} equals Eq. 2 (V = 0)."""
    J, U, mu = 1.1, 2.3, 0.4
    d = n_max + 1
    Hb = np.zeros((d ** L, d ** L), dtype=np.complex128)
    for j in range(1, L):
        c1, c2 = bh.bond_weights(L, j)
        h = bh.bond_hamiltonian(n_max, J, U, c1, c2, mu)
        Hb += np.kron(np.kron(np.eye(d ** (j - 1)), h), np.eye(d ** (L - j - 1)))
    Hf = full_ed_matrix(L, n_max, J, U, mu, 0.0, 0.0)
    assert np.abs(Hb - Hf).max() < 1e-13


def test_gate_is_matrix_exponential_and_unitary():
    h = bh.bond_hamiltonian(4, 1.0, 2.0, 0.5, 1.0)
    for tau in (0.005, 0.01, 0.3):
        G = bh.gate(h, tau)
        assert np.abs(G - scipy.linalg.expm(-1j * tau * h)).max() < 1e-13
        assert np.abs(G @ G.conj().T - np.eye(25)).max() < 1e-13


def test_local_operators():
    b, bd, n, _ = bh.local_ops(3)
    assert np.allclose(bd @ b, n)
    # [b, b+] = 1 except on the truncated top level
    comm = b @ bd - bd @ b
    assert np.allclose(np.diag(comm)[:-1], 1.0)
