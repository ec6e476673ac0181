"""Pins of the oracle's spin-S Heisenberg pieces (the model of Sec. 6, Tables 1 and 2):
spin algebra, the hand-built MPO against a Kronecker-product Hamiltonian built from Sx and
Sy, two-site and free-fermion closed forms, and the oracle's DMRG and TEBD on the model."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bose_hubbard as bh
from oracle import contract as C
from oracle import dmrg, spin, tebd
from oracle.svd import TruncParams
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.cpu


@pytest.mark.parametrize("two_s", [1, 2, 3])
def test_spin_algebra(two_s):
    sp_, sm, sz, sx, sy, ident = spin.spin_ops(two_s)
    S = two_s / 2
    assert np.abs(sx @ sy - sy @ sx - 1j * sz).max() < 1e-14
    assert np.abs(sp_ @ sm - sm @ sp_ - 2 * sz).max() < 1e-14
    assert np.abs(sx @ sx + sy @ sy + sz @ sz - S * (S + 1) * ident).max() < 1e-13
    assert np.allclose(np.diag(sz).real, np.arange(two_s + 1) - S)


@pytest.mark.parametrize("L,two_s,J,Jz,hz", [(4, 2, 1.0, 1.0, 0.0), (4, 2, 1.0, 0.7, 0.3),
                                             (5, 1, 0.8, -0.4, 0.2)])
def test_mpo_equals_kronecker_hamiltonian(L, two_s, J, Jz, hz):
    Ws, l, r, _ = spin.heisenberg_mpo(L, two_s, J, Jz, hz)
    H1 = bh.mpo_to_matrix(Ws, l, r)
    H2 = spin.full_hamiltonian(L, two_s, J, Jz, hz).toarray()
    assert np.abs(H1 - H2).max() < 1e-13


def test_mpo_charges_are_conserved():
    """W[w, w', s', s] is non-zero only where s' - s = wq[w'] - wq[w] (each channel carries
    the charge its operator moved)."""
    Ws, _, _, wq = spin.heisenberg_mpo(3, 2, 1.0, 1.0, 0.5)
    W = Ws[0]
    for w in range(5):
        for v in range(5):
            for so in range(3):
                for si in range(3):
                    if abs(W[w, v, so, si]) > 0:
                        assert so - si == wq[v] - wq[w]


def test_two_spin1_spectrum_closed_form():
    """Two spin-1 sites: S1.S2 = [S_tot(S_tot + 1) - 4] / 2, S_tot = 0, 1, 2 with
    multiplicities 1, 3, 5."""
    h = spin.bond_hamiltonian(2, 1.0, 1.0, 0.0, 1.0, 1.0)
    lam = np.sort(np.linalg.eigvalsh(h))
    ref = np.array([-2.0] + [-1.0] * 3 + [1.0] * 5)
    assert np.abs(lam - ref).max() < 1e-13


def test_spin_half_singlet():
    e, v = spin.ground_state(2, 1, 1.0, 1.0, 0.0, 1)
    assert abs(e + 0.75) < 1e-14
    # singlet (|01> - |10>) / sqrt 2 in the basis s = m + 1/2
    assert abs(abs(v[1]) - 2 ** -0.5) < 1e-14 and abs(v[1] + v[2]) < 1e-14


@pytest.mark.parametrize("L", [6, 8, 10])
def test_xx_chain_free_fermion_energy(L):
    """Spin-1/2 XX chain (Jz = 0): Jordan-Wigner free fermions with hopping J/2, single
    particle energies J cos(k pi / (L + 1)); the ground state fills the negative ones."""
    e, _ = spin.ground_state(L, 1, 1.0, 0.0, 0.0, L // 2)
    ek = np.cos(np.arange(1, L + 1) * np.pi / (L + 1))
    assert abs(e - ek[ek < 0].sum()) < 1e-12


def test_bond_terms_sum_to_hamiltonian():
    """The Trotter split: the bond terms with weights c = 1 at the ends and 1/2 inside add
    up to H (field included)."""
    L, two_s, J, Jz, hz = 5, 2, 1.0, 0.6, 0.4
    d = two_s + 1
    H = np.zeros((d ** L, d ** L), dtype=np.complex128)
    for j in range(1, L):
        c1, c2 = bh.bond_weights(L, j)
        h = spin.bond_hamiltonian(two_s, J, Jz, hz, c1, c2)
        H += np.kron(np.kron(np.eye(d ** (j - 1)), h), np.eye(d ** (L - j - 1)))
    assert np.abs(H - spin.full_hamiltonian(L, two_s, J, Jz, hz).toarray()).max() < 1e-13


def test_oracle_dmrg_spin1_matches_ed():
    """Spin-1 chain, L = 8, S^z_total = 0 (N = 8 quanta), chi = 81 (exact): the oracle's
    DMRG reaches the ED ground state."""
    L, two_s = 8, 2
    E0, v0 = spin.ground_state(L, two_s, 1.0, 1.0, 0.0, L)
    g = synth.rng(3)
    A, q = synth.random_charged_mps(g, L, 3, L, 81)
    Ws, l, r, _ = spin.heisenberg_mpo(L, two_s, 1.0, 1.0)
    A2, q2, hist = dmrg.dmrg(A, q, Ws, l, r, 81, 3)
    assert abs(hist[-1]["E"] - E0) < 1e-10 * abs(E0)
    assert abs(1 - abs(np.vdot(v0, C.mps_to_state(A2)))) < 1e-8


def test_oracle_tebd_xx_chain_free_fermions():
    """Spin-1/2 XX chain from the Neel state |1010...>: <S^z_j + 1/2>(t) follows the free
    fermion closed form; second-order Trotter at dt = 0.05 stays within 3e-4 at t = 1."""
    L, steps, dt = 10, 20, 0.05
    occ = [1, 0] * (L // 2)
    A, q = tebd.product_state(occ, 1)
    hs = [spin.bond_hamiltonian(1, 1.0, 0.0, 0.0, *bh.bond_weights(L, j + 1))
          for j in range(L - 1)]
    ev = tebd.Tebd.from_bond_hamiltonians(A, q, hs, dt, TruncParams(chi_max=32, err_tol=1e-14))
    for _ in range(steps):
        ev.step()
    h1 = np.zeros((L, L))
    for j in range(L - 1):
        h1[j, j + 1] = h1[j + 1, j] = 0.5
    lam, Q = np.linalg.eigh(h1)
    Ut = (Q * np.exp(-1j * lam * dt * steps)) @ Q.conj().T
    exact = (np.abs(Ut) ** 2) @ np.array(occ, dtype=float)
    dens = C.density(ev.A, 1)
    assert np.abs(dens - exact).max() < 3e-4


def test_oracle_tebd_spin1_against_exact_evolution():
    """Spin-1 chain, L = 6, from a Neel-like product state: the Trotter state after t = 0.4
    matches exp(-iHt)|psi> to the O(dt^2) Trotter bound."""
    L, two_s, dt, steps = 6, 2, 0.02, 20
    occ = [2, 0, 2, 0, 2, 0]
    A, q = tebd.product_state(occ, two_s)
    hs = [spin.bond_hamiltonian(two_s, 1.0, 1.0, 0.0, *bh.bond_weights(L, j + 1))
          for j in range(L - 1)]
    ev = tebd.Tebd.from_bond_hamiltonians(A, q, hs, dt, TruncParams(chi_max=81, err_tol=1e-14))
    for _ in range(steps):
        ev.step()
    psi0 = C.mps_to_state(A)
    H = spin.full_hamiltonian(L, two_s, 1.0, 1.0, 0.0)
    exact = spla.expm_multiply(-1j * dt * steps * H, psi0)
    assert abs(1 - abs(np.vdot(exact, C.mps_to_state(ev.A)))) < 1e-5
