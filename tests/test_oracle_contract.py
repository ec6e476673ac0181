"""Pins of the oracle's contractions: H_eff.theta, environments, theta formation and the
gate, checked against exact-diagonalisation expectation values, explicit matrices and
Hermiticity."""
import numpy as np
import pytest

from oracle import bose_hubbard as bh
from oracle import contract as C
from oracle import dmrg, ed
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.cpu


def full_hamiltonian(L, n_max, J, U, mu=0.0):
    Ws, l, r = bh.bh_mpo(L, n_max, J, U, mu)
    d = n_max + 1
    # independent of the MPO: assemble the sectors of the Fock-space ED builder
    Hf = np.zeros((d ** L, d ** L), dtype=np.complex128)
    for N in range(L * n_max + 1):
        basis, _ = ed.fock_basis(L, N, n_max)
        idx = [sum(n * d ** (L - 1 - j) for j, n in enumerate(c)) for c in basis]
        Hf[np.ix_(idx, idx)] = ed.hamiltonian(L, N, n_max, J, U, mu).toarray()
    return Ws, l, r, Hf


@pytest.mark.parametrize("seed", [0, 1])
def test_energy_through_environments_matches_ed(seed):
    """<theta|H_eff theta> at every bond of a mixed-canonical random MPS equals
    <psi|H|psi> computed on the full Fock-space vector."""
    L, n_max, N, chi = 6, 2, 5, 7
    g = synth.rng(seed)
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, chi)
    A, q = dmrg.right_canonicalize(A, q)
    Ws, l, r, Hf = full_hamiltonian(L, n_max, 0.9, 1.6, 0.2)
    psi = C.mps_to_state(A)
    E_ed = np.vdot(psi, Hf @ psi).real
    assert abs(np.linalg.norm(psi) - 1) < 1e-12
    Renv = dmrg.build_right_envs(A, Ws, r)
    Lenv = C.boundary_left(l)
    for i in range(L - 1):
        theta = C.theta_form(A[i], A[i + 1])
        y = C.heff_apply(Lenv, Ws[i], Ws[i + 1], Renv[i + 2], theta)
        assert abs(np.vdot(theta, y).real - E_ed) < 1e-12
        # move the centre right by an exact SVD of the site (gauge change only)
        chl, d, _ = A[i].shape
        M = theta.reshape(chl * d, -1)
        U, S, Vh = np.linalg.svd(M, full_matrices=False)
        k = int(np.sum(S > 1e-14 * S[0]))
        A[i] = U[:, :k].reshape(chl, d, k)
        A[i + 1] = (S[:k, None] * Vh[:k]).reshape(k, d, -1)
        Lenv = C.env_left(Lenv, Ws[i], A[i])
    # the left environment of the whole chain closes on the right boundary
    E_full = C.mps_expect_mpo(A, Ws, l, r).real
    assert abs(E_full - E_ed) < 1e-12


def test_heff_staged_equals_single_einsum_and_is_hermitian():
    g = synth.rng(3)
    chi, d = 5, 3
    Ws, _, _ = bh.bh_mpo(4, d - 1, 1.0, 2.0)
    Le = synth.hermitian_env(g, chi)
    Re = synth.hermitian_env(g, chi + 1)
    H = C.heff_dense(Le, Ws[1], Ws[2], Re)
    assert np.abs(H - H.conj().T).max() < 1e-12
    theta = synth.complex_gaussian(g, (chi, d, d, chi + 1))
    y = C.heff_apply(Le, Ws[1], Ws[2], Re, theta)
    assert np.abs(y.reshape(-1) - H @ theta.reshape(-1)).max() < 1e-12


def test_theta_and_gate_against_kron():
    g = synth.rng(4)
    A = synth.complex_gaussian(g, (3, 4, 5))
    B = synth.complex_gaussian(g, (5, 4, 2))
    th = C.theta_form(A, B)
    ref = (A.reshape(12, 5) @ B.reshape(5, 8)).reshape(3, 4, 4, 2)
    assert np.abs(th - ref).max() < 1e-13
    G = bh.gate(bh.bond_hamiltonian(3, 1.0, 2.0, 0.5, 0.5), 0.1)
    out = C.gate_apply(G, th)
    big = np.kron(np.kron(np.eye(3), G), np.eye(2))
    assert np.abs(out.reshape(-1) - big @ th.reshape(-1)).max() < 1e-13


def test_density_and_overlap():
    g = synth.rng(5)
    L, n_max, N = 5, 2, 4
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, 6)
    psi = C.mps_to_state(A)
    nrm = np.vdot(psi, psi).real
    assert abs(C.mps_overlap(A, A).real - nrm) < 1e-10 * nrm
    dens = C.density(A, n_max)
    for j in range(1, L + 1):
        nj = ed.number_operator_full(L, n_max, j)
        assert abs(dens[j - 1] - np.vdot(psi, nj * psi).real / nrm) < 1e-12
    assert abs(dens.sum() - N) < 1e-12


def _apply_site(psi, op, site, L, d):
    """op acting on one site of a full state vector (sites most significant first)."""
    t = psi.reshape((d,) * L)
    t = np.moveaxis(np.tensordot(op, t, axes=([1], [site])), 0, site)
    return t.reshape(-1)


def test_bdagb_against_full_state_vector():
    """rho_ij = <b+_i b_j> by transfer matrices equals the brute-force value on the full
    d^L vector (operators applied by reshaping), is Hermitian, has the density on its
    diagonal and trace N (the random MPS lives in the N = 4 sector)."""
    L, n_max, N = 5, 2, 4
    d = n_max + 1
    g = synth.rng(9)
    A, _ = synth.random_charged_mps(g, L, d, N, 8)
    psi = C.mps_to_state(A)
    b = np.diag(np.sqrt(np.arange(1, d, dtype=float)), k=1)
    rho = C.bdagb(A, n_max)
    nrm = np.vdot(psi, psi).real
    for i in range(L):
        for j in range(L):
            phi = _apply_site(_apply_site(psi, b, j, L, d), b.T, i, L, d)
            assert abs(rho[i, j] - np.vdot(psi, phi) / nrm) < 1e-12
    assert np.allclose(rho, rho.conj().T, atol=1e-13)
    assert np.allclose(np.diag(rho).real, C.density(A, n_max), atol=1e-13)
    assert abs(np.trace(rho).real - N) < 1e-12


def test_bdagb_fock_state_is_diagonal():
    from oracle import tebd
    occ = [2, 0, 1, 1, 0]
    A, _ = tebd.product_state(occ, 2)
    assert np.allclose(C.bdagb(A, 2), np.diag(occ), atol=1e-15)
