"""Pins of the oracle's algorithms: two-site DMRG against exact diagonalisation and closed
forms, TEBD against exact time evolution, free fermions and invariants."""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg as spla

from oracle import bose_hubbard as bh
from oracle import contract as C
from oracle import dmrg, ed, svd, tebd
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.cpu


def test_dmrg_bose_hubbard_L8_matches_ed():
    """The 8-site, 8-boson, n_max = 3, U = 2 chain at chi = 64: energy and state match ED
    (the N = 8 sector has 3823 states; the middle-bond discarded weight at chi = 64 is
    ~1e-14)."""
    L, N, n_max = 8, 8, 3
    Es, V = ed.lowest(ed.hamiltonian(L, N, n_max, 1.0, 2.0))
    g = synth.rng(0)
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, 64)
    Ws, l, r = bh.bh_mpo(L, n_max, 1.0, 2.0)
    A, q, hist = dmrg.dmrg(A, q, Ws, l, r, 64, 3)
    E = hist[-1]["E"]
    assert abs(E - Es[0]) < 1e-10 * abs(Es[0])
    psi = C.mps_to_state(A)
    ov = abs(np.vdot(ed.embed(V[:, 0], L, N, n_max), psi))
    assert abs(1 - ov) < 1e-8
    energies = [h["E"] for h in hist]
    assert all(b <= a + 1e-12 for a, b in zip(energies, energies[1:]))
    assert abs(np.linalg.norm(psi) - 1) < 1e-12
    assert abs(C.density(A, n_max).sum() - N) < 1e-12


def test_dmrg_free_bosons_closed_form():
    L, N, n_max, J = 6, 2, 2, 1.0
    g = synth.rng(1)
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, 16)
    Ws, l, r = bh.bh_mpo(L, n_max, J, 0.0)
    _, _, hist = dmrg.dmrg(A, q, Ws, l, r, 16, 3)
    assert abs(hist[-1]["E"] - (-2 * J * N * np.cos(np.pi / (L + 1)))) < 1e-10


def test_dmrg_hard_core_closed_form():
    L, N, J = 8, 4, 1.0
    g = synth.rng(2)
    A, q = synth.random_charged_mps(g, L, 2, N, 16)
    Ws, l, r = bh.bh_mpo(L, 1, J, 3.0)
    _, _, hist = dmrg.dmrg(A, q, Ws, l, r, 16, 3)
    exact = -2 * J * sum(np.cos(k * np.pi / (L + 1)) for k in range(1, N + 1))
    assert abs(hist[-1]["E"] - exact) < 1e-10


def exact_evolution(occ, n_max, J, U, t):
    L, N = len(occ), int(sum(occ))
    H = ed.hamiltonian(L, N, n_max, J, U)
    basis, index = ed.fock_basis(L, N, n_max)
    v0 = np.zeros(len(basis), dtype=np.complex128)
    v0[index[tuple(occ)]] = 1.0
    return ed.embed(spla.expm_multiply(-1j * t * H, v0), L, N, n_max)


def test_tebd_second_order_against_exact_evolution():
    occ, n_max, J, U, t = [1, 0, 2, 0, 1, 1], 2, 1.0, 1.3, 0.4
    ex = exact_evolution(occ, n_max, J, U, t)
    errs = []
    for dt in (0.04, 0.02):
        A, q = tebd.product_state(occ, n_max)
        T = tebd.Tebd(A, q, n_max, J, U, dt, svd.TruncParams(chi_max=64, err_tol=1e-14))
        for _ in range(int(round(t / dt))):
            T.step()
        errs.append(np.linalg.norm(C.mps_to_state(T.A) - ex))
    assert errs[1] < 5e-4
    assert 3.5 < errs[0] / errs[1] < 4.5  # error O(dt^2)


def test_tebd_hard_core_free_fermion_densities():
    """Hard-core bosons from a charge-density wave: <n_j(t)> = sum_k |[e^{-iht}]_jk|^2 n_k(0)
    with h the single-particle hopping matrix (the quench of Sec. 5 in miniature)."""
    L, J, dt, t = 8, 1.0, 0.01, 0.5
    occ = [1, 0] * (L // 2)
    h = -J * (np.eye(L, k=1) + np.eye(L, k=-1))
    Uc = scipy.linalg.expm(-1j * t * h)
    exact = (np.abs(Uc) ** 2) @ np.array(occ, dtype=float)
    A, q = tebd.product_state(occ, 1)
    T = tebd.Tebd(A, q, 1, J, 4.0, dt, svd.TruncParams(chi_max=32, err_tol=1e-14))
    for _ in range(int(round(t / dt))):
        T.step()
    dens = C.density(T.A, 1)
    assert np.abs(dens - exact).max() < 1e-4
    assert abs(dens.sum() - L // 2) < 1e-12


def test_tebd_norm_loss_equals_discarded_weight_and_energy_drift():
    occ, n_max, J, U, dt = [1] * 8, 2, 1.0, 2.0, 0.05
    A, q = tebd.product_state(occ, n_max)
    T = tebd.Tebd(A, q, n_max, J, U, dt, svd.TruncParams(chi_max=4, err_tol=1e-12))
    Ws, l, r = bh.bh_mpo(8, n_max, J, U)
    E0 = C.mps_expect_mpo(T.A, Ws, l, r).real
    for _ in range(10):
        T.step()
    nrm = C.mps_overlap(T.A, T.A).real
    assert T.disc_sum > 1e-6  # chi = 4 really truncates
    # truncating at the orthogonality centre removes exactly the discarded weight
    assert abs((1 - nrm) - T.disc_sum) < 1e-3 * T.disc_sum + 1e-13
    E1 = C.mps_expect_mpo(T.A, Ws, l, r).real / nrm
    assert abs(E1 - E0) < 0.05
    assert abs(C.density(T.A, n_max).sum() - 8) < 1e-12
