"""Pins of the oracle's single-site DMRG with subspace expansion (direct sums of App. B):
the expansion term lies in the charge blocks its labels claim, the direct sums leave the
state unchanged, the sweeps reach exact diagonalisation, and without the expansion a
one-site sweep cannot enlarge its bonds."""
import numpy as np
import pytest

from oracle import bose_hubbard as bh
from oracle import contract as C
from oracle import dmrg, dmrg1, ed, spin
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.cpu

BH_WQ = [0, 1, -1, 0]


def _charged_centre(seed=0, L=6, n_max=2, N=6, chi=9):
    g = synth.rng(seed)
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, chi)
    dmrg.right_canonicalize(A, q)
    Ws, l, r = bh.bh_mpo(L, n_max, 1.0, 2.0)
    return A, q, Ws, l, r


def test_expansion_terms_respect_the_charge_rules():
    A, q, Ws, l, r = _charged_centre()
    i = 2
    d = A[i].shape[1]
    Lenv = C.boundary_left(l)
    for j in range(i):
        Lenv = C.env_left(Lenv, Ws[j], A[j])
    P = dmrg1.expansion_right(Lenv, Ws[i], A[i], 0.5)
    qP = (q[i + 1][None, :] + np.array(BH_WQ)[:, None]).reshape(-1)
    allowed = synth.charge_mask(q[i], d, qP)
    assert np.abs(P).max() > 0
    assert np.abs(P[~allowed]).max() == 0.0
    Renv = dmrg.build_right_envs(A, Ws, r)
    Pl = dmrg1.expansion_left(Ws[i], Renv[i + 1], A[i], 0.5)
    qPl = (q[i][None, :] + np.array(BH_WQ)[:, None]).reshape(-1)
    allowed = synth.charge_mask(qPl, d, q[i + 1])
    assert np.abs(Pl).max() > 0
    assert np.abs(Pl[~allowed]).max() == 0.0


def test_direct_sums_leave_the_state_unchanged():
    A, q, Ws, l, r = _charged_centre(1)
    i = 2
    P = 0.3 * synth.complex_gaussian(synth.rng(5), (A[i].shape[0], A[i].shape[1], 7))
    Mt = dmrg1.direct_sum_right(A[i], P)
    Bt = dmrg1.direct_sum_left(A[i + 1], np.zeros((7,) + A[i + 1].shape[1:], dtype=np.complex128))
    assert Mt.shape[2] == A[i].shape[2] + 7 and Bt.shape[0] == A[i + 1].shape[0] + 7
    assert np.abs(C.theta_form(Mt, Bt) - C.theta_form(A[i], A[i + 1])).max() < 1e-15


def test_dmrg1_bose_hubbard_L8_matches_ed():
    """From a chi = 4 start the expansion grows the bonds to the exact ground state."""
    L, N, n_max = 8, 8, 3
    Es, V = ed.lowest(ed.hamiltonian(L, N, n_max, 1.0, 2.0))
    g = synth.rng(2)
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, 4)
    Ws, l, r = bh.bh_mpo(L, n_max, 1.0, 2.0)
    A2, q2, hist = dmrg1.dmrg1(A, q, Ws, l, r, BH_WQ, 64, 10, alpha0=1e-2)
    assert hist[-1]["max_chi"] > 4
    assert abs(hist[-1]["E"] - Es[0]) < 1e-10 * abs(Es[0])
    psi = C.mps_to_state(A2)
    assert abs(1 - abs(np.vdot(ed.embed(V[:, 0], L, N, n_max), psi))) < 1e-8
    assert abs(C.density(A2, n_max).sum() - N) < 1e-12
    tail = [h["E"] for h in hist if h["alpha"] == 0.0]
    assert all(b <= a + 1e-12 for a, b in zip(tail, tail[1:]))


def test_dmrg1_without_expansion_keeps_its_bonds():
    """alpha = 0: a one-site update hands over no new directions, the bonds of a chi = 2
    start never grow and the energy stays well above the ground state."""
    L, N, n_max = 8, 8, 3
    Es, _ = ed.lowest(ed.hamiltonian(L, N, n_max, 1.0, 2.0))
    g = synth.rng(3)
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, 2)
    Ws, l, r = bh.bh_mpo(L, n_max, 1.0, 2.0)
    _, _, hist = dmrg1.dmrg1(A, q, Ws, l, r, BH_WQ, 64, 4, alpha0=0.0)
    assert hist[-1]["max_chi"] <= 2
    assert hist[-1]["E"] - Es[0] > 1e-3 * abs(Es[0])


def test_dmrg1_spin1_matches_ed():
    """The spin-1 chain of Sec. 6 (L = 8, S^z = 0, D = 5 MPO): exact ground state."""
    L = 8
    E0, v0 = spin.ground_state(L, 2, 1.0, 1.0, 0.0, L)
    g = synth.rng(6)
    A, q = synth.random_charged_mps(g, L, 3, L, 6)
    Ws, l, r, wq = spin.heisenberg_mpo(L, 2, 1.0, 1.0)
    A2, _, hist = dmrg1.dmrg1(A, q, Ws, l, r, wq, 81, 10, alpha0=1e-2)
    assert abs(hist[-1]["E"] - E0) < 1e-10 * abs(E0)
    assert abs(1 - abs(np.vdot(v0, C.mps_to_state(A2)))) < 1e-8
