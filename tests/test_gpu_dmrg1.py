"""Single-site DMRG with subspace expansion on the GPU (tnt_dmrg_sweep1) against exact
diagonalisation and the FP64 oracle (oracle/dmrg1.py, the same sweep): from a small start
the expansion grows the bonds to the exact ground state; without it the bonds never grow."""
import numpy as np
import pytest

from oracle import bose_hubbard as bh
from oracle import contract as oc
from oracle import dmrg1 as odmrg1
from oracle import ed
from oracle import spin as ospin
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu

L, N, N_MAX = 8, 8, 3


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def _alphas(alpha0, sweeps, zero_sweeps=2):
    return [0.0 if s >= sweeps - zero_sweeps else alpha0 * 10.0 ** (-s) for s in range(sweeps)]


def _run(ctx, A, q, mpo, chi, alphas):
    from paper_1610_02244_gb300 import tnt
    ctx.set_params(chi_max=chi, precision=tnt.TNT_PREC_FP64)
    try:
        mps = ctx.mps_create(A, q, chi_cap=chi)
        dm = ctx.dmrg_create(mps, mpo)
        stats = [dm.sweep1(a) for a in alphas]
        return stats, mps
    finally:
        ctx.set_params(chi_max=1 << 40)


def test_dmrg1_bose_hubbard_reaches_ed(ctx):
    Es, V = ed.lowest(ed.hamiltonian(L, N, N_MAX, 1.0, 2.0))
    g = synth.rng(2)
    A, q = synth.random_charged_mps(g, L, N_MAX + 1, N, 4)
    alphas = _alphas(1e-2, 10)
    stats, mps = _run(ctx, A, q, ctx.mpo_bose_hubbard(L, N_MAX, 1.0, 2.0), 64, alphas)
    assert max(mps.bond_dim(k) for k in range(L + 1)) > 4
    assert abs(stats[-1]["E"] - Es[0]) <= 1e-10 * abs(Es[0])
    psi = oc.mps_to_state(mps.tensors())
    assert abs(1 - abs(np.vdot(ed.embed(V[:, 0], L, N, N_MAX), psi))) <= 1e-8
    assert abs(mps.norm2() - 1) < 1e-12
    # the oracle's sweep from the same start ends on the same energy
    Ws, l, r = bh.bh_mpo(L, N_MAX, 1.0, 2.0)
    _, _, hist = odmrg1.dmrg1(A, q, Ws, l, r, [0, 1, -1, 0], 64, 10, alpha0=1e-2)
    assert abs(stats[-1]["E"] - hist[-1]["E"]) <= 1e-10 * abs(hist[-1]["E"])


def test_dmrg1_without_expansion_keeps_its_bonds(ctx):
    Es, _ = ed.lowest(ed.hamiltonian(L, N, N_MAX, 1.0, 2.0))
    g = synth.rng(3)
    A, q = synth.random_charged_mps(g, L, N_MAX + 1, N, 2)
    stats, mps = _run(ctx, A, q, ctx.mpo_bose_hubbard(L, N_MAX, 1.0, 2.0), 64, [0.0] * 4)
    assert max(mps.bond_dim(k) for k in range(L + 1)) <= 2
    assert stats[-1]["E"] - Es[0] > 1e-3 * abs(Es[0])


def test_dmrg1_spin1_reaches_ed(ctx):
    E0, v0 = ospin.ground_state(L, 2, 1.0, 1.0, 0.0, L)
    g = synth.rng(6)
    A, q = synth.random_charged_mps(g, L, 3, L, 6)
    stats, mps = _run(ctx, A, q, ctx.mpo_spin_heisenberg(L, 2, 1.0), 81, _alphas(1e-2, 10))
    assert abs(stats[-1]["E"] - E0) <= 1e-10 * abs(E0)
    assert abs(1 - abs(np.vdot(v0, oc.mps_to_state(mps.tensors())))) <= 1e-8
