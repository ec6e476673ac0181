"""End-to-end two-site DMRG on the GPU (C-ABI sweep driver) against the FP64 oracle and
exact diagonalisation: the 8-site Bose-Hubbard chain (N = 8, n_max = 3, J = 1, U = 2),
random-normal initial MPS inside the N = 8 blocks, 4 sweeps at chi_max = 32.
Targets: |dE| <= 1e-10 |E| and |1 - |<psi|psi_ref>|| <= 1e-8."""
import numpy as np
import pytest

from oracle import bose_hubbard as bh
from oracle import contract as oc
from oracle import dmrg as odmrg
from oracle import ed
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu

L, N, N_MAX, J, U = 8, 8, 3, 1.0, 2.0


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


@pytest.fixture(scope="module")
def ed_ground():
    E, V = ed.lowest(ed.hamiltonian(L, N, N_MAX, J, U), 1)
    return E[0], ed.embed(V[:, 0], L, N, N_MAX)


@pytest.fixture(scope="module")
def oracle_chi32():
    g = synth.rng(0)
    A, q = synth.random_charged_mps(g, L, N_MAX + 1, N, 32)
    Ws, l, r = bh.bh_mpo(L, N_MAX, J, U)
    A2, q2, hist = odmrg.dmrg(A, q, Ws, l, r, 32, 4)
    return hist, oc.mps_to_state(A2)


def run_gpu(ctx, chi, sweeps, precision, seed=0):
    from paper_1610_02244_gb300 import tnt
    g = synth.rng(seed)
    A, q = synth.random_charged_mps(g, L, N_MAX + 1, N, chi)
    ctx.set_params(chi_max=chi, precision=precision)
    try:
        mps = ctx.mps_create(A, q, chi_cap=chi)
        mpo = ctx.mpo_bose_hubbard(L, N_MAX, J, U)
        dm = ctx.dmrg_create(mps, mpo)
        stats = [dm.sweep() for _ in range(sweeps)]
        psi = oc.mps_to_state(mps.tensors())
        E_expect = mps.expect_mpo(mpo)
        n2 = mps.norm2()
        charges = [mps.charges(k) for k in range(L + 1)]
    finally:
        ctx.set_params(chi_max=1 << 40, precision=tnt.TNT_PREC_FP64)
    return stats, psi, E_expect, n2, charges


@pytest.mark.parametrize("precision", [0, 1])
def test_dmrg_cfg1_matches_oracle(ctx, oracle_chi32, ed_ground, precision):
    hist, psi_ref = oracle_chi32
    stats, psi, E_expect, n2, charges = run_gpu(ctx, 32, 4, precision)
    E_ref = hist[-1]["E"]
    E = stats[-1]["E"]
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref), (E, E_ref)
    assert abs(E_expect - E_ref) <= 1e-10 * abs(E_ref)
    assert abs(1 - abs(np.vdot(psi_ref, psi))) <= 1e-8
    assert abs(n2 - 1) < 1e-12
    # N = 8 exactly: the state lives in the sector, bond labels are boson counts
    full = psi.reshape(-1)
    counts = np.array([sum(int(c) for c in np.base_repr(i, 4).zfill(L)) for i in range(4 ** L)])
    assert np.abs(full[counts != N]).max() == 0.0
    assert all(np.all(charges[k] >= 0) for k in range(L + 1))
    # against exact diagonalisation: chi = 32 truncation leaves ~1e-9 relative
    E0, _ = ed_ground
    assert abs(E - E0) <= 1e-8 * abs(E0)
    energies = [s["E"] for s in stats]
    assert all(b <= a + 1e-10 for a, b in zip(energies, energies[1:]))


def test_dmrg_chi64_matches_ed(ctx, ed_ground):
    stats, psi, _, _, _ = run_gpu(ctx, 64, 3, 0, seed=1)
    E0, v0 = ed_ground
    assert abs(stats[-1]["E"] - E0) <= 1e-10 * abs(E0)
    assert abs(1 - abs(np.vdot(v0, psi))) <= 1e-8
