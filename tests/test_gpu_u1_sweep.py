"""The U(1) DMRG sweep of the chi = 1024 chain (d = 5, U/J = 3.4, unit filling) at a size the
FP64 oracle finishes in seconds: 12 sites, N = 12, chi_max = 40, from a seeded random start
with a Gaussian sector profile, three sweeps, in FP64 and in split TF32 (with the sweep's
FP64 finish).  Every update's energy of the last sweep against the oracle's sweeps from the
same start, the final state's overlap, the particle number and energy monotonicity.
Targets: |dE| <= 1e-10 |E|, |1 - |<psi|psi_ref>|| <= 1e-8."""
import numpy as np
import pytest

from oracle import bose_hubbard as bh
from oracle import contract as oc
from oracle import dmrg as odmrg
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu

L, N, N_MAX, U, CHI, SWEEPS = 12, 12, 4, 3.4, 40, 3


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def start():
    return synth.random_charged_mps(synth.rng(64), L, N_MAX + 1, N, CHI, "gauss", 2.0)


@pytest.fixture(scope="module")
def oracle_run():
    A, q = start()
    Ws, l, r = bh.bh_mpo(L, N_MAX, 1.0, U)
    A2, _, hist = odmrg.dmrg(A, q, Ws, l, r, CHI, SWEEPS)
    return [h["E"] for h in hist], np.array([u["E"] for u in hist[-1]["updates"]]), oc.mps_to_state(A2)


@pytest.mark.parametrize("precision", [0, 1])
def test_u1_sweep_unit_filling_matches_oracle(ctx, oracle_run, precision):
    from paper_1610_02244_gb300 import tnt
    E_ref, Eu_ref, psi_ref = oracle_run
    A, q = start()
    ctx.set_params(chi_max=CHI, precision=precision)
    try:
        mps = ctx.mps_create(A, q, chi_cap=CHI)
        mpo = ctx.mpo_bose_hubbard(L, N_MAX, 1.0, U)
        dm = ctx.dmrg_create(mps, mpo)
        E = [dm.sweep()["E"] for _ in range(SWEEPS)]
        Eu = dm.update_energies()
        psi = oc.mps_to_state(mps.tensors())
        n = mps.density()
    finally:
        ctx.set_params(chi_max=1 << 40, precision=tnt.TNT_PREC_FP64)
    assert np.abs(np.array(E) - E_ref).max() <= 1e-10 * abs(E_ref[-1]), (E, E_ref)
    assert np.abs(Eu - Eu_ref).max() <= 1e-10 * np.abs(Eu_ref).max()
    assert abs(1 - abs(np.vdot(psi_ref, psi))) <= 1e-8
    assert abs(n.sum() - N) < 1e-10
    assert all(b <= a + 1e-10 * abs(a) for a, b in zip(E[1:], E[2:]))
