"""Independent chains swept in lock step (tnt_dmrg_sweep_batched): every bond's eigensolves of
all chains in one grouped Lanczos, then each chain's SVD and environment growth.  Three
8-site Bose-Hubbard chains (N = 8, n_max = 3) at U/J = 1, 4 and 8 from their own seeded
random starts, chi_max = 16, three sweeps, against the FP64 oracle's sweeps of each chain from
the same start (every update's energy of the last sweep, the final state's overlap) and
against the single-chain GPU sweep.  Targets: |dE| <= 1e-10 |E|, |1 - |<psi|psi_ref>|| <= 1e-8."""
import numpy as np
import pytest

from oracle import bose_hubbard as bh
from oracle import contract as oc
from oracle import dmrg as odmrg
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu

L, N, N_MAX, CHI, SWEEPS = 8, 8, 3, 16, 3
US = (1.0, 4.0, 8.0)


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def starts():
    return [synth.random_charged_mps(synth.rng(40 + k), L, N_MAX + 1, N, CHI) for k in range(len(US))]


@pytest.fixture(scope="module")
def oracle_runs():
    out = []
    for (A, q), U in zip(starts(), US):
        Ws, l, r = bh.bh_mpo(L, N_MAX, 1.0, U)
        A2, _, hist = odmrg.dmrg(A, q, Ws, l, r, CHI, SWEEPS)
        out.append((np.array([u["E"] for u in hist[-1]["updates"]]), oc.mps_to_state(A2)))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_sweep_matches_oracle_per_chain(ctx, oracle_runs, precision):
    from paper_1610_02244_gb300 import tnt
    ctx.set_params(chi_max=CHI, precision=precision)
    try:
        runs, states = [], []
        for (A, q), U in zip(starts(), US):
            mps = ctx.mps_create(A, q, chi_cap=CHI)
            states.append(mps)
            runs.append(ctx.dmrg_create(mps, ctx.mpo_bose_hubbard(L, N_MAX, 1.0, U)))
        for _ in range(SWEEPS):
            st = ctx.dmrg_sweep_batched(runs)
        assert len(st) == len(US) and all(s["E"] == r.update_energies()[-1] for s, r in zip(st, runs))
        for run, mps, (Eu_ref, psi_ref) in zip(runs, states, oracle_runs):
            Eu = run.update_energies()
            assert len(Eu) == 2 * (L - 1)
            assert np.abs(Eu - Eu_ref).max() <= 1e-10 * np.abs(Eu_ref).max(), (Eu, Eu_ref)
            psi = oc.mps_to_state(mps.tensors())
            assert abs(1 - abs(np.vdot(psi_ref, psi))) <= 1e-8
    finally:
        ctx.set_params(chi_max=1 << 40, precision=tnt.TNT_PREC_FP64)


def test_batched_sweep_equals_single_chain_sweeps(ctx):
    """The same chains swept one at a time with tnt_dmrg_sweep: the same energies."""
    from paper_1610_02244_gb300 import tnt
    ctx.set_params(chi_max=CHI, precision=tnt.TNT_PREC_FP64)
    try:
        batched, single = [], []
        for (A, q), U in zip(starts(), US):
            mpo = ctx.mpo_bose_hubbard(L, N_MAX, 1.0, U)
            batched.append(ctx.dmrg_create(ctx.mps_create(A, q, chi_cap=CHI), mpo))
            single.append(ctx.dmrg_create(ctx.mps_create(A, q, chi_cap=CHI), mpo))
        ctx.dmrg_sweep_batched(batched)
        for s in single:
            s.sweep()
        for b, s in zip(batched, single):
            Eb, Es = b.update_energies(), s.update_energies()
            assert np.abs(Eb - Es).max() <= 1e-11 * np.abs(Es).max()
    finally:
        ctx.set_params(chi_max=1 << 40)


def test_batched_sweep_refuses_bad_handles(ctx):
    from paper_1610_02244_gb300 import tnt
    (A, q), = starts()[:1]
    mpo = ctx.mpo_bose_hubbard(L, N_MAX, 1.0, 2.0)
    mps = ctx.mps_create(A, q, chi_cap=CHI)
    a = ctx.dmrg_create(mps, mpo)
    b = ctx.dmrg_create(mps, mpo)
    with pytest.raises(tnt.TntError):  # two handles on one MPS
        ctx.dmrg_sweep_batched([a, b])
    short = ctx.dmrg_create(ctx.mps_product([1, 1, 1, 1], N_MAX + 1, CHI),
                            ctx.mpo_bose_hubbard(4, N_MAX, 1.0, 2.0))
    with pytest.raises(tnt.TntError):  # different lengths
        ctx.dmrg_sweep_batched([a, short])
