"""The first example calculation of Sec. 5 on the GPU: bosons in a harmonic trap,
H of Eq. 2 with the trap term V (j - j_c)^2 n_j, so that every site has its own MPO tensor.

- E1 at the paper's size (L = 100, N = 100, n_max = 3, U/J = 5, V/J = 0.01, j_c at the
  chain centre, chi = 100; Fig. 4): density profile and single-particle density matrix;
- its first DMRG sweep against the FP64 oracle's first sweep from the same seeded start,
  update by update;
- the same Hamiltonian on ten sites with a trap that empties the edges, against exact
  diagonalisation."""
import os

import numpy as np
import pytest

from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def _ed_density(vec, L, N, n_max):
    from oracle import ed
    basis, _ = ed.fock_basis(L, N, n_max)
    occ = np.array(basis, dtype=float)
    return (np.abs(vec)[:, None] ** 2 * occ).sum(axis=0)


@pytest.mark.parametrize("precision", [0, 1])
def test_e1_trap_reduced_to_ten_sites(ctx, precision):
    """The first example's Hamiltonian on L = 10 (N = 10, n_max = 3, U/J = 5) with a trap
    strong enough to empty the edges (V/J = 0.5, every site its own MPO tensor), two-site
    DMRG at chi = 48 against exact diagonalisation of the N = 10 sector: energy, state,
    density, the trap's mirror symmetry, and right-canonical sites after the sweeps."""
    from oracle import contract as oc
    from oracle import ed
    from paper_1610_02244_gb300 import tnt
    Ls, N, n_max, J, U, V, chi = 10, 10, 3, 1.0, 5.0, 0.5, 48
    j_c = (Ls + 1) / 2.0
    Es, Vs = ed.lowest(ed.hamiltonian(Ls, N, n_max, J, U, 0.0, V, j_c), 1)
    n_ref = _ed_density(Vs[:, 0], Ls, N, n_max)
    A, q = synth.random_charged_mps(synth.rng(11), Ls, n_max + 1, N, chi)
    ctx.set_params(chi_max=chi, precision=precision)
    try:
        mps = ctx.mps_create(A, q, chi_cap=chi)
        mpo = ctx.mpo_bose_hubbard(Ls, n_max, J, U, 0.0, V, j_c)
        dm = ctx.dmrg_create(mps, mpo)
        E = [dm.sweep()["E"] for _ in range(4)]
        E_mpo = mps.expect_mpo(mpo)
    finally:
        ctx.set_params(chi_max=1 << 40, precision=tnt.TNT_PREC_FP64)
    # chi = 48 leaves ~4e-11 relative in the FP64 oracle's sweep from the same start
    assert abs(E[-1] - Es[0]) <= 1e-9 * abs(Es[0]), (E, Es[0])
    assert abs(E_mpo - Es[0]) <= 1e-9 * abs(Es[0])
    psi = oc.mps_to_state(mps.tensors())
    assert abs(1 - abs(np.vdot(ed.embed(Vs[:, 0], Ls, N, n_max), psi))) <= 1e-8
    # a split-TF32 eigensolve stops at a residual of ~10 u |E| (u = 2^-22), which leaves the
    # state, and so the density, correct to about 1e-6 where FP64 gives 1e-9
    dtol = 1e-7 if precision == 0 else 1e-5
    n = mps.density()
    assert np.abs(n - n_ref).max() < dtol and abs(n.sum() - N) < 1e-9
    assert np.abs(n - n[::-1]).max() < dtol
    assert n[0] < 0.05 and n[Ls // 2] > 1.5  # empty edges, doubly occupied centre
    Eu = dm.update_energies()  # the last sweep's 2(L - 1) updates, the last one its E
    assert len(Eu) == 2 * (Ls - 1) and Eu[-1] == E[-1]
    # a sweep ends moving left: every site but the first is right-canonical
    for B in mps.tensors()[1:]:
        Bm = B.reshape(B.shape[0], -1)
        assert np.abs(Bm @ Bm.conj().T - np.eye(B.shape[0])).max() < 1e-10


def _golden(name):
    vals = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = float(v)
    return vals


@pytest.mark.parametrize("precision", [0, 1])
def test_e1_first_sweep_matches_oracle(ctx, precision):
    """The first sweep of E1 at the paper's size from the seeded start, against the FP64
    oracle's first sweep from the same start (tests/golden/e1_trap_sweep0.txt, written by
    tests/golden/make_e1_sweep0.py), update by update.  Same algorithm and truncation on
    both sides, but from a random start at chi = 100 every cut falls among near-equal
    Schmidt values (a random state's spectrum is flat), so rounding decides part of the
    kept subspace: the two runs agree to 1e-6 for the first hundred updates and drift to a
    few 1e-6 by the end of the sweep.  Every update is compared at 1e-5 (a defective update,
    like the former non-orthonormal eigenvectors, is off by far more); 1e-10 parity of the
    trapped Hamiltonian at convergence is held by the ten-site test above."""
    from paper_1610_02244_gb300 import tnt
    ref = _golden("e1_trap_sweep0.txt")["E_sweep0"]
    Ls, N, n_max, J, U, V = 100, 100, 3, 1.0, 5.0, 0.01
    A, q = synth.random_charged_mps(synth.rng(4), Ls, n_max + 1, N, 100, "gauss", 2.0)
    ctx.set_params(chi_max=100, precision=precision)
    try:
        mps = ctx.mps_create(A, q, chi_cap=100)
        mpo = ctx.mpo_bose_hubbard(Ls, n_max, J, U, 0.0, V, (Ls + 1) / 2.0)
        dm = ctx.dmrg_create(mps, mpo)
        E = dm.sweep()["E"]
        Eu = dm.update_energies()
    finally:
        ctx.set_params(chi_max=1 << 40, precision=tnt.TNT_PREC_FP64)
    g = _golden("e1_trap_sweep0.txt")
    Eu_ref = np.array([g[f"E_u{k:03d}"] for k in range(2 * (Ls - 1))])
    assert len(Eu) == len(Eu_ref) and Eu[-1] == E
    off = np.abs(Eu - Eu_ref) > 1e-5 * np.abs(Eu_ref)
    first = int(np.argmax(off)) if off.any() else -1  # first update off the oracle
    assert first == -1, (first, Eu[first], Eu_ref[first])
    assert abs(E - ref) <= 1e-5 * abs(ref), (E, ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_e1_trapped_bosons_L100(ctx, precision):
    """E1 at the paper's size (L = N = 100, n_max = 3, U/J = 5, V/J = 0.01, chi = 100) from
    the seeded random start, swept until successive sweep energies differ by less than 1e-4
    (the paper's default DMRG precision, Sec. 5), at most 24 sweeps: the energy falls
    monotonically, the trap pulls the bosons to the centre (Fig. 4(b)), and the density
    matrix is Hermitian with the density on its diagonal."""
    from paper_1610_02244_gb300 import tnt
    Ls, N, n_max, J, U, V = 100, 100, 3, 1.0, 5.0, 0.01
    j_c = (Ls + 1) / 2.0  # sites are numbered 1..L in the trap term of Eq. 2
    g = synth.rng(4)
    A, q = synth.random_charged_mps(g, Ls, n_max + 1, N, 100, "gauss", 2.0)
    ctx.set_params(chi_max=100, precision=precision)
    try:
        mps = ctx.mps_create(A, q, chi_cap=100)
        mpo = ctx.mpo_bose_hubbard(Ls, n_max, J, U, 0.0, V, j_c)
        dm = ctx.dmrg_create(mps, mpo)
        E = [dm.sweep()["E"], dm.sweep()["E"]]
        while abs(E[-1] - E[-2]) > 1e-4 and len(E) < 24:
            E.append(dm.sweep()["E"])
    finally:
        ctx.set_params(chi_max=1 << 40, precision=tnt.TNT_PREC_FP64)
    assert all(b <= a + 1e-8 * abs(a) for a, b in zip(E, E[1:])), E
    assert abs(E[-1] - E[-2]) <= 1e-4, E
    assert abs(mps.expect_mpo(mpo) - E[-1]) <= 1e-8 * abs(E[-1])
    n = mps.density()
    rho = mps.bdagb()
    assert abs(n.sum() - N) < 1e-9
    assert np.abs(n - n[::-1]).max() < 1e-4  # the trap is symmetric about the centre
    assert np.abs(np.diag(rho).real - n).max() < 1e-10
    assert np.abs(rho - rho.conj().T).max() < 1e-10
    # the trap pulls the bosons to the centre: the edges are depleted
    assert n[Ls // 2] > n[0] and n[Ls // 2] > n[-1]
