"""The C-ABI calls around the two-site update: MPS overlap, file output and input, setting
U(1) labels, single DMRG updates, single TEBD gates, and a context whose device memory comes
from a caller-supplied allocator (PyTorch's caching allocator).  Each is checked against the
FP64 CPU oracle or against the composite call it is a piece of."""
import numpy as np
import pytest
import torch

from oracle import bose_hubbard as bh
from oracle import contract as oc
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def test_mps_overlap_matches_oracle(ctx):
    """<a|b> of two random labelled MPS (L = 6, d = 3, N = 6) against the full state
    vectors' inner product; <a|a> against tnt_mps_norm2."""
    Ls, d, N, chi = 6, 3, 6, 7
    A, qa = synth.random_charged_mps(synth.rng(5), Ls, d, N, chi)
    B, qb = synth.random_charged_mps(synth.rng(6), Ls, d, N, chi)
    ma = ctx.mps_create(A, qa, chi_cap=chi)
    mb = ctx.mps_create(B, qb, chi_cap=chi)
    ref = np.vdot(oc.mps_to_state(A), oc.mps_to_state(B))
    got = ma.overlap(mb)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))
    assert abs(ma.overlap(ma) - ma.norm2()) <= 1e-12 * ma.norm2()
    assert abs(mb.overlap(ma) - np.conj(ref)) <= 1e-12 * max(1.0, abs(ref))


def test_mps_overlap_refuses_mismatched_chains(ctx):
    from paper_1610_02244_gb300 import tnt
    a = ctx.mps_product([1, 0, 1, 0], 2, 4)
    b = ctx.mps_product([1, 0, 1], 2, 4)
    with pytest.raises(tnt.TntError):
        a.overlap(b)


def test_mps_save_load_round_trip(ctx, tmp_path):
    """Save, then load with and without the saved parameters: same tensors, same labels,
    unit overlap, and the parameters of the saving context restored on request."""
    from paper_1610_02244_gb300 import tnt
    Ls, d, N, chi = 7, 4, 7, 9
    A, q = synth.random_charged_mps(synth.rng(8), Ls, d, N, chi)
    m = ctx.mps_create(A, q, chi_cap=chi)
    path = tmp_path / "state.tnt"
    ctx.set_params(chi_max=77, trunc_err=3e-9)
    try:
        m.save(path)
    finally:
        ctx.set_params(chi_max=1 << 40, trunc_err=1e-8)
    m2 = ctx.mps_load(path, chi_cap=chi)
    assert ctx.params()["chi_max"] == 1 << 40
    for j in range(Ls):
        assert np.array_equal(m2.site(j), A[j])
    for k in range(Ls + 1):
        assert np.array_equal(m2.charges(k), q[k])
    assert abs(m.overlap(m2) - m.norm2()) <= 1e-13 * m.norm2()
    try:
        ctx.mps_load(path, chi_cap=chi, restore_params=True)
        assert ctx.params()["chi_max"] == 77 and ctx.params()["trunc_err"] == 3e-9
    finally:
        ctx.set_params(chi_max=1 << 40, trunc_err=1e-8)
    bad = tmp_path / "not_an_mps"
    bad.write_bytes(b"hello")
    with pytest.raises(tnt.TntError):
        ctx.mps_load(bad, chi_cap=chi)
    with pytest.raises(tnt.TntError):  # a bond above the storage cap
        ctx.mps_load(path, chi_cap=2)


def test_mps_set_charges_checks_the_blocks(ctx):
    """Relabelling a bond: an equivalent labelling is accepted; one that would put non-zero
    entries of the neighbouring sites outside their blocks is refused and changes nothing."""
    from paper_1610_02244_gb300 import tnt
    m = ctx.mps_product([1, 2, 0, 1], 3, 4)  # bond labels 0, 1, 3, 3, 4
    assert list(m.charges(2)) == [3]
    m.set_charges(2, [3])
    with pytest.raises(tnt.TntError) as ei:
        m.set_charges(2, [2])
    assert "break the new labels" in str(ei.value)
    assert list(m.charges(2)) == [3]


def test_dmrg_single_updates_equal_the_sweep(ctx):
    """A sweep done as 2(L-1) single updates gives the energies of tnt_dmrg_sweep from the
    same start, update by update; an update on a bond away from the centre is refused."""
    from paper_1610_02244_gb300 import tnt
    Ls, n_max, N, chi = 6, 3, 6, 16
    A, q = synth.random_charged_mps(synth.rng(2), Ls, n_max + 1, N, chi)
    ctx.set_params(chi_max=chi, precision=tnt.TNT_PREC_FP64)
    try:
        mpo = ctx.mpo_bose_hubbard(Ls, n_max, 1.0, 2.0)
        ref = ctx.dmrg_create(ctx.mps_create(A, q, chi_cap=chi), mpo)
        ref.sweep()
        Eref = ref.update_energies()
        mps = ctx.mps_create(A, q, chi_cap=chi)
        dm = ctx.dmrg_create(mps, mpo)
        with pytest.raises(tnt.TntError):
            dm.update(3, +1)  # the centre is on site 0
        E = []
        for i in range(Ls - 1):
            lz, _ = dm.update(i, +1)
            E.append(lz["E_rq"])
        for i in range(Ls - 2, -1, -1):
            lz, _ = dm.update(i, -1)
            E.append(lz["E_rq"])
        assert np.abs(np.array(E) - Eref).max() <= 1e-12 * np.abs(Eref).max()
        dm.sweep()  # the centre is back on site 0
    finally:
        ctx.set_params(chi_max=1 << 40)


def test_tebd_single_gates_equal_the_step(ctx):
    """The first Trotter step of a quench done gate by gate (odd bonds at dt/2 ascending,
    even bonds at dt descending, odd bonds at dt/2 ascending, the order of tnt_tebd_step)
    against tnt_tebd_step from the same start: same densities and unit fidelity."""
    Ls, n_max, J, U, dt = 6, 2, 1.0, 2.0, 0.05
    d = n_max + 1
    ctx.set_params(chi_max=64, trunc_err=1e-12)
    try:
        a = ctx.mps_product([1, 0, 2, 1, 0, 1], d, 64)
        b = ctx.mps_product([1, 0, 2, 1, 0, 1], d, 64)
        ta = ctx.tebd_create(a, n_max, J, U, dt)
        ta.step()
        tb = ctx.tebd_create(b, n_max, J, U, dt)
        G = {}
        for i in range(Ls - 1):
            c1, c2 = bh.bond_weights(Ls, i + 1)
            h = bh.bond_hamiltonian(n_max, J, U, c1, c2, 0.0)
            G[i] = (bh.gate(h, dt / 2), bh.gate(h, dt))
        for i in range(0, Ls - 1, 2):
            tb.gate(i, G[i][0], +1)
        for i in reversed(range(1, Ls - 1, 2)):
            tb.gate(i, G[i][1], -1)
        for i in range(0, Ls - 1, 2):
            tb.gate(i, G[i][0], +1)
        assert tb.centre() in range(Ls)
    finally:
        ctx.set_params(chi_max=1 << 40, trunc_err=1e-8)
    assert np.abs(a.density() - b.density()).max() < 1e-12
    assert abs(abs(a.overlap(b)) - 1.0) < 1e-12


def test_context_with_caller_allocator(ctx):
    """Every device allocation of a context made with tnt_ctx_create_with_allocator goes
    through the caller's callbacks (here PyTorch's caching allocator), and its results are
    those of a default context."""
    from paper_1610_02244_gb300 import tnt
    calls = {"alloc": 0, "free": 0}
    st = torch.cuda.current_stream(0)
    alloc0, free0 = tnt.torch_allocator(0, st)

    def alloc(n):
        calls["alloc"] += 1
        return alloc0(n)

    def free(p):
        calls["free"] += 1
        free0(p)
    c2 = tnt.Context(0, allocator=(alloc, free))
    g = synth.rng(4)
    Ws, _, _ = bh.bh_mpo(4, 3, 1.0, 2.0)
    Le, Re = synth.hermitian_env(g, 40), synth.hermitian_env(g, 40)
    th = synth.complex_gaussian(g, (40, 4, 4, 40))
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")
    args = [dev(x) for x in (Le, Ws[1], Ws[2], Re, th)]
    y1 = ctx.heff_apply(*args).cpu().numpy()
    y2 = c2.heff_apply(*args).cpu().numpy()
    assert np.array_equal(y1, y2)
    A, q = synth.random_charged_mps(synth.rng(3), 6, 4, 6, 16)
    c2.set_params(chi_max=16)
    dm = c2.dmrg_create(c2.mps_create(A, q, chi_cap=16), c2.mpo_bose_hubbard(6, 3, 1.0, 2.0))
    E = dm.sweep()["E"]
    assert np.isfinite(E)
    assert calls["alloc"] > 0
    del dm
    c2.close()
    assert calls["free"] > 0
