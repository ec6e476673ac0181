"""Grouped U(1) block-sparse H_eff.theta and its Lanczos solve on the GPU against the FP64
oracle, through the C-ABI.

The oracle contracts the dense, masked tensors (Sec. 4.2 Listing 1 order): with U(1)
labels (App. A.1.1) every entry outside the allowed blocks of L, R and theta is zero, so
the dense result restricted to the blocks is the block-sparse result, and is zero outside
them.  The GPU side packs theta into its compact block layout, runs every block of every
problem in grouped launches, and unpacks.  Tolerances as for the dense kernels: FP64 1e-12
and split TF32 2e-5, relative to max|y|."""
import numpy as np
import pytest
import torch

from oracle import bose_hubbard as bh
from oracle import contract as oc
from oracle import lanczos as olz
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def u1_inputs(seed, qa, qb, d, U=2.0, J=1.0):
    g = synth.rng(seed)
    Ws, _, _ = bh.bh_mpo(4, d - 1, J, U)
    Le = synth.hermitian_env(g, len(qa)) * synth.env_mask(qa, qa)
    Re = synth.hermitian_env(g, len(qb)) * synth.env_mask(qb, qb)
    th = synth.complex_gaussian(g, (len(qa), d, d, len(qb))) * synth.theta_mask(qa, d, qb)
    return Le, Ws[1], Ws[2], Re, th


def problem(Le, W1, W2, Re, qa, qb):
    from paper_1610_02244_gb300 import tnt
    return tnt.U1Problem(dev(Le), dev(W1), dev(W2), dev(Re), qa, qb, synth.BH_WQ)


LABELS = {
    "small": (np.array([0, 0, 1, 1, 1, 2]), np.array([1, 2, 2, 3, 3, 3, 4, 4]), 3),
    "gaps": (np.array([0, 2, 2, 5]), np.array([3, 3, 4, 7, 7, 7, 9]), 3),
    "one_sector": (np.array([4] * 9), np.array([6] * 11), 3),
    "gauss96": (synth.gaussian_sector_labels(96, 7, 1.5, 10),
                synth.gaussian_sector_labels(130, 9, 2.0, 12), 4),
    "gauss_cfg3_profile": (synth.gaussian_sector_labels(256, 15, 2.0, 32),
                           synth.gaussian_sector_labels(256, 15, 2.0, 34), 5),
}


def test_sector_profile_shape():
    q = synth.gaussian_sector_labels(1024, 15, 2.0, 32)
    sizes = np.bincount(q - q.min())
    assert len(q) == 1024 and np.all(np.diff(q) >= 0)
    assert len(sizes) == 15 and sizes.min() >= 1 and 150 <= sizes.max() <= 220


@pytest.mark.parametrize("name", list(LABELS))
def test_pack_roundtrip_and_size(ctx, name):
    qa, qb, d = LABELS[name]
    Le, W1, W2, Re, th = u1_inputs(1, qa, qb, d)
    p = problem(Le, W1, W2, Re, qa, qb)
    n = ctx.u1_size(p)
    assert n == int(synth.theta_mask(qa, d, qb).sum())
    x = ctx.u1_pack(p, dev(th))
    back = ctx.u1_unpack(p, x).cpu().numpy()
    assert np.array_equal(back, th)  # bit-exact: integer index work only


@pytest.mark.parametrize("name", list(LABELS))
@pytest.mark.parametrize("precision", [0, 1])
def test_heff_u1_matches_oracle(ctx, name, precision):
    qa, qb, d = LABELS[name]
    Le, W1, W2, Re, th = u1_inputs(7, qa, qb, d)
    p = problem(Le, W1, W2, Re, qa, qb)
    x = ctx.u1_pack(p, dev(th))
    y, flops = ctx.heff_apply_u1([p], x, precision=precision)
    got = ctx.u1_unpack(p, y).cpu().numpy()
    ref = oc.heff_apply(Le, W1, W2, Re, th)
    assert rel(got, ref) < (FP64_TOL if precision == 0 else MIXED_TOL)
    # the oracle's result has no weight outside the blocks (charge conservation)
    assert np.abs(ref * ~synth.theta_mask(qa, d, qb)).max() <= 1e-12 * np.abs(ref).max()
    dense = 8.0 * (4 * len(qa) * d * d * len(qb) * len(qa) + len(qa) * d * d * len(qb) * 4 * len(qb))
    assert 0 < flops < dense + 8.0 * len(qa) * len(qb) * 16 * d ** 4


def test_heff_u1_batched_chains(ctx):
    """Three chains with different U / J and block structures in one grouped call."""
    cases = [(LABELS["small"], 1.0, 1.0), (LABELS["gauss96"], 3.4, 1.0), (LABELS["gaps"], 8.0, 0.5)]
    probs, refs, xs = [], [], []
    for i, ((qa, qb, d), U, J) in enumerate(cases):
        Le, W1, W2, Re, th = u1_inputs(20 + i, qa, qb, d, U=U, J=J)
        p = problem(Le, W1, W2, Re, qa, qb)
        probs.append(p)
        xs.append(ctx.u1_pack(p, dev(th)))
        refs.append(oc.heff_apply(Le, W1, W2, Re, th))
    x = torch.cat(xs)
    for precision, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        y, _ = ctx.heff_apply_u1(probs, x, precision=precision)
        off = 0
        for p, ref, xi in zip(probs, refs, xs):
            got = ctx.u1_unpack(p, y[off: off + xi.numel()]).cpu().numpy()
            off += xi.numel()
            assert rel(got, ref) < tol
    t = ctx.u1_tiles(probs)
    assert t[0] in (64, 128) and t[1] in (64, 128) and t[2] in (1, 2, 4)


def test_graph_replay_equals_plain_launches(ctx):
    qa, qb, d = LABELS["gauss96"]
    Le, W1, W2, Re, th = u1_inputs(3, qa, qb, d)
    p = problem(Le, W1, W2, Re, qa, qb)
    x = ctx.u1_pack(p, dev(th))
    for precision in (0, 1):
        ctx.set_graphs(True)
        y1, _ = ctx.heff_apply_u1([p], x, precision=precision)
        ctx.set_graphs(False)
        y2, _ = ctx.heff_apply_u1([p], x, precision=precision)
        ctx.set_graphs(True)
        assert torch.equal(y1, y2)


@pytest.mark.parametrize("precision", [0, 1])
def test_lanczos_u1_matches_oracle(ctx, precision):
    """Ground state of the block-sparse H_eff: |dE| <= 1e-10 |E| for both paths (the mixed
    one through its FP64 win-back), and the same ground vector."""
    qa, qb, d = LABELS["gauss96"]
    Le, W1, W2, Re, th = u1_inputs(11, qa, qb, d)
    ctx.set_params(precision=precision, lanczos_tol=1e-12, lanczos_maxit=300, krylov_cap=32)
    p = problem(Le, W1, W2, Re, qa, qb)
    x = ctx.u1_pack(p, dev(th))
    res = ctx.lanczos_ground_u1(p, x)
    ctx.set_params(precision=0)
    E, v, *_ = olz.lanczos_ground(lambda t: oc.heff_apply(Le, W1, W2, Re, t), th)
    assert abs(res["E_rq"] - E) <= 1e-10 * abs(E)
    got = ctx.u1_unpack(p, x).cpu().numpy()
    assert abs(np.linalg.norm(got) - 1) < 1e-12
    assert abs(1 - abs(np.vdot(v.ravel() / np.linalg.norm(v), got.ravel()))) < 1e-8


def test_u1_rejects_unsorted_labels(ctx):
    from paper_1610_02244_gb300 import tnt
    qa, qb, d = LABELS["small"]
    Le, W1, W2, Re, th = u1_inputs(1, qa, qb, d)
    p = problem(Le, W1, W2, Re, qa[::-1].copy(), qb)
    with pytest.raises(tnt.TntError):
        ctx.u1_size(p)


@pytest.mark.parametrize("precision", [0, 1])
def test_lanczos_u1_batched_chains(ctx, precision):
    """Independent chains (different U, J and block structures) solved in lock step, one
    grouped matvec per Krylov step: each ground state as the oracle's, to 1e-10 in E."""
    cases = [(LABELS["gauss96"], 3.4, 1.0), (LABELS["small"], 1.0, 1.0),
             (LABELS["gauss96"], 8.0, 0.7), (LABELS["gaps"], 2.0, 1.0)]
    ctx.set_params(precision=precision, lanczos_tol=1e-12, lanczos_maxit=300, krylov_cap=32)
    probs, xs, refs, cases_inputs = [], [], [], []
    for i, ((qa, qb, d), U, J) in enumerate(cases):
        Le, W1, W2, Re, th = u1_inputs(40 + i, qa, qb, d, U=U, J=J)
        cases_inputs.append((Le, W1, W2, Re))
        p = problem(Le, W1, W2, Re, qa, qb)
        probs.append(p)
        xs.append(ctx.u1_pack(p, dev(th)))
        refs.append(olz.lanczos_ground(lambda t, a=(Le, W1, W2, Re): oc.heff_apply(*a, t), th))
    x = torch.cat(xs)
    res = ctx.lanczos_ground_u1_batched(probs, x)
    ctx.set_params(precision=0)
    off = 0
    for i, (p, xi, (E, v, *_), r) in enumerate(zip(probs, xs, refs, res)):
        assert r["converged"] == 1
        assert abs(r["E_rq"] - E) <= 1e-10 * abs(E), (r, E)
        got = ctx.u1_unpack(p, x[off: off + xi.numel()]).cpu().numpy()
        off += xi.numel()
        assert abs(np.linalg.norm(got) - 1) < 1e-12
        ov = abs(np.vdot(v.ravel() / np.linalg.norm(v), got.ravel()))
        if precision == 0:
            assert abs(1 - ov) < 1e-8
        else:
            # the split-TF32 solve promises |dE| <= 1e-10 |E| through an FP64 residual
            # check ||H x - E x|| <= 1e-5 |E|; the vector is as good as that residual allows
            # (1 - overlap ~ (residual / gap)^2 / 2): check the promise with the oracle
            Le_, W1_, W2_, Re_ = cases_inputs[i]
            Hx = oc.heff_apply(Le_, W1_, W2_, Re_, got)
            assert np.linalg.norm(Hx - r["E_rq"] * got) <= 1e-5 * abs(E)
            assert abs(1 - ov) < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_heff_u1_chi1024_sampled_rows(ctx, precision):
    """The U(1) matvec at the size the U(1) benchmark times (chi = 1024 on both bonds, d = 5,
    15 Gaussian sectors of 1..~200 states, U/J = 3.4): the whole product on the GPU, and
    rows a' of it recomputed one by one by the oracle (the contraction with L restricted to
    one bra index a' is the same formula), in four different left sectors."""
    d, chi = 5, 1024
    qa = synth.gaussian_sector_labels(chi, 15, 2.0, 31)
    qb = synth.gaussian_sector_labels(chi, 15, 2.0, 33)
    g = synth.rng(2000)
    Le = synth.hermitian_env(g, chi) * synth.env_mask(qa, qa)
    Re = synth.hermitian_env(g, chi) * synth.env_mask(qb, qb)
    Ws, _, _ = bh.bh_mpo(4, d - 1, 1.0, 3.4)
    W = Ws[1]
    mask = synth.theta_mask(qa, d, qb)
    th = np.zeros(mask.shape, dtype=np.complex128)
    th[mask] = synth.complex_gaussian(g, (int(mask.sum()),))
    p = problem(Le, W, W, Re, qa, qb)
    x = ctx.u1_pack(p, dev(th))
    y, _ = ctx.heff_apply_u1([p], x, precision=precision)
    rows = [0, 300, 511, 1023]
    got = ctx.u1_unpack(p, y)[rows].cpu().numpy()
    ref = np.concatenate([oc.heff_apply(Le[a:a + 1], W, W, Re, th) for a in rows])
    assert rel(got, ref) < (FP64_TOL if precision == 0 else MIXED_TOL)
    assert len(set(qa[rows])) == 4


def _trapped_chain_bonds(bonds):
    """Environments of the 100-site trapped chain of the first example (N = 100, n_max = 3,
    U/J = 5, V/J = 0.01) for its seeded Gaussian-profile start at chi = 100: right-canonical
    by the oracle's exact moves, then the centre moved right by exact SVDs; per bond i the
    problem (L_i, W_i, W_{i+1}, R_{i+2}, theta = A_i A_{i+1}, labels)."""
    from oracle import dmrg as odmrg
    from oracle.svd import svd_truncate
    Ls, N, n_max = 100, 100, 3
    d = n_max + 1
    A, q = synth.random_charged_mps(synth.rng(4), Ls, d, N, 100, "gauss", 2.0)
    Ws, l, r = bh.bh_mpo(Ls, n_max, 1.0, 5.0, 0.0, 0.01, (Ls + 1) / 2.0)
    odmrg.right_canonicalize(A, q)
    Renv = odmrg.build_right_envs(A, Ws, r)
    Lenv = [oc.boundary_left(l)]
    out = {}
    for j in range(max(bonds) + 1):
        if j in bonds:
            out[j] = (Lenv[j], Ws[j], Ws[j + 1], Renv[j + 2], oc.theta_form(A[j], A[j + 1]),
                      q[j].copy(), q[j + 2].copy())
        chl, _, chr_ = A[j].shape
        rows = (q[j][:, None] + np.arange(d)[None, :]).reshape(-1)
        U, S, Vh, bq, _ = svd_truncate(A[j].reshape(chl * d, chr_), rows, q[j + 1], odmrg.EXACT)
        A[j] = U.reshape(chl, d, len(S))
        A[j + 1] = np.einsum("km,msb->ksb", S[:, None] * Vh, A[j + 1])
        q[j + 1] = bq
        Lenv.append(oc.env_left(Lenv[j], Ws[j], A[j]))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_heff_u1_trapped_chain_bonds(ctx, precision):
    """The U(1) matvec on bonds 12, 30 and 50 of the trapped chain of the first example, with
    its site-dependent MPO tensors and environments whose entries reach several hundred
    (the trap energy accumulated along the chain), against the oracle's dense contraction.
    The split-TF32 tolerance is tight: the same contraction done in exact split-TF32
    arithmetic (operands rounded to TF32 and split in two, three products, FP32
    accumulation) errs by 1.0-1.8e-7 of max|y| on these bonds, so 2e-6 separates rounding
    from a block handled wrongly."""
    for i, (Le, W1, W2, Re, th, qa, qb) in _trapped_chain_bonds([12, 30, 50]).items():
        from paper_1610_02244_gb300 import tnt
        p = tnt.U1Problem(dev(Le), dev(W1), dev(W2), dev(Re), qa, qb, synth.BH_WQ)
        x = ctx.u1_pack(p, dev(th))
        y, _ = ctx.heff_apply_u1([p], x, precision=precision)
        got = ctx.u1_unpack(p, y).cpu().numpy()
        ref = oc.heff_apply(Le, W1, W2, Re, th)
        assert rel(got, ref) < (FP64_TOL if precision == 0 else 2e-6), (i, rel(got, ref))
