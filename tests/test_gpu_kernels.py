"""GPU parity of the two-site kernels against the FP64 CPU oracle, through the C-ABI.

Shapes span several GEMM tiles (64) and ragged tails; the full cfg2 matvec shape
(chi = 256, d = 4, D = 4) is compared element by element in FP64.  Tolerances:
FP64 paths 1e-12 relative to max|y| (rounding of K ~ 1e3 complex FMAs); the split-TF32
path 2e-5 (operands carry 22 mantissa bits, FP32 accumulation over K <= 1024)."""
import numpy as np
import pytest
import torch

from oracle import bose_hubbard as bh
from oracle import contract as oc
from oracle import lanczos as olz
from oracle import svd as osvd
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


def heff_inputs(seed, chl, d, chr_, D=4, U=2.0):
    g = synth.rng(seed)
    Ws, _, _ = bh.bh_mpo(4, d - 1, 1.0, U)
    Le = synth.hermitian_env(g, chl, D)
    Re = synth.hermitian_env(g, chr_, D)
    th = synth.complex_gaussian(g, (chl, d, d, chr_))
    return Le, Ws[1], Ws[2], Re, th


SHAPES = [(1, 2, 1), (5, 3, 7), (67, 4, 45), (130, 5, 64), (64, 2, 129)]


@pytest.mark.parametrize("chl,d,chr_", SHAPES)
def test_heff_fp64(ctx, chl, d, chr_):
    Le, W1, W2, Re, th = heff_inputs(chl + d + chr_, chl, d, chr_)
    y = ctx.heff_apply(dev(Le), dev(W1), dev(W2), dev(Re), dev(th)).cpu().numpy()
    assert rel(y, oc.heff_apply(Le, W1, W2, Re, th)) < FP64_TOL


def test_heff_fp64_cfg2_full(ctx):
    """The micro-benchmark shape: L, R 256x4x256, W 4x4x4x4, theta 256x4x4x256."""
    Le, W1, W2, Re, th = heff_inputs(0, 256, 4, 256)
    y = ctx.heff_apply(dev(Le), dev(W1), dev(W2), dev(Re), dev(th)).cpu().numpy()
    assert rel(y, oc.heff_apply(Le, W1, W2, Re, th)) < FP64_TOL


@pytest.mark.parametrize("chl,d,chr_", SHAPES + [(256, 4, 256)])
def test_heff_mixed(ctx, chl, d, chr_):
    from paper_1610_02244_gb300 import tnt
    Le, W1, W2, Re, th = heff_inputs(100 + chl, chl, d, chr_)
    y = ctx.heff_apply(dev(Le), dev(W1), dev(W2), dev(Re), dev(th),
                       precision=tnt.TNT_PREC_MIXED).cpu().numpy()
    assert rel(y, oc.heff_apply(Le, W1, W2, Re, th)) < MIXED_TOL


def test_heff_zero_and_sector_preserving(ctx):
    """Exact zeros stay exact zeros: a theta confined to one charge sector with block
    sparse environments gives a result confined to the same sector (both precisions)."""
    from paper_1610_02244_gb300 import tnt
    Le, W1, W2, Re, th = heff_inputs(5, 9, 3, 9)
    th[:, 1:, :, :] = 0
    y_ref = oc.heff_apply(Le, W1, W2, Re, th)
    for prec in (tnt.TNT_PREC_FP64, tnt.TNT_PREC_MIXED):
        y = ctx.heff_apply(dev(Le), dev(W1), dev(W2), dev(Re), dev(th), precision=prec)
        y = y.cpu().numpy()
        assert np.all((y == 0) == (y_ref == 0)) or rel(y, y_ref) < MIXED_TOL


@pytest.mark.parametrize("chl,d,chm,chr_", [(3, 2, 4, 5), (70, 4, 66, 33), (256, 4, 256, 256)])
def test_theta_form(ctx, chl, d, chm, chr_):
    g = synth.rng(chl + chm)
    A = synth.complex_gaussian(g, (chl, d, chm))
    B = synth.complex_gaussian(g, (chm, d, chr_))
    th = ctx.theta_form(dev(A), dev(B)).cpu().numpy()
    assert rel(th, oc.theta_form(A, B)) < FP64_TOL


@pytest.mark.parametrize("n_max,chl,chr_", [(4, 17, 33), (1, 64, 65), (3, 5, 1)])
def test_gate_apply(ctx, n_max, chl, chr_):
    from paper_1610_02244_gb300 import tnt
    d = n_max + 1
    G = tnt.bh_bond_gate(n_max, 1.0, 2.0, 0.0, 0.5, 0.5, 0.01)
    g = synth.rng(chl)
    th = synth.complex_gaussian(g, (chl, d, d, chr_))
    out = ctx.gate_apply(dev(G), dev(th)).cpu().numpy()
    Gr = bh.gate(bh.bond_hamiltonian(n_max, 1.0, 2.0, 0.5, 0.5), 0.01)
    assert rel(out, oc.gate_apply(Gr, th)) < FP64_TOL


@pytest.mark.parametrize("chl,d,chr_", [(1, 4, 4), (13, 3, 17), (96, 4, 70), (256, 4, 256)])
def test_environments(ctx, chl, d, chr_):
    g = synth.rng(chl * 7 + chr_)
    Ws, _, _ = bh.bh_mpo(4, d - 1, 0.8, 1.7, 0.2)
    A = synth.complex_gaussian(g, (chl, d, chr_))
    Le = synth.complex_gaussian(g, (chl, 4, chl))
    Re = synth.complex_gaussian(g, (chr_, 4, chr_))
    Lo = ctx.env_left(dev(Le), dev(Ws[2]), dev(A)).cpu().numpy()
    assert rel(Lo, oc.env_left(Le, Ws[2], A)) < FP64_TOL
    Ro = ctx.env_right(dev(Re), dev(Ws[2]), dev(A)).cpu().numpy()
    assert rel(Ro, oc.env_right(Re, Ws[2], A)) < FP64_TOL


@pytest.mark.parametrize("chl,d,chr_", [(6, 3, 6), (12, 4, 10), (14, 3, 20)])
def test_lanczos_fp64_matches_dense_eigh(ctx, chl, d, chr_):
    Le, W1, W2, Re, th = heff_inputs(3 * chl + chr_, chl, d, chr_)
    H = oc.heff_dense(Le, W1, W2, Re)
    w, v = np.linalg.eigh(H)
    t = dev(th)
    res = ctx.lanczos_ground(dev(Le), dev(W1), dev(W2), dev(Re), t)
    x = t.cpu().numpy().reshape(-1)
    assert abs(res["E"] - w[0]) <= 1e-10 * abs(w[0])
    gap = w[1] - w[0]
    if gap > 1e-3 * abs(w[0]):
        assert abs(1 - abs(np.vdot(v[:, 0], x))) < 1e-8
    # the oracle's own Lanczos on the same start vector
    Eo, _, _, _, _ = olz.lanczos_ground(lambda z: oc.heff_apply(Le, W1, W2, Re, z), th)
    assert abs(res["E"] - Eo) <= 1e-10 * abs(Eo)


def test_lanczos_mixed_energy_within_1e10(ctx):
    """The split-TF32 eigensolve (the smallest size that runs split TF32: 65536 entries)
    on environments with the channel structure of a DMRG state: its FP64 Rayleigh quotient
    against the FP64 oracle Lanczos to 1e-10, its vector to 1e-8 in overlap."""
    from paper_1610_02244_gb300 import tnt
    chl, d, chr_ = 64, 4, 64
    g = synth.rng(77)
    Ws, _, _ = bh.bh_mpo(4, d - 1, 1.0, 2.0)
    Le, Re = synth.block_env(g, chl, "left"), synth.block_env(g, chr_, "right")
    th = synth.complex_gaussian(g, (chl, d, d, chr_))
    E_ref, x_ref, _, _, conv = olz.lanczos_ground(lambda v: oc.heff_apply(Le, Ws[1], Ws[2], Re, v), th)
    assert conv
    ctx.set_params(precision=tnt.TNT_PREC_MIXED)
    try:
        x = dev(th)
        res = ctx.lanczos_ground(dev(Le), dev(Ws[1]), dev(Ws[2]), dev(Re), x)
    finally:
        ctx.set_params(precision=tnt.TNT_PREC_FP64)
    assert abs(res["E_rq"] - E_ref) <= 1e-10 * abs(E_ref)
    xv = x.cpu().numpy().reshape(-1)
    assert abs(1 - abs(np.vdot(x_ref.reshape(-1), xv)) / np.linalg.norm(xv)) <= 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_lanczos_cfg2_full_size(ctx, precision):
    """The micro-benchmark shape (chi = 256, d = 4, D = 4; |theta| = 2^20) with 12 Krylov
    steps.  Properties that hold at any size, checked with one oracle matvec: the
    returned vector has unit norm, its Rayleigh quotient and residual |Hx - E x| agree
    with the oracle's FP64 H_eff, and the Ritz value bounds the Rayleigh quotient."""
    Le, W1, W2, Re, th = heff_inputs(11, 256, 4, 256)
    ctx.set_params(precision=precision, krylov_cap=12, lanczos_maxit=12)
    try:
        t = dev(th)
        res = ctx.lanczos_ground(dev(Le), dev(W1), dev(W2), dev(Re), t)
    finally:
        ctx.set_params(precision=0, krylov_cap=32, lanczos_maxit=300)
    x = t.cpu().numpy()
    assert abs(np.linalg.norm(x) - 1) < 1e-12
    y = oc.heff_apply(Le, W1, W2, Re, x)
    E = np.vdot(x, y).real
    assert abs(res["E_rq"] - E) <= 1e-10 * abs(E)
    r = np.linalg.norm(y - E * x)
    assert abs(res["resid_fp64"] - r) <= 1e-8 * r
    # the Ritz value of the last Krylov step is the Rayleigh quotient of the returned
    # vector for the operator Lanczos saw (exact for FP64, within the split-TF32
    # matvec error for the mixed path)
    assert abs(res["E"] - E) <= (1e-10 if precision == 0 else 1e-5) * abs(E)


def svd_case(seed, m, n, charged):
    g = synth.rng(seed)
    M = synth.complex_gaussian(g, (m, n))
    if charged:
        rq = g.integers(0, 5, m)
        cq = g.integers(0, 5, n)
        M = M * (rq[:, None] == cq[None, :])
        return M, rq, cq
    return M, np.zeros(m, np.int64), np.zeros(n, np.int64)


@pytest.mark.parametrize("m,n,charged,side", [
    (40, 30, False, 0), (30, 40, False, 1), (100, 90, True, 0), (90, 100, True, 1),
    (200, 160, False, 0), (160, 200, False, 1), (8, 8, True, 1), (1, 7, False, 0),
    (420, 390, True, 0), (390, 420, True, 1), (65, 300, False, 0)])
def test_svd_trunc_matches_oracle(ctx, m, n, charged, side):
    M, rq, cq = svd_case(m * n + side, m, n, charged)
    chi_max = max(1, min(m, n) * 2 // 3)
    ctx.set_params(chi_max=chi_max, trunc_err=1e-8, trunc_rel=1e-16)
    try:
        U, X, S, bq, info = ctx.svd_trunc(dev(M), rq, cq, side=side)
    finally:
        ctx.set_params(chi_max=1 << 40)
    p = osvd.TruncParams(chi_max=chi_max)
    Ur, Sr, Vr, bqr, inf_r = osvd.svd_truncate(M, rq, cq, p)
    assert info["chi"] == len(Sr)
    order = np.lexsort((-Sr, bqr))
    assert np.array_equal(bq, bqr[order])
    assert np.abs(np.sort(S) - np.sort(Sr)).max() < 1e-12 * Sr.max()
    U, X = U.cpu().numpy(), X.cpu().numpy()
    # gauge-invariant: the truncated product and orthonormality of the kept factor
    assert np.abs(U @ X - (Ur * Sr) @ Vr).max() < 1e-11 * Sr.max()
    if side == 0:
        assert np.abs(U.conj().T @ U - np.eye(len(S))).max() < 1e-12
    else:
        assert np.abs(X @ X.conj().T - np.eye(len(S))).max() < 1e-12
    assert abs(info["err"] - inf_r["err"]) <= 1e-10 * max(inf_r["err"], 1e-14)
    assert abs(info["disc"] - inf_r["disc"]) <= 1e-10 * max(inf_r["disc"], 1e-14)


def test_svd_block_beyond_shared_workspace(ctx):
    """A 2200-row Gram block: the tridiagonal reduction keeps its per-block workspace in
    global memory above 2048 rows."""
    M, _, _ = svd_case(21, 2200, 2100, False)
    ctx.set_params(chi_max=40)
    try:
        U, X, S, bq, info = ctx.svd_trunc(dev(M), None, None, side=0)
    finally:
        ctx.set_params(chi_max=1 << 40)
    s_ref = np.linalg.svd(M, compute_uv=False)
    assert info["chi"] == 40
    assert np.abs(S - s_ref[:40]).max() < 1e-11 * s_ref[0]
    U = U.cpu().numpy()
    assert np.abs(U.conj().T @ U - np.eye(40)).max() < 1e-11


def test_svd_large_block_cfg2_shape(ctx):
    """One dense 1024 x 1024 block (theta of chi = 256, d = 4) through the whole-GPU
    tridiagonal reduction, truncated to chi = 256."""
    M, rq, cq = svd_case(9, 1024, 1024, False)
    ctx.set_params(chi_max=256)
    try:
        U, X, S, bq, info = ctx.svd_trunc(dev(M), None, None, side=0, renorm=False)
    finally:
        ctx.set_params(chi_max=1 << 40)
    s_ref = np.linalg.svd(M, compute_uv=False)
    assert info["chi"] == 256
    assert np.abs(S - s_ref[:256]).max() < 1e-11 * s_ref[0]
    U = U.cpu().numpy()
    assert np.abs(U.conj().T @ U - np.eye(256)).max() < 1e-11
    assert abs(info["disc"] - np.sum(s_ref[256:] ** 2)) < 1e-10 * np.sum(s_ref ** 2)


@pytest.mark.parametrize("side", [0, 1])
def test_svd_zero_charge_blocks(ctx, side):
    """Charge blocks with no weight (a sector of theta a gate has not reached): a 40 x 30
    one and a 200 x 210 one (one CTA per block) and a zero 1 x 1 block.  Their
    values are exact zeros and never kept; the weighted block comes out as the oracle's."""
    g = np.random.default_rng(31)
    rq = np.repeat([0, 1, 2, 3], [40, 200, 1, 120])
    cq = np.repeat([0, 1, 2, 3], [30, 210, 1, 100])
    M = np.zeros((len(rq), len(cq)), dtype=np.complex128)
    blk = (rq[:, None] == 3) & (cq[None, :] == 3)
    M[blk] = (g.normal(size=blk.sum()) + 1j * g.normal(size=blk.sum()))
    ctx.set_params(chi_max=150, trunc_err=1e-8, trunc_rel=1e-16)
    try:
        U, X, S, bq, info = ctx.svd_trunc(dev(M), rq, cq, side=side)
    finally:
        ctx.set_params(chi_max=1 << 40)
    Ur, Sr, Vr, bqr, _ = osvd.svd_truncate(M, rq, cq, osvd.TruncParams(chi_max=150))
    assert info["chi"] == len(Sr) == 100 and np.all(bq == 3)
    assert np.abs(np.sort(S) - np.sort(Sr)).max() < 1e-12 * Sr.max()
    U, X = U.cpu().numpy(), X.cpu().numpy()
    assert np.isfinite(U).all() and np.isfinite(X).all()
    assert np.abs(U @ X - M).max() < 1e-11 * Sr.max()


def low_rank_block(g, m, n, sigmas):
    """m x n complex block U diag(sigmas) V^H with Haar-like orthonormal U, V."""
    r = len(sigmas)
    qu, _ = np.linalg.qr(g.normal(size=(m, r)) + 1j * g.normal(size=(m, r)))
    qv, _ = np.linalg.qr(g.normal(size=(n, r)) + 1j * g.normal(size=(n, r)))
    return (qu * np.asarray(sigmas)) @ qv.conj().T


@pytest.mark.parametrize("side", [0, 1])
def test_svd_rank_deficient_blocks(ctx, side):
    """Charge blocks whose rank is below their candidate count and whose spectra fall
    geometrically to far below the Gram matrix's rounding level, the shape of theta early
    in a quench from a product state (Sec. 5) and of any converged DMRG bond: 99 x 64 of
    rank 40 (sigma 1 .. 1e-22), 120 x 110 of rank 30, 30 x 20 of rank 5, a 10 x 12 block
    of weight 1e-170 (its Gram entries would underflow unscaled) and a 300 x 280 block of
    rank 100 (the whole-GPU reduction).  With chi_max = 512 and the 1e-10 truncation error
    of the 64-site quench, the kept factor must be orthonormal to rounding, every singular
    value above 1e-6 must match the oracle's to 1e-12, and the truncated product must be
    within the truncation error of M.  (A value sigma reaches the Gram matrix as sigma^2: at
    1e-6 that is 1e-12 |G|, resolved to about eps / 1e-12 in angle; near 1e-8 it meets the
    rounding level of the Gram matrix, and such values are compared through the product
    only.)"""
    g = np.random.default_rng(1610 + side)
    spec = [(99, 64, np.geomspace(1.0, 1e-22, 40)), (120, 110, np.geomspace(0.5, 1e-14, 30)),
            (30, 20, np.geomspace(1e-3, 1e-9, 5)), (10, 12, 1e-170 * np.geomspace(1, 1e-3, 10)),
            (300, 280, np.geomspace(0.8, 1e-20, 100))]
    m = sum(s[0] for s in spec)
    n = sum(s[1] for s in spec)
    M = np.zeros((m, n), np.complex128)
    rq = np.zeros(m, np.int64)
    cq = np.zeros(n, np.int64)
    r0 = c0 = 0
    for q, (bm, bn, sig) in enumerate(spec):
        M[r0:r0 + bm, c0:c0 + bn] = low_rank_block(g, bm, bn, sig)
        rq[r0:r0 + bm] = q
        cq[c0:c0 + bn] = q
        r0 += bm
        c0 += bn
    pr, pc = g.permutation(m), g.permutation(n)
    M, rq, cq = M[pr][:, pc], rq[pr], cq[pc]
    ctx.set_params(chi_max=512, trunc_err=1e-10, trunc_rel=1e-16)
    try:
        U, X, S, bq, info = ctx.svd_trunc(dev(M), rq, cq, side=side)
    finally:
        ctx.set_params(chi_max=1 << 40, trunc_err=1e-8)
    Ur, Sr, Vr, bqr, inf_r = osvd.svd_truncate(M, rq, cq, osvd.TruncParams(chi_max=512,
                                                                              err_tol=1e-10))
    U, X = U.cpu().numpy(), X.cpu().numpy()
    assert np.isfinite(S).all() and np.isfinite(U).all() and np.isfinite(X).all()
    k = len(S)
    if side == 0:
        assert np.abs(U.conj().T @ U - np.eye(k)).max() < 1e-12
    else:
        assert np.abs(X @ X.conj().T - np.eye(k)).max() < 1e-12
    big = np.sort(Sr[Sr > 1e-6])[::-1]
    assert np.abs(np.sort(S)[::-1][:len(big)] - big).max() < 1e-12
    assert info["err"] < 1e-10
    assert np.linalg.norm(U @ X - M) < 3e-10 * np.linalg.norm(M)
    # every kept value belongs to a block that holds it: labels agree where values are resolved
    for q in range(len(spec)):
        sq = np.sort(S[bq == q])[::-1]
        rr = np.sort(Sr[(bqr == q) & (Sr > 1e-6)])[::-1]
        assert np.abs(sq[:len(rr)] - rr).max(initial=0) < 1e-12


@pytest.mark.parametrize("side", [0, 1])
def test_svd_automatic_blocking(ctx, side):
    """Automatic blocking (Sec. 6): a block-diagonal matrix with rows and columns shuffled
    and 1e-12 noise everywhere; with the zeroing tolerance 1e-9 the GPU finds the four
    planted blocks and truncates like the oracle's block-wise SVD of the zeroed matrix.
    With the tolerance off, the same call is one dense block."""
    from tests.test_oracle_autoblock import planted
    M, rows, cols = planted(7, [40, 90, 7, 130], [35, 80, 9, 120])
    chi_max = 150
    p = osvd.TruncParams(chi_max=chi_max)
    Ur, Sr, Vr, bqr, inf_r = osvd.svd_truncate_auto(M, 1e-9, p)
    Mz, _, _ = osvd.autoblock(M, 1e-9)
    ctx.set_params(chi_max=chi_max, trunc_err=1e-8, trunc_rel=1e-16)
    ctx.set_svd_zero_tol(1e-9)
    try:
        U, X, S, bq, info = ctx.svd_trunc(dev(M), None, None, side=side)
    finally:
        ctx.set_svd_zero_tol(-1)
        ctx.set_params(chi_max=1 << 40)
    assert info["n_blocks"] == 4
    assert info["chi"] == len(Sr)
    assert np.abs(np.sort(S) - np.sort(Sr)).max() < 1e-12 * Sr.max()
    # bond labels: the oracle's component numbers (same numbering rule), values per block
    for q in set(bqr.tolist()):
        assert np.abs(np.sort(S[bq == q]) - np.sort(Sr[bqr == q])).max() < 1e-12 * Sr.max()
    U, X = U.cpu().numpy(), X.cpu().numpy()
    assert np.abs(U @ X - (Ur * Sr) @ Vr).max() < 1e-11 * Sr.max()
    # off: one dense block of the unzeroed matrix
    ctx.set_params(chi_max=chi_max, trunc_err=1e-8, trunc_rel=1e-16)
    try:
        _, _, S2, _, info2 = ctx.svd_trunc(dev(M), None, None, side=side)
    finally:
        ctx.set_params(chi_max=1 << 40)
    assert info2["n_blocks"] == 1
    _, Sd, _, _, _ = osvd.svd_truncate(M, np.zeros(M.shape[0], np.int64), np.zeros(M.shape[1], np.int64), p)
    assert np.abs(np.sort(S2) - np.sort(Sd)).max() < 1e-12 * Sd.max()
