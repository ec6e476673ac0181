"""FP64 matrix products on the GPU (the contraction-as-GEMM of App. B.1.1) through the
C-ABI, for both FP64 engines: FP64 FMA, and exact integer slices on the TF32 tensor cores.

Pins that do not depend on either implementation:
  * integer-valued operands (|entries| <= 2^10, so every partial sum is an exactly
    representable integer): the product is exact, bit for bit, in both engines;
  * random complex operands: the error against an extended-precision product (numpy
    longdouble) stays within an FP64-sized bound 32 K 2^-53 max|A_i.| max|B_.j| (the
    slice engine's worst case is 22 K 2^-53 of the same product of maxima);
  * rows spanning twelve decades: the error of small rows is measured against their own
    scale (each row is scaled separately);
  * conjugated, transposed and ragged (non-multiple-of-tile) shapes."""
import numpy as np
import pytest
import torch

from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu

ENGINES = [0, 1]  # TNT_FP64_GEMM_FMA, TNT_FP64_GEMM_TC


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def ref_product(A, B):
    """A @ B with longdouble accumulation (real and imaginary parts separately)."""
    ld = np.longdouble
    Ar, Ai = A.real.astype(ld), A.imag.astype(ld)
    Br, Bi = B.real.astype(ld), B.imag.astype(ld)
    return (Ar @ Br - Ai @ Bi), (Ar @ Bi + Ai @ Br)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("M,N,K", [(256, 384, 700), (130, 200, 1000), (1024, 512, 256)])
def test_integer_operands_exact(ctx, engine, M, N, K):
    g = synth.rng(M + N + K)
    A = (g.integers(-1024, 1025, (M, K)) + 1j * g.integers(-1024, 1025, (M, K))).astype(np.complex128)
    B = (g.integers(-1024, 1025, (K, N)) + 1j * g.integers(-1024, 1025, (K, N))).astype(np.complex128)
    ctx.set_fp64_gemm(engine)
    C = ctx.matmul(dev(A), dev(B)).cpu().numpy()
    ctx.set_fp64_gemm(1)
    Ar_, Ai_ = A.real.astype(np.int64), A.imag.astype(np.int64)
    Br_, Bi_ = B.real.astype(np.int64), B.imag.astype(np.int64)
    exact_re = Ar_ @ Br_ - Ai_ @ Bi_
    exact_im = Ar_ @ Bi_ + Ai_ @ Br_
    assert np.array_equal(C.real, exact_re.astype(np.float64))
    assert np.array_equal(C.imag, exact_im.astype(np.float64))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("M,N,K,conj_a,trans_b", [(300, 260, 512, False, False),
                                                  (128, 1024, 1024, True, False),
                                                  (520, 130, 224, False, True)])
def test_random_within_fp64_bound(ctx, engine, M, N, K, conj_a, trans_b):
    g = synth.rng(7 + M)
    A = synth.complex_gaussian(g, (M, K))
    B = synth.complex_gaussian(g, (K, N))
    # with conj_a the stored operand is conj(A), passed as a transposed (column-major) view
    Ad = dev(A.conj().T.copy()).T if conj_a else dev(A)
    Bd = dev(B.T.copy()).T if trans_b else dev(B)
    ctx.set_fp64_gemm(engine)
    C = ctx.matmul(Ad, Bd, conj_a=conj_a).cpu().numpy()
    ctx.set_fp64_gemm(1)
    rr, ri = ref_product(A, B)
    bound = 32 * K * 2.0 ** -53 * np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]
    err = np.maximum(np.abs(C.real - rr.astype(np.float64)), np.abs(C.imag - ri.astype(np.float64)))
    assert np.all(err <= bound)


@pytest.mark.parametrize("engine", ENGINES)
def test_rows_of_different_scales(ctx, engine):
    g = synth.rng(3)
    M, N, K = 256, 256, 640
    A = synth.complex_gaussian(g, (M, K)) * (10.0 ** -np.linspace(0, 12, M))[:, None]
    B = synth.complex_gaussian(g, (K, N))
    ctx.set_fp64_gemm(engine)
    C = ctx.matmul(dev(A), dev(B)).cpu().numpy()
    ctx.set_fp64_gemm(1)
    rr, ri = ref_product(A, B)
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]
    err = np.maximum(np.abs(C.real - rr.astype(np.float64)), np.abs(C.imag - ri.astype(np.float64)))
    assert np.all(err <= 32 * K * 2.0 ** -53 * scale)


def test_engines_agree_on_heff(ctx):
    """The FP64 H_eff.theta at the micro-benchmark shape with both engines: the same to
    FP64 rounding (1e-13 of max|y|)."""
    from oracle import bose_hubbard as bh
    from paper_1610_02244_gb300 import tnt
    g = synth.rng(5)
    Ws, _, _ = bh.bh_mpo(4, 3, 1.0, 2.0)
    Le, Re = dev(synth.hermitian_env(g, 256)), dev(synth.hermitian_env(g, 256))
    th = dev(synth.complex_gaussian(g, (256, 4, 4, 256)))
    W1, W2 = dev(Ws[1]), dev(Ws[2])
    ys = []
    for e in ENGINES:
        ctx.set_fp64_gemm(e)
        ys.append(ctx.heff_apply(Le, W1, W2, Re, th, precision=tnt.TNT_PREC_FP64).cpu().numpy())
    ctx.set_fp64_gemm(1)
    assert np.abs(ys[0] - ys[1]).max() <= 1e-13 * np.abs(ys[0]).max()
