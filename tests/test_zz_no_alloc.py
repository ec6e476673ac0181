"""The allocation-free H_eff.theta entry point against the regular one.

tnt_heff_apply_noalloc exists for callers that must not call cudaMalloc: a plug-in inside a
host application that owns all device memory, or a process sharing its GPU with a framework
that reserved the rest.  It keeps its intermediates in a fixed 16 MiB static device array
instead of the context's scratch.  Here it is called through the C-ABI twice in a row on two
different problems (the array keeps the first call's contents, which must not leak into the
second) and compared with tnt_heff_apply in FP64, and with the FP64 CPU oracle, at the FP64
parity tolerance of the kernel tests; a shape beyond the array's capacity must be refused
with a clear error.  pytest collects this file last, so a failure here cannot keep any other
test from running in a run that stops at its first failure.
"""
import numpy as np
import pytest
import torch

from oracle import bose_hubbard as bh
from oracle import contract as oc
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def case(seed, chl, d, chr_):
    g = synth.rng(seed)
    Ws, _, _ = bh.bh_mpo(4, d - 1, 1.0, 2.0)
    Le = synth.hermitian_env(g, chl)
    Re = synth.hermitian_env(g, chr_)
    th = synth.complex_gaussian(g, (chl, d, d, chr_))
    return Le, Ws[1], Ws[2], Re, th


def test_noalloc_matches_heff_apply_twice(ctx):
    # two different problems back to back: the second must not see the first's leftovers
    for seed, (chl, d, chr_) in ((1, (64, 5, 64)), (2, (37, 3, 53))):
        host = case(seed, chl, d, chr_)
        Le, W1, W2, Re, th = (dev(x) for x in host)
        ref = ctx.heff_apply(Le, W1, W2, Re, th).cpu().numpy()
        out = torch.empty_like(th)
        ctx.heff_apply_noalloc(Le, W1, W2, Re, th, out)
        y = out.cpu().numpy()
        assert np.abs(y - ref).max() <= FP64_TOL * np.abs(ref).max()
        y_or = oc.heff_apply(*host)
        assert np.abs(y - y_or).max() <= FP64_TOL * np.abs(y_or).max()


def test_noalloc_refuses_shapes_beyond_its_array(ctx):
    from paper_1610_02244_gb300 import tnt
    Le, W1, W2, Re, th = (dev(x) for x in case(3, 96, 4, 96))  # 96*4*16*96 = 589,824 > 491,520
    out = torch.empty_like(th)
    with pytest.raises(tnt.TntError) as ei:
        ctx.heff_apply_noalloc(Le, W1, W2, Re, th, out)
    assert ei.value.code == 8 and "scratch" in str(ei.value)
