"""Observables of the device MPS (Sec. 5 examples: <n_j> and <b+_i b_j>) against the FP64
oracle on the very same tensors: a random, unnormalised MPS in a fixed-N sector and a
truncated TEBD state."""
import numpy as np
import pytest

from oracle import contract as oc
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt
    return tnt.Context(0)


def test_density_and_bdagb_random_mps(ctx):
    L, n_max, N, chi = 7, 3, 6, 12
    g = synth.rng(21)
    A, q = synth.random_charged_mps(g, L, n_max + 1, N, chi)
    mps = ctx.mps_create(A, q, chi_cap=chi)
    T = mps.tensors()
    dens = mps.density()
    rho = mps.bdagb()
    assert np.abs(dens - oc.density(T, n_max)).max() < 1e-12
    ref = oc.bdagb(T, n_max)
    assert np.abs(rho - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    assert abs(np.trace(rho).real - N) < 1e-10


def test_density_after_truncated_tebd(ctx):
    n_max = 2
    ctx.set_params(chi_max=6, trunc_err=1e-12, trunc_abs=-1.0, trunc_rel=1e-16, trunc_type=0)
    mps = ctx.mps_product([1] * 7, n_max + 1, 6)
    tb = ctx.tebd_create(mps, n_max, 1.0, 2.0, 0.05)
    for _ in range(8):
        tb.step()
    T = mps.tensors()
    assert np.abs(mps.density() - oc.density(T, n_max)).max() < 1e-12
    assert np.abs(mps.bdagb() - oc.bdagb(T, n_max)).max() < 1e-12
