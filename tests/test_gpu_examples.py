"""The paper's second example calculation (Sec. 5) at its own size on the GPU, checked by
properties that hold at any size and by the free-fermion closed form (the first example,
the trapped chain, is in test_gpu_trap.py).

E2: hard-core bosons (n_max = 1) on L = 51 sites from the CDW state |0101...0>, chi = 200
    (Fig. 5): <n_j(t)> against exp(-iht) of the free-fermion hopping matrix h."""
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


def test_e2_hardcore_cdw_quench_L51(ctx):
    Ls, J, dt, steps = 51, 1.0, 0.05, 20
    occ = [0, 1] * (Ls // 2) + [0]  # 25 bosons, filling 0.49 (the asymptote of Fig. 5)
    ctx.set_params(chi_max=200, trunc_err=1e-10, trunc_abs=-1.0, trunc_rel=1e-16, trunc_type=0)
    try:
        mps = ctx.mps_product(occ, 2, 200)
        tb = ctx.tebd_create(mps, 1, J, 4.0, dt)
        disc = 0.0
        for _ in range(steps):
            disc += tb.step()["disc_sum"]
    finally:
        ctx.set_params(chi_max=1 << 40, trunc_err=1e-8)
    h = np.zeros((Ls, Ls))
    for j in range(Ls - 1):
        h[j, j + 1] = h[j + 1, j] = -J
    lam, Q = np.linalg.eigh(h)
    Ut = (Q * np.exp(-1j * lam * dt * steps)) @ Q.conj().T
    exact = (np.abs(Ut) ** 2) @ np.array(occ, dtype=float)
    dens = mps.density()
    assert np.abs(dens - exact).max() < 3e-4  # second-order Trotter at dt = 0.05, t = 1
    assert abs(dens.sum() - 25) < 1e-10
    assert max(mps.bond_dim(k) for k in range(Ls + 1)) <= 200
    # no renormalisation: the norm loss is the discarded weight, up to the rounding of
    # ~1500 gates and centre moves
    assert abs((1 - mps.norm2()) - disc) <= 1e-3 * disc + 1e-10
