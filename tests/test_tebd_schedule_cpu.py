"""The TEBD layer schedule (alternating directions, reading of Sec. 3's Trotterised
update): the oracle's centre moves per step match the count the benchmark's CPU baseline
scales by, and the alternating order gives the same state as the ascending one when no
truncation acts (the gates of a layer commute)."""
import numpy as np
import pytest

import bench
from oracle import contract as oc
from oracle import svd as osvd
from oracle import tebd as otebd

pytestmark = pytest.mark.cpu


class _Counting(otebd.Tebd):
    moves = 0

    def _move_right(self):
        _Counting.moves += 1
        super()._move_right()

    def _move_left(self):
        _Counting.moves += 1
        super()._move_left()


@pytest.mark.parametrize("L", [6, 7, 9])
def test_moves_per_step_match_the_model(L):
    A, q = otebd.product_state([1, 0] * (L // 2) + [1] * (L % 2), 1)
    ev = _Counting(A, q, 1, 1.0, 0.0, 0.05, osvd.TruncParams(chi_max=64, err_tol=1e-14))
    ev.step()  # the first step starts from the left end
    _Counting.moves = 0
    ev.step()
    assert _Counting.moves == bench._tebd_moves_per_step(L)


def test_alternating_order_equals_ascending_without_truncation():
    L, n_max = 6, 2
    A, q = otebd.product_state([2, 0, 1, 1, 0, 2], n_max)
    p = osvd.TruncParams(chi_max=1000, err_tol=0.0)
    alt = otebd.Tebd(A, q, n_max, 1.0, 2.0, 0.05, p)
    asc = otebd.Tebd(A, q, n_max, 1.0, 2.0, 0.05, p)
    for _ in range(4):
        alt.step()
        for layer, key in ((range(0, L - 1, 2), "half"), (range(1, L - 1, 2), "full"),
                           (range(0, L - 1, 2), "half")):
            for i in layer:
                asc.apply_gate(i, asc.gates[(key, i)], True)
    psi, phi = oc.mps_to_state(alt.A), oc.mps_to_state(asc.A)
    assert abs(1 - abs(np.vdot(psi, phi))) < 1e-12
