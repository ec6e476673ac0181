"""The host half of automatic blocking (tnt_autoblock_components, no GPU needed) against the
oracle's connected components of the zeroed matrix (scipy), on planted block matrices and
random sparse patterns: identical labels, including the numbering rule."""
import numpy as np
import pytest

from oracle import svd as osvd

pytestmark = pytest.mark.cpu


@pytest.fixture(scope="module")
def tnt():
    from paper_1610_02244_gb300 import build as b
    b.build()
    from paper_1610_02244_gb300 import tnt as t
    return t


@pytest.mark.parametrize("seed", range(6))
def test_components_match_oracle(tnt, seed):
    g = np.random.default_rng(seed)
    m, n = int(g.integers(1, 90)), int(g.integers(1, 130))
    M = np.where(g.random((m, n)) < g.choice([0.005, 0.02, 0.08]), 1.0 + 0j, 0.0)
    _, rq_ref, cq_ref = osvd.autoblock(M, 0.5)
    rq, cq, cnt = tnt.autoblock_components(np.abs(M) > 0.5)
    assert np.array_equal(rq, rq_ref) and np.array_equal(cq, cq_ref)
    assert cnt == len(set(rq_ref.tolist()) | set(cq_ref.tolist()))


def test_components_of_planted_blocks(tnt):
    from tests.test_oracle_autoblock import planted
    M, rows, cols = planted(9, [3, 40, 1, 70], [5, 33, 2, 64])
    _, rq_ref, cq_ref = osvd.autoblock(M, 1e-9)
    rq, cq, cnt = tnt.autoblock_components(np.abs(M) > 1e-9)
    assert np.array_equal(rq, rq_ref) and np.array_equal(cq, cq_ref) and cnt == 4


def test_rejects_bad_sizes(tnt):
    from paper_1610_02244_gb300 import _lib
    with pytest.raises(_lib.TntError):
        tnt.autoblock_components(np.zeros((0, 3), bool))
