"""Pins of the oracle's automatic blocking (Sec. 6: zero the entries below a tolerance,
reorder rows and columns into blocks, SVD block by block): the blocks found are the
planted ones, and the block-wise singular values are those of the zeroed matrix."""
import numpy as np
import pytest

from oracle import svd as osvd

pytestmark = pytest.mark.cpu


def planted(seed, sizes_r, sizes_c, noise=1e-12):
    g = np.random.default_rng(seed)
    m, n = sum(sizes_r), sum(sizes_c)
    M = noise * (g.normal(size=(m, n)) + 1j * g.normal(size=(m, n)))
    r0 = c0 = 0
    for a, b in zip(sizes_r, sizes_c):
        M[r0:r0 + a, c0:c0 + b] = g.normal(size=(a, b)) + 1j * g.normal(size=(a, b))
        r0 += a
        c0 += b
    pr, pc = g.permutation(m), g.permutation(n)
    rows = np.repeat(np.arange(len(sizes_r)), sizes_r)[pr]
    cols = np.repeat(np.arange(len(sizes_c)), sizes_c)[pc]
    return M[pr][:, pc], rows, cols


def same_partition(a, b):
    """Labels a and b describe the same grouping (up to renumbering)."""
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


def test_autoblock_finds_planted_blocks():
    M, rows, cols = planted(1, [5, 9, 3, 12], [7, 4, 3, 10])
    Mz, rq, cq = osvd.autoblock(M, 1e-9)
    assert same_partition(rq, rows) and same_partition(cq, cols)
    assert set(rq.tolist()) == set(cq.tolist()) == {0, 1, 2, 3}
    assert rq[0] == 0  # numbered in order of first row
    # nothing of the zeroed matrix lies outside the blocks
    assert np.all(Mz[rq[:, None] != cq[None, :]] == 0)


def test_autoblock_values_are_those_of_the_zeroed_matrix():
    M, _, _ = planted(2, [6, 11, 8], [9, 5, 8])
    Mz, _, _ = osvd.autoblock(M, 1e-9)
    _, S, _, _, _ = osvd.svd_truncate_auto(M, 1e-9, osvd.TruncParams(chi_max=1000, err_tol=0.0))
    ref = np.linalg.svd(Mz, compute_uv=False)
    ref = ref[ref > 1e-16 * ref[0]]
    assert np.abs(np.sort(S)[::-1] - ref).max() < 1e-12 * ref[0]


def test_autoblock_dense_and_empty_lines():
    g = np.random.default_rng(3)
    M = g.normal(size=(6, 5)) + 1j * g.normal(size=(6, 5))
    _, rq, cq = osvd.autoblock(M, 1e-9)
    assert np.all(rq == 0) and np.all(cq == 0)  # one block
    M[2, :] = 1e-15  # a row below the tolerance stands alone
    _, rq, cq = osvd.autoblock(M, 1e-9)
    assert rq[2] not in set(cq.tolist()) and len(set(rq.tolist())) == 2
