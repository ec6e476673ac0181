"""Pins of the oracle's eigensolver and truncated SVD: library routines on special cases,
brute force over the four truncation rules, reconstruction and block structure."""
import numpy as np
import pytest

from oracle import lanczos, svd
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.cpu


def rand_herm(g, n):
    X = synth.complex_gaussian(g, (n, n))
    return (X + X.conj().T) / 2


@pytest.mark.parametrize("n,cap", [(60, 32), (200, 32), (200, 8)])
def test_lanczos_lowest_matches_eigh(n, cap):
    g = synth.rng(n + cap)
    H = rand_herm(g, n)
    H[np.arange(n), np.arange(n)] += np.linspace(0, 3, n)  # open a gap at the bottom
    H[0, 0] -= 4.0
    E, x, nmv, resid, conv = lanczos.lanczos_ground(lambda v: H @ v,
                                                    synth.complex_gaussian(g, n))
    w, v = np.linalg.eigh(H)
    assert conv
    assert abs(E - w[0]) < 1e-12 * abs(w[0])
    assert abs(abs(np.vdot(v[:, 0], x)) - 1) < 1e-10
    assert np.linalg.norm(H @ x - E * x) < 1e-9
    assert nmv <= 300


def test_lanczos_invariant_subspace_stops_early():
    """A start vector inside a 3-dimensional invariant subspace converges in 3 steps."""
    H = np.diag([-2.0, 1.0, 3.0, 5.0, 7.0]).astype(np.complex128)
    x0 = np.array([1, 1, 1, 0, 0], dtype=np.complex128)
    E, x, nmv, _, conv = lanczos.lanczos_ground(lambda v: H @ v, x0)
    assert conv and nmv == 3 and abs(E + 2.0) < 1e-14


def test_tridiag_lowest_matches_eigvalsh():
    g = synth.rng(7)
    a = g.standard_normal(9)
    b = np.abs(g.standard_normal(8))
    E, y = lanczos.tridiag_lowest(a, b)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    assert abs(E - np.linalg.eigvalsh(T)[0]) < 1e-13
    assert np.linalg.norm(T @ y - E * y) < 1e-12


def brute_chi(sig_desc, chi_max, a, r, eps_tol, typ):
    """Largest chi allowed by each rule, read literally, then the smallest (min 1)."""
    n = len(sig_desc)
    nrm = np.sqrt(sum(s * s for s in sig_desc))
    allowed = []
    # rule 1
    allowed.append(min(n, chi_max))
    # rule 2: every kept value must be >= a
    c = n
    if a > 0:
        c = 0
        for s in sig_desc:
            if s >= a:
                c += 1
    allowed.append(c)
    # rule 3
    c = 0
    for s in sig_desc:
        if s / sig_desc[0] >= r:
            c += 1
    allowed.append(c)
    # rule 4: smallest chi whose discarded tail has error < eps_tol
    best = n
    for chi in range(n, -1, -1):
        tail = [s / nrm for s in sig_desc[chi:]]
        if typ == svd.TRUNC_2NORM:
            e = sum(t * t for t in tail) ** 0.5
        elif typ == svd.TRUNC_SUMSQ:
            e = sum(t * t for t in tail)
        else:
            e = sum(abs(t) for t in tail)
        if e < eps_tol:
            best = chi
    allowed.append(best)
    return max(1, min(allowed))


@pytest.mark.parametrize("seed", range(12))
def test_truncation_rules_brute_force(seed):
    g = synth.rng(100 + seed)
    n = int(g.integers(1, 40))
    sig = np.sort(np.exp(g.uniform(-25, 0, n)))[::-1]
    chi_max = int(g.integers(1, 45))
    a = float(g.choice([-1.0, 1e-6, 1e-3]))
    r = float(g.choice([1e-16, 1e-8, 1e-2]))
    eps = float(g.choice([1e-12, 1e-8, 1e-4, 1e-2]))
    typ = int(g.integers(0, 3))
    p = svd.TruncParams(chi_max=chi_max, abs_tol=a, rel_tol=r, err_tol=eps, err_type=typ)
    assert svd.choose_chi(sig, p) == brute_chi(list(sig), chi_max, a, r, eps, typ)


def test_block_svd_reconstructs_and_matches_dense_spectrum():
    g = synth.rng(11)
    rq = g.integers(0, 4, 30)
    cq = g.integers(1, 5, 25)
    M = synth.complex_gaussian(g, (30, 25)) * (rq[:, None] == cq[None, :])
    p = svd.TruncParams(chi_max=1000, rel_tol=1e-16, err_tol=0.0)
    U, S, Vh, bq, info = svd.svd_truncate(M, rq, cq, p)
    assert np.abs((U * S) @ Vh - M).max() < 1e-12
    dense = np.linalg.svd(M, compute_uv=False)
    dense = dense[dense > 1e-12]
    assert np.allclose(np.sort(S)[::-1], dense, atol=1e-12)
    assert np.abs(U.conj().T @ U - np.eye(len(S))).max() < 1e-12
    assert np.abs(Vh @ Vh.conj().T - np.eye(len(S))).max() < 1e-12
    # every kept index couples only rows and columns of its own charge
    assert np.all((np.abs(U) < 1e-15) | (rq[:, None] == bq[None, :]))
    assert np.all(np.diff(bq) >= 0)


def test_truncation_error_definition():
    g = synth.rng(12)
    M = synth.complex_gaussian(g, (20, 20))
    p = svd.TruncParams(chi_max=7, err_tol=0.0)
    U, S, Vh, bq, info = svd.svd_truncate(M, np.zeros(20, int), np.zeros(20, int), p)
    full = np.linalg.svd(M, compute_uv=False)
    assert len(S) == 7
    assert abs(info["err"] - np.sqrt(np.sum(full[7:] ** 2)) / np.linalg.norm(full)) < 1e-13
    assert abs(info["disc"] - np.sum(full[7:] ** 2)) < 1e-11
    # Eckart-Young: the rank-7 truncation error in Frobenius norm is the discarded tail
    assert abs(np.linalg.norm(M - (U * S) @ Vh) ** 2 - info["disc"]) < 1e-10


def test_defaults_match_the_printed_system_information():
    golden = {}
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_defaults.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            golden[k] = v
    p = svd.TruncParams()
    assert p.rel_tol == float(golden["rel_trunc_tol"])
    assert p.abs_tol == float(golden["abs_trunc_tol"])
    assert p.err_tol == float(golden["trunc_err_tol"])
    assert golden["trunc_type"] == "2norm" and p.err_type == svd.TRUNC_2NORM
    import inspect
    assert inspect.signature(lanczos.lanczos_ground).parameters["max_matvec"].default == \
        int(golden["eig_max_iter"])
