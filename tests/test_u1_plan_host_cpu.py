"""The grouped U(1) H_eff.theta plan replayed on the host (no GPU).

The library turns the U(1) block structure of a two-site problem (App. A.1.1 labels, the
Listing 1 contraction of Sec. 4.2) into tables: packed L and R blocks, transposed theta
slabs, stage-1 and stage-4 GEMM tasks, the W1 W2 contraction over block pairs, and the
output rows that gather the result back into compact theta.  `tests/u1_plan_host.cu`
builds those tables with the library's own `u1_layout` and carries them out in FP64 on
the host, exactly as the device kernels read them; here the result is compared with the
oracle's dense contraction restricted to the allowed blocks.  A table that sends a block
to the wrong place, or misses a sector pairing, fails here without a GPU: this covers
structures the GPU tests do not reach, among them the site-dependent MPO tensors of the
trapped chain of Sec. 5 and bond sectors far from the filling of a long chain."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import bose_hubbard as bh
from oracle import contract as oc
from oracle import spin as ospin
from paper_1610_02244_gb300 import synth

pytestmark = pytest.mark.cpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1610_02244_gb300")


@pytest.fixture(scope="module")
def replay(tmp_path_factory):
    from paper_1610_02244_gb300 import build as b
    b.build()
    if not os.path.isdir(b.OBJ) or len([f for f in os.listdir(b.OBJ) if f.endswith(".o")]) < len(b.sources()):
        b.build(force=True)  # the library is current but its objects are gone
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("u1host") / "u1_plan_host")
    objs = sorted(os.path.join(b.OBJ, f) for f in os.listdir(b.OBJ) if f.endswith(".o"))
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
           "--expt-relaxed-constexpr", "-I", os.path.join(PKG, "csrc"), "-I",
           os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "u1_plan_host.cu"),
           *objs, "-o", out, "-cudart", "static", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def run_replay(exe, tmp_path, probs):
    """probs: list of (qa, qb, wq, L, W1, W2, R, theta_dense).  Returns the replayed
    compact y (all problems back to back) and the number of compact entries the gather
    did not write exactly once."""
    xs = []
    with open(tmp_path / "in.bin", "wb") as f:
        np.array([len(probs)], dtype=np.int64).tofile(f)
        for qa, qb, wq, L, W1, W2, R, th in probs:
            d, D = W1.shape[2], W1.shape[0]
            np.array([len(qa), len(qb), d, D], dtype=np.int64).tofile(f)
            for a in (qa, qb, wq):
                np.asarray(a, dtype=np.int64).tofile(f)
            for a in (L, W1, W2, R):
                np.ascontiguousarray(a, dtype=np.complex128).tofile(f)
            xs.append(th[synth.theta_mask(qa, d, qb)])
        x = np.concatenate(xs)
        np.array([len(x)], dtype=np.int64).tofile(f)
        x.astype(np.complex128).tofile(f)
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")],
                       capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    raw = np.fromfile(tmp_path / "out.bin", dtype=np.uint8)
    n = int(raw[:8].view(np.int64)[0])
    y = raw[8:8 + 16 * n].view(np.complex128)
    bad = int(raw[8 + 16 * n:].view(np.int64)[0])
    return y, bad


def oracle_compact(probs):
    ys = []
    for qa, qb, wq, L, W1, W2, R, th in probs:
        y = oc.heff_apply(L, W1, W2, R, th)
        m = synth.theta_mask(qa, W1.shape[2], qb)
        assert np.abs(y[~m]).max(initial=0.0) <= 1e-12 * np.abs(y).max()  # charge conserved
        ys.append(y[m])
    return np.concatenate(ys)


def bh_problem(seed, qa, qb, Ws, i):
    """Environments with the allowed blocks of random Hermitian-paired channels, the MPO
    tensors of sites i, i+1, theta random inside its allowed blocks."""
    g = synth.rng(seed)
    d = Ws[i].shape[2]
    L = synth.hermitian_env(g, len(qa)) * synth.env_mask(qa, qa)
    R = synth.hermitian_env(g, len(qb)) * synth.env_mask(qb, qb)
    th = synth.complex_gaussian(g, (len(qa), d, d, len(qb))) * synth.theta_mask(qa, d, qb)
    return (qa, qb, synth.BH_WQ, L, Ws[i], Ws[i + 1], R, th)


def check(exe, tmp_path, probs):
    y, bad = run_replay(exe, tmp_path, probs)
    ref = oracle_compact(probs)
    assert bad == 0
    assert len(y) == len(ref)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


TRAP = dict(L=100, n_max=3, J=1.0, U=5.0, mu=0.0, V=0.01, j_c=50.5)


def trap_mpo():
    p = TRAP
    return bh.bh_mpo(p["L"], p["n_max"], p["J"], p["U"], p["mu"], p["V"], p["j_c"])[0]


@pytest.mark.parametrize("bond", [1, 12, 40, 49, 90])
def test_trapped_chain_bonds(replay, tmp_path, bond):
    """Bonds of the 100-site trapped chain (N = 100, n_max = 3, chi = 100, the Gaussian
    sector profile of its random start): theta over sites (bond, bond + 1), so the left
    labels are those of bond `bond` and the right ones of bond `bond + 2`, with the
    site-dependent MPO tensors of those two sites."""
    q = synth.bond_charges(100, 4, 100, 100, "gauss", 2.0)
    Ws = trap_mpo()
    check(replay, tmp_path, [bh_problem(bond, q[bond], q[bond + 2], Ws, bond)])


def test_depleted_edge_labels(replay, tmp_path):
    """Labels the trapped ground state has at its empty edge: almost every state of the
    left bond carries no boson, the right bond a few; most sector pairs have no block."""
    qa = np.array([0] * 30 + [1] * 12 + [2] * 3 + [3])
    qb = np.array([0] * 20 + [1] * 25 + [2] * 10 + [3] * 4 + [5, 6])
    Ws = trap_mpo()
    check(replay, tmp_path, [bh_problem(7, qa, qb, Ws, 3)])


def test_label_gaps_and_far_sectors(replay, tmp_path):
    """Sectors with gaps between charges and sectors with no partner on the other side."""
    Ws, _, _ = bh.bh_mpo(6, 2, 1.0, 2.0)
    qa = np.array([0, 2, 2, 5, 9, 9])
    qb = np.array([3, 3, 4, 7, 7, 7, 9, 20])
    check(replay, tmp_path, [bh_problem(3, qa, qb, Ws, 2)])


def test_spin1_mpo(replay, tmp_path):
    """The D = 5 spin-1 MPO with charges (0, +1, -1, 0, 0) on Gaussian sectors."""
    Ws, _, _, wq = ospin.heisenberg_mpo(6, 2, 1.0, 0.7, 0.2)
    g = synth.rng(5)
    qa = synth.gaussian_sector_labels(60, 9, 2.0, 20)
    qb = synth.gaussian_sector_labels(70, 11, 2.0, 22)
    L = synth.hermitian_env(g, len(qa), 5, pair=(1, 2)) * synth.env_mask(qa, qa, wq)
    R = synth.hermitian_env(g, len(qb), 5, pair=(1, 2)) * synth.env_mask(qb, qb, wq)
    th = synth.complex_gaussian(g, (len(qa), 3, 3, len(qb))) * synth.theta_mask(qa, 3, qb)
    check(replay, tmp_path, [(qa, qb, wq, L, Ws[2], Ws[3], R, th)])


def test_several_problems_in_one_plan(replay, tmp_path):
    """Three problems of different shapes in one plan: their tables and compact vectors
    are offset against each other."""
    q = synth.bond_charges(100, 4, 100, 100, "gauss", 2.0)
    Ws = trap_mpo()
    Wu, _, _ = bh.bh_mpo(6, 3, 1.0, 2.0)
    probs = [bh_problem(20, q[20], q[22], Ws, 20),
             bh_problem(21, np.array([0, 0, 1, 1, 1, 2]), np.array([1, 2, 2, 3, 3, 3, 4, 4]), Wu, 1),
             bh_problem(22, q[60], q[62], Ws, 60)]
    check(replay, tmp_path, probs)
