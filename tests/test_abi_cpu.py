"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, exports every
declared symbol, its host-side model builders agree with the oracle, and it refuses to
run without a GPU instead of falling back to anything."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import bose_hubbard as bh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import _lib
    b.build()
    return _lib.load()


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^(?:int|int64_t|const char\*)\s+(tnt_\w+)\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_1610_02244_gb300 import _lib
    declared = declared_symbols()
    assert len(declared) >= 30
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert declared <= exported, declared - exported
    # and nothing undeclared leaks out
    assert {e for e in exported if e.startswith("tnt_")} == declared
    # the binding wraps exactly the declared calls
    assert set(_lib.SIGNATURES) == declared


def test_params_default_are_the_paper_defaults(lib):
    from paper_1610_02244_gb300 import tnt
    p = tnt.params_default()
    golden = dict(ln.split() for ln in open(os.path.join(ROOT, "tests", "golden",
                                                          "paper_defaults.txt"))
                  if ln.strip() and not ln.startswith("#"))
    assert p["trunc_rel"] == float(golden["rel_trunc_tol"])
    assert p["trunc_abs"] == float(golden["abs_trunc_tol"])
    assert p["trunc_err"] == float(golden["trunc_err_tol"])
    assert p["trunc_type"] == 0 and golden["trunc_type"] == "2norm"
    assert p["lanczos_maxit"] == int(golden["eig_max_iter"])


@pytest.mark.parametrize("n_max", [1, 3, 4])
def test_mpo_builder_matches_oracle(lib, n_max):
    from paper_1610_02244_gb300 import tnt
    L, J, U, mu, V, jc = 7, 0.9, 2.7, 0.3, 0.05, 3.5
    Ws, _, _ = bh.bh_mpo(L, n_max, J, U, mu, V, jc)
    for j in (1, 4, 7):
        W = tnt.bh_mpo_site(n_max, J, U, mu, V, float(j), jc)
        assert np.abs(W - Ws[j - 1]).max() < 1e-14


@pytest.mark.parametrize("n_max,c1,c2,tau", [(4, 0.5, 0.5, 0.01), (3, 1.0, 0.5, 0.005),
                                             (1, 0.5, 1.0, 0.3)])
def test_gate_builder_matches_oracle(lib, n_max, c1, c2, tau):
    from paper_1610_02244_gb300 import tnt
    G = tnt.bh_bond_gate(n_max, 1.0, 2.0, 0.1, c1, c2, tau)
    Gr = bh.gate(bh.bond_hamiltonian(n_max, 1.0, 2.0, c1, c2, 0.1), tau)
    assert np.abs(G - Gr).max() < 1e-13


def test_context_refuses_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    code = lib.tnt_ctx_create(0, None, ctypes.byref(h))
    assert code == 3 and not h.value  # TNT_E_CUDA, no handle


def test_argument_errors_are_reported(lib):
    # null handles are rejected without touching the GPU
    assert lib.tnt_ctx_destroy(None) == 1
    assert lib.tnt_params_set(None, None) == 1
    assert lib.tnt_bh_mpo_site(-1, 1.0, 1.0, 0.0, 0.0, 1.0, 0.0, None) == 1


@pytest.mark.parametrize("two_s,J,Jz,hz", [(2, 1.0, 1.0, 0.0), (1, 0.8, -0.3, 0.25),
                                           (3, 1.0, 0.5, 0.1)])
def test_spin_builders_match_oracle(lib, two_s, J, Jz, hz):
    """The spin-S MPO tensor and bond term of Sec. 6 built by the library's host code equal
    the oracle's, and the gate of each bond term equals the oracle's eigh-route gate."""
    from oracle import spin as ospin
    from paper_1610_02244_gb300 import tnt
    Ws, _, _, _ = ospin.heisenberg_mpo(2, two_s, J, Jz, hz)
    assert np.abs(tnt.spin_mpo_site(two_s, J, Jz, hz) - Ws[0]).max() < 1e-15
    for c1, c2 in ((1.0, 0.5), (0.5, 0.5), (0.5, 1.0)):
        h = ospin.bond_hamiltonian(two_s, J, Jz, hz, c1, c2)
        assert np.abs(tnt.spin_bond_h(two_s, J, Jz, hz, c1, c2) - h).max() < 1e-15
        assert np.abs(tnt.bond_gate(h, 0.07) - bh.gate(h, 0.07)).max() < 1e-13


@pytest.mark.parametrize("n", [1, 4, 9, 25, 49])
def test_bond_gate_is_the_matrix_exponential(lib, n):
    """exp(-i tau h) of a random complex Hermitian h by the library's host eigensolver,
    against scipy's Pade exponential (a route with no eigendecomposition): equal to rounding,
    unitary, the identity at tau = 0, and blind to an anti-Hermitian part of its input."""
    import scipy.linalg as sla
    from paper_1610_02244_gb300 import tnt
    tol = 10 * n * np.finfo(float).eps  # rotations accumulate O(n eps) in the eigenvectors
    g = np.random.default_rng(n)
    X = g.normal(size=(n, n)) + 1j * g.normal(size=(n, n))
    h = 0.5 * (X + X.conj().T)
    for tau in (0.01, 0.3):
        G = tnt.bond_gate(h, tau)
        Gr = sla.expm(-1j * tau * h)
        assert np.abs(G - Gr).max() < tol
        assert np.abs(G.conj().T @ G - np.eye(n)).max() < tol
    assert np.abs(tnt.bond_gate(h, 0.0) - np.eye(n)).max() < tol
    K = g.normal(size=(n, n)) + 1j * g.normal(size=(n, n))
    assert np.abs(tnt.bond_gate(h + 0.5 * (K - K.conj().T), 0.3) - tnt.bond_gate(h, 0.3)).max() < tol


def test_bond_gate_of_a_degenerate_term(lib):
    """A bond term with a highly degenerate spectrum (the isotropic spin-1 exchange S.S has
    only three distinct eigenvalues on nine states) still gives the exact gate."""
    import scipy.linalg as sla
    from oracle import spin as ospin
    from paper_1610_02244_gb300 import tnt
    h = ospin.bond_hamiltonian(2, 1.0, 1.0, 0.0, 0.0, 0.0)
    assert len(np.unique(np.round(np.linalg.eigvalsh(h), 10))) == 3
    assert np.abs(tnt.bond_gate(h, 0.2) - sla.expm(-0.2j * h)).max() < 1e-13


def test_bond_gate_argument_errors(lib):
    h = np.eye(4, dtype=np.complex128)
    G = np.zeros_like(h)
    assert lib.tnt_bond_gate(0, h.ctypes.data, 0.1, G.ctypes.data) == 1
    assert lib.tnt_bond_gate(257, h.ctypes.data, 0.1, G.ctypes.data) == 1
    assert lib.tnt_bond_gate(4, None, 0.1, G.ctypes.data) == 1
    assert lib.tnt_bond_gate(4, h.ctypes.data, float("nan"), G.ctypes.data) == 1


def test_host_builders_refuse_non_finite_input(lib):
    """A NaN or infinite model parameter, or a non-finite entry of a bond term, is an
    argument error, not a gate or MPO full of NaN."""
    nan, inf = float("nan"), float("inf")
    out = np.zeros(16 * 16 * 16, dtype=np.complex128)
    p = out.ctypes.data
    assert lib.tnt_bh_mpo_site(3, nan, 1.0, 0.0, 0.0, 1.0, 0.0, p) == 1
    assert lib.tnt_bh_mpo_site(3, 1.0, 1.0, 0.0, inf, 1.0, 0.0, p) == 1
    assert lib.tnt_bh_mpo_site(3, 1.0, 1.0, 0.0, 0.01, 1.0, 50.5, p) == 0
    assert lib.tnt_bh_bond_gate(2, 1.0, nan, 0.0, 0.5, 0.5, 0.1, p) == 1
    assert lib.tnt_bh_bond_gate(2, 1.0, 2.0, 0.0, 0.5, 0.5, inf, p) == 1
    assert lib.tnt_spin_mpo_site(2, 1.0, nan, 0.0, p) == 1
    assert lib.tnt_spin_bond_h(2, 1.0, 1.0, 0.0, 0.5, -inf, p) == 1
    assert lib.tnt_spin_bond_h(2, 1.0, 1.0, 0.0, 0.5, 0.5, p) == 0
    h = np.eye(9, dtype=np.complex128)
    h[3, 4] = complex(0.0, nan)
    assert lib.tnt_bond_gate(9, h.ctypes.data, 0.1, p) == 1
    h[3, 4] = 0.0
    assert lib.tnt_bond_gate(9, h.ctypes.data, 0.1, p) == 0


def test_update_energies_argument_errors(lib):
    """The per-update energies call is host only; without a handle it is an argument
    error (the values themselves are checked on the GPU after a sweep)."""
    n = ctypes.c_int64(-1)
    assert lib.tnt_dmrg_update_energies(None, None, 0, ctypes.byref(n)) == 1
    assert lib.tnt_dmrg_update_energies(None, None, 0, None) == 1
