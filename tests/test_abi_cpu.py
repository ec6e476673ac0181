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
