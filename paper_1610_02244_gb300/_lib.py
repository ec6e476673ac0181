"""ctypes binding of libtntgb.so (the C-ABI in include/tnt_gb300.h).

Argument marshalling only: every step of the computation runs in the CUDA library.  If
the library has not been built, loading fails with an error instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtntgb.so")

TNT_OK, TNT_E_INVALID, TNT_E_ALLOC, TNT_E_CUDA, TNT_E_NOCONV = 0, 1, 2, 3, 4
TNT_E_TIMEOUT, TNT_E_BOUNDS, TNT_E_NAN, TNT_E_UNSUPPORTED = 5, 6, 7, 8
TNT_PREC_FP64, TNT_PREC_MIXED = 0, 1
TNT_FP64_GEMM_FMA, TNT_FP64_GEMM_TC = 0, 1
TNT_TRUNC_2NORM, TNT_TRUNC_SUMSQ, TNT_TRUNC_1NORM = 0, 1, 2
TNT_SVD_LEFT, TNT_SVD_RIGHT = 0, 1

STATUS_NAMES = {0: "TNT_OK", 1: "TNT_E_INVALID", 2: "TNT_E_ALLOC", 3: "TNT_E_CUDA",
                4: "TNT_E_NOCONV", 5: "TNT_E_TIMEOUT", 6: "TNT_E_BOUNDS", 7: "TNT_E_NAN",
                8: "TNT_E_UNSUPPORTED"}


class TntError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class tnt_cplx(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class tnt_params(C.Structure):
    _fields_ = [("chi_max", C.c_int64), ("trunc_abs", C.c_double), ("trunc_rel", C.c_double),
                ("trunc_err", C.c_double), ("trunc_type", C.c_int), ("lanczos_tol", C.c_double),
                ("lanczos_maxit", C.c_int), ("krylov_cap", C.c_int), ("precision", C.c_int),
                ("seed", C.c_uint64)]


class tnt_lanczos_result(C.Structure):
    _fields_ = [("E", C.c_double), ("E_rq", C.c_double), ("resid", C.c_double),
                ("resid_fp64", C.c_double), ("n_matvec", C.c_int), ("converged", C.c_int)]


class tnt_trunc_result(C.Structure):
    _fields_ = [("chi", C.c_int64), ("err", C.c_double), ("disc", C.c_double),
                ("norm2", C.c_double), ("n_blocks", C.c_int), ("tie_at_cut", C.c_int)]


class tnt_sweep_stats(C.Structure):
    _fields_ = [("E", C.c_double), ("max_err", C.c_double), ("max_disc", C.c_double),
                ("max_chi", C.c_int64), ("total_matvecs", C.c_int), ("unconverged", C.c_int),
                ("seconds", C.c_double), ("t_plan", C.c_double), ("t_eig", C.c_double),
                ("t_svd", C.c_double), ("t_env", C.c_double)]


class tnt_u1_problem(C.Structure):
    _fields_ = [("d_L", C.c_void_p), ("d_W1", C.c_void_p), ("d_W2", C.c_void_p),
                ("d_R", C.c_void_p), ("chl", C.c_int64), ("d", C.c_int64), ("D", C.c_int64),
                ("chr", C.c_int64), ("h_qa", C.c_void_p), ("h_qb", C.c_void_p),
                ("h_wq", C.c_void_p)]


class tnt_step_stats(C.Structure):
    _fields_ = [("err_sum", C.c_double), ("disc_sum", C.c_double), ("max_chi", C.c_int64),
                ("seconds", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class tnt_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


P = C.c_void_p
I64 = C.c_int64
I = C.c_int
D = C.c_double
PI64 = C.POINTER(C.c_int64)
PD = C.POINTER(C.c_double)

# name -> argtypes (all return int unless listed in _RESTYPE)
SIGNATURES = {
    "tnt_ctx_create": [I, P, C.POINTER(P)],
    "tnt_ctx_create_with_allocator": [I, P, C.POINTER(tnt_allocator), C.POINTER(P)],
    "tnt_ctx_destroy": [P],
    "tnt_set_stream": [P, P],
    "tnt_last_error": [P],
    "tnt_launch_count": [P],
    "tnt_profile_select": [P, C.c_char_p],
    "tnt_profile_read": [P, PD, PI64, PD],
    "tnt_params_default": [C.POINTER(tnt_params)],
    "tnt_params_set": [P, C.POINTER(tnt_params)],
    "tnt_params_get": [P, C.POINTER(tnt_params)],
    "tnt_sys_info": [P, C.c_char_p, C.c_size_t],
    "tnt_bh_mpo_site": [I, D, D, D, D, D, D, P],
    "tnt_bh_bond_gate": [I, D, D, D, D, D, D, P],
    "tnt_spin_mpo_site": [I, D, D, D, P],
    "tnt_spin_bond_h": [I, D, D, D, D, D, P],
    "tnt_bond_gate": [I, P, D, P],
    "tnt_theta_form": [P, P, P, I64, I64, I64, I64, P],
    "tnt_gate_apply": [P, P, P, I64, I64, I64, P],
    "tnt_heff_apply": [P, P, P, P, P, P, I64, I64, I64, I64, I, P],
    "tnt_heff_apply_noalloc": [P, P, P, P, P, P, I64, I64, I64, I64, P],
    "tnt_env_left": [P, P, P, P, I64, I64, I64, I64, P],
    "tnt_env_right": [P, P, P, P, I64, I64, I64, I64, P],
    "tnt_lanczos_ground": [P, P, P, P, P, I64, I64, I64, I64, P,
                           C.POINTER(tnt_lanczos_result)],
    "tnt_svd_trunc": [P, P, I64, I64, P, P, I, I, P, P, P, P, C.POINTER(tnt_trunc_result)],
    "tnt_mpo_bose_hubbard": [P, I, I, D, D, D, D, D, C.POINTER(P)],
    "tnt_mpo_spin_heisenberg": [P, I, I, D, D, D, C.POINTER(P)],
    "tnt_mpo_create": [P, I, I, I, C.POINTER(P), P, P, P, C.POINTER(P)],
    "tnt_mpo_destroy": [P],
    "tnt_mps_create": [P, I, I, I64, P, P, P, C.POINTER(P)],
    "tnt_mps_product": [P, I, I, I64, P, C.POINTER(P)],
    "tnt_mps_destroy": [P],
    "tnt_mps_length": [P, C.POINTER(I), C.POINTER(I)],
    "tnt_mps_bond_dim": [P, I, PI64],
    "tnt_mps_get_site": [P, P, I, P, I64],
    "tnt_mps_get_charges": [P, I, P, I64],
    "tnt_mps_expect_mpo": [P, P, P, PD],
    "tnt_mps_norm2": [P, P, PD],
    "tnt_mps_overlap": [P, P, P, C.POINTER(tnt_cplx)],
    "tnt_mps_set_charges": [P, P, I, P],
    "tnt_mps_save": [P, P, C.c_char_p],
    "tnt_mps_load": [P, C.c_char_p, I64, I, C.POINTER(P)],
    "tnt_dmrg_create": [P, P, P, C.POINTER(P)],
    "tnt_dmrg_sweep": [P, P, C.POINTER(tnt_sweep_stats)],
    "tnt_dmrg_sweep1": [P, P, D, C.POINTER(tnt_sweep_stats)],
    "tnt_dmrg_update_energies": [P, C.POINTER(D), I64, C.POINTER(I64)],
    "tnt_dmrg_sweep_batched": [P, I, C.POINTER(P), C.POINTER(tnt_sweep_stats)],
    "tnt_dmrg_update": [P, P, I, I, C.POINTER(tnt_lanczos_result), C.POINTER(tnt_trunc_result)],
    "tnt_dmrg_destroy": [P],
    "tnt_mps_density": [P, P, PD],
    "tnt_mps_bdagb": [P, P, P],
    "tnt_tebd_create": [P, P, I, D, D, D, D, C.POINTER(P)],
    "tnt_tebd_create_spin": [P, P, I, D, D, D, D, C.POINTER(P)],
    "tnt_tebd_create_bonds": [P, P, C.POINTER(P), D, C.POINTER(P)],
    "tnt_u1_size": [C.POINTER(tnt_u1_problem), PI64],
    "tnt_u1_pack": [P, C.POINTER(tnt_u1_problem), P, P],
    "tnt_u1_unpack": [P, C.POINTER(tnt_u1_problem), P, P],
    "tnt_heff_apply_u1": [P, I, C.POINTER(tnt_u1_problem), P, P, I, PD],
    "tnt_lanczos_ground_u1": [P, C.POINTER(tnt_u1_problem), P, C.POINTER(tnt_lanczos_result)],
    "tnt_lanczos_ground_u1_batched": [P, I, C.POINTER(tnt_u1_problem), P,
                                      C.POINTER(tnt_lanczos_result)],
    "tnt_set_graphs": [P, I],
    "tnt_set_svd_zero_tol": [P, D],
    "tnt_autoblock_components": [C.c_int64, C.c_int64, P, P, P, P],
    "tnt_matmul": [P, I64, I64, I64, P, I64, I64, I, P, I64, I64, I, P, I64],
    "tnt_set_fp64_gemm": [P, I],
    "tnt_u1_tiles": [P, I, C.POINTER(tnt_u1_problem), C.POINTER(C.c_int)],
    "tnt_tebd_step": [P, P, C.POINTER(tnt_step_stats)],
    "tnt_tebd_gate": [P, P, I, P, I, C.POINTER(tnt_trunc_result)],
    "tnt_tebd_centre": [P, C.POINTER(I)],
    "tnt_tebd_destroy": [P],
}
_RESTYPE = {"tnt_last_error": C.c_char_p, "tnt_launch_count": C.c_int64}

_lib = None


def load():
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA extension first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    for name, argt in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = argt
        fn.restype = _RESTYPE.get(name, C.c_int)
    _lib = lib
    return lib


def check(ctx, code: int, ok=(TNT_OK,)):
    if code not in ok:
        msg = load().tnt_last_error(ctx).decode() if ctx else ""
        raise TntError(code, msg)
    return code
