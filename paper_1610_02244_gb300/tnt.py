"""Python API over the C-ABI: same names as the C calls, argument marshalling only.

Device tensors are torch complex128 CUDA tensors in the leg orders of include/tnt_gb300.h;
PyTorch only provides memory and the stream.  Every computation runs in libtntgb.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from ._lib import (TNT_FP64_GEMM_FMA, TNT_FP64_GEMM_TC, TNT_PREC_FP64,  # noqa: F401
                   TNT_PREC_MIXED, TNT_SVD_LEFT, TNT_SVD_RIGHT, TNT_TRUNC_1NORM,
                   TNT_TRUNC_2NORM, TNT_TRUNC_SUMSQ, TntError)

CDT = torch.complex128


def _ptr(t: torch.Tensor) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != CDT or not t.is_contiguous():
        raise ValueError("expected a contiguous complex128 CUDA tensor")
    return t.data_ptr()


def _struct_dict(s) -> dict:
    return {k: getattr(s, k) for k, _ in s._fields_}


def bh_mpo_site(n_max, J, U, mu=0.0, V=0.0, j=1.0, j_c=0.0) -> np.ndarray:
    """Host builder of one Bose-Hubbard MPO tensor W[4,4,d,d] (C call tnt_bh_mpo_site)."""
    d = n_max + 1
    out = np.zeros((4, 4, d, d), dtype=np.complex128)
    L.check(None, L.load().tnt_bh_mpo_site(n_max, J, U, mu, V, j, j_c, out.ctypes.data))
    return out


def bh_bond_gate(n_max, J, U, mu, c1, c2, tau) -> np.ndarray:
    """Host builder of the Trotter gate exp(-i tau h_bond), d^2 x d^2 (tnt_bh_bond_gate)."""
    d = n_max + 1
    out = np.zeros((d * d, d * d), dtype=np.complex128)
    L.check(None, L.load().tnt_bh_bond_gate(n_max, J, U, mu, c1, c2, tau, out.ctypes.data))
    return out


def spin_mpo_site(two_s, J, Jz, hz=0.0) -> np.ndarray:
    """Host builder of one spin-S Heisenberg MPO tensor W[5,5,d,d] (tnt_spin_mpo_site)."""
    d = two_s + 1
    out = np.zeros((5, 5, d, d), dtype=np.complex128)
    L.check(None, L.load().tnt_spin_mpo_site(two_s, J, Jz, hz, out.ctypes.data))
    return out


def spin_bond_h(two_s, J, Jz, hz, c1, c2) -> np.ndarray:
    """Host builder of the spin-S Heisenberg bond term, d^2 x d^2 (tnt_spin_bond_h)."""
    d = two_s + 1
    out = np.zeros((d * d, d * d), dtype=np.complex128)
    L.check(None, L.load().tnt_spin_bond_h(two_s, J, Jz, hz, c1, c2, out.ctypes.data))
    return out


def bond_gate(h, tau) -> np.ndarray:
    """exp(-i tau h) of a Hermitian host matrix (tnt_bond_gate)."""
    h = np.ascontiguousarray(h, dtype=np.complex128)
    out = np.zeros_like(h)
    L.check(None, L.load().tnt_bond_gate(h.shape[0], h.ctypes.data, tau, out.ctypes.data))
    return out


def autoblock_components(nonzero: np.ndarray):
    """Component labels of a boolean non-zero pattern (tnt_autoblock_components, host only):
    (row labels, column labels, count)."""
    nz = np.asarray(nonzero, dtype=bool)
    m, n = nz.shape
    W = (n + 31) // 32
    pad = np.zeros((m, W * 32), dtype=bool)
    pad[:, :n] = nz
    mask = np.packbits(pad.reshape(m, W, 4, 8)[..., ::-1], axis=-1).reshape(m, W, 4)
    mask = np.ascontiguousarray(mask.view(np.uint32).reshape(m, W))  # little endian words
    rq = np.zeros(m, dtype=np.int64)
    cq = np.zeros(n, dtype=np.int64)
    cnt = C.c_int64()
    L.check(None, L.load().tnt_autoblock_components(m, n, mask.ctypes.data, rq.ctypes.data,
                                                     cq.ctypes.data, C.byref(cnt)))
    return rq, cq, cnt.value


def params_default() -> dict:
    p = L.tnt_params()
    L.check(None, L.load().tnt_params_default(C.byref(p)))
    return _struct_dict(p)


def torch_allocator(device: int, stream: torch.cuda.Stream):
    """(alloc, free) callables that take the library's device memory from PyTorch's caching
    allocator on `stream` (for Context(allocator=...))."""
    def alloc(nbytes):
        return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)
    return alloc, free


class Context:
    """A library context on one GPU, enqueueing on torch's current stream.

    allocator: optional (alloc(nbytes) -> device pointer as int, free(ptr)) pair through
    which every device allocation of the context and its handles is made
    (tnt_ctx_create_with_allocator); by default the library calls cudaMalloc."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None,
                 allocator=None):
        self.lib = L.load()
        self.device = device
        torch.cuda.set_device(device)
        st = stream if stream is not None else torch.cuda.current_stream(device)
        self.stream = st
        h = C.c_void_p()
        if allocator is None:
            code = self.lib.tnt_ctx_create(device, C.c_void_p(st.cuda_stream), C.byref(h))
        else:
            alloc, free = allocator

            def _alloc(nbytes, _user):
                try:
                    return int(alloc(nbytes)) or None
                except Exception:
                    return None

            def _free(ptr, _user):
                free(ptr)
            # the callbacks must outlive the context (the library calls them until destroy)
            self._cb = L.tnt_allocator(L.ALLOC_FN(_alloc), L.FREE_FN(_free), None)
            code = self.lib.tnt_ctx_create_with_allocator(device, C.c_void_p(st.cuda_stream),
                                                          C.byref(self._cb), C.byref(h))
        if code != 0:
            raise TntError(code, "tnt_ctx_create failed (no usable CUDA device?)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.tnt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, code, ok=(0,)):
        return L.check(self.h, code, ok)

    # ---------------------------------------------------------------- params
    def params(self) -> dict:
        p = L.tnt_params()
        self._chk(self.lib.tnt_params_get(self.h, C.byref(p)))
        return _struct_dict(p)

    def set_params(self, **kw):
        p = L.tnt_params()
        self._chk(self.lib.tnt_params_get(self.h, C.byref(p)))
        for k, v in kw.items():
            setattr(p, k, v)
        self._chk(self.lib.tnt_params_set(self.h, C.byref(p)))

    def sys_info(self) -> str:
        buf = C.create_string_buffer(2048)
        self._chk(self.lib.tnt_sys_info(self.h, buf, 2048))
        return buf.value.decode()

    def launch_count(self) -> int:
        return int(self.lib.tnt_launch_count(self.h))

    def profile_select(self, kernel_class: str | None):
        self._chk(self.lib.tnt_profile_select(self.h, (kernel_class or "").encode()))

    def profile_read(self):
        """(summed ms, launches, summed algorithmic work) of the selected kernel class
        since the last read; work is FLOPs or bytes depending on the class."""
        ms, n, w = C.c_double(), C.c_int64(), C.c_double()
        self._chk(self.lib.tnt_profile_read(self.h, C.byref(ms), C.byref(n), C.byref(w)))
        return ms.value, n.value, w.value

    # ---------------------------------------------------------------- kernels
    def theta_form(self, A, B, out=None):
        chl, d, chm = A.shape
        chr_ = B.shape[2]
        out = out if out is not None else torch.empty((chl, d, d, chr_), dtype=CDT, device=A.device)
        self._chk(self.lib.tnt_theta_form(self.h, _ptr(A), _ptr(B), chl, d, chm, chr_, _ptr(out)))
        return out

    def gate_apply(self, G, theta, out=None):
        chl, d, _, chr_ = theta.shape
        out = out if out is not None else torch.empty_like(theta)
        self._chk(self.lib.tnt_gate_apply(self.h, _ptr(G), _ptr(theta), chl, d, chr_, _ptr(out)))
        return out

    def heff_apply(self, Lenv, W1, W2, Renv, theta, precision=TNT_PREC_FP64, out=None):
        chl, d, _, chr_ = theta.shape
        D = W1.shape[0]
        out = out if out is not None else torch.empty_like(theta)
        self._chk(self.lib.tnt_heff_apply(self.h, _ptr(Lenv), _ptr(W1), _ptr(W2), _ptr(Renv),
                                          _ptr(theta), chl, d, D, chr_, precision, _ptr(out)))
        return out

    def heff_apply_noalloc(self, Lenv, W1, W2, Renv, theta, out):
        """FP64 H_eff.theta that makes no device allocation (fixed 16 MiB static scratch);
        `out` must be supplied by the caller."""
        chl, d, _, chr_ = theta.shape
        D = W1.shape[0]
        self._chk(self.lib.tnt_heff_apply_noalloc(self.h, _ptr(Lenv), _ptr(W1), _ptr(W2),
                                                  _ptr(Renv), _ptr(theta), chl, d, D, chr_,
                                                  _ptr(out)))
        return out

    def env_left(self, Lenv, W, A, out=None):
        chl, d, chr_ = A.shape
        D = W.shape[0]
        out = out if out is not None else torch.empty((chr_, D, chr_), dtype=CDT, device=A.device)
        self._chk(self.lib.tnt_env_left(self.h, _ptr(Lenv), _ptr(W), _ptr(A), chl, d, D, chr_,
                                        _ptr(out)))
        return out

    def env_right(self, Renv, W, B, out=None):
        chl, d, chr_ = B.shape
        D = W.shape[0]
        out = out if out is not None else torch.empty((chl, D, chl), dtype=CDT, device=B.device)
        self._chk(self.lib.tnt_env_right(self.h, _ptr(Renv), _ptr(W), _ptr(B), chl, d, D, chr_,
                                         _ptr(out)))
        return out

    def lanczos_ground(self, Lenv, W1, W2, Renv, theta):
        """theta (device) is overwritten by the eigenvector; returns the result dict."""
        chl, d, _, chr_ = theta.shape
        D = W1.shape[0]
        res = L.tnt_lanczos_result()
        self._chk(self.lib.tnt_lanczos_ground(self.h, _ptr(Lenv), _ptr(W1), _ptr(W2), _ptr(Renv),
                                              chl, d, D, chr_, _ptr(theta), C.byref(res)),
                  ok=(0, L.TNT_E_NOCONV))
        return _struct_dict(res)

    def svd_trunc(self, M, row_q=None, col_q=None, side=TNT_SVD_LEFT, renorm=False):
        """Truncated SVD of the m x n device matrix M; returns (U, X, S, bond_q, info)."""
        m, n = M.shape
        chi_max = self.params()["chi_max"]
        cap = int(min(m, n, chi_max))
        U = torch.empty(m * cap, dtype=CDT, device=M.device)
        X = torch.empty(cap * n, dtype=CDT, device=M.device)
        S = np.zeros(cap)
        bq = np.zeros(cap, dtype=np.int64)
        res = L.tnt_trunc_result()
        if row_q is not None:
            rq = np.ascontiguousarray(row_q, dtype=np.int64)
            cq = np.ascontiguousarray(col_q, dtype=np.int64)
            prq, pcq = rq.ctypes.data, cq.ctypes.data
        else:
            prq = pcq = None
        self._chk(self.lib.tnt_svd_trunc(self.h, _ptr(M), m, n, prq, pcq, side, int(renorm),
                                         _ptr(U), _ptr(X), S.ctypes.data, bq.ctypes.data,
                                         C.byref(res)))
        k = res.chi
        return (U[: m * k].view(m, k), X[: k * n].view(k, n), S[:k].copy(), bq[:k].copy(),
                _struct_dict(res))

    # ---------------------------------------------------------------- U(1) blocks
    def u1_size(self, prob: "U1Problem") -> int:
        n = C.c_int64()
        self._chk(self.lib.tnt_u1_size(C.byref(prob.s), C.byref(n)))
        return n.value

    def u1_pack(self, prob: "U1Problem", theta):
        x = torch.empty(self.u1_size(prob), dtype=torch.complex128, device=theta.device)
        self._chk(self.lib.tnt_u1_pack(self.h, C.byref(prob.s), _ptr(theta), _ptr(x)))
        return x

    def u1_unpack(self, prob: "U1Problem", x):
        th = torch.empty((prob.chl, prob.d, prob.d, prob.chr), dtype=torch.complex128,
                         device=x.device)
        self._chk(self.lib.tnt_u1_unpack(self.h, C.byref(prob.s), _ptr(x), _ptr(th)))
        return th

    def heff_apply_u1(self, probs, x, precision=TNT_PREC_FP64, out=None):
        """y = H_eff x for the problems' compact vectors back to back; returns (y, flops)."""
        probs = list(probs)
        arr = (L.tnt_u1_problem * len(probs))(*[p.s for p in probs])
        y = torch.empty_like(x) if out is None else out
        fl = C.c_double()
        self._chk(self.lib.tnt_heff_apply_u1(self.h, len(probs), arr, _ptr(x), _ptr(y),
                                             precision, C.byref(fl)))
        return y, fl.value

    def lanczos_ground_u1(self, prob: "U1Problem", x):
        """x (compact, device) is overwritten by the eigenvector; returns the result dict."""
        res = L.tnt_lanczos_result()
        self._chk(self.lib.tnt_lanczos_ground_u1(self.h, C.byref(prob.s), _ptr(x), C.byref(res)),
                  ok=(0, L.TNT_E_NOCONV))
        return _struct_dict(res)

    def lanczos_ground_u1_batched(self, probs, x):
        """x: the problems' compact start vectors back to back (overwritten by the ground
        states); returns one result dict per problem."""
        probs = list(probs)
        arr = (L.tnt_u1_problem * len(probs))(*[p.s for p in probs])
        res = (L.tnt_lanczos_result * len(probs))()
        self._chk(self.lib.tnt_lanczos_ground_u1_batched(self.h, len(probs), arr, _ptr(x), res),
                  ok=(0, L.TNT_E_NOCONV))
        return [_struct_dict(r) for r in res]

    def matmul(self, A, B, conj_a=False, conj_b=False, out=None):
        """C = op(A) op(B) (FP64 accuracy) for 2-D complex128 device tensors; A may be a
        transposed view (any strides)."""
        M, K = A.shape
        K2, N = B.shape
        if K != K2:
            raise ValueError("inner dimensions differ")
        C = torch.empty((M, N), dtype=torch.complex128, device=A.device) if out is None else out
        self._chk(self.lib.tnt_matmul(self.h, M, N, K, A.data_ptr(), A.stride(0), A.stride(1),
                                      int(conj_a), B.data_ptr(), B.stride(0), B.stride(1),
                                      int(conj_b), _ptr(C), C.stride(0)))
        return C

    def set_fp64_gemm(self, engine: int):
        self._chk(self.lib.tnt_set_fp64_gemm(self.h, engine))

    def set_svd_zero_tol(self, tol: float):
        """Automatic blocking of unlabelled SVDs (tol < 0: off)."""
        self._chk(self.lib.tnt_set_svd_zero_tol(self.h, float(tol)))

    def set_graphs(self, on: bool):
        self._chk(self.lib.tnt_set_graphs(self.h, 1 if on else 0))

    def u1_tiles(self, probs):
        probs = list(probs)
        arr = (L.tnt_u1_problem * len(probs))(*[p.s for p in probs])
        t = (C.c_int * 3)()
        self._chk(self.lib.tnt_u1_tiles(self.h, len(probs), arr, t))
        return tuple(t)

    # ---------------------------------------------------------------- objects
    def mpo_bose_hubbard(self, L_, n_max, J, U, mu=0.0, V=0.0, j_c=0.0) -> "Mpo":
        h = C.c_void_p()
        self._chk(self.lib.tnt_mpo_bose_hubbard(self.h, L_, n_max, J, U, mu, V, j_c, C.byref(h)))
        return Mpo(self, h)

    def mpo_spin_heisenberg(self, L_, two_s, J=1.0, Jz=None, hz=0.0) -> "Mpo":
        h = C.c_void_p()
        Jz = J if Jz is None else Jz
        self._chk(self.lib.tnt_mpo_spin_heisenberg(self.h, L_, two_s, J, Jz, hz, C.byref(h)))
        return Mpo(self, h)

    def mpo_create(self, Ws, left, right, wq=None) -> "Mpo":
        Ws = [np.ascontiguousarray(W, dtype=np.complex128) for W in Ws]
        D, d = Ws[0].shape[0], Ws[0].shape[2]
        lb = np.ascontiguousarray(left, dtype=np.complex128)
        rb = np.ascontiguousarray(right, dtype=np.complex128)
        wp = None
        if wq is not None:
            wqa = np.ascontiguousarray(wq, dtype=np.int32)
            wp = wqa.ctypes.data
        sp = (C.c_void_p * len(Ws))(*[W.ctypes.data for W in Ws])
        h = C.c_void_p()
        self._chk(self.lib.tnt_mpo_create(self.h, len(Ws), d, D, sp, lb.ctypes.data,
                                          rb.ctypes.data, wp, C.byref(h)))
        return Mpo(self, h)

    def mps_create(self, tensors, charges=None, chi_cap=None) -> "Mps":
        Ls = len(tensors)
        d = tensors[0].shape[1]
        chi = np.array([1] + [t.shape[2] for t in tensors], dtype=np.int64)
        cap = int(chi_cap if chi_cap is not None else chi.max())
        arrs = [np.ascontiguousarray(t, dtype=np.complex128) for t in tensors]
        sp = (C.c_void_p * Ls)(*[a.ctypes.data for a in arrs])
        qp = None
        if charges is not None:
            qa = [np.ascontiguousarray(q, dtype=np.int64) for q in charges]
            qp = (C.c_void_p * (Ls + 1))(*[a.ctypes.data for a in qa])
        h = C.c_void_p()
        self._chk(self.lib.tnt_mps_create(self.h, Ls, d, cap, chi.ctypes.data, sp, qp, C.byref(h)))
        return Mps(self, h)

    def mps_product(self, occupations, d, chi_cap) -> "Mps":
        occ = np.ascontiguousarray(occupations, dtype=np.int32)
        h = C.c_void_p()
        self._chk(self.lib.tnt_mps_product(self.h, len(occ), d, chi_cap, occ.ctypes.data,
                                           C.byref(h)))
        return Mps(self, h)

    def mps_load(self, path: str, chi_cap: int, restore_params: bool = False) -> "Mps":
        """MPS from a file written by Mps.save (tnt_mps_load)."""
        h = C.c_void_p()
        self._chk(self.lib.tnt_mps_load(self.h, str(path).encode(), int(chi_cap),
                                        int(restore_params), C.byref(h)))
        return Mps(self, h)

    def dmrg_sweep_batched(self, runs) -> list:
        """One lock-step sweep of several chains' Dmrg handles (tnt_dmrg_sweep_batched);
        returns each chain's sweep statistics."""
        n = len(runs)
        hs = (C.c_void_p * n)(*[r.h.value for r in runs])
        st = (L.tnt_sweep_stats * n)()
        self._chk(self.lib.tnt_dmrg_sweep_batched(self.h, n, hs, st))
        return [_struct_dict(x) for x in st]

    def dmrg_create(self, mps: "Mps", mpo: "Mpo") -> "Dmrg":
        h = C.c_void_p()
        self._chk(self.lib.tnt_dmrg_create(self.h, mps.h, mpo.h, C.byref(h)))
        return Dmrg(self, h, mps, mpo)

    def tebd_create(self, mps: "Mps", n_max, J, U, dt, mu=0.0) -> "Tebd":
        h = C.c_void_p()
        self._chk(self.lib.tnt_tebd_create(self.h, mps.h, n_max, J, U, mu, dt, C.byref(h)))
        return Tebd(self, h, mps)

    def tebd_create_spin(self, mps: "Mps", two_s, J, dt, Jz=None, hz=0.0) -> "Tebd":
        h = C.c_void_p()
        Jz = J if Jz is None else Jz
        self._chk(self.lib.tnt_tebd_create_spin(self.h, mps.h, two_s, J, Jz, hz, dt, C.byref(h)))
        return Tebd(self, h, mps)

    def tebd_create_bonds(self, mps: "Mps", bond_hs, dt) -> "Tebd":
        hs = [np.ascontiguousarray(x, dtype=np.complex128) for x in bond_hs]
        hp = (C.c_void_p * len(hs))(*[x.ctypes.data for x in hs])
        h = C.c_void_p()
        self._chk(self.lib.tnt_tebd_create_bonds(self.h, mps.h, hp, dt, C.byref(h)))
        return Tebd(self, h, mps)


class Mpo:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def __del__(self):
        if getattr(self, "h", None):
            self.ctx.lib.tnt_mpo_destroy(self.h)
            self.h = None


class Mps:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        Ls, d = C.c_int(), C.c_int()
        ctx._chk(ctx.lib.tnt_mps_length(h, C.byref(Ls), C.byref(d)))
        self.L, self.d = Ls.value, d.value

    def bond_dim(self, k) -> int:
        v = C.c_int64()
        self.ctx._chk(self.ctx.lib.tnt_mps_bond_dim(self.h, k, C.byref(v)))
        return v.value

    def site(self, j) -> np.ndarray:
        shape = (self.bond_dim(j), self.d, self.bond_dim(j + 1))
        out = np.zeros(shape, dtype=np.complex128)
        self.ctx._chk(self.ctx.lib.tnt_mps_get_site(self.ctx.h, self.h, j, out.ctypes.data,
                                                    out.size))
        return out

    def charges(self, k) -> np.ndarray:
        out = np.zeros(self.bond_dim(k), dtype=np.int64)
        self.ctx._chk(self.ctx.lib.tnt_mps_get_charges(self.h, k, out.ctypes.data, out.size))
        return out

    def tensors(self):
        return [self.site(j) for j in range(self.L)]

    def expect_mpo(self, mpo: Mpo) -> float:
        v = C.c_double()
        self.ctx._chk(self.ctx.lib.tnt_mps_expect_mpo(self.ctx.h, self.h, mpo.h, C.byref(v)))
        return v.value

    def density(self) -> np.ndarray:
        out = np.zeros(self.L)
        self.ctx._chk(self.ctx.lib.tnt_mps_density(self.ctx.h, self.h, out.ctypes.data_as(L.PD)))
        return out

    def bdagb(self) -> np.ndarray:
        """<b+_i b_j> / <psi|psi> as an L x L complex matrix."""
        out = np.zeros((self.L, self.L), dtype=np.complex128)
        self.ctx._chk(self.ctx.lib.tnt_mps_bdagb(self.ctx.h, self.h, out.ctypes.data))
        return out

    def norm2(self) -> float:
        v = C.c_double()
        self.ctx._chk(self.ctx.lib.tnt_mps_norm2(self.ctx.h, self.h, C.byref(v)))
        return v.value

    def overlap(self, other: "Mps") -> complex:
        """<self|other> (tnt_mps_overlap)."""
        v = L.tnt_cplx()
        self.ctx._chk(self.ctx.lib.tnt_mps_overlap(self.ctx.h, self.h, other.h, C.byref(v)))
        return complex(v.re, v.im)

    def set_charges(self, bond: int, q):
        """Replace the U(1) labels of one bond (tnt_mps_set_charges)."""
        qa = np.ascontiguousarray(q, dtype=np.int64)
        self.ctx._chk(self.ctx.lib.tnt_mps_set_charges(self.ctx.h, self.h, bond, qa.ctypes.data))

    def save(self, path: str):
        """Write the MPS and the context's parameters to a file (tnt_mps_save)."""
        self.ctx._chk(self.ctx.lib.tnt_mps_save(self.ctx.h, self.h, str(path).encode()))

    def __del__(self):
        if getattr(self, "h", None):
            self.ctx.lib.tnt_mps_destroy(self.h)
            self.h = None


class Dmrg:
    def __init__(self, ctx: Context, h, mps: Mps, mpo: Mpo):
        self.ctx, self.h, self.mps, self.mpo = ctx, h, mps, mpo

    def sweep(self) -> dict:
        st = L.tnt_sweep_stats()
        self.ctx._chk(self.ctx.lib.tnt_dmrg_sweep(self.ctx.h, self.h, C.byref(st)))
        return _struct_dict(st)

    def sweep1(self, alpha: float) -> dict:
        """One single-site sweep with subspace expansion (mixing factor alpha)."""
        st = L.tnt_sweep_stats()
        self.ctx._chk(self.ctx.lib.tnt_dmrg_sweep1(self.ctx.h, self.h, float(alpha), C.byref(st)))
        return _struct_dict(st)

    def update(self, bond: int, direction: int) -> tuple:
        """One two-site update (tnt_dmrg_update): (Lanczos result, truncation result);
        an eigensolve that hit its cap is returned, not raised."""
        lz, tr = L.tnt_lanczos_result(), L.tnt_trunc_result()
        self.ctx._chk(self.ctx.lib.tnt_dmrg_update(self.ctx.h, self.h, bond, direction,
                                                   C.byref(lz), C.byref(tr)), ok=(0, 4))
        return _struct_dict(lz), _struct_dict(tr)

    def update_energies(self) -> np.ndarray:
        """Energy of every update of the last sweep, in update order
        (tnt_dmrg_update_energies)."""
        n = C.c_int64()
        self.ctx._chk(self.ctx.lib.tnt_dmrg_update_energies(self.h, None, 0, C.byref(n)))
        out = np.zeros(n.value, dtype=np.float64)
        self.ctx._chk(self.ctx.lib.tnt_dmrg_update_energies(
            self.h, out.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n)))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            self.ctx.lib.tnt_dmrg_destroy(self.h)
            self.h = None


class Tebd:
    def __init__(self, ctx: Context, h, mps: Mps):
        self.ctx, self.h, self.mps = ctx, h, mps

    def step(self) -> dict:
        st = L.tnt_step_stats()
        self.ctx._chk(self.ctx.lib.tnt_tebd_step(self.ctx.h, self.h, C.byref(st)))
        return _struct_dict(st)

    def gate(self, bond: int, G, direction: int = 1) -> dict:
        """One gate G[(s1' s2'), (s1 s2)] on bond (bond, bond+1) (tnt_tebd_gate)."""
        g = np.ascontiguousarray(G, dtype=np.complex128)
        tr = L.tnt_trunc_result()
        self.ctx._chk(self.ctx.lib.tnt_tebd_gate(self.ctx.h, self.h, bond, g.ctypes.data,
                                                 direction, C.byref(tr)))
        return _struct_dict(tr)

    def centre(self) -> int:
        v = C.c_int()
        self.ctx._chk(self.ctx.lib.tnt_tebd_centre(self.h, C.byref(v)))
        return v.value

    def __del__(self):
        if getattr(self, "h", None):
            self.ctx.lib.tnt_tebd_destroy(self.h)
            self.h = None


class U1Problem:
    """One U(1) H_eff problem for the grouped calls: device L, W1, W2, R and host labels
    (kept alive here while the C struct points at them)."""

    def __init__(self, Lenv, W1, W2, Renv, qa, qb, wq=(0, 1, -1, 0)):
        self.chl, D, _ = Lenv.shape
        self.chr = Renv.shape[0]
        self.d = W1.shape[2]
        self.qa = np.ascontiguousarray(qa, dtype=np.int64)
        self.qb = np.ascontiguousarray(qb, dtype=np.int64)
        self.wq = np.ascontiguousarray(wq, dtype=np.int32)
        self.tensors = (Lenv, W1, W2, Renv)
        self.s = L.tnt_u1_problem(_ptr(Lenv), _ptr(W1), _ptr(W2), _ptr(Renv), self.chl, self.d,
                                  D, self.chr, self.qa.ctypes.data, self.qb.ctypes.data,
                                  self.wq.ctypes.data)
