"""Python binding of libpwh: the plane-wave Kohn-Sham Hamiltonian H|psi> and a
block Davidson eigensolver on one GB300.

Argument marshalling only: every step of the computation runs in the CUDA
library ``_lib/libpwh.so`` (built by ``paper_1709_10010_gb300.build``).  PyTorch
supplies device memory and the CUDA stream.  There is no CPU fallback: if the
library is missing, loading it raises.

Band blocks are torch complex128 tensors of shape (nb, npw) with unit stride
along npw: row b is band b, i.e. column-major npw x nb with ld = stride(0).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpwh.so")

PWH_FP64, PWH_MIXED, PWH_MIXED_FAST = 0, 1, 2
PRECISIONS = {"fp64": PWH_FP64, "mixed": PWH_MIXED, "mixed_fast": PWH_MIXED_FAST}
STATUS = {0: "PWH_OK", 1: "PWH_ERR_ARG", 2: "PWH_ERR_CUDA", 3: "PWH_ERR_OOM",
          4: "PWH_ERR_NOT_CONVERGED", 5: "PWH_ERR_NONFINITE", 6: "PWH_ERR_TIMEOUT",
          7: "PWH_ERR_STATE"}

_c_i32, _c_i64, _c_p, _c_d = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double


class SystemDesc(ctypes.Structure):
    _fields_ = [("lattice", _c_d * 9), ("kpoint", _c_d * 3), ("ecut_ha", _c_d),
                ("fft", _c_i32 * 3), ("precision", _c_i32), ("stream", _c_p)]


class DavidsonOpts(ctypes.Structure):
    _fields_ = [("nb", _c_i32), ("max_iter", _c_i32), ("max_subspace_mult", _c_i32),
                ("precond", _c_i32), ("mixed", _c_i32), ("jd_inner", _c_i32),
                ("tol", _c_d), ("switch_tol", _c_d)]


class DavidsonStats(ctypes.Structure):
    _fields_ = [("iters", _c_i32), ("n_apply", _c_i32), ("n_apply_fp64", _c_i32),
                ("switch_iter", _c_i32), ("t_total_s", _c_d), ("t_mixed_s", _c_d),
                ("t_fp64_s", _c_d), ("max_resid", _c_d)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PRECOND = {"tpa": 0, "mlp": 1, "none": 2}


class TraceEntry(ctypes.Structure):
    _fields_ = [("iter", _c_i32), ("fp64", _c_i32), ("m", _c_i32), ("n_above", _c_i32),
                ("max_resid", _c_d), ("t_s", _c_d)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", _c_i64), ("total_ms", _c_d),
                ("flops", _c_d), ("bytes", _c_d)]


class PwhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


# name -> (restype, argtypes); must match include/pwh.h
SIGNATURES = {
    "pwh_create_system": (_c_i32, [ctypes.POINTER(SystemDesc), ctypes.POINTER(_c_p)]),
    "pwh_destroy_system": (_c_i32, [_c_p]),
    "pwh_get_dims": (_c_i32, [_c_p, ctypes.POINTER(_c_i64), ctypes.POINTER(_c_i32),
                              ctypes.POINTER(_c_i64)]),
    "pwh_get_miller": (_c_i32, [_c_p, _c_p]),
    "pwh_get_kinetic": (_c_i32, [_c_p, _c_p]),
    "pwh_get_internal_order": (_c_i32, [_c_p, _c_p]),
    "pwh_set_potential": (_c_i32, [_c_p, _c_p, _c_i32]),
    "pwh_set_projectors": (_c_i32, [_c_p, _c_i32, _c_p, _c_p, _c_i32, _c_i32]),
    "pwh_set_precision": (_c_i32, [_c_p, _c_i32]),
    "pwh_apply_h": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_i64]),
    "pwh_apply_h_host": (_c_i32, [_c_p, _c_i32, _c_p, _c_p]),
    "pwh_apply_h_internal": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_i64]),
    "pwh_get_gamma_half": (_c_i32, [_c_p, ctypes.POINTER(_c_i64), _c_p]),
    "pwh_apply_h_gamma": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_i64]),
    "pwh_sync": (_c_i32, [_c_p]),
    "pwh_batch_davidson_solve": (_c_i32, [_c_i32, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_i32]),
    "pwh_subspace_eigh": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_i32, _c_p, _c_p, _c_p, _c_i64,
                                   _c_i32, _c_i32]),
    "pwh_mlp_num_params": (_c_i32, [ctypes.POINTER(_c_i32)]),
    "pwh_mlp_forward": (_c_i32, [_c_p, _c_p, _c_p, _c_i64, _c_p]),
    "pwh_mlp_loss_grad": (_c_i32, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_i64, _c_d, _c_p, _c_p]),
    "pwh_mlp_adam": (_c_i32, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_i32, ctypes.c_float]),
    "pwh_mlp_training_rows": (_c_i32, [_c_p, _c_i32, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "pwh_set_mlp": (_c_i32, [_c_p, _c_p, _c_i32]),
    "pwh_get_shells": (_c_i32, [_c_p, ctypes.POINTER(_c_i32), _c_p, _c_p]),
    "pwh_set_kernel_timing": (_c_i32, [_c_p, _c_i32]),
    "pwh_get_kernel_times": (_c_i32, [_c_p, _c_p, _c_i32, ctypes.POINTER(_c_i32)]),
    "pwh_launch_count": (_c_i32, [ctypes.POINTER(_c_i64)]),
    "pwh_davidson_solve": (_c_i32, [_c_p, ctypes.POINTER(DavidsonOpts), _c_p, _c_i64, _c_p,
                                    ctypes.POINTER(DavidsonStats)]),
    "pwh_davidson_solve_host": (_c_i32, [_c_p, ctypes.POINTER(DavidsonOpts), _c_p, _c_p,
                                         ctypes.POINTER(DavidsonStats)]),
    "pwh_davidson_solve_gamma": (_c_i32, [_c_p, ctypes.POINTER(DavidsonOpts), _c_p, _c_i64, _c_p,
                                          ctypes.POINTER(DavidsonStats)]),
    "pwh_get_davidson_trace": (_c_i32, [_c_p, _c_i32, _c_p, ctypes.POINTER(_c_i32)]),
    "pwh_set_overlap": (_c_i32, [_c_p, _c_p, _c_i32, _c_i32]),
    "pwh_apply_s": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_i64]),
    "pwh_exx_apply": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_i32, _c_p, _c_i64, _c_p,
                               _c_i64]),
    "pwh_set_ace": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_d, ctypes.POINTER(_c_i32)]),
    "pwh_density": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_p]),
    "pwh_hartree_xc": (_c_i32, [_c_p, _c_p, _c_p, _c_p, _c_p]),
    "pwh_apply_local_noalloc": (_c_i32, [_c_p, _c_i32, _c_p, _c_i64, _c_p, _c_i64]),
    "pwh_subspace_cholqr": (_c_i32, [_c_p, _c_i32, _c_i32, _c_p, _c_p, _c_d, _c_p,
                                     ctypes.POINTER(_c_i32)]),
    "pwh_subspace_gemm": (_c_i32, [_c_p, _c_i32, _c_i32, _c_i32, _c_i32, _c_i32, _c_p, _c_p, _c_i64,
                                   _c_p, _c_i64, _c_p, _c_p, _c_i64]),
    "pwh_last_error": (ctypes.c_char_p, []),
}

_lib = None
MLP_PARAMS = 4545   # network parameters; the blob adds 8 feature-range floats
MLP_BLOB = MLP_PARAMS + 8


def lib():
    """The loaded libpwh (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpwh not built: {LIB_PATH} is missing "
                               "(run python -m paper_1709_10010_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise PwhError(status, lib().pwh_last_error().decode())


def launch_count() -> int:
    """Kernels launched by libpwh in this process so far."""
    c = _c_i64()
    _check(lib().pwh_launch_count(ctypes.byref(c)))
    return int(c.value)


def _torch():
    import torch
    return torch


def _band_ptr(t, npw: int):
    """Device pointer and leading dimension of a (nb, npw) complex128 tensor."""
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128):
        raise TypeError("band blocks must be CUDA complex128 tensors")
    if t.dim() != 2 or t.shape[1] != npw or t.stride(1) != 1:
        raise ValueError(f"expected shape (nb, {npw}) with unit stride along npw")
    ld = t.stride(0) if t.shape[0] > 1 else npw
    return ctypes.c_void_p(t.data_ptr()), ld


class System:
    """One plane-wave system (cell, k-point, cutoff) living on the current GPU."""

    def __init__(self, lattice, kpoint=(0.0, 0.0, 0.0), ecut_ha=10.0, fft=(0, 0, 0),
                 precision="fp64", stream=None):
        d = SystemDesc()
        lat = np.asarray(lattice, dtype=np.float64).reshape(9)
        for i in range(9):
            d.lattice[i] = float(lat[i])
        for i in range(3):
            d.kpoint[i] = float(kpoint[i])
            d.fft[i] = int(fft[i])
        d.ecut_ha = float(ecut_ha)
        d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        d.stream = ctypes.c_void_p(int(stream))
        h = ctypes.c_void_p()
        _check(lib().pwh_create_system(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        n = _c_i64()
        f = (_c_i32 * 3)()
        ns = _c_i64()
        _check(lib().pwh_get_dims(h, ctypes.byref(n), f, ctypes.byref(ns)))
        self.npw, self.fft, self.nsticks = int(n.value), tuple(int(x) for x in f), int(ns.value)
        self.nproj = 0

    @classmethod
    def from_cell(cls, cell, **kw):
        return cls(cell.lattice, cell.kpoint, cell.ecut_ha, **kw)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pwh_destroy_system(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- basis
    def miller(self) -> np.ndarray:
        out = np.empty((self.npw, 3), dtype=np.int32)
        _check(lib().pwh_get_miller(self._h, out.ctypes.data_as(_c_p)))
        return out

    def kinetic(self) -> np.ndarray:
        out = np.empty(self.npw, dtype=np.float64)
        _check(lib().pwh_get_kinetic(self._h, out.ctypes.data_as(_c_p)))
        return out

    def internal_order(self) -> np.ndarray:
        out = np.empty(self.npw, dtype=np.int32)
        _check(lib().pwh_get_internal_order(self._h, out.ctypes.data_as(_c_p)))
        return out

    # ---------------------------------------------------------------- inputs
    def set_potential(self, v_r):
        torch = _torch()
        if isinstance(v_r, torch.Tensor):
            t = v_r.contiguous()
            assert t.dtype == torch.float64 and t.numel() == int(np.prod(self.fft))
            _check(lib().pwh_set_potential(self._h, ctypes.c_void_p(t.data_ptr()), int(t.is_cuda)))
            torch.cuda.current_stream().synchronize() if t.is_cuda else None
        else:
            a = np.ascontiguousarray(v_r, dtype=np.float64)
            assert a.size == int(np.prod(self.fft))
            _check(lib().pwh_set_potential(self._h, a.ctypes.data_as(_c_p), 0))

    def set_projectors(self, beta, D):
        """beta: (P, npw) complex128 in public order; D: (P,) real diagonal or
        (P, P) complex Hermitian."""
        beta = np.ascontiguousarray(beta, dtype=np.complex128)
        P = beta.shape[0] if beta.ndim == 2 else 0
        if P == 0:
            _check(lib().pwh_set_projectors(self._h, 0, None, None, 1, 0))
            self.nproj = 0
            return
        assert beta.shape == (P, self.npw)
        D = np.asarray(D)
        if D.ndim == 1:
            Dd = np.ascontiguousarray(D, dtype=np.float64)
            diag = 1
        else:
            Dd = np.asfortranarray(D, dtype=np.complex128)  # column-major
            diag = 0
        _check(lib().pwh_set_projectors(self._h, P, beta.ctypes.data_as(_c_p),
                                        Dd.ctypes.data_as(_c_p), diag, 0))
        self.nproj = P

    def set_precision(self, precision):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib().pwh_set_precision(self._h, p))

    def set_kernel_timing(self, on: bool):
        _check(lib().pwh_set_kernel_timing(self._h, int(bool(on))))

    def kernel_times(self) -> dict:
        """{family: dict(launches, ms, flops, bytes)} accumulated while timing is on."""
        arr = (KernelTime * 32)()
        n = _c_i32()
        _check(lib().pwh_get_kernel_times(self._h, arr, 32, ctypes.byref(n)))
        return {arr[i].name.decode(): {"launches": int(arr[i].launches), "ms": float(arr[i].total_ms),
                                       "flops": float(arr[i].flops), "bytes": float(arr[i].bytes)}
                for i in range(min(n.value, 32))}

    def subspace_eigh(self, H, nk, Q=None, warm=0, precision="fp64"):
        """Lowest nk eigenpairs of a Hermitian matrix given as an (n, n) CUDA
        complex128 tensor Ht with Ht[j, i] = H[i, j] (column-major H).  Returns
        (theta, C) CUDA tensors, C of shape (nk, n) holding eigenvectors as
        rows.  Q: optional (n_max, n_max) tensor (row j = eigenvector j) that
        receives all n eigenvectors; with warm > 0 it must hold on entry the
        eigenvectors of the leading warm x warm block.  precision: "fp64"
        (FP64-accurate) or "mixed" (the FP32 result)."""
        torch = _torch()
        n = int(H.shape[0])
        Hc = H.contiguous()
        theta = torch.empty(nk, dtype=torch.float64, device=H.device)
        C = torch.empty((nk, n), dtype=torch.complex128, device=H.device)
        qp = ctypes.c_void_p(Q.data_ptr()) if Q is not None else None
        ldq = int(Q.shape[1]) if Q is not None else 0
        _check(lib().pwh_subspace_eigh(self._h, n, ctypes.c_void_p(Hc.data_ptr()), n, int(nk),
                                       ctypes.c_void_p(theta.data_ptr()),
                                       ctypes.c_void_p(C.data_ptr()), qp, ldq, int(warm),
                                       PRECISIONS[precision]))
        return theta, C

    def cholqr(self, S, t0=None, drop_rel=0.0, precision="fp64"):
        """Cholesky-QR factor of a Gram matrix S = T^H T given as a (k, k) CUDA
        complex128 tensor holding S^T (column-major S); returns (Tr as a (k, k)
        tensor holding Tr^T, kept) with T Tr orthonormal in its first kept
        columns."""
        torch = _torch()
        k = int(S.shape[0])
        Sc = S.contiguous()
        Tr = torch.empty((k, k), dtype=torch.complex128, device=S.device)
        kept = _c_i32()
        tp = ctypes.c_void_p(t0.data_ptr()) if t0 is not None else None
        _check(lib().pwh_subspace_cholqr(self._h, PRECISIONS[precision], k,
                                         ctypes.c_void_p(Sc.data_ptr()), tp, float(drop_rel),
                                         ctypes.c_void_p(Tr.data_ptr()), ctypes.byref(kept)))
        return Tr, kept.value

    def gemm(self, A, B, C=None, conj_a=False, alpha=1.0, beta=0.0, precision="fp64"):
        """C = alpha op(A) B + beta C on the device (the eigensolver's subspace
        GEMM).  Matrices are CUDA complex128 tensors holding column-major
        matrices as their transposes (row j of the tensor = column j), like
        subspace_eigh: A has shape (cols, rows) of the stored A, op(A) = A^H
        when conj_a.  Returns C (shape (N, M))."""
        torch = _torch()
        ka, ra = int(A.shape[0]), int(A.shape[1])     # stored A: ra rows x ka columns
        M, K = (ka, ra) if conj_a else (ra, ka)
        N = int(B.shape[0])
        assert int(B.shape[1]) == K, "inner dimensions differ"
        if C is None:
            C = torch.zeros((N, M), dtype=torch.complex128, device=A.device)
        al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
        be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
        _check(lib().pwh_subspace_gemm(self._h, PRECISIONS[precision], int(bool(conj_a)), M, N, K, al,
                                       ctypes.c_void_p(A.data_ptr()), max(1, ra),
                                       ctypes.c_void_p(B.data_ptr()), max(1, K), be,
                                       ctypes.c_void_p(C.data_ptr()), max(1, M)))
        return C

    def sync(self):
        """Wait for the stream; raises PwhError(PWH_ERR_TIMEOUT) if a bounded
        device wait gave up."""
        _check(lib().pwh_sync(self._h))

    # ---------------------------------------------------------------- apply
    def apply_h(self, psi, hpsi=None):
        """hpsi = H psi on the device; psi (nb, npw) complex128 CUDA tensor."""
        torch = _torch()
        if hpsi is None:
            hpsi = torch.empty_like(psi, memory_format=torch.contiguous_format)
        p, ldp = _band_ptr(psi, self.npw)
        h, ldh = _band_ptr(hpsi, self.npw)
        _check(lib().pwh_apply_h(self._h, int(psi.shape[0]), p, ldp, h, ldh))
        return hpsi

    def apply_h_internal(self, psi, hpsi=None):
        torch = _torch()
        if hpsi is None:
            hpsi = torch.empty_like(psi, memory_format=torch.contiguous_format)
        p, ldp = _band_ptr(psi, self.npw)
        h, ldh = _band_ptr(hpsi, self.npw)
        _check(lib().pwh_apply_h_internal(self._h, int(psi.shape[0]), p, ldp, h, ldh))
        return hpsi

    def gamma_half(self) -> np.ndarray:
        """Public indices of the half sphere that stores real bands at k = 0."""
        n = _c_i64()
        _check(lib().pwh_get_gamma_half(self._h, ctypes.byref(n), None))
        idx = np.empty(n.value, dtype=np.int32)
        _check(lib().pwh_get_gamma_half(self._h, ctypes.byref(n), idx.ctypes.data_as(_c_p)))
        return idx

    def apply_h_gamma(self, psi, hpsi=None):
        """hpsi = H psi for real bands on the half sphere; psi (nb, npw_half)
        complex128 CUDA tensor."""
        torch = _torch()
        n = _c_i64()
        _check(lib().pwh_get_gamma_half(self._h, ctypes.byref(n), None))
        if hpsi is None:
            hpsi = torch.empty_like(psi, memory_format=torch.contiguous_format)
        p, ldp = _band_ptr(psi, n.value)
        h, ldh = _band_ptr(hpsi, n.value)
        _check(lib().pwh_apply_h_gamma(self._h, int(psi.shape[0]), p, ldp, h, ldh))
        return hpsi

    def apply_local_noalloc(self, psi, hpsi):
        """(kinetic + local potential) psi in FP64, internal order, into the
        caller's hpsi; the library allocates nothing during the call."""
        p, ldp = _band_ptr(psi, self.npw)
        h, ldh = _band_ptr(hpsi, self.npw)
        _check(lib().pwh_apply_local_noalloc(self._h, int(psi.shape[0]), p, ldp, h, ldh))
        return hpsi

    def apply_h_host(self, psi: np.ndarray, hpsi: np.ndarray | None = None) -> np.ndarray:
        """Host (nb, npw) complex128 in, host out; copies inside the call."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        if hpsi is None:
            hpsi = np.empty_like(psi)
        assert psi.shape[1] == self.npw and hpsi.shape == psi.shape and hpsi.flags.c_contiguous
        _check(lib().pwh_apply_h_host(self._h, int(psi.shape[0]), psi.ctypes.data_as(_c_p),
                                      hpsi.ctypes.data_as(_c_p)))
        return hpsi

    # ------------------------------------------------------------- overlap
    def set_overlap(self, q=None):
        """S = 1 + sum_ij |beta_i> q_ij <beta_j| over the projectors: q a host
        array of nproj reals (diagonal) or an (nproj, nproj) complex matrix;
        None removes it.  The eigensolvers then solve H x = e S x."""
        if q is None:
            _check(lib().pwh_set_overlap(self._h, None, 0, 0))
            return
        q = np.asarray(q)
        if q.ndim == 1:
            d = np.ascontiguousarray(q, dtype=np.float64)
            _check(lib().pwh_set_overlap(self._h, d.ctypes.data_as(_c_p), 1, 0))
        else:
            m = np.asfortranarray(q, dtype=np.complex128)
            _check(lib().pwh_set_overlap(self._h, m.ctypes.data_as(_c_p), 0, 0))

    def apply_s(self, psi, spsi=None):
        """spsi = S psi on the device; psi (nb, npw) complex128 CUDA tensor."""
        torch = _torch()
        if spsi is None:
            spsi = torch.empty_like(psi, memory_format=torch.contiguous_format)
        p, ldp = _band_ptr(psi, self.npw)
        h, ldh = _band_ptr(spsi, self.npw)
        _check(lib().pwh_apply_s(self._h, int(psi.shape[0]), p, ldp, h, ldh))
        return spsi

    # ------------------------------------------------------- exact exchange
    def exx_apply(self, psi_occ, occ, phi, out=None):
        """V_x phi (Fock exchange of the occupied bands psi_occ with weights
        occ) for bands phi; (n, npw) CUDA complex128 tensors, public order."""
        torch = _torch()
        if out is None:
            out = torch.empty_like(phi, memory_format=torch.contiguous_format)
        po, ldo = _band_ptr(psi_occ, self.npw)
        pp, ldp = _band_ptr(phi, self.npw)
        op, ldr = _band_ptr(out, self.npw)
        w = np.ascontiguousarray(occ, dtype=np.float64)
        _check(lib().pwh_exx_apply(self._h, int(psi_occ.shape[0]), po, ldo, w.ctypes.data_as(_c_p),
                                   int(phi.shape[0]), pp, ldp, op, ldr))
        return out

    def set_ace(self, psi_occ=None, occ=None, alpha=1.0):
        """Adaptively compressed exchange of the occupied bands psi_occ (CUDA
        complex128 (nocc, npw)) added to H from now on; None removes it.
        Returns the rank kept."""
        r = _c_i32()
        if psi_occ is None:
            _check(lib().pwh_set_ace(self._h, 0, None, self.npw, None, 1.0, ctypes.byref(r)))
            return 0
        po, ldo = _band_ptr(psi_occ, self.npw)
        w = np.ascontiguousarray(occ, dtype=np.float64)
        _check(lib().pwh_set_ace(self._h, int(psi_occ.shape[0]), po, ldo, w.ctypes.data_as(_c_p),
                                 float(alpha), ctypes.byref(r)))
        return r.value

    # ------------------------------------------------------------ SCF steps
    def density(self, psi, occ):
        """rho on the FFT grid (CUDA float64 tensor of shape fft) from bands psi
        ((nb, npw) CUDA complex128, public order) with occupations occ."""
        torch = _torch()
        nb = int(psi.shape[0])
        rho = torch.empty(self.fft, dtype=torch.float64, device="cuda")
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        assert occ.size == nb
        if nb:
            p, ld = _band_ptr(psi, self.npw)
        else:
            p, ld = None, self.npw
        _check(lib().pwh_density(self._h, nb, p, ld, occ.ctypes.data_as(_c_p),
                                 ctypes.c_void_p(rho.data_ptr())))
        return rho

    def hartree_xc(self, rho, v_ion=None):
        """(v_ion + V_H + v_xc as a CUDA float64 grid, dict of E_H, E_xc and
        int v_xc rho) from the density rho (CUDA float64 grid)."""
        torch = _torch()
        rho = rho.contiguous()
        assert rho.dtype == torch.float64 and rho.numel() == int(np.prod(self.fft))
        out = torch.empty_like(rho)
        vi = ctypes.c_void_p(v_ion.contiguous().data_ptr()) if v_ion is not None else None
        en = np.zeros(3, dtype=np.float64)
        _check(lib().pwh_hartree_xc(self._h, ctypes.c_void_p(rho.data_ptr()), vi,
                                    ctypes.c_void_p(out.data_ptr()), en.ctypes.data_as(_c_p)))
        return out, {"e_hartree": float(en[0]), "e_xc": float(en[1]), "int_vxc_rho": float(en[2])}

    # ----------------------------------------------------- learned precond
    def shells(self):
        """(shell index of every public plane wave, kinetic energy of every shell)."""
        n = _c_i32()
        _check(lib().pwh_get_shells(self._h, ctypes.byref(n), None, None))
        sh = np.empty(self.npw, dtype=np.int32)
        T = np.empty(n.value, dtype=np.float64)
        _check(lib().pwh_get_shells(self._h, ctypes.byref(n), sh.ctypes.data_as(_c_p),
                                    T.ctypes.data_as(_c_p)))
        return sh, T

    def set_mlp(self, blob):
        b = np.ascontiguousarray(blob, dtype=np.float32)
        _check(lib().pwh_set_mlp(self._h, b.ctypes.data_as(_c_p), int(b.size)))

    def mlp_forward(self, params, feats):
        torch = _torch()
        out = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
        _check(lib().pwh_mlp_forward(self._h, ctypes.c_void_p(params.data_ptr()),
                                     ctypes.c_void_p(feats.data_ptr()), int(feats.shape[0]),
                                     ctypes.c_void_p(out.data_ptr())))
        return out

    def mlp_loss_grad(self, params, feats, y, w, wsum=None):
        torch = _torch()
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=feats.device)
        loss = torch.empty(1, dtype=torch.float32, device=feats.device)
        wsum = float(w.double().sum().item()) if wsum is None else float(wsum)
        _check(lib().pwh_mlp_loss_grad(self._h, ctypes.c_void_p(params.data_ptr()),
                                       ctypes.c_void_p(feats.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(w.data_ptr()), int(feats.shape[0]), wsum,
                                       ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(loss.data_ptr())))
        return loss, g

    def mlp_adam(self, params, g, m, v, step, lr):
        _check(lib().pwh_mlp_adam(self._h, ctypes.c_void_p(params.data_ptr()),
                                  ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                                  ctypes.c_void_p(v.data_ptr()), int(step), float(lr)))

    def mlp_training_rows(self, X, HX, theta, Xstar):
        """Rows of (features, target, weight) from one trajectory point; X, HX,
        Xstar: (nb, npw) CUDA complex128 (public order), theta: numpy (nb,)."""
        torch = _torch()
        nb = int(X.shape[0])
        nsh = int(self.shells()[1].size)
        F = torch.empty((nb * nsh, 4), dtype=torch.float32, device=X.device)
        y = torch.empty(nb * nsh, dtype=torch.float32, device=X.device)
        w = torch.empty(nb * nsh, dtype=torch.float32, device=X.device)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        for t in (X, HX, Xstar):
            _band_ptr(t, self.npw)
        _check(lib().pwh_mlp_training_rows(self._h, nb, ctypes.c_void_p(X.data_ptr()),
                                           ctypes.c_void_p(HX.data_ptr()), th.ctypes.data_as(_c_p),
                                           ctypes.c_void_p(Xstar.data_ptr()),
                                           ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           ctypes.c_void_p(w.data_ptr())))
        return F, y, w

    # ---------------------------------------------------------- eigensolver
    def davidson(self, psi, tol=1e-8, max_iter=200, mult=3, precond="tpa", mixed=False,
                 switch_tol=1e-5, jd_inner=0, check=True):
        """Lowest nb = psi.shape[0] eigenpairs; psi (nb, npw) CUDA complex128
        holds the starting bands and receives the eigenvectors.  Returns
        (eigenvalues as numpy, stats dict, status)."""
        p, ld = _band_ptr(psi, self.npw)
        nb = int(psi.shape[0])
        o = DavidsonOpts(nb=nb, max_iter=int(max_iter), max_subspace_mult=int(mult),
                         precond=PRECOND[precond], mixed=int(bool(mixed)), jd_inner=int(jd_inner),
                         tol=float(tol), switch_tol=float(max(switch_tol, tol)))
        st = DavidsonStats()
        eig = np.zeros(nb, dtype=np.float64)
        status = lib().pwh_davidson_solve(self._h, ctypes.byref(o), p, ld,
                                          eig.ctypes.data_as(_c_p), ctypes.byref(st))
        if check and status not in (0,):
            _check(status)
        return eig, st.as_dict(), status

    def davidson_gamma(self, psi, tol=1e-8, max_iter=200, mult=3, precond="tpa", mixed=False,
                       switch_tol=1e-5, jd_inner=0, check=True):
        """davidson() for real bands at k = 0: psi (nb, npw_half) CUDA complex128
        on the half sphere (gamma_half()), starting bands in, eigenvectors out."""
        n = _c_i64()
        _check(lib().pwh_get_gamma_half(self._h, ctypes.byref(n), None))
        p, ld = _band_ptr(psi, n.value)
        nb = int(psi.shape[0])
        o = DavidsonOpts(nb=nb, max_iter=int(max_iter), max_subspace_mult=int(mult),
                         precond=PRECOND[precond], mixed=int(bool(mixed)), jd_inner=int(jd_inner),
                         tol=float(tol), switch_tol=float(max(switch_tol, tol)))
        st = DavidsonStats()
        eig = np.zeros(nb, dtype=np.float64)
        status = lib().pwh_davidson_solve_gamma(self._h, ctypes.byref(o), p, ld,
                                                eig.ctypes.data_as(_c_p), ctypes.byref(st))
        if check and status not in (0,):
            _check(status)
        return eig, st.as_dict(), status

    def davidson_trace(self):
        """Per-iteration record of the last solve: a list of dicts (iter, fp64,
        m, n_above, max_resid, t_s)."""
        n = _c_i32()
        _check(lib().pwh_get_davidson_trace(self._h, 0, None, ctypes.byref(n)))
        arr = (TraceEntry * max(1, n.value))()
        _check(lib().pwh_get_davidson_trace(self._h, n.value, arr, ctypes.byref(n)))
        return [{k: getattr(arr[i], k) for k, _ in TraceEntry._fields_} for i in range(n.value)]

    def davidson_host(self, psi: np.ndarray, tol=1e-8, max_iter=200, mult=3, precond="tpa",
                      mixed=False, switch_tol=1e-5, jd_inner=0, check=True):
        """davidson() with the bands in host memory: psi (nb, npw) C-contiguous
        complex128 numpy array (pinned memory copies fastest), starting bands
        in, eigenvectors out; the copies run inside the library call."""
        if not (isinstance(psi, np.ndarray) and psi.dtype == np.complex128 and psi.ndim == 2
                and psi.shape[1] == self.npw and psi.flags.c_contiguous):
            raise ValueError(f"expected a C-contiguous complex128 array of shape (nb, {self.npw})")
        nb = int(psi.shape[0])
        o = DavidsonOpts(nb=nb, max_iter=int(max_iter), max_subspace_mult=int(mult),
                         precond=PRECOND[precond], mixed=int(bool(mixed)), jd_inner=int(jd_inner),
                         tol=float(tol), switch_tol=float(max(switch_tol, tol)))
        st = DavidsonStats()
        eig = np.zeros(nb, dtype=np.float64)
        status = lib().pwh_davidson_solve_host(self._h, ctypes.byref(o), psi.ctypes.data_as(_c_p),
                                               eig.ctypes.data_as(_c_p), ctypes.byref(st))
        if check and status not in (0,):
            _check(status)
        return eig, st.as_dict(), status


def batch_davidson(systems, psis, tol=1e-8, max_iter=200, mult=3, precond="tpa", mixed=True,
                   switch_tol=1e-3, jd_inner=20, nthreads=16):
    """Solve many independent systems concurrently (pwh_batch_davidson_solve).
    systems: list of System (each created with its own stream); psis: list of
    (nb_i, npw_i) CUDA complex128 tensors (starting bands in, eigenvectors
    out).  Returns (list of eigenvalue arrays, list of stats dicts, statuses)."""
    n = len(systems)
    hs = (_c_p * n)(*[s._h.value for s in systems])
    opts = (DavidsonOpts * n)()
    ptrs = (_c_p * n)()
    lds = (_c_i64 * n)()
    eigs = [np.zeros(int(p.shape[0]), dtype=np.float64) for p in psis]
    eptr = (_c_p * n)(*[e.ctypes.data for e in eigs])
    stats = (DavidsonStats * n)()
    status = (_c_i32 * n)()
    for i, (s, p) in enumerate(zip(systems, psis)):
        ptr, ld = _band_ptr(p, s.npw)
        ptrs[i] = ptr.value
        lds[i] = ld
        opts[i] = DavidsonOpts(nb=int(p.shape[0]), max_iter=int(max_iter), max_subspace_mult=int(mult),
                               precond=PRECOND[precond], mixed=int(bool(mixed)), jd_inner=int(jd_inner),
                               tol=float(tol), switch_tol=float(max(switch_tol, tol)))
    st = lib().pwh_batch_davidson_solve(n, hs, opts, ptrs, lds, eptr, stats, status, int(nthreads))
    return eigs, [stats[i].as_dict() for i in range(n)], [int(status[i]) for i in range(n)], st

