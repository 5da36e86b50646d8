"""GB300 direct-SCF Fock build (J, K <- P) and its drivers.

Thin Python binding over the C ABI of ``libcq.so`` (declared in
``include/cq.h``): argument marshalling only.  Device memory and streams
come from PyTorch; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing, importing a
function that needs it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcq.so")
_lib = None

CQ_DENS_REAL_SYM, CQ_DENS_COMPLEX_HERM, CQ_DENS_PAULI4 = 0, 1, 2
CQ_PREC_FP64, CQ_PREC_MIXED = 0, 1


class CQError(RuntimeError):
    pass


class FockOpts(ctypes.Structure):
    _fields_ = [("schwarz_tol", ctypes.c_double), ("mixed_tol", ctypes.c_double),
                ("prec", ctypes.c_int), ("want_J", ctypes.c_int), ("want_K", ctypes.c_int)]


class FockStats(ctypes.Structure):
    _fields_ = [("quartets_fp64", ctypes.c_ulonglong), ("quartets_fp32", ctypes.c_ulonglong),
                ("prim_fp64", ctypes.c_ulonglong), ("prim_fp32", ctypes.c_ulonglong),
                ("ms", ctypes.c_double)]


def build():
    from . import buildlib as _b
    return _b.build()


def lib():
    """Load libcq.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CQError(f"libcq.so not built ({LIB_PATH}); run paper_1905_01381_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        L.cq_basis_create.argtypes = [ctypes.c_int, dp, ip, ctypes.c_int, ip, ip, ip, dp, dp,
                                      ctypes.POINTER(vp)]
        L.cq_basis_info.argtypes = [vp, ip, ip, ip]
        L.cq_basis_destroy.argtypes = [vp]
        L.cq_basis_destroy.restype = None
        L.cq_schwarz.argtypes = [vp, vp, vp]
        L.cq_fock_build.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(FockOpts),
                                    ctypes.POINTER(FockStats), vp]
        L.cq_nuclear_repulsion.argtypes = [vp, dp]
        L.cq_last_error.restype = ctypes.c_char_p
        L.cq_fock_profile.argtypes = [vp, ctypes.c_int]
        L.cq_fock_class_stats.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp,
                                          ctypes.POINTER(ctypes.c_ulonglong),
                                          ctypes.POINTER(ctypes.c_ulonglong)]
        L.cq_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, dp, vp]
        L.cq_fock_build_noalloc.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(FockOpts), vp]
        L.cq_fock_noalloc_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.cq_fock_noalloc_scratch_bytes.restype = ctypes.c_size_t
        _lib = L
    return _lib


def check(rc: int, what: str = ""):
    if rc != 0:
        msg = lib().cq_last_error().decode()
        raise CQError(f"{what} failed ({rc}): {msg}")


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


PAIR_CLASSES = ["ss", "ps", "pp", "ds", "dp", "dd"]
QUARTET_CLASSES = [(X, Y) for X in range(6) for Y in range(X + 1)]


def peak_fma(fp32: bool, iters: int = 20000, stream=None) -> float:
    """Measured FMA throughput in FLOP/s (an FMA counts 2)."""
    v = ctypes.c_double()
    check(lib().cq_peak_fma(int(fp32), iters, ctypes.byref(v), _stream_ptr(stream)), "cq_peak_fma")
    return v.value


class Basis:
    """A contracted Cartesian Gaussian basis on the current CUDA device."""

    def __init__(self, mol, basis):
        L = lib()
        self.mol, self.basis = mol, basis
        xyz = np.ascontiguousarray(mol.xyz, dtype=np.float64)
        Z = np.ascontiguousarray(mol.Z, dtype=np.int32)
        sa = np.ascontiguousarray(basis.shell_atom, dtype=np.int32)
        sl = np.ascontiguousarray(basis.shell_L, dtype=np.int32)
        sn = np.ascontiguousarray(basis.shell_nprim, dtype=np.int32)
        ex = np.ascontiguousarray(basis.exps, dtype=np.float64)
        co = np.ascontiguousarray(basis.coefs, dtype=np.float64)
        dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        h = ctypes.c_void_p()
        check(L.cq_basis_create(int(Z.shape[0]), xyz.ctypes.data_as(dp), Z.ctypes.data_as(ip),
                                int(sl.shape[0]), sa.ctypes.data_as(ip), sl.ctypes.data_as(ip),
                                sn.ctypes.data_as(ip), ex.ctypes.data_as(dp), co.ctypes.data_as(dp),
                                ctypes.byref(h)), "cq_basis_create")
        self.h = h
        n, ns, npair = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(L.cq_basis_info(h, ctypes.byref(n), ctypes.byref(ns), ctypes.byref(npair)))
        self.nbf, self.nshell, self.npair = n.value, ns.value, npair.value

    def close(self):
        if getattr(self, "h", None):
            lib().cq_basis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def schwarz(self, stream=None):
        import torch
        Q = torch.empty((self.nshell, self.nshell), dtype=torch.float64, device="cuda")
        check(lib().cq_schwarz(self.h, _ptr(Q), _stream_ptr(stream)), "cq_schwarz")
        return Q

    def nuclear_repulsion(self) -> float:
        E = ctypes.c_double()
        check(lib().cq_nuclear_repulsion(self.h, ctypes.byref(E)), "cq_nuclear_repulsion")
        return E.value

    def fock_build(self, P, kind=None, schwarz_tol=1e-14, mixed_tol=1e-5, prec=CQ_PREC_FP64,
                   want_J=True, want_K=True, J=None, K=None, stats=False, stream=None):
        """J, K of a density given as a torch CUDA tensor:
        float64 (n, n) real symmetric; complex128 (n, n) Hermitian;
        complex128 (4, n, n) Pauli components P^0..P^3."""
        import torch
        n = self.nbf
        if kind is None:
            if P.dtype == torch.float64:
                kind = CQ_DENS_REAL_SYM
            elif P.dim() == 3:
                kind = CQ_DENS_PAULI4
            else:
                kind = CQ_DENS_COMPLEX_HERM
        P = P.contiguous()
        if want_J and J is None:
            J = torch.empty((n, n), dtype=torch.float64, device=P.device)
        if want_K and K is None:
            if kind == CQ_DENS_REAL_SYM:
                K = torch.empty((n, n), dtype=torch.float64, device=P.device)
            elif kind == CQ_DENS_COMPLEX_HERM:
                K = torch.empty((n, n), dtype=torch.complex128, device=P.device)
            else:
                K = torch.empty((4, n, n), dtype=torch.complex128, device=P.device)
        o = FockOpts(schwarz_tol, mixed_tol, prec, int(want_J), int(want_K))
        st = FockStats()
        check(lib().cq_fock_build(self.h, kind, _ptr(P), _ptr(J) if want_J else None,
                                  _ptr(K) if want_K else None, ctypes.byref(o),
                                  ctypes.byref(st) if stats else None, _stream_ptr(stream)),
              "cq_fock_build")
        if stats:
            return J, K, {"quartets_fp64": st.quartets_fp64, "quartets_fp32": st.quartets_fp32,
                          "prim_fp64": st.prim_fp64, "prim_fp32": st.prim_fp32, "ms": st.ms}
        return J, K

    def profile(self, enable: bool = True):
        check(lib().cq_fock_profile(self.h, int(enable)), "cq_fock_profile")

    def class_stats(self):
        """Per-class (time ms, quartets, primitive quartets) of the last build."""
        out = {}
        for qc, (X, Y) in enumerate(QUARTET_CLASSES):
            for p in (0, 1):
                ms = ctypes.c_double()
                nq, npq = ctypes.c_ulonglong(), ctypes.c_ulonglong()
                check(lib().cq_fock_class_stats(self.h, qc, p, ctypes.byref(ms), ctypes.byref(nq),
                                                ctypes.byref(npq)), "cq_fock_class_stats")
                if nq.value or ms.value:
                    key = f"({PAIR_CLASSES[X]}|{PAIR_CLASSES[Y]})" + ("f32" if p else "f64")
                    out[key] = {"qc": qc, "fp32": p, "ms": ms.value, "quartets": nq.value,
                                "prims": npq.value}
        return out
