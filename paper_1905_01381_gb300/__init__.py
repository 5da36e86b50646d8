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

CQ_DENS_REAL_SYM, CQ_DENS_COMPLEX_HERM, CQ_DENS_PAULI4, CQ_DENS_REAL_GENERAL = 0, 1, 2, 3
CQ_PREC_FP64, CQ_PREC_MIXED = 0, 1


class CQError(RuntimeError):
    pass


class FockOpts(ctypes.Structure):
    _fields_ = [("schwarz_tol", ctypes.c_double), ("mixed_tol", ctypes.c_double),
                ("prec", ctypes.c_int), ("want_J", ctypes.c_int), ("want_K", ctypes.c_int),
                ("fp64_tol", ctypes.c_double)]


class FockStats(ctypes.Structure):
    _fields_ = [("quartets_fp64", ctypes.c_ulonglong), ("quartets_fp32", ctypes.c_ulonglong),
                ("prim_fp64", ctypes.c_ulonglong), ("prim_fp32", ctypes.c_ulonglong),
                ("ms", ctypes.c_double), ("quartets_df", ctypes.c_ulonglong), ("prim_df", ctypes.c_ulonglong)]


class SCFOpts(ctypes.Structure):
    _fields_ = [("e_tol", ctypes.c_double), ("d_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("diis_size", ctypes.c_int), ("prec", ctypes.c_int), ("mixed_tol", ctypes.c_double),
                ("schwarz_tol", ctypes.c_double), ("incremental", ctypes.c_int), ("full_every", ctypes.c_int),
                ("switch_tol", ctypes.c_double), ("graph", ctypes.c_int), ("guess_fallback", ctypes.c_int),
                ("fp64_tol", ctypes.c_double)]


class SCFStats(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("last_rms", ctypes.c_double), ("quartets_fp64", ctypes.c_ulonglong),
                ("quartets_fp32", ctypes.c_ulonglong), ("ms", ctypes.c_double), ("graph", ctypes.c_int),
                ("quartets_df", ctypes.c_ulonglong)]


class RTOpts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("field", ctypes.c_double * 3), ("t_on", ctypes.c_double),
                ("t_off", ctypes.c_double), ("restart_every", ctypes.c_int), ("prec", ctypes.c_int),
                ("mixed_tol", ctypes.c_double), ("schwarz_tol", ctypes.c_double), ("fp64_tol", ctypes.c_double)]


class RTObs(ctypes.Structure):
    _fields_ = [("dipole", ctypes.c_double * 3), ("trPS", ctypes.c_double), ("energy", ctypes.c_double),
                ("em2", ctypes.c_int)]


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
        L.cq_one_electron.argtypes = [vp, vp, vp, vp, vp, dp, vp]
        L.cq_scf.argtypes = [vp, ctypes.c_int, ctypes.POINTER(SCFOpts), vp, vp, vp, ctypes.POINTER(SCFStats), vp]
        L.cq_scf_ghf.argtypes = [vp, ctypes.c_int, ctypes.POINTER(SCFOpts), vp, vp, vp, ctypes.POINTER(SCFStats),
                                 vp]
        L.cq_rt_step.argtypes = [vp, ctypes.POINTER(RTOpts), ctypes.c_int, vp, vp, ctypes.POINTER(RTObs), vp]
        L.cq_dense_info.argtypes = [vp, ip, ip, vp]
        L.cq_autotune.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(FockOpts), ip, dp, vp]
        L.cq_basis_create_batch.argtypes = [ctypes.c_int, dp, ip, ip, ctypes.c_int, ip, ip, ip, dp, dp,
                                            ctypes.POINTER(vp)]
        L.cq_basis_layout.argtypes = [vp, ip, ip, ip]
        L.cq_scf_batch.argtypes = [vp, ip, ctypes.POINTER(SCFOpts), vp, vp, dp, ip, ctypes.POINTER(SCFStats), vp]
        L.cq_nuclear_repulsion_batch.argtypes = [vp, dp]
        L.cq_mlp_param_count.restype = ctypes.c_size_t
        L.cq_mlp_init.argtypes = [vp, ctypes.c_ulonglong, vp]
        L.cq_guess_dataset.argtypes = [vp, vp, vp, vp, vp, ip, vp]
        L.cq_mlp_loss_grad.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, dp, vp]
        L.cq_mlp_train.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                   ctypes.c_ulonglong, dp, vp]
        L.cq_guess_density.argtypes = [vp, vp, ip, ctypes.c_int, ctypes.c_int, vp, vp]
        L.cq_fock_set_variant.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.cq_fock_get_variant.argtypes = [vp, ctypes.c_int, ctypes.c_int, ip]
        L.cq_fock_set_list_split.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.cq_fock_build_noalloc.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(FockOpts), vp]
        L.cq_fock_noalloc_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.cq_fock_noalloc_scratch_bytes.restype = ctypes.c_size_t
        L.cq_boys.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.cq_set_list_capacity.argtypes = [ctypes.c_longlong]
        L.cq_get_list_capacity.restype = ctypes.c_longlong
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


def set_list_capacity(entries: int):
    """Largest quartet list (entries) a basis created afterwards keeps; larger
    bases build in passes (see cq_set_list_capacity)."""
    check(lib().cq_set_list_capacity(int(entries)), "cq_set_list_capacity")


def get_list_capacity() -> int:
    return int(lib().cq_get_list_capacity())


def peak_fma(fp32: bool, iters: int = 20000, stream=None) -> float:
    """Measured FMA throughput in FLOP/s (an FMA counts 2)."""
    v = ctypes.c_double()
    check(lib().cq_peak_fma(int(fp32), iters, ctypes.byref(v), _stream_ptr(stream)), "cq_peak_fma")
    return v.value


class Basis:
    """A contracted Cartesian Gaussian basis on the current CUDA device.

    Basis(mol, basis) holds one molecule; Basis.batch([(mol, basis), ...])
    holds many independent molecules whose matrices use the batched layout
    (nmol slots of ld x ld)."""

    def __init__(self, mol, basis, atom_mol=None):
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
        if atom_mol is None:
            check(L.cq_basis_create(int(Z.shape[0]), xyz.ctypes.data_as(dp), Z.ctypes.data_as(ip),
                                    int(sl.shape[0]), sa.ctypes.data_as(ip), sl.ctypes.data_as(ip),
                                    sn.ctypes.data_as(ip), ex.ctypes.data_as(dp), co.ctypes.data_as(dp),
                                    ctypes.byref(h)), "cq_basis_create")
        else:
            am = np.ascontiguousarray(atom_mol, dtype=np.int32)
            check(L.cq_basis_create_batch(int(Z.shape[0]), xyz.ctypes.data_as(dp), Z.ctypes.data_as(ip),
                                          am.ctypes.data_as(ip), int(sl.shape[0]), sa.ctypes.data_as(ip),
                                          sl.ctypes.data_as(ip), sn.ctypes.data_as(ip),
                                          ex.ctypes.data_as(dp), co.ctypes.data_as(dp), ctypes.byref(h)),
                  "cq_basis_create_batch")
        self.h = h
        n, ns, npair = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(L.cq_basis_info(h, ctypes.byref(n), ctypes.byref(ns), ctypes.byref(npair)))
        self.nbf, self.nshell, self.npair = n.value, ns.value, npair.value
        nm, ld = ctypes.c_int(), ctypes.c_int()
        check(L.cq_basis_layout(h, ctypes.byref(nm), ctypes.byref(ld), None))
        self.nmol, self.ld = nm.value, ld.value
        mn = (ctypes.c_int * self.nmol)()
        check(L.cq_basis_layout(h, None, None, mn))
        self.mol_n = list(mn)

    @classmethod
    def batch(cls, items):
        """One batched basis from a list of (Molecule, Basis) pairs."""
        import synth
        Zs, xyzs, am = [], [], []
        sa, sl, sn, ex, co = [], [], [], [], []
        aoff = 0
        for m, (mol, bas) in enumerate(items):
            Zs.append(mol.Z); xyzs.append(mol.xyz); am.append(np.full(mol.natom, m))
            sa.append(bas.shell_atom + aoff); sl.append(bas.shell_L); sn.append(bas.shell_nprim)
            ex.append(bas.exps); co.append(bas.coefs)
            aoff += mol.natom
        mol = synth.Molecule(np.concatenate(Zs).astype(np.int32), np.concatenate(xyzs))
        bas = synth.Basis(np.concatenate(sa).astype(np.int32), np.concatenate(sl).astype(np.int32),
                          np.concatenate(sn).astype(np.int32), np.concatenate(ex), np.concatenate(co))
        out = cls(mol, bas, atom_mol=np.concatenate(am))
        out.items = items
        return out

    def pack(self, mats):
        """List of per-molecule (n_m, n_m[, ...]) arrays -> batched-layout tensor."""
        import torch
        first = torch.as_tensor(mats[0])
        out = torch.zeros((self.nmol, self.ld, self.ld), dtype=first.dtype)
        for m, M in enumerate(mats):
            n = self.mol_n[m]
            out[m, :n, :n] = torch.as_tensor(M)
        return out.cuda()

    def unpack(self, T):
        """Batched-layout tensor -> list of per-molecule numpy arrays."""
        T = T.reshape(self.nmol, self.ld, self.ld).cpu().numpy()
        return [T[m, :self.mol_n[m], :self.mol_n[m]].copy() for m in range(self.nmol)]

    def scf_batch(self, nocc, e_tol=1e-10, d_tol=1e-8, max_iter=128, diis_size=8, prec=CQ_PREC_FP64,
                  mixed_tol=1e-5, schwarz_tol=1e-14, switch_tol=1e-5, D0=None, stream=None,
                  raise_on_fail=True, graph=True, guess_fallback=40, fp64_tol=0.0):
        """Batched RHF; returns (D batched tensor, energies, iterations, stats).
        With D0, a molecule still open after guess_fallback iterations restarts
        from the core guess (0: never)."""
        import torch
        D = torch.empty((self.nmol, self.ld, self.ld), dtype=torch.float64, device="cuda")
        no = np.ascontiguousarray(nocc, dtype=np.int32)
        E = np.zeros(self.nmol)
        it = np.zeros(self.nmol, dtype=np.int32)
        o = SCFOpts(e_tol, d_tol, max_iter, diis_size, prec, mixed_tol, schwarz_tol, 0, 8, switch_tol, int(bool(graph)),
                    int(guess_fallback), fp64_tol)
        st = SCFStats()
        ip, dp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        rc = lib().cq_scf_batch(self.h, no.ctypes.data_as(ip), ctypes.byref(o),
                                _ptr(D0) if D0 is not None else None, _ptr(D), E.ctypes.data_as(dp),
                                it.ctypes.data_as(ip), ctypes.byref(st), _stream_ptr(stream))
        if raise_on_fail:
            check(rc, "cq_scf_batch")
        return D, E, it, {"iterations": st.iterations, "converged": st.converged, "ms": st.ms,
                          "quartets_fp64": st.quartets_fp64, "quartets_fp32": st.quartets_fp32,
                          "quartets_df": st.quartets_df, "rc": rc, "graph": st.graph}

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

    def boys(self, T, mmax: int, fp32=False, stream=None):
        """F_0..F_mmax(T) for a CUDA float64 tensor T, evaluated by the
        integral kernels' device Boys function: fp32 = False / 0 in FP64,
        True / 1 in FP32, 2 in double-float."""
        import torch
        T = T.contiguous()
        F = torch.empty((T.numel(), mmax + 1), dtype=torch.float64, device=T.device)
        check(lib().cq_boys(self.h, int(fp32), int(mmax), int(T.numel()), _ptr(T), _ptr(F),
                            _stream_ptr(stream)), "cq_boys")
        return F

    def nuclear_repulsion(self) -> float:
        E = ctypes.c_double()
        check(lib().cq_nuclear_repulsion(self.h, ctypes.byref(E)), "cq_nuclear_repulsion")
        return E.value

    def nuclear_repulsion_batch(self):
        """Nuclear repulsion of every molecule of a batched basis."""
        E = np.zeros(self.nmol)
        check(lib().cq_nuclear_repulsion_batch(self.h, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
              "cq_nuclear_repulsion_batch")
        return E

    def fock_build(self, P, kind=None, schwarz_tol=1e-14, mixed_tol=1e-5, prec=CQ_PREC_FP64,
                   want_J=True, want_K=True, J=None, K=None, stats=False, stream=None, fp64_tol=0.0):
        """J, K of a density given as a torch CUDA tensor:
        float64 (n, n) real symmetric; complex128 (n, n) Hermitian;
        complex128 (4, n, n) Pauli components P^0..P^3; with
        kind=CQ_DENS_REAL_GENERAL, float64 (n, n) of any symmetry (real J and
        K, e.g. of a transition density).  In mixed precision,
        fp64_tol > mixed_tol adds the double-float tier for bounds in
        [mixed_tol, fp64_tol)."""
        import torch
        n = self.ld
        if kind is None:
            if P.dtype == torch.float64:
                kind = CQ_DENS_REAL_SYM
            elif P.dim() == 3 and self.nmol == 1 or P.dim() == 4:
                kind = CQ_DENS_PAULI4
            else:
                kind = CQ_DENS_COMPLEX_HERM
        P = P.contiguous()
        shape = (n, n) if self.nmol == 1 else (self.nmol, n, n)
        if want_J and J is None:
            J = torch.empty(shape, dtype=torch.float64, device=P.device)
        if want_K and K is None:
            if kind in (CQ_DENS_REAL_SYM, CQ_DENS_REAL_GENERAL):
                K = torch.empty(shape, dtype=torch.float64, device=P.device)
            elif kind == CQ_DENS_COMPLEX_HERM:
                K = torch.empty(shape, dtype=torch.complex128, device=P.device)
            else:
                K = torch.empty((4,) + shape, dtype=torch.complex128, device=P.device)
        o = FockOpts(schwarz_tol, mixed_tol, prec, int(want_J), int(want_K), fp64_tol)
        st = FockStats()
        check(lib().cq_fock_build(self.h, kind, _ptr(P), _ptr(J) if want_J else None,
                                  _ptr(K) if want_K else None, ctypes.byref(o),
                                  ctypes.byref(st) if stats else None, _stream_ptr(stream)),
              "cq_fock_build")
        if stats:
            return J, K, {"quartets_fp64": st.quartets_fp64, "quartets_fp32": st.quartets_fp32,
                          "prim_fp64": st.prim_fp64, "prim_fp32": st.prim_fp32, "ms": st.ms,
                          "quartets_df": st.quartets_df, "prim_df": st.prim_df}
        return J, K

    def profile(self, enable: bool = True):
        check(lib().cq_fock_profile(self.h, int(enable)), "cq_fock_profile")

    def class_stats(self):
        """Per-class (time ms, quartets, primitive quartets) of the last build."""
        out = {}
        for qc, (X, Y) in enumerate(QUARTET_CLASSES):
            for p in (0, 1, 2):
                ms = ctypes.c_double()
                nq, npq = ctypes.c_ulonglong(), ctypes.c_ulonglong()
                check(lib().cq_fock_class_stats(self.h, qc, p, ctypes.byref(ms), ctypes.byref(nq),
                                                ctypes.byref(npq)), "cq_fock_class_stats")
                if nq.value or ms.value:
                    key = f"({PAIR_CLASSES[X]}|{PAIR_CLASSES[Y]})" + ("f64", "f32", "df")[p]
                    out[key] = {"qc": qc, "fp32": int(p == 1), "prec": p, "ms": ms.value, "quartets": nq.value,
                                "prims": npq.value}
        return out

    def one_electron(self, origin=(0.0, 0.0, 0.0), stream=None):
        """S, T, V (nbf x nbf) and dipole moment integrals M (3, nbf, nbf)."""
        import torch
        n = self.ld
        shape = (n, n) if self.nmol == 1 else (self.nmol, n, n)
        S, T, V = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3))
        M = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
        o = (ctypes.c_double * 3)(*origin)
        check(lib().cq_one_electron(self.h, _ptr(S), _ptr(T), _ptr(V), _ptr(M), o, _stream_ptr(stream)),
              "cq_one_electron")
        return S, T, V, M

    def scf(self, nocc, e_tol=1e-10, d_tol=1e-8, max_iter=128, diis_size=8, prec=CQ_PREC_FP64,
            mixed_tol=1e-5, schwarz_tol=1e-14, incremental=False, full_every=8, switch_tol=1e-5,
            D0=None, stream=None, raise_on_fail=True, fp64_tol=0.0):
        """RHF SCF; returns (D, F, stats dict).  fp64_tol > mixed_tol adds the
        double-float tier to the mixed builds."""
        import torch
        n = self.nbf
        D = torch.empty((n, n), dtype=torch.float64, device="cuda")
        F = torch.empty((n, n), dtype=torch.float64, device="cuda")
        o = SCFOpts(e_tol, d_tol, max_iter, diis_size, prec, mixed_tol, schwarz_tol, int(incremental),
                    full_every, switch_tol, 0, 0, fp64_tol)
        st = SCFStats()
        rc = lib().cq_scf(self.h, int(nocc), ctypes.byref(o), _ptr(D0) if D0 is not None else None,
                          _ptr(D), _ptr(F), ctypes.byref(st), _stream_ptr(stream))
        if raise_on_fail:
            check(rc, "cq_scf")
        stats = {"energy": st.energy, "iterations": st.iterations, "converged": bool(st.converged),
                 "last_rms": st.last_rms, "quartets_fp64": st.quartets_fp64,
                 "quartets_fp32": st.quartets_fp32, "quartets_df": st.quartets_df, "ms": st.ms, "rc": rc}
        return D, F, stats

    def scf_ghf(self, nelec, e_tol=1e-10, d_tol=1e-8, max_iter=128, diis_size=8, prec=CQ_PREC_FP64,
                mixed_tol=1e-5, schwarz_tol=1e-14, switch_tol=1e-5, P0=None, stream=None, raise_on_fail=True,
                fp64_tol=0.0):
        """Two-component GHF SCF; P0 and the returned P, F are (4, nbf, nbf)
        complex128 Pauli components.  Returns (P, F, stats dict)."""
        import torch
        n = self.nbf
        P = torch.empty((4, n, n), dtype=torch.complex128, device="cuda")
        F = torch.empty((4, n, n), dtype=torch.complex128, device="cuda")
        o = SCFOpts(e_tol, d_tol, max_iter, diis_size, prec, mixed_tol, schwarz_tol, 0, 8, switch_tol, 0, 0, fp64_tol)
        st = SCFStats()
        rc = lib().cq_scf_ghf(self.h, int(nelec), ctypes.byref(o),
                              _ptr(P0.contiguous()) if P0 is not None else None, _ptr(P), _ptr(F),
                              ctypes.byref(st), _stream_ptr(stream))
        if raise_on_fail:
            check(rc, "cq_scf_ghf")
        stats = {"energy": st.energy, "iterations": st.iterations, "converged": bool(st.converged),
                 "last_rms": st.last_rms, "quartets_fp64": st.quartets_fp64,
                 "quartets_fp32": st.quartets_fp32, "quartets_df": st.quartets_df, "ms": st.ms, "rc": rc}
        return P, F, stats

    def rt_step(self, step, P_prev, P_cur, dt=0.05, field=(0.0, 0.0, 0.0), t_on=0.0, t_off=0.0,
                restart_every=50, prec=CQ_PREC_FP64, mixed_tol=1e-5, schwarz_tol=1e-14, obs=True,
                stream=None, fp64_tol=0.0):
        """One MMUT/EM2 step; P_prev, P_cur complex128 (nbf, nbf) CUDA tensors updated in
        place.  Returns the observables of the density on entry (dict) or None."""
        o = RTOpts(dt, (ctypes.c_double * 3)(*field), t_on, t_off, restart_every, prec, mixed_tol,
                   schwarz_tol, fp64_tol)
        ob = RTObs()
        check(lib().cq_rt_step(self.h, ctypes.byref(o), int(step), _ptr(P_prev), _ptr(P_cur),
                               ctypes.byref(ob) if obs else None, _stream_ptr(stream)), "cq_rt_step")
        if not obs:
            return None
        return {"dipole": list(ob.dipole), "trPS": ob.trPS, "energy": ob.energy, "em2": bool(ob.em2)}

    def dense_info(self, stream=None):
        m, d = ctypes.c_int(), ctypes.c_int()
        check(lib().cq_dense_info(self.h, ctypes.byref(m), ctypes.byref(d), _stream_ptr(stream)),
              "cq_dense_info")
        return m.value, d.value

    def set_variant(self, qc, prec, variant):
        """Kernel variant of class qc at precision prec (0 FP64, 1 FP32, 2
        double-float): 0 lane groups, 1 cooperative (task mode), 2 axis
        permutation, 3 cooperative on the screened list."""
        check(lib().cq_fock_set_variant(self.h, int(qc), int(prec), int(variant)), "cq_fock_set_variant")

    def set_list_split(self, prec, split, chunk):
        """Work split of variant 3 at precision prec (cq_fock_set_list_split)."""
        check(lib().cq_fock_set_list_split(self.h, int(prec), int(split), int(chunk)), "cq_fock_set_list_split")

    def get_variant(self, qc, prec):
        v = ctypes.c_int()
        check(lib().cq_fock_get_variant(self.h, int(qc), int(prec), ctypes.byref(v)), "cq_fock_get_variant")
        return v.value

    def autotune(self, P, prec=CQ_PREC_MIXED, mixed_tol=1e-3, schwarz_tol=1e-14, fp64_tol=0.0, cache=True,
                 stream=None, kind=None):
        """Pick the fastest kernel variant per class and precision (see
        cq_autotune) for builds with these options.  With cache=True the
        choice is stored per GPU model and split in _build/tuning.json and
        reused by later calls instead of re-timing."""
        import json
        import torch
        key = f"{torch.cuda.get_device_name()} prec={prec} mixed_tol={mixed_tol:g} fp64_tol={fp64_tol:g}"
        path = os.path.join(_HERE, "_build", "tuning.json")
        if cache and os.path.exists(path):
            try:
                tab = json.load(open(path)).get(key)
            except Exception:
                tab = None
            if tab and all(len(row) == 3 for row in tab["variant"]):
                for qc, row in enumerate(tab["variant"]):
                    for p, v in enumerate(row):
                        self.set_variant(qc, p, v)
                return tab
        if kind is None:
            kind = (CQ_DENS_REAL_SYM if P.dtype == torch.float64 else
                    CQ_DENS_PAULI4 if P.dim() == 3 else CQ_DENS_COMPLEX_HERM)
        o = FockOpts(schwarz_tol, mixed_tol, prec, 1, 1, fp64_tol)
        tab = (ctypes.c_int * 63)()
        ms = (ctypes.c_double * 63)()
        check(lib().cq_autotune(self.h, kind, _ptr(P.contiguous()), ctypes.byref(o), tab, ms,
                                _stream_ptr(stream)), "cq_autotune")
        out = {"variant": [[tab[3 * q + p] for p in range(3)] for q in range(21)],
               "best_ms": [[ms[3 * q + p] for p in range(3)] for q in range(21)]}
        if cache:
            data = {}
            if os.path.exists(path):
                try:
                    data = json.load(open(path))
                except Exception:
                    data = {}
            data[key] = out
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(data, fh, indent=1)
        return out


class DensityGuessMLP:
    """Learned initial density (see cq_mlp_* / cq_guess_* in include/cq.h)."""

    def __init__(self, seed: int = 0, stream=None):
        import torch
        self.n = int(lib().cq_mlp_param_count())
        self.params = torch.empty(self.n, dtype=torch.float32, device="cuda")
        check(lib().cq_mlp_init(_ptr(self.params), seed, _stream_ptr(stream)), "cq_mlp_init")

    @staticmethod
    def dataset(basis, D=None, stream=None):
        """(X, T, head) of every atom pair of a batched basis; T from D."""
        import torch
        npair = ctypes.c_int()
        check(lib().cq_guess_dataset(basis.h, None, None, None, None, ctypes.byref(npair),
                                     _stream_ptr(stream)), "cq_guess_dataset")
        n = npair.value
        X = torch.empty((n, 40), dtype=torch.float32, device="cuda")
        H = torch.empty(n, dtype=torch.int32, device="cuda")
        T = torch.empty((n, 1472), dtype=torch.float32, device="cuda") if D is not None else None
        check(lib().cq_guess_dataset(basis.h, _ptr(D) if D is not None else None, _ptr(X),
                                     _ptr(T) if T is not None else None, _ptr(H), ctypes.byref(npair),
                                     _stream_ptr(stream)), "cq_guess_dataset")
        return X, T, H

    def loss_grad(self, X, T, H, stream=None):
        import torch
        g = torch.empty_like(self.params)
        loss = ctypes.c_double()
        check(lib().cq_mlp_loss_grad(_ptr(self.params), int(X.shape[0]), _ptr(X), _ptr(T), _ptr(H),
                                     _ptr(g), ctypes.byref(loss), _stream_ptr(stream)), "cq_mlp_loss_grad")
        return loss.value, g

    def train(self, X, T, H, epochs=20, batch=2048, lr=1e-3, seed=0, stream=None):
        loss = ctypes.c_double()
        check(lib().cq_mlp_train(_ptr(self.params), int(X.shape[0]), _ptr(X), _ptr(T), _ptr(H), epochs,
                                 batch, lr, seed, ctypes.byref(loss), _stream_ptr(stream)), "cq_mlp_train")
        return loss.value

    def guess(self, basis, nocc, npurify=0, onsite_only=False, stream=None):
        import torch
        D = torch.empty((basis.nmol, basis.ld, basis.ld), dtype=torch.float64, device="cuda")
        no = np.ascontiguousarray(nocc, dtype=np.int32)
        check(lib().cq_guess_density(basis.h, _ptr(self.params), no.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     npurify, int(bool(onsite_only)), _ptr(D), _stream_ptr(stream)),
              "cq_guess_density")
        return D
