"""Oracle -- test infrastructure, not part of the product.

A plain, slow, obviously correct FP64 CPU restatement of what the GPU path
computes: integrals over contracted Cartesian Gaussians (McMurchie-Davidson,
in ``oracle_ints.c``), Coulomb/exchange matrices by their definitions, the
Pauli spin-basis split (Eq. pauli_sep), the Hartree-Fock Fock matrix in the
Pauli basis (Eq. 2c_fock), RHF/GHF SCF with DIIS, and RT-TDHF with the MMUT
and EM2 propagators (Sec. "Real-Time Electronic Dynamics").

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` leg may import this package.  It shares no code with
``paper_1905_01381_gb300`` and imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP)."""
    src = os.path.join(_HERE, "oracle_ints.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                           "-std=gnu11", src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def nthreads_default() -> int:
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


class OBasis:
    """Flat shell arrays in the layout the C oracle expects."""

    def __init__(self, mol, basis):
        self.mol = mol
        self.ctr = np.ascontiguousarray(mol.xyz[basis.shell_atom], dtype=np.float64)
        self.L = np.ascontiguousarray(basis.shell_L, dtype=np.int32)
        self.np_ = np.ascontiguousarray(basis.shell_nprim, dtype=np.int32)
        self.poff = np.ascontiguousarray(
            np.concatenate([[0], np.cumsum(self.np_)[:-1]]), dtype=np.int32)
        self.ex = np.ascontiguousarray(basis.exps, dtype=np.float64)
        self.co = np.ascontiguousarray(basis.coefs, dtype=np.float64)
        self.nsh = int(self.L.shape[0])
        self.nbf = int(lib().or_nbf(self.nsh, _i(self.L)))
        self.axyz = np.ascontiguousarray(mol.xyz, dtype=np.float64)
        self.Zc = np.ascontiguousarray(mol.Z, dtype=np.float64)
        self.bfo = np.concatenate([[0], np.cumsum((self.L + 1) * (self.L + 2) // 2)])

    def args(self):
        return (self.nsh, _d(self.ctr), _i(self.L), _i(self.np_), _i(self.poff),
                _d(self.ex), _d(self.co))


def boys(mmax: int, T: float) -> np.ndarray:
    F = np.zeros(mmax + 1)
    lib().or_boys(ctypes.c_int(mmax), ctypes.c_double(T), _d(F))
    return F


def boys_quadrature(m: int, T: float, dps: int = 40) -> str:
    """F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt (the Boys function's
    definition, Boys 1950) by mpmath quadrature at `dps` digits, returned as
    a decimal string with 25 significant digits."""
    import mpmath
    with mpmath.workdps(dps):
        T = mpmath.mpf(T)
        v = mpmath.quad(lambda t: t ** (2 * m) * mpmath.exp(-T * t * t), [0, mpmath.mpf(1) / 2, 1])
        return mpmath.nstr(v, 25, min_fixed=-1, max_fixed=-1)


def _one(ob: OBasis, kind: int, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    M = np.zeros((ob.nbf, ob.nbf))
    O = np.ascontiguousarray(origin, dtype=np.float64)
    lib().or_one_electron(ctypes.c_int(kind), *ob.args(), ctypes.c_int(ob.mol.natom),
                          _d(ob.axyz), _d(ob.Zc), _d(O), _d(M))
    return M


def overlap(ob):
    return _one(ob, 0)


def kinetic(ob):
    return _one(ob, 1)


def nuclear(ob):
    return _one(ob, 2)


def dipole(ob, origin=(0.0, 0.0, 0.0)):
    """Moment integrals <m| r_d - O_d |n> for d = x, y, z (no charge sign)."""
    return np.stack([_one(ob, 3 + d, origin) for d in range(3)])


def core_hamiltonian(ob):
    return kinetic(ob) + nuclear(ob)


def nuclear_repulsion(mol) -> float:
    E = 0.0
    for a in range(mol.natom):
        for b in range(a):
            E += mol.Z[a] * mol.Z[b] / np.linalg.norm(mol.xyz[a] - mol.xyz[b])
    return float(E)


def eri_shell(ob, a, b, c, d) -> np.ndarray:
    n = [(ob.L[s] + 1) * (ob.L[s] + 2) // 2 for s in (a, b, c, d)]
    out = np.zeros(n)
    lib().or_eri_shell(*ob.args(), a, b, c, d, _d(out))
    return out


def eri_full(ob) -> np.ndarray:
    n = ob.nbf
    T = np.zeros((n, n, n, n))
    lib().or_eri_full(*ob.args(), _d(T))
    return T


def schwarz(ob) -> np.ndarray:
    Q = np.zeros((ob.nsh, ob.nsh))
    lib().or_schwarz(*ob.args(), _d(Q))
    return Q


def norm_factors(ob) -> np.ndarray:
    f = np.zeros(ob.nbf)
    lib().or_norm_factors(*ob.args(), _d(f))
    return f


def jk_real(ob, Ds, nthreads: int | None = None):
    """J and K of a list of real nbf x nbf matrices (any symmetry)."""
    Ds = [np.ascontiguousarray(D, dtype=np.float64) for D in Ds]
    nd = len(Ds)
    D = np.ascontiguousarray(np.stack(Ds))
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    lib().or_jk(*ob.args(), nd, _d(D), _d(J), _d(K),
                nthreads if nthreads is not None else nthreads_default())
    return J, K


def jk(ob, P, nthreads: int | None = None):
    """J[P], K[P] for a real or complex matrix P (linear in P)."""
    if np.iscomplexobj(P):
        J, K = jk_real(ob, [P.real, P.imag], nthreads)
        return J[0] + 1j * J[1], K[0] + 1j * K[1]
    J, K = jk_real(ob, [P], nthreads)
    return J[0], K[0]


def jk_elements(ob, Ds, mu, nu, nthreads: int | None = None):
    """Selected J/K elements from the definitions (for large cases)."""
    Ds = [np.ascontiguousarray(D, dtype=np.float64) for D in Ds]
    D = np.ascontiguousarray(np.stack(Ds))
    mu = np.ascontiguousarray(mu, dtype=np.int32)
    nu = np.ascontiguousarray(nu, dtype=np.int32)
    ne = int(mu.shape[0])
    Jo = np.zeros((len(Ds), ne))
    Ko = np.zeros((len(Ds), ne))
    lib().or_jk_elements(*ob.args(), len(Ds), _d(D), ne, _i(mu), _i(nu), _d(Jo), _d(Ko),
                         nthreads if nthreads is not None else nthreads_default())
    return Jo, Ko


def jk_sample(ob, Ds, stride: int, offset: int = 0, nthreads: int | None = None):
    """J'/K' partial sums over the bra shell pairs p % stride == offset;
    returns (J, K, shell quartets visited).  Timing support only."""
    Ds = [np.ascontiguousarray(D, dtype=np.float64) for D in Ds]
    D = np.ascontiguousarray(np.stack(Ds))
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    f = lib().or_jk_sample
    f.restype = ctypes.c_long
    nq = f(*ob.args(), len(Ds), _d(D), _d(J), _d(K),
           nthreads if nthreads is not None else nthreads_default(), stride, offset)
    return J, K, int(nq)


def jk_sample_pairs(ob, Ds, pairs, nthreads: int | None = None):
    """J'/K' partial sums over an explicit set of bra shell pairs (pair index
    a(a+1)/2 + b, a >= b); returns (J, K, shell quartets visited).  Timing
    support only."""
    Ds = [np.ascontiguousarray(D, dtype=np.float64) for D in Ds]
    D = np.ascontiguousarray(np.stack(Ds))
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    sel = np.zeros(ob.nsh * (ob.nsh + 1) // 2, dtype=np.uint8)
    sel[np.asarray(pairs, dtype=np.int64)] = 1
    f = lib().or_jk_pairs
    f.restype = ctypes.c_long
    nq = f(*ob.args(), len(Ds), _d(D), _d(J), _d(K),
           nthreads if nthreads is not None else nthreads_default(),
           sel.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return J, K, int(nq)


def jk_blocks(ob, Ds, pa, pb, nthreads: int | None = None):
    """Whole J and K blocks of shell pairs (pa[i], pb[i]) from their
    definitions, for a list of real densities: returns lists (one entry per
    pair) of (J, K) arrays of shape (len(Ds), n_a, n_b)."""
    Ds = [np.ascontiguousarray(D, dtype=np.float64) for D in Ds]
    D = np.ascontiguousarray(np.stack(Ds))
    pa = np.ascontiguousarray(pa, dtype=np.int32)
    pb = np.ascontiguousarray(pb, dtype=np.int32)
    npairs = int(pa.shape[0])
    Jo = np.zeros((len(Ds), npairs, 36))
    Ko = np.zeros((len(Ds), npairs, 36))
    lib().or_jk_blocks(*ob.args(), len(Ds), _d(D), npairs, _i(pa), _i(pb), _d(Jo), _d(Ko),
                       nthreads if nthreads is not None else nthreads_default())
    nc = [(int(l) + 1) * (int(l) + 2) // 2 for l in ob.L]
    out = []
    for p in range(npairs):
        na, nb = nc[pa[p]], nc[pb[p]]
        out.append((Jo[:, p, :na * nb].reshape(len(Ds), na, nb), Ko[:, p, :na * nb].reshape(len(Ds), na, nb)))
    return out
