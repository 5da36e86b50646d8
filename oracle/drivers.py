"""Oracle drivers (test infrastructure): Pauli split, Fock matrices, RHF and
GHF SCF with DIIS, and RT-TDHF with MMUT/EM2.

Readings of the paper used here (each also listed in the design notes):
  * Eq. 2c_fock with the Pauli split of Eq. pauli_sep (X^0 = (X^aa+X^bb)/2):
    F^0 = h + 2 J[P^0] - K[P^0],  F^k = -K[P^k]  (k = 1, 2, 3); the factor 2
    makes a collinear closed-shell P^{2C} = diag(D, D) reproduce RHF.
  * Energy: E = sum_I Tr[(h^I + F^I) P^I] + E_nuc (Eq. 2c_expectation gives
    Tr[O^{2C} P^{2C}] = 2 sum_I Tr[O^I P^I]; the HF energy is half of
    Tr[(h+F)P] in the 2C basis).  RHF: E = Tr[(h + F) D] + E_nuc, D = C_occ C_occ^T.
  * K_{mn} = sum_{ls} (ml|sn) P_{ls} with P = C C^dagger.
  * SCF: core guess, DIIS on e = X^T (F D S - S D F) X, subspace 8; converged
    when |dE| and rms(e) are below the requested thresholds.
  * RT (Sec. Real-Time Electronic Dynamics): Loewdin orthonormal basis,
    MMUT P'_{k+1} = U P'_{k-1} U^+, U = exp(-2i dt F'(P_k, t_k)); EM2 for the
    first step and every ``restart`` steps; exponentials by Hermitian
    eigendecomposition; field V(t) = E(t) . r (electron charge -1, length
    gauge) with the step envelope on [t_on, t_off).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import (OBasis, core_hamiltonian, dipole, jk, nuclear_repulsion,
               overlap)


# ---------------- Pauli spin basis (Eq. pauli_sep) ----------------

def pauli_split(X2c: np.ndarray) -> np.ndarray:
    """2n x 2n spin-blocked matrix -> (4, n, n) components X^0..X^3."""
    n = X2c.shape[0] // 2
    aa, ab = X2c[:n, :n], X2c[:n, n:]
    ba, bb = X2c[n:, :n], X2c[n:, n:]
    X0 = 0.5 * (aa + bb)
    X1 = 0.5 * (ab + ba)
    X2 = (ab - ba) / (-2j)
    X3 = 0.5 * (aa - bb)
    return np.stack([X0, X1, X2, X3])


def pauli_join(X: np.ndarray) -> np.ndarray:
    """(4, n, n) -> 2n x 2n, X^{2C} = sum_I X^I (x) sigma_I."""
    s = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]),
         np.array([[1, 0], [0, -1]])]
    return sum(np.kron(s[I], X[I]) for I in range(4))


# ---------------- helpers ----------------

def orthogonalizer(S: np.ndarray, lin_dep: float = 1e-8):
    w, V = np.linalg.eigh(S)
    if w.min() >= lin_dep:
        return (V * w ** -0.5) @ V.T, 0
    keep = w >= lin_dep
    return V[:, keep] * w[keep] ** -0.5, int((~keep).sum())


@dataclasses.dataclass
class SCFResult:
    energy: float
    D: np.ndarray
    F: np.ndarray
    iterations: int
    converged: bool
    energies: list


class _DIIS:
    def __init__(self, nvec=8):
        self.nvec = nvec
        self.F, self.e = [], []

    def push(self, F, e):
        self.F.append(F); self.e.append(e)
        if len(self.F) > self.nvec:
            self.F.pop(0); self.e.pop(0)

    def extrapolate(self):
        m = len(self.F)
        if m < 2:
            return self.F[-1]
        B = -np.ones((m + 1, m + 1), dtype=complex if np.iscomplexobj(self.e[0]) else float)
        B[m, m] = 0
        for i in range(m):
            for j in range(m):
                B[i, j] = np.vdot(self.e[i], self.e[j])
        rhs = np.zeros(m + 1); rhs[m] = -1
        c = np.linalg.solve(B, rhs)
        return sum(c[i] * self.F[i] for i in range(m))


class System:
    """One-electron data of a molecule in a basis (oracle side)."""

    def __init__(self, mol, basis):
        self.mol, self.basis = mol, basis
        self.ob = OBasis(mol, basis)
        self.S = overlap(self.ob)
        self.h = core_hamiltonian(self.ob)
        self.Enuc = nuclear_repulsion(mol)
        self.X, self.ndrop = orthogonalizer(self.S)
        self.n = self.ob.nbf


def rhf_fock(sysm: System, D: np.ndarray, nthreads=None):
    J, K = jk(sysm.ob, D, nthreads)
    F = sysm.h + 2.0 * J - K
    E = float(np.real(np.sum((sysm.h + F) * D.T))) + sysm.Enuc
    return F, E


def rhf(sysm: System, nocc: int, e_tol=1e-10, d_tol=1e-8, max_iter=128,
        nthreads=None, D0=None) -> SCFResult:
    S, X = sysm.S, sysm.X

    def dens(F):
        w, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp[:, :nocc]
        return C @ C.T

    D = dens(sysm.h) if D0 is None else D0
    diis = _DIIS()
    Eold, energies = None, []
    for it in range(1, max_iter + 1):
        F, E = rhf_fock(sysm, D, nthreads)
        energies.append(E)
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        rms = float(np.sqrt(np.mean(err ** 2)))
        if Eold is not None and abs(E - Eold) < e_tol and rms < d_tol:
            return SCFResult(E, D, F, it, True, energies)
        Eold = E
        diis.push(F, err)
        D = dens(diis.extrapolate())
    return SCFResult(E, D, F, max_iter, False, energies)


# ---------------- GHF in the Pauli basis ----------------

def ghf_fock(sysm: System, P: np.ndarray, nthreads=None):
    """P: (4, n, n) complex Pauli components -> (F (4,n,n), E)."""
    J0, K0 = jk(sysm.ob, P[0], nthreads)
    F = np.zeros_like(P, dtype=complex)
    F[0] = sysm.h + 2.0 * J0 - K0
    for k in (1, 2, 3):
        _, Kk = jk(sysm.ob, P[k], nthreads)
        F[k] = -Kk
    hI = [sysm.h, 0, 0, 0]
    E = sysm.Enuc
    for I in range(4):
        E += float(np.real(np.sum((hI[I] + F[I]) * P[I].T)))
    return F, E


def ghf(sysm: System, nelec: int, e_tol=1e-10, d_tol=1e-8, max_iter=200,
        P0=None, nthreads=None) -> SCFResult:
    n = sysm.n
    S2 = np.kron(np.eye(2), sysm.S)
    X2 = np.kron(np.eye(2), sysm.X)

    def dens(F2):
        w, Cp = np.linalg.eigh(X2.conj().T @ F2 @ X2)
        C = X2 @ Cp[:, :nelec]
        return C @ C.conj().T

    if P0 is None:
        P2 = dens(np.kron(np.eye(2), sysm.h).astype(complex))
    else:
        P2 = P0
    diis = _DIIS()
    Eold, energies = None, []
    for it in range(1, max_iter + 1):
        F, E = ghf_fock(sysm, pauli_split(P2), nthreads)
        F2 = pauli_join(F)
        energies.append(E)
        err = X2.conj().T @ (F2 @ P2 @ S2 - S2 @ P2 @ F2) @ X2
        rms = float(np.sqrt(np.mean(np.abs(err) ** 2)))
        if Eold is not None and abs(E - Eold) < e_tol and rms < d_tol:
            return SCFResult(E, P2, F2, it, True, energies)
        Eold = E
        diis.push(F2, err)
        P2 = dens(diis.extrapolate())
    return SCFResult(E, P2, F2, max_iter, False, energies)


# ---------------- RT-TDHF (closed shell) ----------------

@dataclasses.dataclass
class Field:
    amp: tuple = (0.0, 0.0, 0.0)
    t_on: float = 0.0
    t_off: float = 0.0

    def at(self, t: float) -> np.ndarray:
        on = self.t_on <= t < self.t_off
        return np.asarray(self.amp, dtype=float) * (1.0 if on else 0.0)


def _expm_herm(Fp: np.ndarray, a: float) -> np.ndarray:
    """exp(-i a Fp) for Hermitian Fp by eigendecomposition."""
    w, V = np.linalg.eigh(Fp)
    return (V * np.exp(-1j * a * w)) @ V.conj().T


class RT:
    """Closed-shell RT-TDHF in the orthonormal basis (oracle)."""

    def __init__(self, sysm: System, D0: np.ndarray, dt: float, field: Field,
                 restart: int = 50, nthreads=None, two_electron: bool = True):
        self.s = sysm
        self.dt, self.field, self.restart = dt, field, restart
        self.nthreads = nthreads
        self.two_electron = two_electron
        # two_electron=False propagates under h + V(t) alone (no J, K): a
        # test-only switch whose exact solution is a plain unitary rotation
        S, X = sysm.S, sysm.X
        self.Xinv = X.T @ S          # X^dagger S maps AO density to ortho: P' = X^+ S P S X
        self.mu = dipole(sysm.ob)    # moment integrals about the origin
        self.P_cur = self._to_ortho(D0.astype(complex))
        self.P_prev = None
        self.k = 0

    def _to_ortho(self, P):
        return self.Xinv @ P @ self.Xinv.T

    def _to_ao(self, Pp):
        X = self.s.X
        return X @ Pp @ X.T

    def fock(self, Pp, t):
        P = self._to_ao(Pp)
        if self.two_electron:
            F0, E = rhf_fock(self.s, P, self.nthreads)
        else:
            F0, E = self.s.h, None
        V = np.tensordot(self.field.at(t), self.mu, axes=1)
        X = self.s.X
        return X.T @ (F0 + V) @ X, E

    def observables(self, Pp):
        P = self._to_ao(Pp)
        mol = self.s.mol
        nuc = (mol.Z[:, None] * mol.xyz).sum(axis=0)
        dip = -2.0 * np.real(np.einsum('dij,ji->d', self.mu, P)) + nuc
        trPS = float(np.real(np.sum(P * self.s.S.T)))
        _, E = rhf_fock(self.s, P, self.nthreads)
        return dip, trPS, E

    def step(self):
        t = self.k * self.dt
        dt = self.dt
        if self.P_prev is None or (self.restart > 0 and self.k % self.restart == 0):
            Fk, _ = self.fock(self.P_cur, t)
            U = _expm_herm(Fk, dt)
            Pfe = U @ self.P_cur @ U.conj().T
            Fk1, _ = self.fock(Pfe, t + dt)
            U = _expm_herm(0.5 * (Fk + Fk1), dt)
            Pn = U @ self.P_cur @ U.conj().T
        else:
            Fk, _ = self.fock(self.P_cur, t)
            U = _expm_herm(Fk, 2.0 * dt)
            Pn = U @ self.P_prev @ U.conj().T
        self.P_prev, self.P_cur = self.P_cur, Pn
        self.k += 1
        return self.observables(Pn)
