"""Seeded synthetic inputs: molecules, even-tempered Cartesian basis sets and
random densities.

This module is shared by the oracle side and the GPU side and therefore holds
none of the method's arithmetic: it only draws coordinates, exponents,
contraction coefficients and random orbital matrices.  Normalisation,
integrals, the Pauli split of a two-component density, and everything else
the method computes live separately in ``oracle/`` and in the package.

Workload recipe (all numbers in atomic units, bohr):

* water-like triatomic: O at the origin, two H at 1.8*(1+U(-0.05,0.05)),
  H-O-H angle 104.5 deg*(1+U(-0.05,0.05)).
* clusters: rejection sampling in a cube of side (N*12)^(1/3) with a minimum
  pair distance of 1.7.
* basis "triatomic": per atom three s shells with centre exponents
  0.2*3^k (k=0,1,2), each contracted over three primitives
  alpha_k*3^((j-1)/3), equal coefficients, plus one single-primitive p shell
  of exponent 0.8.
* basis "spd": heavy atoms (Z>1) 4 s (0.2*3^k, k<4), 3 p (k<3), 2 d
  (0.4, 1.2); hydrogen 3 s (k<3) and 1 p (0.8).  Each shell draws a
  contraction depth d in {1..6}; primitives alpha*3^((j-(d-1)/2)/d),
  coefficients U[0.5, 1].
"""
from __future__ import annotations

import dataclasses
import numpy as np

L_MAX = 2


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclasses.dataclass
class Molecule:
    Z: np.ndarray      # (natom,) int32 nuclear charges
    xyz: np.ndarray    # (natom, 3) float64, bohr

    @property
    def natom(self) -> int:
        return int(self.Z.shape[0])

    def n_electrons(self, charge: int = 0) -> int:
        return int(self.Z.sum()) - charge

    def closed_shell_charge(self) -> int:
        """Neutral if the electron count is even, else +1."""
        return int(self.Z.sum()) % 2


@dataclasses.dataclass
class Basis:
    """Shells of contracted Cartesian Gaussians (raw, unnormalised coefs)."""
    shell_atom: np.ndarray   # (nshell,) int32
    shell_L: np.ndarray      # (nshell,) int32, 0..2
    shell_nprim: np.ndarray  # (nshell,) int32
    exps: np.ndarray         # (sum nprim,) float64
    coefs: np.ndarray        # (sum nprim,) float64

    @property
    def nshell(self) -> int:
        return int(self.shell_L.shape[0])

    @property
    def nbf(self) -> int:
        L = self.shell_L
        return int(((L + 1) * (L + 2) // 2).sum())

    def shell_centers(self, mol: Molecule) -> np.ndarray:
        return np.ascontiguousarray(mol.xyz[self.shell_atom])


def triatomic(seed: int) -> Molecule:
    g = rng(seed)
    r1 = 1.8 * (1 + g.uniform(-0.05, 0.05))
    r2 = 1.8 * (1 + g.uniform(-0.05, 0.05))
    th = np.deg2rad(104.5 * (1 + g.uniform(-0.05, 0.05)))
    xyz = np.array([[0.0, 0.0, 0.0],
                    [r1, 0.0, 0.0],
                    [r2 * np.cos(th), r2 * np.sin(th), 0.0]])
    return Molecule(np.array([8, 1, 1], dtype=np.int32), xyz)


def _place(g: np.random.Generator, n: int, dmin: float = 1.7,
           v0: float = 12.0) -> np.ndarray:
    side = (n * v0) ** (1.0 / 3.0)
    pts: list[np.ndarray] = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("cluster placement failed")
        p = g.uniform(0.0, side, size=3)
        if all(np.linalg.norm(p - q) >= dmin for q in pts):
            pts.append(p)
    xyz = np.array(pts)
    return xyz - xyz.mean(axis=0)


def cluster(natom: int, seed: int, p_h: float = 0.25,
            heavy=(6, 7, 8), counts: dict | None = None) -> Molecule:
    """Seeded cluster.  ``counts`` (element -> number) fixes the composition;
    otherwise each atom is H with probability p_h, else uniform over heavy."""
    g = rng(seed)
    if counts is not None:
        Z = np.concatenate([np.full(c, z) for z, c in counts.items()])
        g.shuffle(Z)
        assert Z.shape[0] == natom
    else:
        Z = np.where(g.uniform(size=natom) < p_h, 1,
                     g.choice(np.array(heavy), size=natom))
    xyz = _place(g, natom)
    return Molecule(Z.astype(np.int32), xyz)


def _depth_prims(g, alpha, depth):
    j = np.arange(depth)
    ex = alpha * 3.0 ** ((j - (depth - 1) / 2.0) / depth)
    co = g.uniform(0.5, 1.0, size=depth)
    return ex, co


def basis_triatomic(mol: Molecule) -> Basis:
    atoms, Ls, nps, ex, co = [], [], [], [], []
    for a in range(mol.natom):
        for k in range(3):
            al = 0.2 * 3.0 ** k
            e = al * 3.0 ** ((np.arange(3) - 1) / 3.0)
            atoms.append(a); Ls.append(0); nps.append(3)
            ex.append(e); co.append(np.ones(3))
        atoms.append(a); Ls.append(1); nps.append(1)
        ex.append(np.array([0.8])); co.append(np.ones(1))
    return Basis(np.array(atoms, np.int32), np.array(Ls, np.int32),
                 np.array(nps, np.int32), np.concatenate(ex),
                 np.concatenate(co))


def basis_spd(mol: Molecule, seed: int, max_depth: int = 6,
              min_depth: int = 1) -> Basis:
    g = rng(seed)
    atoms, Ls, nps, ex, co = [], [], [], [], []

    def add(a, L, alpha):
        d = int(g.integers(min_depth, max_depth + 1))
        e, c = _depth_prims(g, alpha, d)
        atoms.append(a); Ls.append(L); nps.append(d); ex.append(e); co.append(c)

    for a in range(mol.natom):
        if mol.Z[a] > 1:
            for k in range(4):
                add(a, 0, 0.2 * 3.0 ** k)
            for k in range(3):
                add(a, 1, 0.2 * 3.0 ** k)
            add(a, 2, 0.4)
            add(a, 2, 1.2)
        else:
            for k in range(3):
                add(a, 0, 0.2 * 3.0 ** k)
            add(a, 1, 0.8)
    return Basis(np.array(atoms, np.int32), np.array(Ls, np.int32),
                 np.array(nps, np.int32), np.concatenate(ex),
                 np.concatenate(co))


def orbitals(n: int, nocc: int, seed: int, complex_: bool = False,
             scale: float = 1.0) -> np.ndarray:
    """Random orthonormal (Euclidean) columns, n x nocc."""
    g = rng(seed)
    A = g.standard_normal((n, nocc))
    if complex_:
        A = A + 1j * g.standard_normal((n, nocc))
    Q, _ = np.linalg.qr(A)
    return Q * scale


def density(n: int, nocc: int, seed: int, complex_: bool = False,
            scale: float = 1.0) -> np.ndarray:
    """P = C C^dagger from random orthonormal orbitals (Hermitian PSD)."""
    C = orbitals(n, nocc, seed, complex_, scale)
    return C @ C.conj().T


def spinor_density(n: int, nocc: int, seed: int) -> np.ndarray:
    """2n x 2n P^{2C} = C C^dagger from random unitary occupied spinors,
    rows/columns ordered (alpha block, beta block)."""
    return density(2 * n, nocc, seed, complex_=True)


def hermitian_component(n: int, seed: int, complex_: bool = True,
                        scale: float = 1.0) -> np.ndarray:
    """A random Hermitian matrix (not tied to any wavefunction)."""
    g = rng(seed)
    A = g.standard_normal((n, n))
    if complex_:
        A = A + 1j * g.standard_normal((n, n))
    return scale * 0.5 * (A + A.conj().T)


# ---- named workloads -----------------------------------------------------

def workload_triatomic(rep: int = 0):
    mol = triatomic(1000 * 1 + rep)
    return mol, basis_triatomic(mol)


def workload_rt16(rep: int = 0):
    seed = 1000 * 2 + rep
    mol = cluster(16, seed, counts={8: 6, 1: 10})
    return mol, basis_spd(mol, seed + 7)


def workload_large100(rep: int = 0):
    seed = 1000 * 3 + rep
    mol = cluster(100, seed, p_h=0.25)
    return mol, basis_spd(mol, seed + 7)


def workload_ghf40(rep: int = 0):
    seed = 1000 * 4 + rep
    mol = cluster(40, seed, counts={8: 10, 7: 10, 6: 10, 1: 10})
    return mol, basis_spd(mol, seed + 7)


def workload_batch(nmol: int = 512, rep: int = 0, max_depth: int = 6):
    out = []
    g = rng(1000 * 5 + rep)
    for i in range(nmol):
        na = int(g.integers(4, 13))
        s = int(g.integers(0, 2 ** 31))
        mol = cluster(na, s, p_h=0.5)
        out.append((mol, basis_spd(mol, s + 7, max_depth=max_depth)))
    return out


def small_cluster(natom: int, seed: int, p_h: float = 0.5,
                  max_depth: int = 3):
    """Small mixed s,p,d cases for parity tests that the oracle finishes in
    seconds."""
    mol = cluster(natom, seed, p_h=p_h)
    return mol, basis_spd(mol, seed + 7, max_depth=max_depth)
