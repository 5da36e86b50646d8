"""Pins on the paper's own sample molecule (the water geometry of its input
specification figure): the mirror symmetry of that geometry fixes two
dipole components and the equivalence of the two hydrogens.  CPU only."""
import numpy as np
import pytest

import synth
from golden import water_sample_input


@pytest.fixture(scope="module")
def water(oracle_lib):
    from oracle import drivers
    Z, xyz = water_sample_input()
    mol = synth.Molecule(Z, xyz)
    bas = synth.basis_triatomic(mol)
    s = drivers.System(mol, bas)
    r = drivers.rhf(s, 5)
    assert r.converged
    return mol, bas, s, r


def test_sample_geometry(water):
    mol = water[0]
    d1 = np.linalg.norm(mol.xyz[1] - mol.xyz[0]) / golden_angstrom()
    d2 = np.linalg.norm(mol.xyz[2] - mol.xyz[0]) / golden_angstrom()
    v1, v2 = mol.xyz[1] - mol.xyz[0], mol.xyz[2] - mol.xyz[0]
    ang = np.degrees(np.arccos(v1 @ v2 / np.linalg.norm(v1) / np.linalg.norm(v2)))
    assert abs(d1 - d2) < 1e-12
    # the printed coordinates encode r(OH) = 1.1 Angstrom, angle HOH = 104 degrees
    assert abs(d1 - 1.1) < 1e-9 and abs(ang - 104.0) < 1e-7


def golden_angstrom():
    from golden import ANGSTROM
    return ANGSTROM


def test_mirror_symmetry_fixes_dipole(water, oracle_lib):
    """x -> -x and z -> -z map the molecule onto itself: the x and z dipole
    components vanish, the y component does not."""
    mol, bas, s, r = water
    M = oracle_lib.dipole(s.ob)
    nuc = (mol.Z[:, None] * mol.xyz).sum(0)
    mu = np.array([-2 * np.sum(M[k] * r.D) + nuc[k] for k in range(3)])
    assert abs(mu[0]) < 1e-10 and abs(mu[2]) < 1e-10
    assert abs(mu[1]) > 1e-3


def test_hydrogens_equivalent(water, oracle_lib):
    """Exchanging the two hydrogens (atoms and their basis functions) leaves
    the energy unchanged and permutes the density blocks."""
    from oracle import drivers
    mol, bas, s, r = water
    perm_atoms = [0, 2, 1]
    mol2 = synth.Molecule(mol.Z[perm_atoms], mol.xyz[perm_atoms])
    s2 = drivers.System(mol2, synth.basis_triatomic(mol2))
    r2 = drivers.rhf(s2, 5)
    assert abs(r2.energy - r.energy) < 1e-10
    n1 = s.n // 3
    p = np.r_[0:n1, 2 * n1:3 * n1, n1:2 * n1]
    assert np.abs(r2.D - r.D[np.ix_(p, p)]).max() < 1e-8
