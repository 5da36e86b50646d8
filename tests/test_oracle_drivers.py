"""Pins of the oracle's drivers against identities of the method (Pauli spin
basis, RHF as a special case of GHF, invariances, conservation laws of the
propagators).  CPU only."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def dr(oracle_lib):
    from oracle import drivers
    return drivers


@pytest.fixture(scope="module")
def water(dr):
    mol, bas = synth.workload_triatomic()
    s = dr.System(mol, bas)
    r = dr.rhf(s, 5)
    assert r.converged
    return s, r


def test_pauli_roundtrip_and_expectation(dr):
    g = synth.rng(1)
    n = 5
    X = g.standard_normal((2 * n, 2 * n)) + 1j * g.standard_normal((2 * n, 2 * n))
    assert np.abs(dr.pauli_join(dr.pauli_split(X)) - X).max() < 1e-14
    O = g.standard_normal((2 * n, 2 * n)) + 1j * g.standard_normal((2 * n, 2 * n))
    lhs = np.trace(O @ X)
    Oi, Xi = dr.pauli_split(O), dr.pauli_split(X)
    rhs = 2 * sum(np.trace(Oi[I] @ Xi[I]) for I in range(4))
    assert abs(lhs - rhs) < 1e-12
    # Hermitian X^{2C} -> Hermitian components
    H = X + X.conj().T
    for C in dr.pauli_split(H):
        assert np.abs(C - C.conj().T).max() < 1e-14


def test_scf_properties(dr, water):
    s, r = water
    D, S = r.D, s.S
    assert abs(np.trace(D @ S) - 5) < 1e-12
    assert np.abs(D @ S @ D - D).max() < 1e-10
    assert np.abs(r.F @ D @ S - S @ D @ r.F).max() < 1e-6
    X = s.X
    assert np.abs(X.T @ S @ X - np.eye(X.shape[1])).max() < 1e-12


def test_ghf_reduces_to_rhf(dr, water):
    s, r = water
    P2 = np.kron(np.eye(2), r.D).astype(complex)
    F, E = dr.ghf_fock(s, dr.pauli_split(P2))
    Frhf, Erhf = dr.rhf_fock(s, r.D)
    assert abs(E - Erhf) < 1e-12
    assert np.abs(F[0] - Frhf).max() < 1e-12
    assert np.abs(F[1:]).max() < 1e-14


def test_ghf_collinear_equals_uhf_formula(dr, water, oracle_lib):
    s, r = water
    n = s.n
    Pa = synth.density(n, 5, 3)
    Pb = synth.density(n, 4, 4)
    P2 = np.zeros((2 * n, 2 * n), complex)
    P2[:n, :n], P2[n:, n:] = Pa, Pb
    F, E = dr.ghf_fock(s, dr.pauli_split(P2))
    F2 = dr.pauli_join(F)
    Ja, Ka = oracle_lib.jk(s.ob, Pa)
    Jb, Kb = oracle_lib.jk(s.ob, Pb)
    Faa = s.h + Ja + Jb - Ka
    Fbb = s.h + Ja + Jb - Kb
    assert np.abs(F2[:n, :n] - Faa).max() < 1e-12
    assert np.abs(F2[n:, n:] - Fbb).max() < 1e-12
    Euhf = 0.5 * (np.sum((s.h + Faa) * Pa.T) + np.sum((s.h + Fbb) * Pb.T)) + s.Enuc
    assert abs(E - Euhf.real) < 1e-12


def test_ghf_spin_rotation_invariance(dr, water):
    s, r = water
    n = s.n
    P2 = synth.spinor_density(n, 10, 5)
    F, E = dr.ghf_fock(s, dr.pauli_split(P2))
    th, nv = 0.7, np.array([0.3, -0.5, 0.81])
    nv = nv / np.linalg.norm(nv)
    sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
    Ns = sum(nv[i] * sig[i] for i in range(3))
    U2 = np.cos(th / 2) * np.eye(2) - 1j * np.sin(th / 2) * Ns
    U = np.kron(U2, np.eye(n))
    Fr, Er = dr.ghf_fock(s, dr.pauli_split(U @ P2 @ U.conj().T))
    assert abs(E - Er) < 1e-11


def test_rhf_energy_invariances(dr, water):
    s, r = water
    mol, bas = s.mol, s.basis
    Q, _ = np.linalg.qr(synth.rng(8).standard_normal((3, 3)))
    for xyz in [mol.xyz + np.array([0.3, -1.1, 2.0]), mol.xyz @ Q.T]:
        s2 = dr.System(synth.Molecule(mol.Z, xyz), bas)
        r2 = dr.rhf(s2, 5)
        assert abs(r2.energy - r.energy) < 1e-9


def test_rt_zero_field_is_stationary(dr, water):
    s, r = water
    rt = dr.RT(s, r.D, 0.05, dr.Field((0, 0, 0), 0, 0))
    P0 = rt.P_cur.copy()
    for _ in range(10):
        rt.step()
    assert np.abs(rt.P_cur - P0).max() < 1e-8


def test_rt_conservation_and_linearity(dr, water):
    s, r = water
    out = {}
    for amp in (1e-4, 2e-4):
        rt = dr.RT(s, r.D, 0.05, dr.Field((0, amp, 0), 0, 0.05), restart=50)
        ys, trs, Es = [], [], []
        for _ in range(60):
            d, tr, E = rt.step()
            ys.append(d[1]); trs.append(tr); Es.append(E)
        P = rt._to_ao(rt.P_cur)
        assert np.abs(P @ s.S @ P - P).max() < 1e-10          # idempotency
        assert np.abs(np.array(trs) - 5).max() < 1e-10          # Tr(PS)
        assert np.ptp(Es[1:]) < 1e-9                             # field-free energy after kick
        out[amp] = np.array(ys)
    y0 = dr.RT(s, r.D, 0.05, dr.Field((0, 0, 0), 0, 0)).observables(
        dr.RT(s, r.D, 0.05, dr.Field()).P_cur)[0][1]
    d1, d2 = out[1e-4] - y0, out[2e-4] - y0
    m = np.abs(d1).max()
    assert m > 1e-7
    assert np.abs(d2 - 2 * d1).max() < 1e-2 * m     # second-order response only
