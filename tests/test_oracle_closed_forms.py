"""Pins of the oracle's energy expression and of its real-time propagator's
time scale against results fixed by mathematics alone.  CPU only.

* Energy (Eq. 2c_fock, Eq. 2c_expectation): one normalised s Gaussian of
  exponent a on a nucleus of charge Z, doubly occupied, has the closed-shell
  Hartree-Fock energy E(a) = 2 h + (ss|ss) with the textbook one-centre
  integrals T = 3a/2, <1/r> = 2 sqrt(2a/pi) and (ss|ss) = 2 sqrt(a/pi), i.e.
      E(a) = 3a - 4 Z sqrt(2a/pi) + 2 sqrt(a/pi),
  minimised at sqrt(a*) = (2 sqrt(2) Z - 1) / (3 sqrt(pi)) with
  E(a*) = -(2 sqrt(2) Z - 1)^2 / (3 pi)  (-2.3009 Eh for helium).  A common
  factor error in the energy (half a trace, a per-spin / total density
  mix-up, a factor on J) moves E(a) off this curve.
* Time scale (Eq. lvn, Sec. "Real-Time Electronic Dynamics", MMUT and EM2):
  with J and K switched off the Fock matrix is the constant h, the
  Liouville-von Neumann equation i dP'/dt = [F', P'] has the exact solution
  P'(t) = exp(-i F' t) P'(0) exp(i F' t), and both propagators are exact
  for a constant F' -- so the oracle's trajectory must equal it to round-off
  at every step.  A wrong step length (dt instead of 2 dt in the MMUT
  exponent), a wrong sign of the exponent or a wrong time in EM2 fails.
  With J and K on, MMUT and EM2 are second-order methods: the trajectories
  at dt, dt/2 and dt/4 approach one limit with successive differences
  shrinking by about 4.
"""
import copy

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def dr(oracle_lib):
    from oracle import drivers
    return drivers


def _one_gaussian(alpha, Z=2):
    mol = synth.Molecule(np.array([Z], np.int32), np.zeros((1, 3)))
    bas = synth.Basis(np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                      np.array([alpha], float), np.array([1.0]))
    return mol, bas


def _e_closed(alpha, Z):
    return 3 * alpha - 4 * Z * np.sqrt(2 * alpha / np.pi) + 2 * np.sqrt(alpha / np.pi)


@pytest.mark.parametrize("alpha", [0.05, 0.3, 0.7670, 1.9, 12.0])
def test_single_gaussian_rhf_energy(dr, alpha):
    Z = 2
    s = dr.System(*_one_gaussian(alpha, Z))
    ref = _e_closed(alpha, Z)
    # the SCF (one function, one doubly occupied orbital) and the Fock
    # expression on D = 1 must both give the closed form
    r = dr.rhf(s, 1)
    assert r.converged
    assert abs(r.energy - ref) < 1e-12, (r.energy, ref)
    F, E = dr.rhf_fock(s, np.ones((1, 1)))
    assert abs(E - ref) < 1e-12
    # F = h + 2J - K = h + (ss|ss) for the single function
    h = 1.5 * alpha - Z * 2 * np.sqrt(2 * alpha / np.pi)
    assert abs(F[0, 0] - (h + 2 * np.sqrt(alpha / np.pi))) < 1e-12
    # the same through the two-component Fock build with P^2C = diag(D, D)
    P2 = np.kron(np.eye(2), np.ones((1, 1))).astype(complex)
    Fg, Eg = dr.ghf_fock(s, dr.pauli_split(P2))
    assert abs(Eg - ref) < 1e-12


def test_single_gaussian_variational_minimum(dr):
    Z = 2
    a_star = ((2 * np.sqrt(2) * Z - 1) / (3 * np.sqrt(np.pi))) ** 2
    e_star = -(2 * np.sqrt(2) * Z - 1) ** 2 / (3 * np.pi)
    assert abs(e_star - (-2.30099)) < 1e-5       # one-Gaussian helium
    es = [dr.rhf(dr.System(*_one_gaussian(a, Z)), 1).energy for a in (0.98 * a_star, a_star, 1.02 * a_star)]
    assert abs(es[1] - e_star) < 1e-12
    assert es[0] > es[1] and es[2] > es[1]
    # E(a) = 3a - c sqrt(a), c = (4 sqrt(2) Z - 2)/sqrt(pi): the symmetric
    # second difference equals E''(a*) = c / (4 a*^{3/2}) to O(h^2)
    c = (4 * np.sqrt(2) * Z - 2) / np.sqrt(np.pi)
    e2 = c / (4 * a_star ** 1.5)
    assert abs((es[0] + es[2] - 2 * es[1]) / (0.02 * a_star) ** 2 - e2) < 1e-3 * e2


@pytest.fixture(scope="module")
def water(dr):
    mol, bas = synth.workload_triatomic()
    s = dr.System(mol, bas)
    r = dr.rhf(s, 5)
    assert r.converged
    return s, r


def test_rt_pure_h_is_exact_rotation(dr, water):
    s, r = water
    dt = 0.05
    rt = dr.RT(s, r.D, dt, dr.Field(), restart=7, two_electron=False)
    Fp = s.X.T @ s.h @ s.X
    w, V = np.linalg.eigh(Fp)
    P0 = rt.P_cur.copy()
    assert np.abs(Fp @ P0 - P0 @ Fp).max() > 1e-2       # P(0) does not commute with h
    worst = 0.0
    for k in range(1, 41):
        rt.step()
        U = (V * np.exp(-1j * w * k * dt)) @ V.conj().T
        worst = max(worst, np.abs(rt.P_cur - U @ P0 @ U.conj().T).max())
    assert worst < 1e-10, worst


def _quenched(dr, s, amp):
    """SCF density in a static field E_z = amp (the initial state of a
    field-free propagation that is not stationary)."""
    from oracle import dipole
    sf = copy.copy(s)
    sf.h = s.h + amp * dipole(s.ob)[2]
    r = dr.rhf(sf, 5)
    assert r.converged
    return r.D


def test_rt_second_order_time_convergence(dr, water):
    s, _ = water
    D0 = _quenched(dr, s, 0.02)
    T = 1.6
    traj = {}
    for dt in (0.1, 0.05, 0.025):
        rt = dr.RT(s, D0, dt, dr.Field(), restart=50)
        every = int(round(0.2 / dt))
        mu = []
        for k in range(1, int(round(T / dt)) + 1):
            d, _, _ = rt.step()
            if k % every == 0:
                mu.append(d[2])
        traj[dt] = np.array(mu)
    d1 = np.abs(traj[0.1] - traj[0.05]).max()
    d2 = np.abs(traj[0.05] - traj[0.025]).max()
    assert np.ptp(traj[0.025]) > 1e-3              # the dipole really moves
    assert 3.5 < d1 / d2 < 4.5, (d1, d2)
