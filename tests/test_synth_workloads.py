"""The seeded workload generators: reproducible, and the sizes the
benchmark and the parity tests state.  CPU only."""
import numpy as np

import synth


def _nbf(bas):
    return int(sum((bas.shell_L + 1) * (bas.shell_L + 2) // 2))


def test_generators_are_deterministic():
    a, b = synth.workload_rt16(), synth.workload_rt16()
    assert np.array_equal(a[0].xyz, b[0].xyz) and np.array_equal(a[1].exps, b[1].exps)
    assert np.array_equal(synth.density(20, 4, 3), synth.density(20, 4, 3))
    assert not np.array_equal(synth.density(20, 4, 3), synth.density(20, 4, 4))


def test_rt16_workload():
    mol, bas = synth.workload_rt16()
    assert sorted(mol.Z.tolist()) == [1] * 10 + [8] * 6
    assert _nbf(bas) == 210
    assert mol.n_electrons() == 58
    d = np.linalg.norm(mol.xyz[:, None] - mol.xyz[None], axis=-1) + 1e9 * np.eye(16)
    assert d.min() >= 1.7 - 1e-12
    depth = np.unique(bas.shell_nprim)
    assert depth.min() >= 1 and depth.max() <= 6


def test_density_is_an_idempotent_projector_in_the_orthonormal_sense():
    P = synth.density(30, 7, 11, complex_=True)
    assert np.abs(P - P.conj().T).max() < 1e-13
    assert abs(np.trace(P).real - 7) < 1e-10
    assert np.abs(P @ P - P).max() < 1e-10


def test_batch_workload_depth_and_sizes():
    items = synth.workload_batch(16, max_depth=1)
    assert len(items) == 16
    for mol, bas in items:
        assert 4 <= mol.natom <= 12
        assert np.all(bas.shell_nprim == 1)
