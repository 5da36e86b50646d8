"""Parity at full workload sizes on sampled outputs: the oracle computes the
sampled J/K elements one by one from their definitions, the GPU builds the
whole matrices in the configuration the benchmark times (autotuned kernel
variants, FP64 and mixed precision).  Properties that hold at any size
(symmetry, Hermiticity, the mixed-precision energy error) are checked on
the full matrices."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10
MIXED_TOL = 3e-3      # the precision split the benchmark times


@pytest.fixture(scope="module")
def cq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_01381_gb300 as cq
    cq.build()
    return cq


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _sample(n, k, seed):
    g = synth.rng(seed)
    mu = np.concatenate([[0, n - 1, 0, n - 1], g.integers(0, n, k)])
    nu = np.concatenate([[0, n - 1, n - 1, 0], g.integers(0, n, k)])
    return mu.astype(np.int32), nu.astype(np.int32)


def test_rt16_benchmark_configuration(cq, orc):
    """The 16-atom, 210-function workload with its complex-Hermitian
    density, exactly as the benchmark builds it."""
    import torch
    mol, bas = synth.workload_rt16()
    b = cq.Basis(mol, bas)
    n = b.nbf
    Ph = synth.density(n, 29, 5, complex_=True)
    P = torch.as_tensor(Ph, device="cuda")
    b.autotune(P, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, cache=False)
    J, K = b.fock_build(P)
    Jm, Km = b.fock_build(P, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL)
    mu, nu = _sample(n, 12, 3)
    Jo, Ko = orc.jk_elements(orc.OBasis(mol, bas), [Ph.real, Ph.imag], mu, nu)
    Jg, Kg = J.cpu().numpy(), K.cpu().numpy()
    assert np.abs(Jg[mu, nu] - Jo[0]).max() < TOL
    assert np.abs(Jo[1]).max() < 1e-12          # J of the antisymmetric part vanishes
    assert np.abs(Kg[mu, nu] - (Ko[0] + 1j * Ko[1])).max() < TOL
    assert np.abs(Jg - Jg.T).max() < 1e-12
    assert np.abs(Kg - Kg.conj().T).max() < 1e-12
    Jmg, Kmg = Jm.cpu().numpy(), Km.cpu().numpy()
    assert np.abs(Jmg[mu, nu] - Jo[0]).max() < 1e-6
    assert np.abs(Kmg[mu, nu] - (Ko[0] + 1j * Ko[1])).max() < 1e-6
    dE = np.sum((2 * (Jmg - Jg) - (Kmg - Kg)) * Ph.T).real
    assert abs(dE) < 1e-6
