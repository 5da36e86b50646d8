"""Parity at full workload sizes on sampled outputs.

The oracle computes whole J and K blocks of 16 seeded shell pairs straight
from the definitions (every shell quartet, no screening); the GPU builds the
whole matrices in the configuration the benchmark times.  Properties that
hold at any size (symmetry, Hermiticity, the energy error of the precision
split against the GPU's all-FP64 build) are checked on the full matrices.

Tolerances: 1e-10 max-abs for all-FP64 builds (the method's FP64 target);
for mixed builds 5e-6 max-abs per element (FP32 quartets carry bounds
below mixed_tol = 3e-3 or 5e-3 and relative rounding ~1e-7; their errors add up over
the quartets touching an element) and |dE| <= 1e-6 Eh against all-FP64.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10
MIXED_TOL = 5e-3      # the benchmark's split of the rt16 build
FP64_TOL = 1.0        # double-float below, FP64 above (the benchmark's three tiers)
TOL_MIXED_ELEM = 5e-6


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


def _pairs(nsh, k, seed):
    """k seeded shell pairs a >= b, including the first and last shells."""
    g = synth.rng(seed)
    out = [(0, 0), (nsh - 1, 0), (nsh - 1, nsh - 1)]
    while len(out) < k:
        a, b = sorted(g.integers(0, nsh, 2), reverse=True)
        if (int(a), int(b)) not in out:
            out.append((int(a), int(b)))
    return out


def _bfo(bas):
    nc = [(int(l) + 1) * (int(l) + 2) // 2 for l in bas.shell_L]
    return np.concatenate([[0], np.cumsum(nc)])


def _blk(M, bfo, a, b):
    return M[..., bfo[a]:bfo[a + 1], bfo[b]:bfo[b + 1]]


def test_rt16_benchmark_configuration(cq, orc):
    """The 16-atom, 210-function workload with its complex-Hermitian
    density, as the benchmark builds it (autotuned kernel variants; FP32,
    double-float and FP64 tiers): whole blocks of 16 shell pairs, FP64 and
    mixed."""
    import torch
    mol, bas = synth.workload_rt16()
    b = cq.Basis(mol, bas)
    n = b.nbf
    Ph = synth.density(n, 29, 5, complex_=True)
    P = torch.as_tensor(Ph, device="cuda")
    b.autotune(P, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL, cache=False)
    J, K = b.fock_build(P)
    Jm, Km = b.fock_build(P, prec=cq.CQ_PREC_MIXED, mixed_tol=MIXED_TOL, fp64_tol=FP64_TOL)
    pairs = _pairs(b.nshell, 16, 3)
    ref = orc.jk_blocks(orc.OBasis(mol, bas), [Ph.real, Ph.imag], [p[0] for p in pairs], [p[1] for p in pairs])
    bfo = _bfo(bas)
    Jg, Kg, Jmg, Kmg = (x.cpu().numpy() for x in (J, K, Jm, Km))
    for (a, c), (Jo, Ko) in zip(pairs, ref):
        assert np.abs(Jo[1]).max() < 1e-12            # J of the antisymmetric part vanishes
        assert np.abs(_blk(Jg, bfo, a, c) - Jo[0]).max() < TOL
        assert np.abs(_blk(Kg, bfo, a, c) - (Ko[0] + 1j * Ko[1])).max() < TOL
        assert np.abs(_blk(Jmg, bfo, a, c) - Jo[0]).max() < TOL_MIXED_ELEM
        assert np.abs(_blk(Kmg, bfo, a, c) - (Ko[0] + 1j * Ko[1])).max() < TOL_MIXED_ELEM
    assert np.abs(Jg - Jg.T).max() < 1e-12
    assert np.abs(Kg - Kg.conj().T).max() < 1e-12
    dE = np.sum((2 * (Jmg - Jg) - (Kmg - Kg)) * Ph.T).real
    assert abs(dE) < 1e-6


def test_large100_mixed(cq, orc):
    """The 100-atom, 1930-function single build with the benchmark's
    split for it (FP32 below 3e-3, Schwarz 1e-12): whole blocks of 16 shell pairs
    against the oracle, and the symmetry of the full matrices."""
    import torch
    mol, bas = synth.workload_large100()
    b = cq.Basis(mol, bas)
    n = b.nbf
    assert n == 1930
    Ph = synth.density(n, 200, 11)
    P = torch.as_tensor(Ph, device="cuda")
    J, K, st = b.fock_build(P, prec=cq.CQ_PREC_MIXED, mixed_tol=3e-3, fp64_tol=FP64_TOL, schwarz_tol=1e-12,
                            stats=True)
    assert st["quartets_fp32"] > 100 * st["quartets_df"] > 0
    pairs = _pairs(b.nshell, 16, 4)
    ref = orc.jk_blocks(orc.OBasis(mol, bas), [Ph], [p[0] for p in pairs], [p[1] for p in pairs])
    bfo = _bfo(bas)
    Jg, Kg = J.cpu().numpy(), K.cpu().numpy()
    for (a, c), (Jo, Ko) in zip(pairs, ref):
        assert np.abs(_blk(Jg, bfo, a, c) - Jo[0]).max() < TOL_MIXED_ELEM, (a, c)
        assert np.abs(_blk(Kg, bfo, a, c) - Ko[0]).max() < TOL_MIXED_ELEM, (a, c)
    assert np.abs(Jg - Jg.T).max() < 1e-12
    assert np.abs(Kg - Kg.T).max() < 1e-12


def _pauli_split(X2c):
    n = X2c.shape[0] // 2
    aa, ab, ba, bb = X2c[:n, :n], X2c[:n, n:], X2c[n:, :n], X2c[n:, n:]
    return np.stack([0.5 * (aa + bb), 0.5 * (ab + ba), (ab - ba) / (-2j), 0.5 * (aa - bb)])


def test_ghf40_pauli_fp64_and_mixed(cq, orc):
    """The 40-atom two-component build (810 spatial functions, scalar + 3
    spin components of a random spinor density): whole blocks of 16 shell
    pairs for J and all eight real K matrices, FP64 and mixed, and the
    mixed energy error against the FP64 build."""
    import torch
    mol, bas = synth.workload_ghf40()
    b = cq.Basis(mol, bas)
    n = b.nbf
    Pc = _pauli_split(synth.spinor_density(n, int(mol.Z.sum()), 12))
    P = torch.as_tensor(np.ascontiguousarray(Pc), device="cuda")
    J, K = b.fock_build(P, schwarz_tol=1e-12)
    Jm, Km = b.fock_build(P, prec=cq.CQ_PREC_MIXED, mixed_tol=3e-3, schwarz_tol=1e-12)
    pairs = _pairs(b.nshell, 16, 5)
    Ds = [Pc[0].real] + [x for I in range(4) for x in (Pc[I].real, Pc[I].imag)]
    ref = orc.jk_blocks(orc.OBasis(mol, bas), Ds, [p[0] for p in pairs], [p[1] for p in pairs])
    bfo = _bfo(bas)
    Jg, Kg, Jmg, Kmg = (x.cpu().numpy() for x in (J, K, Jm, Km))
    for (a, c), (Jo, Ko) in zip(pairs, ref):
        assert np.abs(_blk(Jg, bfo, a, c) - Jo[0]).max() < TOL
        assert np.abs(_blk(Jmg, bfo, a, c) - Jo[0]).max() < TOL_MIXED_ELEM
        for I in range(4):
            ko = Ko[1 + 2 * I] + 1j * Ko[2 + 2 * I]
            assert np.abs(_blk(Kg[I], bfo, a, c) - ko).max() < TOL, (a, c, I)
            assert np.abs(_blk(Kmg[I], bfo, a, c) - ko).max() < TOL_MIXED_ELEM, (a, c, I)
    dE = np.sum(2 * (Jmg - Jg) * Pc[0].T).real - sum(np.sum((Kmg[I] - Kg[I]) * Pc[I].T).real for I in range(4))
    assert abs(dE) < 1e-6


@pytest.fixture(scope="module")
def dr(orc):
    from oracle import drivers
    return drivers


def test_rt_1000_steps_against_oracle(cq, dr):
    """1000 MMUT steps (EM2 start and restart every 50 steps) on the
    triatomic after a delta kick of 1e-4 au along z, dt = 0.05 au: dipole,
    Tr(PS) and energy equal to the oracle's at every step (FP64)."""
    import torch
    mol, bas = synth.workload_triatomic()
    b = cq.Basis(mol, bas)
    D, _, _ = b.scf(5)
    Pc = D.to(torch.complex128).clone()
    Pp = Pc.clone()
    s = dr.System(mol, bas)
    rt = dr.RT(s, D.cpu().numpy(), 0.05, dr.Field((0.0, 0.0, 1e-4), 0.0, 0.05), restart=50)
    field = dict(field=(0.0, 0.0, 1e-4), t_on=0.0, t_off=0.05)
    worst = [0.0, 0.0, 0.0]
    g = b.rt_step(0, Pp, Pc, dt=0.05, restart_every=50, **field)
    for k in range(1, 1001):
        o = rt.step()
        g = b.rt_step(k, Pp, Pc, dt=0.05, restart_every=50, **field)
        worst[0] = max(worst[0], float(np.abs(np.array(g["dipole"]) - o[0]).max()))
        worst[1] = max(worst[1], abs(g["trPS"] - o[1]))
        worst[2] = max(worst[2], abs(g["energy"] - o[2]))
    assert worst[0] < 1e-9 and worst[1] < 1e-10 and worst[2] < 1e-9, worst


def test_rt16_kick_response(cq):
    """RT-TDHF on the 16-atom workload (210 functions, FP64): after delta
    kicks of 1e-4 and 2e-4 au along z, Tr(PS) stays N_occ, the field-free
    energy is conserved, and the dipole response is linear in the kick."""
    import torch
    mol, bas = synth.workload_rt16()
    b = cq.Basis(mol, bas)
    nocc = int(mol.Z.sum()) // 2
    D, E0, st = b.scf(nocc)
    assert st["converged"]
    resp = {}
    for amp in (1e-4, 2e-4):
        Pc = D.to(torch.complex128).clone()
        Pp = Pc.clone()
        mu, tr, en = [], [], []
        for k in range(40):
            o = b.rt_step(k, Pp, Pc, dt=0.05, field=(0.0, 0.0, amp), t_on=0.0, t_off=0.05)
            mu.append(o["dipole"][2]); tr.append(o["trPS"]); en.append(o["energy"])
        assert np.abs(np.array(tr) - nocc).max() < 1e-9
        # MMUT conserves the field-free energy to O(dt^2) of the motion the
        # kick starts: 1e-7 Eh on -349.5 Eh (3e-10 relative) over 40 steps
        assert np.ptp(en[2:]) < 1e-7
        resp[amp] = np.array(mu)
    d1 = resp[1e-4] - resp[1e-4][0]
    d2 = resp[2e-4] - resp[2e-4][0]
    assert np.abs(d1).max() > 1e-7
    assert np.abs(d2 - 2 * d1).max() < 1e-2 * np.abs(d1).max()
