"""GPU one-electron integrals, RHF SCF and RT-TDHF steps against the oracle
(FP64 targets: 1e-10 Eh in energy; one-electron matrices to 1e-12)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_01381_gb300 as cq
    cq.build()
    return cq


@pytest.fixture(scope="module")
def dr():
    import oracle
    oracle.build()
    from oracle import drivers
    return drivers


def _mixed_case():
    mol = synth.cluster(4, 91, counts={8: 1, 7: 1, 1: 2})
    return mol, synth.basis_spd(mol, 92, max_depth=3)


def test_one_electron(cq):
    import oracle
    mol, bas = _mixed_case()
    b = cq.Basis(mol, bas)
    ob = oracle.OBasis(mol, bas)
    S, T, V, M = (x.cpu().numpy() for x in b.one_electron(origin=(0.2, -0.1, 0.3)))
    assert np.abs(S - oracle.overlap(ob)).max() < 1e-12
    assert np.abs(T - oracle.kinetic(ob)).max() < 1e-11
    assert np.abs(V - oracle.nuclear(ob)).max() < 1e-10
    assert np.abs(M - oracle.dipole(ob, origin=(0.2, -0.1, 0.3))).max() < 1e-12
    assert abs(b.nuclear_repulsion() - oracle.nuclear_repulsion(mol)) < 1e-12


def _paper_water():
    from golden import water_sample_input
    mol = synth.Molecule(*water_sample_input())
    return mol, synth.basis_triatomic(mol)


@pytest.mark.parametrize("case", ["triatomic", "mixed", "paper_water"])
def test_rhf_energy_matches_oracle(cq, dr, case):
    mol, bas = {"triatomic": synth.workload_triatomic, "mixed": _mixed_case,
                "paper_water": _paper_water}[case]()
    nocc = mol.n_electrons(mol.closed_shell_charge()) // 2
    b = cq.Basis(mol, bas)
    D, F, st = b.scf(nocc)
    ref = dr.rhf(dr.System(mol, bas), nocc)
    assert st["converged"] and ref.converged
    assert abs(st["energy"] - ref.energy) < 1e-10, (st["energy"], ref.energy)
    Dg = D.cpu().numpy()
    assert np.abs(Dg - ref.D).max() < 1e-6
    S = b.one_electron()[0].cpu().numpy()
    assert abs(np.trace(Dg @ S) - nocc) < 1e-10


@pytest.mark.parametrize("fp64_tol", [0.0, 1e-2])
def test_rhf_mixed_incremental_same_energy(cq, fp64_tol):
    """Mixed and incremental builds (two tiers, or three with a double-float
    band up to 1e-2) converge to the all-FP64 energy: the last iterations
    are all-FP64 builds."""
    mol, bas = _mixed_case()
    nocc = mol.n_electrons(mol.closed_shell_charge()) // 2
    b = cq.Basis(mol, bas)
    _, _, st64 = b.scf(nocc)
    _, _, stm = b.scf(nocc, prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4, incremental=True, fp64_tol=fp64_tol)
    assert stm["converged"]
    assert stm["quartets_fp32"] > 0
    assert (stm["quartets_df"] > 0) == (fp64_tol > 0)
    assert abs(stm["energy"] - st64["energy"]) < 1e-10


def test_rt_matches_oracle_step_by_step(cq, dr):
    import torch
    mol, bas = synth.workload_triatomic()
    b = cq.Basis(mol, bas)
    D, _, _ = b.scf(5)
    Pc = D.to(torch.complex128).clone()
    Pp = Pc.clone()
    s = dr.System(mol, bas)
    r = dr.rhf(s, 5)
    field = dict(field=(0.0, 0.0, 1e-3), t_on=0.0, t_off=0.05)
    rt = dr.RT(s, D.cpu().numpy(), 0.05, dr.Field((0.0, 0.0, 1e-3), 0.0, 0.05), restart=5)
    gobs, oobs = [], []
    for k in range(12):
        gobs.append(b.rt_step(k, Pp, Pc, dt=0.05, restart_every=5, **field))
        oobs.append(rt.step())
    for k in range(11):
        g, o = gobs[k + 1], oobs[k]
        assert np.abs(np.array(g["dipole"]) - o[0]).max() < 1e-9, k
        assert abs(g["trPS"] - o[1]) < 1e-10
        assert abs(g["energy"] - o[2]) < 1e-10
    assert gobs[0]["em2"] and gobs[5]["em2"] and not gobs[1]["em2"]
    assert abs(gobs[0]["energy"] - r.energy) < 1e-10


def test_rt_double_float_matches_oracle(cq, dr):
    """RT steps whose Fock builds run every quartet in double-float (mixed
    precision with mixed_tol 0 and no FP64 tier) follow the FP64 oracle at
    the FP64 tolerances."""
    import torch
    mol, bas = synth.workload_triatomic()
    b = cq.Basis(mol, bas)
    D, _, _ = b.scf(5)
    Pc = D.to(torch.complex128).clone()
    Pp = Pc.clone()
    s = dr.System(mol, bas)
    field = dict(field=(0.0, 0.0, 1e-3), t_on=0.0, t_off=0.05)
    rt = dr.RT(s, D.cpu().numpy(), 0.05, dr.Field((0.0, 0.0, 1e-3), 0.0, 0.05), restart=5)
    kw = dict(prec=cq.CQ_PREC_MIXED, mixed_tol=0.0, fp64_tol=1e300)
    gobs, oobs = [], []
    for k in range(12):
        gobs.append(b.rt_step(k, Pp, Pc, dt=0.05, restart_every=5, **field, **kw))
        oobs.append(rt.step())
    for k in range(11):
        g, o = gobs[k + 1], oobs[k]
        assert np.abs(np.array(g["dipole"]) - o[0]).max() < 1e-9, k
        assert abs(g["trPS"] - o[1]) < 1e-10
        assert abs(g["energy"] - o[2]) < 1e-9


def test_rt_zero_field_stationary(cq):
    import torch
    mol, bas = synth.workload_triatomic()
    b = cq.Basis(mol, bas)
    D, _, _ = b.scf(5, e_tol=1e-12, d_tol=1e-11, max_iter=200)
    Pc = D.to(torch.complex128).clone()
    Pp = Pc.clone()
    P0 = Pc.clone()
    for k in range(6):
        b.rt_step(k, Pp, Pc, dt=0.05)
    assert (Pc - P0).abs().max().item() < 1e-8


def test_ghf_scf_matches_oracle(cq, dr):
    """Two-component SCF: a cation (9 electrons) from a random spinor guess
    reaches the oracle's GHF energy; the neutral molecule from the
    (collinear) core guess reaches the RHF energy."""
    import torch
    mol, bas = synth.workload_triatomic()
    sysm = dr.System(mol, bas)
    b = cq.Basis(mol, bas)
    P2 = synth.spinor_density(sysm.n, 9, 21)
    ref = dr.ghf(sysm, 9, P0=P2)
    assert ref.converged
    P0 = torch.as_tensor(np.ascontiguousarray(dr.pauli_split(P2)), device="cuda")
    P, F, st = b.scf_ghf(9, P0=P0)
    assert st["converged"]
    assert abs(st["energy"] - ref.energy) < 1e-10, (st["energy"], ref.energy)
    # the energy of the returned density by the oracle's GHF Fock
    Pc = P.cpu().numpy()
    _, E = dr.ghf_fock(sysm, Pc)
    assert abs(E - st["energy"]) < 1e-10
    Pn, _, stn = b.scf_ghf(10)
    assert abs(stn["energy"] - dr.rhf(sysm, 5).energy) < 1e-10
    assert np.abs(Pn[1:].cpu().numpy()).max() < 1e-10      # collinear, unpolarised
