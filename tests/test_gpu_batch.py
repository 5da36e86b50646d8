"""Batched execution: many molecules in one basis, one Fock build and one
batched SCF for all of them, against the oracle molecule by molecule."""
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


def _items():
    out = [synth.workload_triatomic()]
    for k, (counts, depth) in enumerate([({8: 1, 1: 2}, 4), ({8: 1, 6: 1, 1: 2}, 3), ({7: 1, 1: 3}, 2)]):
        mol = synth.cluster(sum(counts.values()), 500 + k, counts=counts)
        out.append((mol, synth.basis_spd(mol, 600 + k, max_depth=depth)))
    return out


def test_batched_jk_and_overlap(cq):
    import oracle
    items = _items()
    b = cq.Basis.batch(items)
    assert b.nmol == len(items)
    Ds = [synth.density(sum((bas.shell_L + 1) * (bas.shell_L + 2) // 2), 3, 40 + m)
          for m, (mol, bas) in enumerate(items)]
    J, K = b.fock_build(b.pack(Ds))
    S = b.one_electron()[0]
    Jl, Kl, Sl = b.unpack(J), b.unpack(K), b.unpack(S)
    for m, (mol, bas) in enumerate(items):
        ob = oracle.OBasis(mol, bas)
        Jo, Ko = oracle.jk(ob, Ds[m])
        assert np.abs(Jl[m] - Jo).max() < 1e-10, m
        assert np.abs(Kl[m] - Ko).max() < 1e-10, m
        assert np.abs(Sl[m] - oracle.overlap(ob)).max() < 1e-12
    # padding stays zero
    Jt = J.cpu().numpy()
    for m, n in enumerate(b.mol_n):
        assert np.abs(Jt[m, n:, :]).max(initial=0.0) == 0.0


def test_batched_scf_matches_single_and_oracle(cq):
    from oracle import drivers
    items = _items()
    nocc = [mol.n_electrons(mol.closed_shell_charge()) // 2 for mol, _ in items]
    b = cq.Basis.batch(items)
    D, E, it, st = b.scf_batch(nocc)
    assert st["converged"] == len(items)
    for m, (mol, bas) in enumerate(items):
        ref = drivers.rhf(drivers.System(mol, bas), nocc[m])
        assert abs(E[m] - ref.energy) < 1e-9, (m, E[m], ref.energy)
        single = cq.Basis(mol, bas)
        _, _, s1 = single.scf(nocc[m])
        assert abs(E[m] - s1["energy"]) < 1e-9
    Dm, Em, _, stm = b.scf_batch(nocc, prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4)
    assert stm["quartets_fp32"] > 0
    assert np.abs(Em - E).max() < 1e-9
