"""Learned initial density: GPU gradients against the FP64 reference, and
what the trained network gains over the core-Hamiltonian guess."""
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


def _mols(n, seed, lo=4, hi=8, depth=3):
    g = synth.rng(seed)
    out = []
    for i in range(n):
        na = int(g.integers(lo, hi + 1))
        s = int(g.integers(0, 2 ** 31))
        mol = synth.cluster(na, s, p_h=0.5)
        if mol.closed_shell_charge():
            continue
        out.append((mol, synth.basis_spd(mol, s + 7, max_depth=depth)))
    return out


def test_gradient_matches_fp64_reference(cq):
    import torch
    from oracle import mlp
    items = _mols(6, 11)
    b = cq.Basis.batch(items)
    net = cq.DensityGuessMLP(seed=5)
    X, _, H = net.dataset(b)
    n = min(48, X.shape[0])
    X, H = X[:n].contiguous(), H[:n].contiguous()
    T = (torch.randn((n, 1472), generator=torch.Generator().manual_seed(1)) * 0.1).float().cuda()
    loss, g = net.loss_grad(X, T, H)
    lref, gref = mlp.loss_and_grad(net.params.cpu().numpy(), X.cpu().numpy(), T.cpu().numpy(),
                                   H.cpu().numpy().tolist())
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    ga = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(ga - gref) <= 1e-4 * np.linalg.norm(gref)


def test_learned_guess_reduces_iterations(cq):
    """Single-primitive shells (the learnable case: the AO density blocks
    then depend on the geometry only); training on converged molecules."""
    train = _mols(320, 21, depth=1)
    test = _mols(64, 22, depth=1)
    nocc_tr = [m.n_electrons() // 2 for m, _ in train]
    btr = cq.Basis.batch(train)
    Dtr, Etr, ittr, st = btr.scf_batch(nocc_tr, raise_on_fail=False)
    ok = [i for i in range(len(train)) if ittr[i] < 128]
    assert len(ok) >= 0.9 * len(train)
    # training data from the converged molecules only
    keep = [train[i] for i in ok]
    bk = cq.Basis.batch(keep)
    Dk, _, _, stk = bk.scf_batch([nocc_tr[i] for i in ok],
                                 D0=bk.pack([btr.unpack(Dtr)[i] for i in ok]))
    net = cq.DensityGuessMLP(seed=7)
    X, T, H = net.dataset(bk, Dk)
    loss0, _ = net.loss_grad(X, T, H)
    loss = net.train(X, T, H, epochs=150, batch=256, lr=2e-3, seed=3)
    print("training pairs", X.shape[0], "loss", loss0, "->", loss)
    assert loss < 0.2 * loss0, (loss, loss0)
    nocc = [m.n_electrons() // 2 for m, _ in test]
    bte = cq.Basis.batch(test)
    _, Ecore, itcore, _ = bte.scf_batch(nocc, raise_on_fail=False)
    D0 = net.guess(bte, nocc)
    _, Elrn, itlrn, _ = bte.scf_batch(nocc, D0=D0, raise_on_fail=False)
    both = (itcore < 128) & (itlrn < 128)
    assert both.sum() >= 0.8 * len(test)
    same = both & (np.abs(Ecore - Elrn) < 1e-8)
    print("converged", both.sum(), "same solution", same.sum(), "learned lower",
          int((both & (Elrn < Ecore - 1e-8)).sum()), "core lower", int((both & (Ecore < Elrn - 1e-8)).sum()))
    print("dE", (Elrn - Ecore)[both])
    print("iterations core", itcore[same].mean(), "learned", itlrn[same].mean())
    assert same.sum() >= 0.75 * both.sum()
    assert itlrn[same].mean() < itcore[same].mean(), (itlrn[same].mean(), itcore[same].mean())
