"""The allocation-free Fock build (cq_fock_build_noalloc), called through the
C ABI, must give the same J and K as cq_fock_build, twice in a row (its
scratch array keeps the previous call's contents), and must refuse a basis
too large for its fixed scratch.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def cq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_01381_gb300 as cq
    cq.build()
    return cq


def _noalloc(cq, b, kind, P, J, K):
    import torch
    o = cq.FockOpts(1e-14, 1e-5, cq.CQ_PREC_FP64, 1, 1)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = cq.lib().cq_fock_build_noalloc(b.h, kind, ctypes.c_void_p(P.data_ptr()),
                                        ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(K.data_ptr()),
                                        ctypes.byref(o), s)
    return rc


def test_noalloc_matches_fock_build_twice(cq):
    import torch
    mol = synth.cluster(5, 311, counts={8: 2, 1: 3})
    bas = synth.basis_spd(mol, 312, max_depth=4)
    b = cq.Basis(mol, bas)
    n = b.nbf
    cases = [(cq.CQ_DENS_REAL_SYM, torch.as_tensor(synth.density(n, 7, 21), device="cuda")),
             (cq.CQ_DENS_COMPLEX_HERM, torch.as_tensor(synth.density(n, 6, 22, complex_=True), device="cuda"))]
    for kind, P in cases:
        Jr, Kr = b.fock_build(P)
        for rep in range(2):
            J = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
            K = torch.full_like(Kr, float("nan"))
            assert _noalloc(cq, b, kind, P, J, K) == 0, cq.lib().cq_last_error()
            torch.cuda.synchronize()
            assert (J - Jr).abs().max().item() < TOL, (kind, rep)
            assert (K - Kr).abs().max().item() < TOL, (kind, rep)


def test_noalloc_rejects_oversize_basis(cq):
    import torch
    mol = synth.cluster(24, 313, counts={8: 14, 1: 10})
    bas = synth.basis_spd(mol, 314, max_depth=1)
    b = cq.Basis(mol, bas)
    need = cq.lib().cq_fock_noalloc_scratch_bytes(cq.CQ_DENS_PAULI4, b.nbf, b.nshell)
    assert need > 16 * 1024 * 1024
    P = torch.zeros((4, b.nbf, b.nbf), dtype=torch.complex128, device="cuda")
    J = torch.zeros((b.nbf, b.nbf), dtype=torch.float64, device="cuda")
    K = torch.zeros_like(P)
    rc = _noalloc(cq, b, cq.CQ_DENS_PAULI4, P, J, K)
    assert rc == -1
    assert b"16 MiB" in cq.lib().cq_last_error()
