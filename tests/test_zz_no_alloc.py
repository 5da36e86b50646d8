"""The allocation-free Fock build (cq_fock_build_noalloc), called through the
C ABI, must give the same J and K as cq_fock_build, twice in a row (its
scratch array keeps the previous call's contents), for every density kind,
both precision modes and a basis that builds in passes; it must work as the
very first build on a fresh basis handle, leave the device's free memory
unchanged once warmed up, and refuse a basis too large for its fixed
scratch.  Collected last on purpose."""
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


def _noalloc(cq, b, kind, P, J, K, prec=None, mixed_tol=1e-5):
    import torch
    o = cq.FockOpts(1e-14, mixed_tol, cq.CQ_PREC_FP64 if prec is None else prec, 1, 1)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = cq.lib().cq_fock_build_noalloc(b.h, kind, ctypes.c_void_p(P.data_ptr()),
                                        ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(K.data_ptr()),
                                        ctypes.byref(o), s)
    return rc


def _small():
    mol = synth.cluster(5, 311, counts={8: 2, 1: 3})
    return mol, synth.basis_spd(mol, 312, max_depth=4)


def _densities(cq, n):
    import torch
    Pp = np.stack([synth.hermitian_component(n, 30 + i, scale=0.1) for i in range(4)])
    return [(cq.CQ_DENS_REAL_SYM, torch.as_tensor(synth.density(n, 7, 21), device="cuda")),
            (cq.CQ_DENS_COMPLEX_HERM, torch.as_tensor(synth.density(n, 6, 22, complex_=True), device="cuda")),
            (cq.CQ_DENS_PAULI4, torch.as_tensor(Pp, device="cuda"))]


def _check_twice(cq, b, kind, P, prec=None, mixed_tol=1e-5):
    import torch
    n = b.nbf
    kw = {} if prec is None else {"prec": prec, "mixed_tol": mixed_tol}
    Jr, Kr = b.fock_build(P, kind=kind, **kw)
    for rep in range(2):
        J = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        K = torch.full_like(Kr, float("nan"))
        assert _noalloc(cq, b, kind, P, J, K, prec, mixed_tol) == 0, cq.lib().cq_last_error()
        torch.cuda.synchronize()
        assert (J - Jr).abs().max().item() < TOL, (kind, prec, rep)
        assert (K - Kr).abs().max().item() < TOL, (kind, prec, rep)


def test_noalloc_first_build_on_fresh_handle(cq):
    """No cq_fock_build before the call: the allocation-free build must not
    rely on scratch an earlier ordinary build left in the handle."""
    import torch
    mol, bas = _small()
    b = cq.Basis(mol, bas)
    n = b.nbf
    P = torch.as_tensor(synth.density(n, 7, 21), device="cuda")
    J = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    K = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(cq, b, cq.CQ_DENS_REAL_SYM, P, J, K) == 0, cq.lib().cq_last_error()
    torch.cuda.synchronize()
    Jr, Kr = cq.Basis(mol, bas).fock_build(P)
    assert (J - Jr).abs().max().item() < TOL
    assert (K - Kr).abs().max().item() < TOL


def test_noalloc_matches_fock_build_twice(cq):
    mol, bas = _small()
    b = cq.Basis(mol, bas)
    for kind, P in _densities(cq, b.nbf):
        _check_twice(cq, b, kind, P)
        _check_twice(cq, b, kind, P, prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4)


def test_noalloc_in_pass_mode(cq):
    """A basis whose candidate quartets exceed the list capacity builds in
    passes; the allocation-free build drains the same lists."""
    mol, bas = _small()
    old = cq.get_list_capacity()
    cq.set_list_capacity(3000)
    try:
        b = cq.Basis(mol, bas)
    finally:
        cq.set_list_capacity(old)
    kind, P = _densities(cq, b.nbf)[1]
    _check_twice(cq, b, kind, P)
    _check_twice(cq, b, kind, P, prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4)


def test_noalloc_leaves_free_memory_unchanged(cq):
    import torch
    mol, bas = _small()
    b = cq.Basis(mol, bas)
    n = b.nbf
    P = torch.as_tensor(synth.density(n, 6, 22, complex_=True), device="cuda")
    J = torch.empty((n, n), dtype=torch.float64, device="cuda")
    K = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    assert _noalloc(cq, b, cq.CQ_DENS_COMPLEX_HERM, P, J, K) == 0     # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _noalloc(cq, b, cq.CQ_DENS_COMPLEX_HERM, P, J, K) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


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
