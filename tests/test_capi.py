"""The C-ABI library loads and exports every symbol include/cq.h declares;
host-side argument validation returns documented status codes.  CPU only
(no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libcq():
    import paper_1905_01381_gb300 as cq
    cq.build()
    return cq.lib()


def declared_symbols():
    out = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            out += re.findall(r"\b(cq_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(out))


def test_every_declared_symbol_is_exported(libcq):
    syms = declared_symbols()
    assert "cq_fock_build" in syms and "cq_basis_create" in syms
    for s in syms:
        assert hasattr(libcq, s), s


def test_invalid_basis_rejected_on_host(libcq):
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    xyz = np.zeros(3)
    Z = np.array([1], np.int32)
    atom = np.array([0], np.int32)
    nprim = np.array([1], np.int32)
    ex = np.array([1.0])
    co = np.array([1.0])
    h = ctypes.c_void_p()
    for L, e in [(3, 1.0), (0, -1.0), (-1, 1.0)]:
        Ls = np.array([L], np.int32)
        exv = np.array([e])
        rc = libcq.cq_basis_create(1, xyz.ctypes.data_as(dp), Z.ctypes.data_as(ip), 1,
                                   atom.ctypes.data_as(ip), Ls.ctypes.data_as(ip),
                                   nprim.ctypes.data_as(ip), exv.ctypes.data_as(dp),
                                   co.ctypes.data_as(dp), ctypes.byref(h))
        assert rc == -1
        assert b"" != libcq.cq_last_error()
    bad_atom = np.array([5], np.int32)
    rc = libcq.cq_basis_create(1, xyz.ctypes.data_as(dp), Z.ctypes.data_as(ip), 1,
                               bad_atom.ctypes.data_as(ip), np.array([0], np.int32).ctypes.data_as(ip),
                               nprim.ctypes.data_as(ip), ex.ctypes.data_as(dp), co.ctypes.data_as(dp),
                               ctypes.byref(h))
    assert rc == -1
    rc = libcq.cq_fock_build(None, 0, None, None, None, None, None, None)
    assert rc == -1


def test_list_capacity_setting(libcq):
    old = libcq.cq_get_list_capacity()
    assert old >= 1024
    assert libcq.cq_set_list_capacity(10) == -1          # below the minimum: rejected
    assert libcq.cq_get_list_capacity() == old
    assert libcq.cq_set_list_capacity(4096) == 0
    assert libcq.cq_get_list_capacity() == 4096
    assert libcq.cq_set_list_capacity(old) == 0


def test_every_entry_point_rejects_null_arguments(libcq):
    """Host-side validation: each entry point returns CQ_ERR_INVALID_ARG (-1)
    with a message, before any device work, when its required pointers are
    NULL or its sizes are out of range."""
    c_int, c_ll, c_u64 = ctypes.c_int, ctypes.c_longlong, ctypes.c_ulonglong
    calls = {
        "cq_basis_layout": (None, None, None, None),
        "cq_basis_info": (None, None, None, None),
        "cq_schwarz": (None, None, None),
        "cq_fock_profile": (None, c_int(1)),
        "cq_fock_class_stats": (None, c_int(0), c_int(0), None, None, None),
        "cq_fock_set_variant": (None, c_int(0), c_int(0), c_int(0)),
        "cq_fock_get_variant": (None, c_int(0), c_int(0), None),
        "cq_fock_set_list_split": (None, c_int(0), c_int(1), c_int(1)),
        "cq_autotune": (None, c_int(0), None, None, None, None, None),
        "cq_one_electron": (None, None, None, None, None, None, None),
        "cq_scf": (None, c_int(1), None, None, None, None, None, None),
        "cq_scf_ghf": (None, c_int(2), None, None, None, None, None, None),
        "cq_scf_batch": (None, None, None, None, None, None, None, None, None),
        "cq_rt_step": (None, None, c_int(0), None, None, None, None),
        "cq_guess_dataset": (None, None, None, None, None, None, None),
        "cq_guess_density": (None, None, None, c_int(0), c_int(0), None, None),
        "cq_dense_info": (None, None, None, None),
        "cq_nuclear_repulsion": (None, None),
        "cq_nuclear_repulsion_batch": (None, None),
        "cq_mlp_init": (None, c_u64(0), None),
        "cq_mlp_loss_grad": (None, c_int(0), None, None, None, None, None, None),
        "cq_fock_build_noalloc": (None, c_int(0), None, None, None, None, None),
        "cq_peak_fma": (c_int(0), c_int(0), None, None),
    }
    for name, args in calls.items():
        f = getattr(libcq, name)
        rc = f(*args)
        assert rc == -1, (name, rc)
        assert libcq.cq_last_error(), name
