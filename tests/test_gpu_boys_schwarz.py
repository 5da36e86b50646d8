"""Device Boys function and Schwarz table, element by element.

* Boys: the device function the integral kernels call (cq_boys), in FP64,
  in FP32 (FP64 below the first table interval) and in double-float,
  against the Boys function's definition F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt evaluated by
  high-precision quadrature (tests/golden/boys_mpmath.txt) on T in [0, 200],
  m <= 8: relative error <= 1e-14 in FP64, <= 1e-13 in double-float
  (48-bit words) and <= 1e-6 in FP32.
* Schwarz (direct-SCF screening, Sec. "Reference Wave Functions"): the
  library's Q_ab = sqrt(max |(mn|mn)|) over the x^L-normalised functions of
  shells a, b, against the oracle's diagonal integrals over unit-normalised
  functions rescaled by the Cartesian component factors
  s = sqrt((2L-1)!! / ((2lx-1)!! (2ly-1)!! (2lz-1)!!)), for every shell pair.
"""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


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


def _golden():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "boys_mpmath.txt")) if not ln.startswith("#")]
    T = sorted({float(r[0]) for r in rows})
    ref = np.zeros((len(T), 9))
    for r in rows:
        ref[T.index(float(r[0])), int(r[1])] = float(r[2])
    return np.array(T), ref


@pytest.mark.parametrize("fp32,tol", [(0, 1e-14), (1, 1e-6), (2, 1e-13)])
def test_device_boys_against_quadrature(cq, fp32, tol):
    import torch
    T, ref = _golden()
    mol, bas = synth.workload_triatomic()
    b = cq.Basis(mol, bas)
    for mmax in (0, 3, 8):
        F = b.boys(torch.as_tensor(T, device="cuda"), mmax, fp32=fp32).cpu().numpy()
        rel = np.abs(F - ref[:, :mmax + 1]) / ref[:, :mmax + 1]
        assert rel.max() < tol, (mmax, T[np.unravel_index(rel.argmax(), rel.shape)[0]], rel.max())


def test_device_boys_special_values(cq):
    import torch
    mol, bas = synth.workload_triatomic()
    b = cq.Basis(mol, bas)
    F = b.boys(torch.zeros(1, dtype=torch.float64, device="cuda"), 8).cpu().numpy()[0]
    assert np.abs(F - 1.0 / (2 * np.arange(9) + 1)).max() < 1e-16
    F32 = b.boys(torch.zeros(1, dtype=torch.float64, device="cuda"), 8, fp32=True).cpu().numpy()[0]
    assert np.array_equal(F32, (1.0 / (2 * np.arange(9) + 1)).astype(np.float32).astype(np.float64))


def _comp_factor(L):
    def df(n):
        return 1 if n <= 0 else n * df(n - 2)
    out = []
    for lx in range(L, -1, -1):
        for ly in range(L - lx, -1, -1):
            lz = L - lx - ly
            out.append(np.sqrt(df(2 * L - 1) / (df(2 * lx - 1) * df(2 * ly - 1) * df(2 * lz - 1))))
    return np.array(out)


@pytest.mark.parametrize("case", ["triatomic", "cluster"])
def test_schwarz_table_elementwise(cq, orc, case):
    if case == "triatomic":
        mol, bas = synth.workload_triatomic()
    else:
        mol, bas = synth.small_cluster(4, 551, max_depth=3)
    b = cq.Basis(mol, bas)
    Q = b.schwarz().cpu().numpy()
    ob = orc.OBasis(mol, bas)
    L = np.asarray(bas.shell_L)
    ns = len(L)
    assert Q.shape == (ns, ns)
    worst = 0.0
    for a in range(ns):
        sa = _comp_factor(L[a])
        for c in range(ns):
            sc = _comp_factor(L[c])
            blk = orc.eri_shell(ob, a, c, a, c)
            na, nc = len(sa), len(sc)
            diag = np.array([[blk[m, k, m, k] for k in range(nc)] for m in range(na)])
            ref = np.sqrt(np.abs(diag / (sa[:, None] * sc[None, :]) ** 2).max())
            worst = max(worst, abs(Q[a, c] - ref) / ref)
    assert worst < 1e-12, worst
