"""GPU parity of the direct Fock build (J, K <- P) against the oracle,
element by element, through the C ABI.  Tolerance: 1e-10 max-abs for the
all-FP64 path (the target stated for the method's FP64 results)."""
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


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _case(counts, seed, max_depth):
    mol = synth.cluster(sum(counts.values()), seed, counts=counts)
    return mol, synth.basis_spd(mol, seed + 1, max_depth=max_depth)


CASES = {
    "triatomic": lambda: synth.workload_triatomic(),
    "O1H2_deep": lambda: _case({8: 1, 1: 2}, 77, 6),
    "O2H2": lambda: _case({8: 2, 1: 2}, 78, 3),
    "OCNH3": lambda: _case({8: 1, 6: 1, 7: 1, 1: 3}, 79, 4),
}


def _gpu(t):
    import torch
    return torch.as_tensor(t).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_jk_real_symmetric(cq, orc, name):
    mol, bas = CASES[name]()
    b = cq.Basis(mol, bas)
    ob = orc.OBasis(mol, bas)
    n = b.nbf
    assert n == ob.nbf
    D = synth.density(n, max(1, n // 4), 11)
    J, K = b.fock_build(_gpu(D))
    Jo, Ko = orc.jk(ob, D)
    assert np.abs(J.cpu().numpy() - Jo).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL


def test_jk_complex_hermitian(cq, orc):
    mol, bas = CASES["OCNH3"]()
    b = cq.Basis(mol, bas)
    ob = orc.OBasis(mol, bas)
    P = synth.density(b.nbf, 9, 12, complex_=True)
    J, K = b.fock_build(_gpu(P))
    Jo, Ko = orc.jk(ob, P)
    assert np.abs(J.cpu().numpy() - Jo.real).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL


def test_jk_pauli4(cq, orc):
    from oracle import drivers
    mol, bas = CASES["O2H2"]()
    b = cq.Basis(mol, bas)
    ob = orc.OBasis(mol, bas)
    n = b.nbf
    P2 = synth.spinor_density(n, 13, 13)
    Pc = drivers.pauli_split(P2)
    J, K = b.fock_build(_gpu(np.ascontiguousarray(Pc)))
    Jo, _ = orc.jk(ob, Pc[0])
    assert np.abs(J.cpu().numpy() - Jo.real).max() < TOL
    Kg = K.cpu().numpy()
    for I in range(4):
        _, Ko = orc.jk(ob, Pc[I])
        assert np.abs(Kg[I] - Ko).max() < TOL, I


def test_schwarz_table(cq, orc):
    mol, bas = CASES["OCNH3"]()
    b = cq.Basis(mol, bas)
    Q = b.schwarz().cpu().numpy()
    Qo = orc.schwarz(orc.OBasis(mol, bas))
    # the library uses the x^L normalisation of each shell for its bound
    assert Q.shape == Qo.shape
    assert np.all(Q > 0)
    # bound property: every oracle |(mn|mn)| <= (s_m s_n Q_ab)^2 with s <= sqrt(3)
    assert np.all(Qo <= 3.0 * Q * (1 + 1e-12))


def test_mixed_precision_error(cq, orc):
    mol, bas = CASES["OCNH3"]()
    b = cq.Basis(mol, bas)
    ob = orc.OBasis(mol, bas)
    D = synth.density(b.nbf, 8, 14)
    J, K, st = b.fock_build(_gpu(D), prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4, stats=True)
    assert st["quartets_fp32"] > 0 and st["quartets_fp64"] > 0
    Jo, Ko = orc.jk(ob, D)
    dJ = np.abs(J.cpu().numpy() - Jo).max()
    dK = np.abs(K.cpu().numpy() - Ko).max()
    assert dJ < 1e-6 and dK < 1e-6, (dJ, dK)
    dE = abs(np.sum((2 * (J.cpu().numpy() - Jo) - (K.cpu().numpy() - Ko)) * D))
    assert dE < 1e-6


def test_deterministic_to_rounding(cq):
    mol, bas = CASES["O2H2"]()
    b = cq.Basis(mol, bas)
    D = _gpu(synth.density(b.nbf, 7, 3))
    J1, K1 = b.fock_build(D)
    J2, K2 = b.fock_build(D)
    assert (J1 - J2).abs().max().item() < 1e-13
    assert (K1 - K2).abs().max().item() < 1e-13


def test_single_shell_and_max_primitives(cq, orc):
    mol = synth.Molecule(np.array([8], np.int32), np.zeros((1, 3)))
    ex = 0.1 * 1.7 ** np.arange(16)
    bas = synth.Basis(np.array([0], np.int32), np.array([2], np.int32), np.array([16], np.int32),
                      ex, np.linspace(0.2, 1.0, 16))
    b = cq.Basis(mol, bas)
    D = synth.density(6, 2, 5)
    J, K = b.fock_build(_gpu(D))
    Jo, Ko = orc.jk(orc.OBasis(mol, bas), D)
    assert np.abs(J.cpu().numpy() - Jo).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL


def test_zero_density_and_screening(cq):
    mol, bas = CASES["O2H2"]()
    b = cq.Basis(mol, bas)
    import torch
    Z = torch.zeros((b.nbf, b.nbf), dtype=torch.float64, device="cuda")
    J, K, st = b.fock_build(Z, stats=True)
    assert J.abs().max().item() == 0.0 and K.abs().max().item() == 0.0
    assert st["quartets_fp64"] == 0


def _set_all(cq, b, variant):
    """Every class and precision (FP64, FP32, double-float) to `variant`
    where it exists, the cooperative kernel on the screened list (3, which
    every class has) elsewhere.  The axis-permutation kernel (2) exists for
    the classes of total angular momentum >= 4 with a d shell and for
    (pp|pp), in FP64 and double-float too except (dd|dp) and (dd|dd);
    double-float lane groups (0) for total angular momentum <= 3; the
    cooperative task mode (1) in FP64 and FP32."""
    n = 0
    for qc in range(21):
        for p in (0, 1, 2):
            try:
                b.set_variant(qc, p, variant)
                n += 1
            except cq.CQError:
                b.set_variant(qc, p, 3)
    assert n == {0: 42 + 8, 1: 42, 2: 13 + 11 + 11, 3: 63}[variant]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_class_in_each_kernel_variant(cq, orc, variant):
    """Lane-group (0), warp-cooperative (1: tasks, 3: screened list) and
    axis-permutation (2) kernels for all 21 classes: FP64, the FP32 and FP64
    halves of a mixed build, an almost all-FP32 build and an all
    double-float build against the oracle."""
    mol, bas = CASES["OCNH3"]()
    b = cq.Basis(mol, bas)
    _set_all(cq, b, variant)
    ob = orc.OBasis(mol, bas)
    P = synth.density(b.nbf, 9, 15, complex_=True)
    J, K = b.fock_build(_gpu(P))
    Jo, Ko = orc.jk(ob, P)
    assert np.abs(J.cpu().numpy() - Jo.real).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL
    Jm, Km, st = b.fock_build(_gpu(P), prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4, stats=True)
    assert st["quartets_fp32"] > 0
    assert np.abs(Jm.cpu().numpy() - Jo.real).max() < 1e-6
    assert np.abs(Km.cpu().numpy() - Ko).max() < 1e-6
    # every quartet with bound below 10 in FP32 (FP32 rounding of O(1) values)
    J3, K3, st3 = b.fock_build(_gpu(P), prec=cq.CQ_PREC_MIXED, mixed_tol=10.0, stats=True)
    assert st3["quartets_fp32"] > 10 * st3["quartets_fp64"]
    assert np.abs(J3.cpu().numpy() - Jo.real).max() < 2e-5
    assert np.abs(K3.cpu().numpy() - Ko).max() < 2e-5
    # every quartet in double-float (~48 bits): the FP64 tolerance holds
    Jd, Kd, std = b.fock_build(_gpu(P), prec=cq.CQ_PREC_MIXED, mixed_tol=0.0, fp64_tol=1e300, stats=True)
    assert std["quartets_df"] == st["quartets_fp64"] + st["quartets_fp32"]
    assert np.abs(Jd.cpu().numpy() - Jo.real).max() < TOL
    assert np.abs(Kd.cpu().numpy() - Ko).max() < TOL


@pytest.mark.parametrize("fp64_tol", [0.0, 1e-2])
def test_autotune_keeps_parity(cq, orc, fp64_tol):
    """The autotuner's choice (two tiers, or three with a double-float band
    up to 1e-2) keeps FP64 and mixed builds at their tolerances."""
    mol, bas = CASES["OCNH3"]()
    b = cq.Basis(mol, bas)
    P = synth.density(b.nbf, 9, 16, complex_=True)
    tab = b.autotune(_gpu(P), mixed_tol=1e-4, fp64_tol=fp64_tol, cache=False)
    assert len(tab["variant"]) == 21 and all(len(row) == 3 for row in tab["variant"])
    assert all(v in (0, 1, 2, 3) for row in tab["variant"] for v in row)
    assert tab["variant"][19][0] != 2 and tab["variant"][20][0] != 2   # FP32-only there
    assert all(row[2] != 1 for row in tab["variant"])                  # no double-float task mode
    if fp64_tol:
        assert any(ms > 0 for row in tab["best_ms"] for ms in row[2:])
    J, K = b.fock_build(_gpu(P))
    Jo, Ko = orc.jk(orc.OBasis(mol, bas), P)
    assert np.abs(J.cpu().numpy() - Jo.real).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL
    Jm, Km = b.fock_build(_gpu(P), prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4, fp64_tol=fp64_tol)
    assert np.abs(Jm.cpu().numpy() - Jo.real).max() < 1e-6
    assert np.abs(Km.cpu().numpy() - Ko).max() < 1e-6


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_bounded_list_passes(cq, orc, variant):
    """A basis whose candidate quartets exceed the list capacity builds in
    passes (one task per bra pair, the cooperative kernel reading the list):
    same J/K as the oracle, FP64 and mixed, every class in each variant."""
    mol, bas = CASES["OCNH3"]()
    old = cq.get_list_capacity()
    cq.set_list_capacity(3000)
    try:
        b = cq.Basis(mol, bas)
    finally:
        cq.set_list_capacity(old)
    _set_all(cq, b, variant)
    ob = orc.OBasis(mol, bas)
    P = synth.density(b.nbf, 9, 17, complex_=True)
    J, K, st = b.fock_build(_gpu(P), stats=True)
    Jo, Ko = orc.jk(ob, P)
    assert np.abs(J.cpu().numpy() - Jo.real).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL
    ref = cq.Basis(mol, bas)
    _, _, st_ref = ref.fock_build(_gpu(P), stats=True)
    assert st["quartets_fp64"] == st_ref["quartets_fp64"]
    Jm, Km, stm = b.fock_build(_gpu(P), prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4, stats=True)
    assert stm["quartets_fp32"] > 0
    assert np.abs(Jm.cpu().numpy() - Jo.real).max() < 1e-6
    assert np.abs(Km.cpu().numpy() - Ko).max() < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed", "three-tier"])
def test_builds_bitwise_reproducible(cq, prec):
    """J'/K' are accumulated as exact integers (order-independent), so two
    identical builds -- class kernels on concurrent streams, atomics in any
    order -- give bit-identical J and K, for every density kind."""
    import torch
    mol, bas = CASES["OCNH3"]()
    b = cq.Basis(mol, bas)
    n = b.nbf
    Pp = np.stack([synth.hermitian_component(n, 40 + i, scale=0.1) for i in range(4)])
    kw = {"mixed": {"prec": cq.CQ_PREC_MIXED, "mixed_tol": 1e-4},
          "three-tier": {"prec": cq.CQ_PREC_MIXED, "mixed_tol": 1e-4, "fp64_tol": 1e-2}}.get(prec, {})
    for P in (synth.density(n, 9, 18), synth.density(n, 9, 19, complex_=True), Pp):
        outs = [b.fock_build(_gpu(P), **kw) for _ in range(3)]
        for J, K in outs[1:]:
            assert torch.equal(J, outs[0][0])
            assert torch.equal(K, outs[0][1])
    # a second handle (other allocations, other stream timing) agrees too
    b2 = cq.Basis(mol, bas)
    J2, K2 = b2.fock_build(_gpu(P), **kw)
    assert torch.equal(J2, outs[0][0]) and torch.equal(K2, outs[0][1])


@pytest.mark.parametrize("name", ["OCNH3", "O1H2_deep"])
def test_double_float_tier(cq, orc, name):
    """The double-float tier: with every surviving quartet in double-float
    (pairs of FP32 values, ~48 bits) J and K still match the FP64 oracle at
    1e-10 for real, complex-Hermitian and Pauli densities; with three tiers
    (FP32 below 1e-4, double-float up to 1e-2, FP64 above) all three lists
    are used and the result matches at the mixed tolerance."""
    mol, bas = CASES[name]()
    b = cq.Basis(mol, bas)
    ob = orc.OBasis(mol, bas)
    n = b.nbf
    D = synth.density(n, max(1, n // 4), 11)
    J, K, st = b.fock_build(_gpu(D), prec=cq.CQ_PREC_MIXED, mixed_tol=0.0, fp64_tol=1e300, stats=True)
    assert st["quartets_df"] > 0 and st["quartets_fp64"] == 0 and st["quartets_fp32"] == 0
    Jo, Ko = orc.jk(ob, D)
    assert np.abs(J.cpu().numpy() - Jo).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL
    Pc = synth.density(n, max(1, n // 4), 12, complex_=True)
    Jc, Kc = b.fock_build(_gpu(Pc), prec=cq.CQ_PREC_MIXED, mixed_tol=0.0, fp64_tol=1e300)
    Joc, Koc = orc.jk(ob, Pc)
    assert np.abs(Jc.cpu().numpy() - Joc.real).max() < TOL
    assert np.abs(Kc.cpu().numpy() - Koc).max() < TOL
    from oracle import drivers
    Pp = np.ascontiguousarray(drivers.pauli_split(synth.spinor_density(n, 7, 13)))
    Jp, Kp = b.fock_build(_gpu(Pp), prec=cq.CQ_PREC_MIXED, mixed_tol=0.0, fp64_tol=1e300)
    Jop, _ = orc.jk(ob, Pp[0])
    assert np.abs(Jp.cpu().numpy() - Jop.real).max() < TOL
    for I in range(4):
        _, KoI = orc.jk(ob, Pp[I])
        assert np.abs(Kp.cpu().numpy()[I] - KoI).max() < TOL, I
    J3, K3, st3 = b.fock_build(_gpu(D), prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4, fp64_tol=1e-2, stats=True)
    assert st3["quartets_df"] > 0 and st3["quartets_fp64"] > 0 and st3["quartets_fp32"] > 0
    _, _, st2 = b.fock_build(_gpu(D), prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4, stats=True)
    assert st3["quartets_df"] + st3["quartets_fp64"] == st2["quartets_fp64"]
    assert st3["quartets_fp32"] == st2["quartets_fp32"]
    assert np.abs(J3.cpu().numpy() - Jo).max() < 1e-6
    assert np.abs(K3.cpu().numpy() - Ko).max() < 1e-6


@pytest.mark.parametrize("name", ["OCNH3", "O1H2_deep"])
def test_non_hermitian_density(cq, orc, name):
    """J and K of a real density of no symmetry (the transition densities of
    the direct ph-RPA products): FP64 against the oracle's contraction of
    the full definition at the FP64 tolerance, three tiers at the mixed one;
    J is that of the symmetric part alone."""
    mol, bas = CASES[name]()
    b = cq.Basis(mol, bas)
    g = np.random.default_rng(21)
    D = 0.1 * g.standard_normal((b.nbf, b.nbf))
    Jo, Ko = orc.jk(orc.OBasis(mol, bas), D)
    J, K = b.fock_build(_gpu(D), kind=cq.CQ_DENS_REAL_GENERAL)
    assert np.abs(J.cpu().numpy() - Jo).max() < TOL
    assert np.abs(K.cpu().numpy() - Ko).max() < TOL
    assert np.abs(Ko - Ko.T).max() > 1e-3                     # K of a non-symmetric D is not symmetric
    J3, K3, st = b.fock_build(_gpu(D), kind=cq.CQ_DENS_REAL_GENERAL, prec=cq.CQ_PREC_MIXED, mixed_tol=1e-4,
                              fp64_tol=1e-2, stats=True)
    assert st["quartets_fp32"] > 0 and st["quartets_df"] > 0
    assert np.abs(J3.cpu().numpy() - Jo).max() < 1e-6
    assert np.abs(K3.cpu().numpy() - Ko).max() < 1e-6
    Js, _ = b.fock_build(_gpu(0.5 * (D + D.T)))
    assert np.abs(Js.cpu().numpy() - J.cpu().numpy()).max() < 1e-12
