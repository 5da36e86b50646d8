"""Pins of the oracle against facts fixed by mathematics, independent of the
oracle's own code: closed forms, high-precision quadrature, derivative
identities of Gaussians, symmetries and invariances.  CPU only."""
import itertools

import numpy as np
import pytest

import synth

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp

CART = {0: [(0, 0, 0)],
        1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
        2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]}


def dfact(n):
    return 1 if n <= 0 else n * dfact(n - 2)


def prim_norm(a, l):
    return ((2 * a / mpmath.pi) ** mpmath.mpf(0.75) * (4 * a) ** (mpmath.mpf(sum(l)) / 2)
            / mpmath.sqrt(dfact(2 * l[0] - 1) * dfact(2 * l[1] - 1) * dfact(2 * l[2] - 1)))


# ------------------------------------------------------------ Boys function
def boys_mp(m, T):
    T = mpmath.mpf(T)
    return mpmath.quad(lambda t: t ** (2 * m) * mpmath.exp(-T * t * t), [0, 1])


def test_boys_against_quadrature(oracle_lib):
    mp.dps = 30
    worst = 0.0
    for T in [0.0, 1e-12, 1e-6, 0.01, 0.3, 1.0, 2.5, 7.7, 15.0, 29.9, 30.0, 30.1,
              45.0, 80.0, 200.0]:
        F = oracle_lib.boys(8, T)
        for m in range(9):
            ref = boys_mp(m, T)
            worst = max(worst, float(abs((F[m] - ref) / ref)))
    assert worst < 1e-14, worst


def test_boys_special_values(oracle_lib):
    F = oracle_lib.boys(8, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(9)], rtol=0, atol=1e-16)
    for T in [0.5, 3.0, 31.0]:
        F0 = oracle_lib.boys(0, T)[0]
        assert abs(F0 - 0.5 * np.sqrt(np.pi / T) * float(mpmath.erf(np.sqrt(T)))) < 1e-15


# ------------------------------------------------ ERIs by Gaussian-transform quadrature
# 1/r = (2/sqrt(pi)) int_0^inf exp(-u^2 r^2) du makes every ERI a 1-D integral
# over u of a product of three separable 2-D Gaussian integrals, each of which
# is a polynomial times a Gaussian and is integrated exactly by a 2-D
# Gauss-Hermite rule after completing the square.
from scipy import integrate  # noqa: E402

_GH_Y, _GH_W = np.polynomial.hermite.hermgauss(10)
_Y1, _Y2 = np.meshgrid(_GH_Y, _GH_Y, indexing="ij")
_W2 = np.outer(_GH_W, _GH_W)


def _gt_factor(u, l, e, c):
    a, b, cc, d = e
    A, B, C, D = c
    u2 = u * u
    M = np.array([[a + b + u2, -u2], [-u2, cc + d + u2]])
    v = np.array([a * A + b * B, cc * C + d * D])
    m = np.linalg.solve(M, v)
    R = np.linalg.cholesky(M).T
    Ri = np.linalg.inv(R)
    x1 = m[0] + Ri[0, 0] * _Y1 + Ri[0, 1] * _Y2
    x2 = m[1] + Ri[1, 0] * _Y1 + Ri[1, 1] * _Y2
    poly = (x1 - A) ** l[0] * (x1 - B) ** l[1] * (x2 - C) ** l[2] * (x2 - D) ** l[3]
    return (np.sum(_W2 * poly) / np.linalg.det(R)
            * np.exp(m @ v - (a * A * A + b * B * B + cc * C * C + d * D * D)))


def eri_gt(ls, exps, ctrs):
    """(ab|cd) over normalised single primitives with Cartesian powers ls."""
    def integrand(t):
        u = t / (1 - t)
        return np.prod([_gt_factor(u, [ls[k][x] for k in range(4)], exps,
                                   [ctrs[k][x] for k in range(4)]) for x in range(3)]) / (1 - t) ** 2
    val, _ = integrate.quad(integrand, 0, 1, epsabs=1e-15, epsrel=1e-13, limit=200)
    nrm = np.prod([float(prim_norm(mpmath.mpf(exps[k]), ls[k])) for k in range(4)])
    return 2 / np.sqrt(np.pi) * val * nrm


def _single_prim_basis(Ls, exps, ctrs):
    mol = synth.Molecule(np.arange(1, 5, dtype=np.int32), np.array(ctrs, float))
    bas = synth.Basis(np.arange(4, dtype=np.int32), np.array(Ls, np.int32),
                      np.ones(4, np.int32), np.array(exps, float), np.ones(4))
    return mol, bas


CLASSES = [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (2, 0, 0, 0),
           (2, 1, 0, 0), (1, 1, 1, 1), (2, 0, 1, 0), (2, 2, 0, 0), (2, 1, 1, 0),
           (2, 0, 2, 0), (2, 1, 1, 1), (2, 2, 1, 0), (2, 1, 2, 0), (2, 2, 1, 1),
           (2, 1, 2, 1), (2, 2, 2, 0), (2, 2, 2, 1), (2, 2, 2, 2), (0, 2, 1, 2),
           (1, 2, 0, 1)]


@pytest.mark.parametrize("cls", CLASSES)
def test_eri_against_gaussian_transform(oracle_lib, cls):
    g = synth.rng(sum((k + 1) * 10 ** k * l for k, l in enumerate(cls)))
    exps = list(g.uniform(0.3, 2.0, size=4))
    ctrs = [list(g.uniform(-1.0, 1.0, size=3)) for _ in range(4)]
    mol, bas = _single_prim_basis(cls, exps, ctrs)
    ob = oracle_lib.OBasis(mol, bas)
    blk = oracle_lib.eri_shell(ob, 0, 1, 2, 3)
    comps = list(itertools.product(*[range(len(CART[l])) for l in cls]))
    pick = comps if len(comps) <= 12 else [comps[i] for i in g.choice(len(comps), 12, replace=False)]
    for idx in pick:
        ls = [CART[cls[k]][idx[k]] for k in range(4)]
        ref = eri_gt(ls, exps, ctrs)
        assert abs(blk[idx] - ref) <= 2e-13 * max(1.0, abs(ref)), (cls, idx, blk[idx], ref)


def ssss(a, b, c, d, A, B, C, D):
    """Closed-form (ss|ss) over unnormalised s primitives."""
    p, q = a + b, c + d
    AB2 = sum((A[i] - B[i]) ** 2 for i in range(3))
    CD2 = sum((C[i] - D[i]) ** 2 for i in range(3))
    P = [(a * A[i] + b * B[i]) / p for i in range(3)]
    Q = [(c * C[i] + d * D[i]) / q for i in range(3)]
    T = p * q / (p + q) * sum((P[i] - Q[i]) ** 2 for i in range(3))
    F0 = mpmath.mpf(1) if T == 0 else mpmath.sqrt(mpmath.pi / T) / 2 * mpmath.erf(mpmath.sqrt(T))
    return (2 * mpmath.pi ** mpmath.mpf(2.5) / (p * q * mpmath.sqrt(p + q))
            * mpmath.exp(-a * b / p * AB2) * mpmath.exp(-c * d / q * CD2) * F0)


def test_ssss_closed_form(oracle_lib):
    g = synth.rng(21)
    for rep in range(5):
        exps = list(g.uniform(0.1, 3.0, size=4))
        ctrs = [list(g.uniform(-1.5, 1.5, size=3)) for _ in range(4)]
        if rep == 0:
            ctrs = [ctrs[0]] * 4          # T = 0 branch
        mol, bas = _single_prim_basis((0, 0, 0, 0), exps, ctrs)
        ob = oracle_lib.OBasis(mol, bas)
        mp.dps = 30
        ref = ssss(*[mpmath.mpf(e) for e in exps], *ctrs)
        ref *= mpmath.fprod([prim_norm(mpmath.mpf(e), (0, 0, 0)) for e in exps])
        assert abs(oracle_lib.eri_shell(ob, 0, 1, 2, 3)[0, 0, 0, 0] - float(ref)) < 1e-15


def _axis_ops(l, alpha):
    """x_A^l G = sum coef * d^k/dA^k G for l <= 2 (Gaussian derivative identity)."""
    if l == 0:
        return [(0, mpmath.mpf(1))]
    if l == 1:
        return [(1, 1 / (2 * alpha))]
    return [(2, 1 / (4 * alpha ** 2)), (0, 1 / (2 * alpha))]


@pytest.mark.parametrize("cls", [(1, 0, 0, 0), (0, 1, 1, 0), (2, 0, 0, 0)])
def test_eri_low_order_by_center_derivatives(oracle_lib, cls):
    """Second, independent pin for low classes: a Cartesian factor on centre A
    is a derivative of the s Gaussian with respect to A."""
    mp.dps = 30
    g = synth.rng(99 + sum(cls))
    exps = list(g.uniform(0.3, 2.0, size=4))
    ctrs = [list(g.uniform(-1.0, 1.0, size=3)) for _ in range(4)]
    mol, bas = _single_prim_basis(cls, exps, ctrs)
    ob = oracle_lib.OBasis(mol, bas)
    blk = oracle_lib.eri_shell(ob, 0, 1, 2, 3)
    ex = [mpmath.mpf(e) for e in exps]
    x0 = [mpmath.mpf(v) for c in ctrs for v in c]

    def f(*x):
        return ssss(*ex, x[0:3], x[3:6], x[6:9], x[9:12])

    for idx in itertools.product(*[range(len(CART[l])) for l in cls]):
        ls = [CART[cls[k]][idx[k]] for k in range(4)]
        terms = [[]]
        for k in range(4):
            for ax in range(3):
                terms = [t + [op] for op in _axis_ops(ls[k][ax], ex[k]) for t in terms]
        tot = 0
        for t in terms:
            orders = tuple(o for o, _ in t)
            coef = mpmath.fprod([c for _, c in t])
            tot += coef * (mpmath.diff(f, x0, orders) if any(orders) else f(*x0))
        ref = float(tot * mpmath.fprod([prim_norm(ex[k], ls[k]) for k in range(4)]))
        assert abs(blk[idx] - ref) < 1e-12, (idx, blk[idx], ref)


# ------------------------------------------------ one-electron integrals
def _1d_overlap_mp(i, j, a, b, A, B):
    return mpmath.quad(lambda x: (x - A) ** i * (x - B) ** j *
                       mpmath.exp(-a * (x - A) ** 2 - b * (x - B) ** 2), [-mpmath.inf, mpmath.inf])


def test_overlap_kinetic_dipole_quadrature(oracle_lib):
    mp.dps = 20
    g = synth.rng(7)
    Ls = [2, 1, 2, 0]
    exps = list(g.uniform(0.4, 1.5, size=4))
    ctrs = [list(g.uniform(-1, 1, size=3)) for _ in range(4)]
    mol, bas = _single_prim_basis(Ls, exps, ctrs)
    ob = oracle_lib.OBasis(mol, bas)
    S = oracle_lib.overlap(ob)
    T = oracle_lib.kinetic(ob)
    O = (0.1, -0.2, 0.3)
    M = oracle_lib.dipole(ob, origin=O)
    bfo = ob.bfo
    for sa, sb in [(0, 2), (1, 3)]:
        for ia, la in enumerate(CART[Ls[sa]]):
            for ib, lb in enumerate(CART[Ls[sb]]):
                a, b = exps[sa], exps[sb]
                A, B = ctrs[sa], ctrs[sb]
                s1 = [_1d_overlap_mp(la[x], lb[x], a, b, A[x], B[x]) for x in range(3)]
                d2 = []
                for x in range(3):
                    j = lb[x]
                    f = lambda y, j=j, x=x: (
                        (j * (j - 1) * (y - B[x]) ** (j - 2) if j >= 2 else 0)
                        - 2 * b * (2 * j + 1) * (y - B[x]) ** j
                        + 4 * b * b * (y - B[x]) ** (j + 2))
                    d2.append(mpmath.quad(lambda y: (y - A[x]) ** la[x] * f(y) *
                                          mpmath.exp(-a * (y - A[x]) ** 2 - b * (y - B[x]) ** 2),
                                          [-mpmath.inf, mpmath.inf]))
                nrm = prim_norm(mpmath.mpf(a), la) * prim_norm(mpmath.mpf(b), lb)
                sref = nrm * s1[0] * s1[1] * s1[2]
                tref = -nrm / 2 * (d2[0] * s1[1] * s1[2] + s1[0] * d2[1] * s1[2] + s1[0] * s1[1] * d2[2])
                i, j = bfo[sa] + ia, bfo[sb] + ib
                assert abs(S[i, j] - float(sref)) < 1e-13
                assert abs(T[i, j] - float(tref)) < 1e-12
                for x in range(3):
                    mx = mpmath.quad(lambda y: (y - A[x]) ** la[x] * (y - B[x]) ** lb[x] * (y - O[x]) *
                                     mpmath.exp(-a * (y - A[x]) ** 2 - b * (y - B[x]) ** 2),
                                     [-mpmath.inf, mpmath.inf])
                    mref = nrm * mx * s1[(x + 1) % 3] * s1[(x + 2) % 3]
                    assert abs(M[x, i, j] - float(mref)) < 1e-13


def _nuc_gt(la, lb, a, b, A, B, C):
    """<a| 1/|r-C| |b> by the same Gaussian transform, 1-D Gauss-Hermite factors."""
    y, w = np.polynomial.hermite.hermgauss(10)

    def fac(u, x):
        s = a + b + u * u
        m = (a * A[x] + b * B[x] + u * u * C[x]) / s
        xs = m + y / np.sqrt(s)
        const = a * A[x] ** 2 + b * B[x] ** 2 + u * u * C[x] ** 2 - s * m * m
        return np.sum(w * (xs - A[x]) ** la[x] * (xs - B[x]) ** lb[x]) / np.sqrt(s) * np.exp(-const)

    val, _ = integrate.quad(lambda t: np.prod([fac(t / (1 - t), x) for x in range(3)]) / (1 - t) ** 2,
                            0, 1, epsabs=1e-15, epsrel=1e-13, limit=200)
    return 2 / np.sqrt(np.pi) * val


def test_nuclear_attraction_quadrature(oracle_lib):
    g = synth.rng(11)
    ex = list(g.uniform(0.4, 1.5, size=2))
    A = list(g.uniform(-1, 1, 3)); B = list(g.uniform(-1, 1, 3)); C = list(g.uniform(-1, 1, 3))
    mol = synth.Molecule(np.array([0, 0, 3], np.int32), np.array([A, B, C]))
    bas = synth.Basis(np.array([0, 1], np.int32), np.array([2, 1], np.int32),
                      np.ones(2, np.int32), np.array(ex), np.ones(2))
    ob = oracle_lib.OBasis(mol, bas)
    V = oracle_lib.nuclear(ob)
    for ia, la in enumerate(CART[2]):
        for ib, lb in enumerate(CART[1]):
            nrm = float(prim_norm(mpmath.mpf(ex[0]), la) * prim_norm(mpmath.mpf(ex[1]), lb))
            ref = -3.0 * nrm * _nuc_gt(la, lb, ex[0], ex[1], A, B, C)
            assert abs(V[ia, 6 + ib] - ref) < 1e-12, (la, lb, V[ia, 6 + ib], ref)


# ------------------------------------------------ contraction, symmetry, J/K
def test_contracted_eri_is_sum_of_primitives(oracle_lib):
    """A contracted, normalised shell quartet equals the coefficient-weighted
    sum of raw primitive quartets, each Cartesian component scaled to unit
    self-overlap by the closed-form same-centre Gaussian overlap."""
    mol, bas = synth.small_cluster(2, 5, max_depth=3)
    ob = oracle_lib.OBasis(mol, bas)
    S = oracle_lib.overlap(ob)
    assert np.allclose(np.diag(S), 1.0, atol=1e-14)
    shells = [0, 4, 1, 5] if ob.nsh > 5 else [0, 1, 2, 3]

    def NL(a, L):
        return (2 * a / np.pi) ** 0.75 * (4 * a) ** (L / 2)

    def same_centre_overlap(a, b, l):
        p = a + b
        return np.prod([dfact(2 * k - 1) / (2 * p) ** k * np.sqrt(np.pi / p) for k in l])

    prim = {}
    comp_scale = {}
    for s in shells:
        o, L = ob.poff[s], bas.shell_L[s]
        prim[s] = [(bas.exps[o + k], bas.coefs[o + k]) for k in range(bas.shell_nprim[s])]
        comp_scale[s] = []
        for l in CART[L]:
            tot = sum(ci * cj * NL(ai, L) * NL(aj, L) * same_centre_overlap(ai, aj, l)
                      for ai, ci in prim[s] for aj, cj in prim[s])
            comp_scale[s].append(tot ** -0.5)
    a, b, c, d = shells
    ref = oracle_lib.eri_shell(ob, a, b, c, d)
    acc = np.zeros_like(ref)
    for ea, ca in prim[a]:
        for eb, cb in prim[b]:
            for ec, cc in prim[c]:
                for ed, cd in prim[d]:
                    Ls = [bas.shell_L[s] for s in shells]
                    m2, b2 = _single_prim_basis(Ls, [ea, eb, ec, ed],
                                                [list(mol.xyz[bas.shell_atom[s]]) for s in shells])
                    blk = oracle_lib.eri_shell(oracle_lib.OBasis(m2, b2), 0, 1, 2, 3)
                    raw = blk / np.einsum('a,b,c,d->abcd', *[
                        np.array([float(prim_norm(mpmath.mpf(e), l)) for l in CART[L]])
                        for e, L in zip([ea, eb, ec, ed], Ls)])
                    w = ca * cb * cc * cd * NL(ea, Ls[0]) * NL(eb, Ls[1]) * NL(ec, Ls[2]) * NL(ed, Ls[3])
                    acc += w * raw
    acc *= np.einsum('a,b,c,d->abcd', *[np.array(comp_scale[s]) for s in shells])
    assert np.allclose(acc, ref, rtol=1e-12, atol=1e-15)


@pytest.fixture(scope="module")
def tiny(oracle_lib):
    mol, bas = synth.small_cluster(2, 3, max_depth=2)
    ob = oracle_lib.OBasis(mol, bas)
    return ob, oracle_lib.eri_full(ob)


def test_eri_eightfold_symmetry_and_psd(tiny):
    ob, G = tiny
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(G - G.transpose(perm)).max() < 1e-14
    n = ob.nbf
    w = np.linalg.eigvalsh(G.reshape(n * n, n * n))
    assert w.min() > -1e-12


def test_schwarz_inequality(oracle_lib, tiny):
    ob, G = tiny
    n = ob.nbf
    diag = np.einsum('ijij->ij', G)
    assert np.all(np.abs(G) <= np.sqrt(np.einsum('ij,kl->ijkl', diag, diag)) + 1e-14)
    Q = oracle_lib.schwarz(ob)
    for a in range(ob.nsh):
        for b in range(ob.nsh):
            blk = diag[ob.bfo[a]:ob.bfo[a + 1], ob.bfo[b]:ob.bfo[b + 1]]
            assert abs(Q[a, b] - np.sqrt(np.abs(blk).max())) < 1e-14


def test_jk_against_full_tensor(oracle_lib, tiny):
    ob, G = tiny
    n = ob.nbf
    g = synth.rng(4)
    D = g.standard_normal((n, n))            # general, non-symmetric
    J, K = oracle_lib.jk(ob, D)
    assert np.abs(J - np.einsum('ijkl,kl->ij', G, D)).max() < 1e-13
    assert np.abs(K - np.einsum('iklj,kl->ij', G, D)).max() < 1e-13


def test_jk_hermitian_and_positive(oracle_lib):
    mol, bas = synth.small_cluster(3, 9, max_depth=2)
    ob = oracle_lib.OBasis(mol, bas)
    P = synth.density(ob.nbf, 4, 3, complex_=True)
    J, K = oracle_lib.jk(ob, P)
    assert np.abs(J - J.conj().T).max() < 1e-13
    assert np.abs(K - K.conj().T).max() < 1e-13
    assert np.abs(J.imag).max() < 1e-13       # J of the antisymmetric Im part vanishes
    eJ = np.sum(J * P.T)
    eK = np.sum(K * P.T)
    assert abs(eJ.imag) < 1e-12 and abs(eK.imag) < 1e-12
    assert eJ.real > 0 and eK.real > 0


def test_jk_elements_match_full(oracle_lib):
    mol, bas = synth.small_cluster(3, 13, max_depth=2)
    ob = oracle_lib.OBasis(mol, bas)
    D = synth.density(ob.nbf, 5, 2)
    J, K = oracle_lib.jk(ob, D)
    mu = np.array([0, 3, ob.nbf - 1, 7]); nu = np.array([0, 5, 2, ob.nbf - 1])
    Jo, Ko = oracle_lib.jk_elements(ob, [D], mu, nu)
    assert np.abs(Jo[0] - J[mu, nu]).max() < 1e-13
    assert np.abs(Ko[0] - K[mu, nu]).max() < 1e-13


def test_jk_sample_partitions_the_build(oracle_lib):
    """The timing sample of the CPU baseline: the bra-pair residue classes
    p % stride partition the unique shell quartets, so the samples add up to
    the full J and K and their quartet counts to npair (npair + 1) / 2."""
    mol, bas = synth.small_cluster(3, 21, max_depth=2)
    ob = oracle_lib.OBasis(mol, bas)
    D = synth.density(ob.nbf, 4, 6)
    J, K = oracle_lib.jk_real(ob, [D])
    stride = 3
    Js, Ks, nq = 0.0, 0.0, 0
    for off in range(stride):
        j, k, n = oracle_lib.jk_sample(ob, [D], stride, off)
        Js, Ks, nq = Js + j, Ks + k, nq + n
    npair = ob.nsh * (ob.nsh + 1) // 2
    assert nq == npair * (npair + 1) // 2
    assert np.abs(Js - J).max() < 1e-12 and np.abs(Ks - K).max() < 1e-12
