"""The cooperative kernel's instruction tables, executed on the CPU.

The generator writes the vertical and horizontal recurrences of each class
as groups of 32-wide instructions over value slots, scheduled into phases
between warp syncs and with slots reused once their last reader has run.
Here a small interpreter runs those tables the way the kernel does (group
by group, every node of a group reading the slots before the group writes)
with random coefficients, and compares every target with the same
recurrence evaluated directly node by node.  A scheduling or slot-reuse
error changes a target; no GPU and no oracle are involved.  CPU only."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1905_01381_gb300", "csrc")
sys.path.insert(0, CSRC)

import gen_coop  # noqa: E402
import gen_eri  # noqa: E402

NCOEF = gen_coop.NCOEF


def _unpack(d):
    w0, w1, w2, w3 = d
    return ((w0 & 0xffff, w0 >> 16, w1 & 0xffff, w1 >> 16, w2 & 0xffff), w2 >> 16,
            [(w3 >> (6 * k)) & 63 for k in range(5)])


def _run_vrr(prog, cf, base):
    V = np.zeros(prog["nslots"] + 1)
    V[:len(base)] = base
    for shape, n, first, _ in prog["groups"]:
        outs = []
        for d in prog["descs"][first:first + n]:
            x, out, c = _unpack(d)
            v = cf[c[0]] * V[x[0]] + cf[c[1]] * V[x[1]]
            if shape in (gen_coop.SHAPE_ABC, gen_coop.SHAPE_ALL):
                v += cf[c[2]] * (V[x[2]] - cf[c[3]] * V[x[3]])
            if shape >= gen_coop.SHAPE_ABE:
                v += cf[c[4]] * V[x[4]]
            outs.append((out, v))
        for out, v in outs:           # a group writes after all its nodes read
            V[out] = v
    return np.array([V[t] for t in prog["targets"]])


def _direct_vrr(cls, cf, base):
    P = gen_coop.VRRPlan(*cls)
    val = {}
    for k, nd in P.nodes.items():
        if "base" in nd:
            val[k] = base[nd["base"]]
    for k in P.order:
        nd = P.nodes[k]
        o, c = nd["ops"], nd["cs"]
        v = cf[c[0]] * val[o[0]] + cf[c[1]] * val[o[1]]
        if o[2] is not None:
            v += cf[c[2]] * (val[o[2]] - cf[c[3]] * val[o[3]])
        if o[4] is not None:
            v += cf[c[4]] * val[o[4]]
        val[k] = v
    return np.array([val[t] for t in P.targets])


@pytest.mark.parametrize("cls", gen_eri.classes())
def test_vrr_tables_match_direct_recurrence(cls):
    g = np.random.default_rng(sum(cls) + 7)
    cf = g.uniform(-1.0, 1.0, NCOEF)
    prog = gen_coop.vrr_program(*cls)
    base = g.uniform(-1.0, 1.0, prog["L"] + 1)
    got = _run_vrr(prog, cf, base)
    ref = _direct_vrr(cls, cf, base)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("cls", [c for c in gen_eri.classes() if sum(c) >= 4])
def test_schedule_respects_dependencies_and_fills_lanes(cls):
    P = gen_coop.VRRPlan(*cls)
    maxlev = max(P.nodes[k]["level"] for k in P.order)
    phases = gen_coop.schedule(P, maxlev)
    where = {}
    for ph, nodes in enumerate(phases):
        for k in nodes:
            assert k not in where
            where[k] = ph
    assert set(where) == set(P.order)
    for k in P.order:
        for d in P.nodes[k]["deps"]:
            if d in where:
                assert where[d] < where[k]
    # groups of one shape per phase: at most one partial group per shape
    for nodes in phases:
        by = {}
        for k in nodes:
            by[P.nodes[k]["shape"]] = by.get(P.nodes[k]["shape"], 0) + 1
        assert all(n > 0 for n in by.values())


def _run_hrr(prog, acc, ab, cd):
    hc = np.concatenate([ab, cd])
    V = np.zeros(prog["nslots"] + 1)
    nacc = len(acc)
    V[prog["N"]:prog["N"] + nacc] = acc
    for kind, n, first, _ in prog["groups"]:
        outs = []
        for d in prog["descs"][first:first + n]:
            x, out, c = _unpack(d)
            v = V[x[1]] * hc[c[0]] + V[x[0]] if kind == 0 else V[x[0]]
            outs.append((out, v))
        for out, v in outs:
            V[out] = v
    return V[:prog["N"]].copy()


def _direct_hrr(cls, E, F, acc, ab, cd):
    la, lb, lc, ld = cls
    A, B, C, D = (gen_eri.comps(l) for l in cls)
    val = {(e, f): acc[i * len(F) + j] for i, e in enumerate(E) for j, f in enumerate(F)}

    def bra(a, b, f):   # (a b| f 0) by (a b+1_i| = (a+1_i b| + AB_i (a b|
        if sum(b) == 0:
            return val[(a, f)]
        i = gen_eri.pick_axis(b)
        b1 = gen_eri.sub(b, i)
        return bra(gen_eri.add(a, i), b1, f) + ab[i] * bra(a, b1, f)

    def ket(a, b, c, d):
        if sum(d) == 0:
            return bra(a, b, c)
        i = gen_eri.pick_axis(d)
        d1 = gen_eri.sub(d, i)
        return ket(a, b, gen_eri.add(c, i), d1) + cd[i] * ket(a, b, c, d1)

    return np.array([ket(a, b, c, d) for a in A for b in B for c in C for d in D])


@pytest.mark.parametrize("cls", gen_eri.classes())
def test_hrr_tables_match_direct_recurrence(cls):
    g = np.random.default_rng(sum(cls) + 11)
    v = gen_coop.vrr_program(*cls)
    h = gen_coop.hrr_program(*cls, v["E"], v["F"])
    acc = g.uniform(-1.0, 1.0, v["nacc"])
    ab, cd = g.uniform(-1.0, 1.0, 3), g.uniform(-1.0, 1.0, 3)
    got = _run_hrr(h, acc, ab, cd)
    ref = _direct_hrr(cls, v["E"], v["F"], acc, ab, cd)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


# ------------------------------------------------ axis-permutation split
import gen_sym  # noqa: E402


@pytest.mark.parametrize("cls", gen_sym.classes_for_sym())
def test_axis_permutation_split_covers_every_target(cls):
    """The G lanes of the split kernel run the recurrence for the
    representatives T0 on permuted inputs; scattered by the generated
    tables, their outputs must be every target of the class, each written
    exactly once, equal to the recurrence evaluated in the original frame."""
    import random
    rel = gen_sym.check_plan(*cls, random.Random(hash(cls) & 0xffff))
    assert rel < 1e-12, rel
    T0, dst, E, F = gen_sym.plan(*cls)
    writes = [d for row in dst for d in row if d != 0xFFFF]
    assert sorted(writes) == list(range(len(E) * len(F)))
    assert len(dst) == cls[4] and all(len(r) == len(T0) for r in dst)


def test_axis_permutation_split_is_cheap():
    """Per lane the split recurrence keeps about 1/G of the accumulators (a
    little more where orbits are smaller than the group) at
    a total cost (G lanes) of at most 1.25x (C3) or 1.6x (S3) the full one."""
    for cls in gen_sym.classes_for_sym():
        la, lb, lc, ld, G = cls
        g = gen_eri.ClassGen(la, lb, lc, ld)
        g.gen("R")
        full = g.flops
        _, st = gen_sym.emit_class(*cls)
        assert st["n0"] <= 1.2 * st["nacc"] / G + 12      # orbits with stabilisers are smaller
        assert G * (st["vrr_flops_lane"] - st["n0"]) <= (1.25 if G == 3 else 1.6) * full, (cls, st)
