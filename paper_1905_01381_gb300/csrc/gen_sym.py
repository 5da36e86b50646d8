"""Generator of the axis-permutation split of the vertical recurrence.

A Cartesian Gaussian integral is unchanged when the coordinate axes are
relabelled together with every Cartesian exponent: the integral [e0|f0]
computed from inputs whose vector components are permuted (PA, QC, W-P,
W-Q with components (v[p0], v[p1], v[p2])) is the integral of the
permuted target (e', f') with e'[p[i]] = e[i], f'[p[i]] = f[i].  So the
targets E x F of a class (la lb|lc ld) split into orbits under a group of
axis permutations (the cyclic group C3 or the full S3), and G lanes -- one
per group element -- that run the SAME straight-line recurrence for one
representative per orbit (the set T0) on permuted inputs together produce
every target.  Per lane the accumulators shrink to |T0| (about a third or a
sixth of the targets) for a recurrence of 1.1-1.2x (C3) or about 1.5x (S3)
the work of the full one, which keeps the FP32 kernels of the high classes
in registers.

The recurrences are those of gen_eri.py (Obara-Saika, same axis choice);
representatives are chosen greedily, highest orbits first, to minimise the
shared closure.  For every lane k and representative i the tables give the
target index (ie * |F| + jf) of its permuted image, or 0xFFFF where another
lane (the first one producing that target) writes it.

Usage: imported by buildlib.py.
"""
from __future__ import annotations

import itertools

from gen_eri import ClassGen, comps

C3 = [(0, 1, 2), (1, 2, 0), (2, 0, 1)]
S3 = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]
GROUPS = {3: C3, 6: S3}


def permute(p, t):
    """Exponents in the original frame of exponents t in the frame whose
    axis i is the original axis p[i]."""
    out = [0, 0, 0]
    for i in range(3):
        out[p[i]] = t[i]
    return tuple(out)


def plan(la, lb, lc, ld, G):
    """(T0, dst, E, F): representatives and per-lane destination tables."""
    perms = GROUPS[G]
    E = [e for l in range(la, la + lb + 1) for e in comps(l)]
    F = [f for l in range(lc, lc + ld + 1) for f in comps(l)]
    index = {(e, f): ie * len(F) + jf for ie, e in enumerate(E) for jf, f in enumerate(F)}
    seen = set()
    orbits = []
    for e in E:
        for f in F:
            if (e, f) in seen:
                continue
            orb = {(permute(p, e), permute(p, f)) for p in perms}
            seen |= orb
            orbits.append(sorted(orb))
    g = ClassGen(la, lb, lc, ld)
    T0 = []
    for orb in sorted(orbits, key=lambda o: -(sum(o[0][0]) + sum(o[0][1]))):
        best = None
        for t in orb:
            trial = ClassGen(la, lb, lc, ld)
            trial.names = dict(g.names)
            trial.n = g.n
            trial.node(t[0], t[1], 0)
            if best is None or len(trial.lines) < best[0]:
                best = (len(trial.lines), t)
        T0.append(best[1])
        g.node(best[1][0], best[1][1], 0)
    written = set()
    dst = []
    for p in perms:
        row = []
        for (e, f) in T0:
            tgt = index[(permute(p, e), permute(p, f))]
            if tgt in written:
                row.append(0xFFFF)
            else:
                written.add(tgt)
                row.append(tgt)
        dst.append(row)
    assert written == set(range(len(E) * len(F))), "orbits do not cover the targets"
    return T0, dst, E, F


def emit_class(la, lb, lc, ld, G):
    """Text of the SymClass<la, lb, lc, ld, G> specialisation and its
    per-class statistics."""
    T0, dst, E, F = plan(la, lb, lc, ld, G)
    g = ClassGen(la, lb, lc, ld)
    names = [g.node(e, f, 0) for (e, f) in T0]
    L = la + lb + lc + ld
    used = " ".join(g.lines)
    consts = []
    for k in range(1, 5):
        for nm in ("oo2z", "oo2e", "oo2ze"):
            if f"{nm}_{k}" in used:
                consts.append(f"    const R {nm}_{k} = {k}.0 * {nm};" if k > 1 else f"    const R {nm}_1 = {nm};")
    perms = GROUPS[G]
    code = 0
    for k, p in enumerate(perms):
        for i in range(3):
            code |= p[i] << (2 * (3 * k + i))
    s = [f"// class ({'spd'[la]}{'spd'[lb]}|{'spd'[lc]}{'spd'[ld]}), {G}-lane axis-permutation split "
         "-- generated by gen_sym.py, do not edit",
         f"template <> struct SymClass<{la}, {lb}, {lc}, {ld}, {G}> {{",
         f"  static constexpr int N0 = {len(T0)};",
         f"  static constexpr unsigned long long PERM = {code}ull;   // 2 bits per (lane, axis)",
         "  template <typename R>",
         "  static __device__ __forceinline__ void prim(const PrimQuartet<R>& q, R* __restrict__ acc) {",
         "    const R PAx = q.PA[0], PAy = q.PA[1], PAz = q.PA[2];",
         "    const R QCx = q.QC[0], QCy = q.QC[1], QCz = q.QC[2];",
         "    const R WPx = q.WP[0], WPy = q.WP[1], WPz = q.WP[2];",
         "    const R WQx = q.WQ[0], WQy = q.WQ[1], WQz = q.WQ[2];",
         "    const R oo2z = q.oo2z, oo2e = q.oo2e, oo2ze = q.oo2ze, roz = q.roz, roe = q.roe;",
         "    (void)PAx; (void)PAy; (void)PAz; (void)QCx; (void)QCy; (void)QCz;",
         "    (void)WPx; (void)WPy; (void)WPz; (void)WQx; (void)WQy; (void)WQz;",
         "    (void)oo2z; (void)oo2e; (void)oo2ze; (void)roz; (void)roe;"]
    for m in range(L + 1):
        s.append(f"    const R S{m} = q.S[{m}]; (void)S{m};")
    s.extend(consts)
    s.extend(g.lines)
    for i, nm in enumerate(names):
        s.append(f"    acc[{i}] += {nm};")
    s.append("  }")
    s.append("};")
    s.append(f"__device__ const unsigned short g_symdst_{la}{lb}{lc}{ld}_{G}[{G * len(T0)}] = {{" +
             ",".join(str(x) for row in dst for x in row) + "};")
    s.append(f"template <> __device__ __forceinline__ const unsigned short* sym_dst<{la}, {lb}, {lc}, {ld}, {G}>() "
             f"{{ return g_symdst_{la}{lb}{lc}{ld}_{G}; }}")
    stats = dict(cls=f"{la}{lb}{lc}{ld}", G=G, n0=len(T0), nacc=len(E) * len(F),
                 vrr_flops_lane=g.flops + len(T0))
    return "\n".join(s) + "\n", stats


def check_plan(la, lb, lc, ld, G, rng):
    """Evaluate the recurrence numerically: the G lanes' permuted outputs,
    scattered by the tables, must equal the full set of targets evaluated in
    the original frame (CPU check of the tables; used by the tests)."""
    import math
    T0, dst, E, F = plan(la, lb, lc, ld, G)
    perms = GROUPS[G]
    L = la + lb + lc + ld
    vec = {k: [rng.uniform(-1, 1) for _ in range(3)] for k in ("PA", "QC", "WP", "WQ")}
    sc = {k: rng.uniform(0.1, 1.0) for k in ("oo2z", "oo2e", "oo2ze", "roz", "roe")}
    S = [rng.uniform(0.1, 1.0) / (m + 1) for m in range(L + 1)]

    def evaluate(targets, v):
        memo = {}

        def val(e, f, m):
            key = (e, f, m)
            if key in memo:
                return memo[key]
            if sum(e) == 0 and sum(f) == 0:
                r = S[m]
            elif sum(f) > 0:
                i = max(range(3), key=lambda a: (f[a], -a))
                f1 = list(f); f1[i] -= 1; f1 = tuple(f1)
                r = v["QC"][i] * val(e, f1, m) + v["WQ"][i] * val(e, f1, m + 1)
                if f1[i] > 0:
                    f2 = list(f1); f2[i] -= 1; f2 = tuple(f2)
                    r += f1[i] * sc["oo2e"] * (val(e, f2, m) - sc["roe"] * val(e, f2, m + 1))
                if e[i] > 0:
                    e1 = list(e); e1[i] -= 1
                    r += e[i] * sc["oo2ze"] * val(tuple(e1), f1, m + 1)
            else:
                i = max(range(3), key=lambda a: (e[a], -a))
                e1 = list(e); e1[i] -= 1; e1 = tuple(e1)
                r = v["PA"][i] * val(e1, f, m) + v["WP"][i] * val(e1, f, m + 1)
                if e1[i] > 0:
                    e2 = list(e1); e2[i] -= 1
                    r += e1[i] * sc["oo2z"] * (val(tuple(e2), f, m) - sc["roz"] * val(tuple(e2), f, m + 1))
            memo[key] = r
            return r
        return [val(e, f, 0) for (e, f) in targets]

    full = evaluate([(e, f) for e in E for f in F], vec)
    out = [None] * len(full)
    for k, p in enumerate(perms):
        vp = {name: [comp[p[i]] for i in range(3)] for name, comp in vec.items()}
        vals = evaluate(T0, vp)
        for i, d in enumerate(dst[k]):
            if d != 0xFFFF:
                assert out[d] is None
                out[d] = vals[i]
    return max(abs(a - b) / max(1e-300, abs(b)) for a, b in zip(out, full)) if full else 0.0


def classes_for_sym():
    """(la, lb, lc, ld, G) of the classes that get the split kernel: every
    class of total angular momentum >= 4 but (ps|ps)-like light ones; the
    six-lane split where the three-lane one would not fit the registers."""
    return [(1, 1, 1, 1, 3), (2, 0, 1, 1, 3), (2, 0, 2, 0, 3), (2, 1, 1, 0, 3), (2, 2, 0, 0, 3),
            (2, 1, 2, 0, 3), (2, 1, 1, 1, 3), (2, 2, 1, 0, 3), (2, 2, 1, 1, 3), (2, 2, 2, 0, 3),
            (2, 1, 2, 1, 3), (2, 2, 2, 1, 6), (2, 2, 2, 2, 6)]


def sym_fp64(la, lb, lc, ld):
    """Whether the split kernel is also built in FP64 (not for (dd|dp) and
    (dd|dd), whose per-lane accumulators would not fit as doubles)."""
    return (la, lb, lc, ld) not in ((2, 2, 2, 1), (2, 2, 2, 2))


if __name__ == "__main__":
    import random
    rng = random.Random(1)
    for c in classes_for_sym():
        code, st = emit_class(*c)
        print(st, "check", check_plan(*c, rng))
    for c in itertools.islice(classes_for_sym(), 0):
        pass
