"""Generator of the instruction tables of the warp-cooperative ERI kernel.

For a class (la lb|lc ld) the Obara-Saika vertical recurrence (same
recurrences and the same axis choice as gen_eri.py) and the Head-Gordon-Pople
horizontal recurrence are written as data: every recurrence node is one
instruction

    out = c0*x0 + c1*x1 [+ c2*(x2 - c3*x3)] [+ c4*x4]        (VRR)
    out = x0 + c0*x1                                          (HRR)

with operands x* naming value slots of a per-warp shared-memory buffer and
coefficients c* naming per-primitive-quartet (VRR) or per-quartet (HRR)
constants.  Nodes are ordered by dependency level; within a level they are
independent, so the 32 lanes of a warp evaluate 32 of them at a time.  Value
slots are reused once the last reader's level has passed.

Coefficient ids (VRR): 0-2 PA, 3-5 QC, 6-8 WP, 9-11 WQ, 12 rho/zeta,
13 rho/eta, 14+k-1 k/(2 zeta), 18+k-1 k/(2 eta), 22+k-1 k/(2(zeta+eta))
(k = 1..4).  HRR: 0-2 AB, 3-5 CD.
"""
from __future__ import annotations

from gen_eri import add, comps, ncart, pick_axis, sub

NCOEF = 26
SHAPE_AB, SHAPE_ABC, SHAPE_ABE, SHAPE_ALL = 0, 1, 2, 3


class VRRPlan:
    def __init__(self, la, lb, lc, ld):
        self.L = la + lb + lc + ld
        self.nodes = {}      # key -> node dict
        self.order = []
        E = [e for l in range(la, la + lb + 1) for e in comps(l)]
        F = [f for l in range(lc, lc + ld + 1) for f in comps(l)]
        self.E, self.F = E, F
        self.targets = []
        for e in E:
            for f in F:
                self.targets.append(self.node(e, f, 0))

    def node(self, e, f, m):
        key = (e, f, m)
        if key in self.nodes:
            return key
        if sum(e) == 0 and sum(f) == 0:
            self.nodes[key] = {"base": m, "deps": [], "level": 0}
            return key
        nd = {"ops": [None] * 5, "cs": [0] * 5, "shape": SHAPE_AB}
        if sum(f) > 0:
            i = pick_axis(f)
            f1 = sub(f, i)
            nd["ops"][0] = self.node(e, f1, m); nd["cs"][0] = 3 + i
            nd["ops"][1] = self.node(e, f1, m + 1); nd["cs"][1] = 9 + i
            has_b = f1[i] > 0
            has_e = e[i] > 0
            if has_b:
                f2 = sub(f1, i)
                nd["ops"][2] = self.node(e, f2, m); nd["ops"][3] = self.node(e, f2, m + 1)
                nd["cs"][2] = 18 + f1[i] - 1; nd["cs"][3] = 13
            if has_e:
                nd["ops"][4] = self.node(sub(e, i), f1, m + 1); nd["cs"][4] = 22 + e[i] - 1
        else:
            i = pick_axis(e)
            e1 = sub(e, i)
            nd["ops"][0] = self.node(e1, f, m); nd["cs"][0] = 0 + i
            nd["ops"][1] = self.node(e1, f, m + 1); nd["cs"][1] = 6 + i
            has_b = e1[i] > 0
            has_e = False
            if has_b:
                e2 = sub(e1, i)
                nd["ops"][2] = self.node(e2, f, m); nd["ops"][3] = self.node(e2, f, m + 1)
                nd["cs"][2] = 14 + e1[i] - 1; nd["cs"][3] = 12
        nd["shape"] = (SHAPE_ALL if has_b and has_e else SHAPE_ABC if has_b else
                       SHAPE_ABE if has_e else SHAPE_AB)
        deps = [o for o in nd["ops"] if o is not None]
        nd["deps"] = deps
        nd["level"] = 1 + max(self.nodes[d]["level"] for d in deps)
        self.nodes[key] = nd
        self.order.append(key)
        return key

    def flops(self):
        fl = {SHAPE_AB: 3, SHAPE_ABC: 7, SHAPE_ABE: 5, SHAPE_ALL: 9}
        return sum(fl[self.nodes[k]["shape"]] for k in self.order)


def allocate(levels, deps_of, fixed, persistent, first_free):
    """Slot allocation by level with reuse.  levels: list of lists of node
    keys; fixed: key -> slot for pre-placed values; persistent: keys never
    freed.  A slot whose last reader sits in level l is reusable from level
    l+1 on.  Returns (slot map, number of slots)."""
    last_use = {}
    for li, lv in enumerate(levels):
        for k in lv:
            for d in deps_of(k):
                last_use[d] = max(last_use.get(d, -1), li)
    slot = dict(fixed)
    free = []
    nslots = first_free
    release_at = {}
    for k, s in fixed.items():
        if k not in persistent and k in last_use:
            release_at.setdefault(last_use[k] + 1, []).append(s)
    for li, lv in enumerate(levels):
        for s in release_at.pop(li, []):
            free.append(s)
        free.sort(reverse=True)
        for k in lv:
            if free:
                s = free.pop()
            else:
                s = nslots
                nslots += 1
            slot[k] = s
            if k not in persistent:
                lu = last_use.get(k)
                if lu is not None:
                    release_at.setdefault(lu + 1, []).append(s)
    return slot, nslots


def pack(x0, x1, x2, x3, x4, out, cs):
    assert all(0 <= v < 65536 for v in (x0, x1, x2, x3, x4, out)), "slot overflow"
    assert all(0 <= c < 64 for c in cs)
    w0 = x0 | (x1 << 16)
    w1 = x2 | (x3 << 16)
    w2 = x4 | (out << 16)
    w3 = cs[0] | (cs[1] << 6) | (cs[2] << 12) | (cs[3] << 18) | (cs[4] << 24)
    return (w0, w1, w2, w3)


def schedule(P, maxlev):
    """Phases (lists of nodes evaluated between two warp syncs) that fill
    whole 32-lane groups where the dependencies allow: every node has a
    window [earliest, latest] phase (latest from its consumers; targets may
    wait for the last phase); a phase takes the nodes whose window closes
    there, then tops up each shape's last group with ready nodes whose
    window is still open (closing soonest first)."""
    nodes = [k for k in P.order]
    consumers = {k: [] for k in nodes}
    for k in nodes:
        for d in P.nodes[k]["deps"]:
            if d in consumers:
                consumers[d].append(k)
    latest = {}
    for k in reversed(nodes):   # P.order lists every node after its deps
        latest[k] = min((latest[c] - 1 for c in consumers[k]), default=maxlev)
    done = {k: 0 for k in P.nodes if "base" in P.nodes[k]}
    remaining = list(nodes)
    phases = []
    for ph in range(1, maxlev + 1):
        ready = [k for k in remaining if all(d in done and done[d] < ph for d in P.nodes[k]["deps"])]
        chosen = []
        by_shape = {}
        for k in ready:
            by_shape.setdefault(P.nodes[k]["shape"], []).append(k)
        for sh, ks in by_shape.items():
            must = [k for k in ks if latest[k] <= ph]
            opt = sorted((k for k in ks if latest[k] > ph), key=lambda k: (latest[k], P.nodes[k]["level"]))
            room = (-len(must)) % 32
            chosen += must + opt[:room]
        assert all(latest[k] > ph for k in remaining if k not in chosen and k in ready)
        for k in chosen:
            done[k] = ph
        cs = set(chosen)
        remaining = [k for k in remaining if k not in cs]
        phases.append(chosen)
    assert not remaining
    return phases


def vrr_program(la, lb, lc, ld):
    P = VRRPlan(la, lb, lc, ld)
    L = P.L
    maxlev = max((P.nodes[k]["level"] for k in P.order), default=0)
    levels = schedule(P, maxlev)
    fixed = {k: P.nodes[k]["base"] for k in P.nodes if "base" in P.nodes[k]}
    targets = set(P.targets)
    slot, nslots = allocate(levels, lambda k: P.nodes[k]["deps"], fixed, targets, L + 1)
    groups, descs = [], []
    for lv in levels:
        by_shape = {}
        for k in lv:
            by_shape.setdefault(P.nodes[k]["shape"], []).append(k)
        shapes = sorted(by_shape)
        for si, sh in enumerate(shapes):
            ks = by_shape[sh]
            for c0 in range(0, len(ks), 32):
                chunk = ks[c0:c0 + 32]
                last = (si == len(shapes) - 1) and (c0 + 32 >= len(ks))
                groups.append((sh, len(chunk), len(descs), 1 if last else 0))
                for k in chunk:
                    nd = P.nodes[k]
                    ops = [slot[o] if o is not None else 0 for o in nd["ops"]]
                    descs.append(pack(*ops, slot[k], nd["cs"]))
    tslots = [slot[t] for t in P.targets]
    return dict(groups=groups, descs=descs, nslots=nslots, targets=tslots, nacc=len(P.targets),
                L=L, nodes=len(P.order), flops=P.flops() + len(P.targets), E=P.E, F=P.F)


def hrr_program(la, lb, lc, ld, E, F):
    """Bra HRR for every ket column f, then ket HRR for every bra pair (a,b).
    Inputs: contracted [e0|f0] at slots NOUT + ie*len(F) + jf; outputs:
    (ab|cd) at slots 0..N-1 in [a][b][c][d] order."""
    A, B, C, D = comps(la), comps(lb), comps(lc), comps(ld)
    N = len(A) * len(B) * len(C) * len(D)
    nodes = {}
    order = []

    def inp(e, f):
        return ("in", e, f)

    def bnode(a, b, f):
        if sum(b) == 0:
            return inp(a, f)
        key = ("b", a, b, f)
        if key in nodes:
            return key
        i = pick_axis(b)
        b1 = sub(b, i)
        x = bnode(add(a, i), b1, f)
        y = bnode(a, b1, f)
        lev = 1 + max(nodes[x]["level"] if x in nodes else 0, nodes[y]["level"] if y in nodes else 0)
        nodes[key] = {"ops": (x, y), "c": i, "level": lev}
        order.append(key)
        return key

    def knode(a, b, c, d):
        if sum(d) == 0:
            return bnode(a, b, c)
        key = ("k", a, b, c, d)
        if key in nodes:
            return key
        i = pick_axis(d)
        d1 = sub(d, i)
        x = knode(a, b, add(c, i), d1)
        y = knode(a, b, c, d1)
        lev = 1 + max(nodes[x]["level"] if x in nodes else 0, nodes[y]["level"] if y in nodes else 0)
        nodes[key] = {"ops": (x, y), "c": 3 + i, "level": lev}
        order.append(key)
        return key

    outs = []
    for a in A:
        for b in B:
            for c in C:
                for d in D:
                    outs.append(knode(a, b, c, d))
    fixed = {}
    for ie, e in enumerate(E):
        for jf, f in enumerate(F):
            fixed[inp(e, f)] = N + ie * len(F) + jf
    # outputs that are pure inputs (no HRR) are copied by a move node
    moves = []
    outslot = {}
    for idx, k in enumerate(outs):
        outslot.setdefault(k, idx)
    maxlev = max((nodes[k]["level"] for k in order), default=0)
    levels = [[] for _ in range(maxlev + 1)]
    for k in order:
        levels[nodes[k]["level"]].append(k)
    levels = levels[1:]
    persistent = set(outs)

    def deps(k):
        return list(nodes[k]["ops"]) if k in nodes else []

    # outputs get fixed slots 0..N-1; intermediates above N + NACC
    fixed_all = dict(fixed)
    for k, idx in outslot.items():
        if k in nodes:
            fixed_all[k] = idx
    first = N + len(E) * len(F)
    # allocate only non-output nodes
    inter_levels = [[k for k in lv if k not in outslot] for lv in levels]
    slot, nslots = allocate(inter_levels, deps, fixed_all, persistent, first)
    for k, idx in outslot.items():
        if k in nodes:
            slot[k] = idx
    groups, descs = [], []
    # outputs equal to an input (no recurrence): move instructions, first,
    # while every input slot still holds its value
    mv = []
    for idx, k in enumerate(outs):
        if k not in nodes:
            mv.append((fixed[k], idx))
    for c0 in range(0, len(mv), 32):
        chunk = mv[c0:c0 + 32]
        groups.append((1, len(chunk), len(descs), 1))
        for src, dst in chunk:
            descs.append(pack(src, 0, 0, 0, 0, dst, [0, 0, 0, 0, 0]))
    for lv in levels:
        for c0 in range(0, len(lv), 32):
            chunk = lv[c0:c0 + 32]
            last = c0 + 32 >= len(lv)
            groups.append((0, len(chunk), len(descs), 1 if last else 0))
            for k in chunk:
                x, y = nodes[k]["ops"]
                descs.append(pack(slot[x] if x in slot else fixed[x], slot[y] if y in slot else fixed[y],
                                  0, 0, 0, slot[k], [nodes[k]["c"], 0, 0, 0, 0]))
    return dict(groups=groups, descs=descs, nslots=max(nslots, N + len(E) * len(F)), N=N,
                flops=2 * len(order))


def emit(outdir, classes):
    """Text of coop_tables.cuh (included by cq_coop.cu) with all tables, the
    device-side class directory and the host-side size table."""
    lines = ["// generated by gen_coop.py -- do not edit", "namespace cq {"]
    dir_entries = []
    stats = {}
    for (la, lb, lc, ld) in classes:
        cls = f"{la}{lb}{lc}{ld}"
        v = vrr_program(la, lb, lc, ld)
        h = hrr_program(la, lb, lc, ld, v["E"], v["F"])
        for tag, prog in (("v", v), ("h", h)):
            lines.append(f"__device__ const int4 g_{tag}desc_{cls}[{max(1, len(prog['descs']))}] = {{")
            lines.append(",".join("{%d,%d,%d,%d}" % d for d in prog["descs"]) or "{0,0,0,0}")
            lines.append("};")
            lines.append(f"__device__ const int4 g_{tag}grp_{cls}[{max(1, len(prog['groups']))}] = {{")
            lines.append(",".join("{%d,%d,%d,%d}" % g for g in prog["groups"]) or "{0,0,0,0}")
            lines.append("};")
        lines.append(f"__device__ const unsigned short g_tgt_{cls}[{v['nacc']}] = {{" +
                     ",".join(str(t) for t in v["targets"]) + "};")
        nslots = max(v["nslots"], h["nslots"])
        dir_entries.append(
            f"{{{la}, {lb}, {lc}, {ld}, {v['L']}, {v['nacc']}, {h['N']}, {nslots}, "
            f"{len(v['groups'])}, {len(h['groups'])}, g_vgrp_{cls}, g_vdesc_{cls}, g_hgrp_{cls}, g_hdesc_{cls}, g_tgt_{cls}}}")
        stats[cls] = dict(vrr_nodes=v["nodes"], vrr_groups=len(v["groups"]), vrr_flops=v["flops"],
                          hrr_flops=h["flops"], nslots=nslots, nacc=v["nacc"], N=h["N"],
                          vslots=v["nslots"], hslots=h["nslots"])
    lines.append("__device__ const CoopClass COOP_CLASSES_D[NQC_COOP] = {")
    lines.append(",\n".join(dir_entries))
    lines.append("};")
    lines.append("const CoopSize COOP_SIZES[NQC_COOP] = {")
    lines.append(",\n".join(f"{{{st['nslots']}, {st['nacc']}, {st['N']}, {st['vslots']}, {st['hslots']}}}"
                            for st in stats.values()))
    lines.append("};")
    lines.append("}  // namespace cq")
    return "\n".join(lines) + "\n", stats


if __name__ == "__main__":
    import json
    import sys
    from gen_eri import classes
    code, st = emit(sys.argv[1] if len(sys.argv) > 1 else ".", classes())
    print(json.dumps(st, indent=1))
