"""Generator of the per-class ERI device functions.

For every angular-momentum class (la lb | lc ld) with la >= lb, lc >= ld and
(la, lb) >= (lc, ld) (21 classes for s, p, d shells) it emits a
straight-line device function that evaluates one contracted shell quartet
over Cartesian Gaussians:

  * per primitive quartet: T, the prefactor, the Boys values F_m(T), and the
    Obara-Saika vertical recurrence (bra build on the axis of the largest
    Cartesian exponent, then ket build with the electron-transfer term) for
    the integrals [e0|f0]^(0), la <= |e| <= la+lb, lc <= |f| <= lc+ld;
  * the primitive sum of those integrals;
  * the Head-Gordon-Pople horizontal recurrence, first on the bra and then
    on the ket, giving the (ab|cd) block in [a][b][c][d] order.

Recurrences (Obara & Saika, J. Chem. Phys. 84, 3963 (1986); Head-Gordon &
Pople, J. Chem. Phys. 89, 5777 (1988)), with zeta = a+b, eta = c+d,
rho = zeta*eta/(zeta+eta), W = (zeta P + eta Q)/(zeta+eta):

  [e+1i 0|f0]^m = PA_i [e0|f0]^m + WP_i [e0|f0]^(m+1)
                  + e_i/(2 zeta) ([e-1i 0|f0]^m - rho/zeta [e-1i 0|f0]^(m+1))
                  + f_i/(2(zeta+eta)) [e0|f-1i 0]^(m+1)
  [e0|f+1i 0]^m = QC_i [e0|f0]^m + WQ_i [e0|f0]^(m+1)
                  + f_i/(2 eta) ([e0|f-1i 0]^m - rho/eta [e0|f-1i 0]^(m+1))
                  + e_i/(2(zeta+eta)) [e-1i 0|f0]^(m+1)
  (a, b+1i| = (a+1i, b| + AB_i (a, b|

The script also prints the number of floating-point operations per
primitive quartet and per contracted quartet for each class, which the
benchmark uses as the algorithmic work of each kernel.

Usage: python gen_eri.py OUTDIR
"""
from __future__ import annotations

import json
import os
import sys


def comps(L):
    return [(lx, ly, L - lx - ly) for lx in range(L, -1, -1) for ly in range(L - lx, -1, -1)]


def ncart(L):
    return (L + 1) * (L + 2) // 2


def sub(t, i, k=1):
    u = list(t); u[i] -= k
    return tuple(u)


def add(t, i, k=1):
    u = list(t); u[i] += k
    return tuple(u)


def pick_axis(t):
    # axis of the largest exponent; ties go to the first (x before y before z)
    best = 0
    for i in (1, 2):
        if t[i] > t[best]:
            best = i
    return best


AX = "xyz"


class ClassGen:
    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.L = la + lb + lc + ld
        self.lines = []
        self.names = {}
        self.n = 0
        self.flops = 0  # per primitive quartet, VRR part

    def tmp(self):
        self.n += 1
        return f"v{self.n}"

    # ---------- VRR ----------
    def node(self, e, f, m):
        key = (e, f, m)
        if key in self.names:
            return self.names[key]
        if sum(e) == 0 and sum(f) == 0:
            name = f"S{m}"
            self.names[key] = name
            return name
        terms = []
        if sum(f) > 0:
            i = pick_axis(f)
            f1 = sub(f, i)
            a0 = self.node(e, f1, m)
            a1 = self.node(e, f1, m + 1)
            expr = f"QC{AX[i]} * {a0}"
            expr = f"fma(WQ{AX[i]}, {a1}, {expr})"
            self.flops += 3
            if f1[i] > 0:
                f2 = sub(f1, i)
                b0 = self.node(e, f2, m)
                b1 = self.node(e, f2, m + 1)
                expr = f"fma(oo2e_{f1[i]}, fma(-roe, {b1}, {b0}), {expr})"
                self.flops += 4
            if e[i] > 0:
                c1 = self.node(sub(e, i), f1, m + 1)
                expr = f"fma(oo2ze_{e[i]}, {c1}, {expr})"
                self.flops += 2
        else:
            i = pick_axis(e)
            e1 = sub(e, i)
            a0 = self.node(e1, f, m)
            a1 = self.node(e1, f, m + 1)
            expr = f"fma(WP{AX[i]}, {a1}, PA{AX[i]} * {a0})"
            self.flops += 3
            if e1[i] > 0:
                e2 = sub(e1, i)
                b0 = self.node(e2, f, m)
                b1 = self.node(e2, f, m + 1)
                expr = f"fma(oo2z_{e1[i]}, fma(-roz, {b1}, {b0}), {expr})"
                self.flops += 4
        name = self.tmp()
        self.lines.append(f"    const R {name} = {expr};")
        self.names[key] = name
        return name

    def gen(self, prec_tag):
        la, lb, lc, ld = self.la, self.lb, self.lc, self.ld
        L = self.L
        E = [e for Le in range(la, la + lb + 1) for e in comps(Le)]
        F = [f for Lf in range(lc, lc + ld + 1) for f in comps(Lf)]
        self.E, self.F = E, F
        acc_names = {}
        for ie, e in enumerate(E):
            for jf, f in enumerate(F):
                acc_names[(e, f)] = f"acc[{ie * len(F) + jf}]"
        body = []
        for e in E:
            for f in F:
                nm = self.node(e, f, 0)
                body.append((acc_names[(e, f)], nm))
        vrr = list(self.lines)
        nacc = len(E) * len(F)
        # which scaled constants are used
        used = " ".join(vrr)
        consts = []
        for k in range(1, 5):
            if f"oo2z_{k}" in used:
                consts.append(f"    const R oo2z_{k} = {k}.0 * oo2z;" if k > 1 else "    const R oo2z_1 = oo2z;")
            if f"oo2e_{k}" in used:
                consts.append(f"    const R oo2e_{k} = {k}.0 * oo2e;" if k > 1 else "    const R oo2e_1 = oo2e;")
            if f"oo2ze_{k}" in used:
                consts.append(f"    const R oo2ze_{k} = {k}.0 * oo2ze;" if k > 1 else "    const R oo2ze_1 = oo2ze;")
        ncon = sum(1 for c in consts if "*" in c)

        # ---------- HRR ----------
        hr = []
        AB = {}
        hflops = 0

        # bra: (a,b| from (e,0|, for every f in F
        bra_names = {}

        def bnode(a, b, jf):
            nonlocal hflops
            key = (a, b, jf)
            if key in bra_names:
                return bra_names[key]
            if sum(b) == 0:
                nm = f"acc[{E.index(a) * len(F) + jf}]"
            else:
                i = pick_axis(b)
                b1 = sub(b, i)
                x = bnode(add(a, i), b1, jf)
                y = bnode(a, b1, jf)
                nm = f"h{len(bra_names)}_{jf}"
                hr.append(f"    const R {nm} = fma(ABv[{i}], {y}, {x});")
                hflops += 2
            bra_names[key] = nm
            return nm

        A_c, B_c, C_c, D_c = comps(la), comps(lb), comps(lc), comps(ld)
        bra_out = {}
        for jf in range(len(F)):
            for a in A_c:
                for b in B_c:
                    bra_out[(a, b, jf)] = bnode(a, b, jf)

        # ket: (cd) from (f,0), per bra component pair
        out_lines = []
        for ia, a in enumerate(A_c):
            for ib, b in enumerate(B_c):
                ket_names = {}

                def knode(c, d):
                    nonlocal hflops
                    key = (c, d)
                    if key in ket_names:
                        return ket_names[key]
                    if sum(d) == 0:
                        nm = bra_out[(a, b, F.index(c))]
                    else:
                        i = pick_axis(d)
                        d1 = sub(d, i)
                        x = knode(add(c, i), d1)
                        y = knode(c, d1)
                        nm = f"k{ia}_{ib}_{len(ket_names)}"
                        hr.append(f"    const R {nm} = fma(CDv[{i}], {y}, {x});")
                        hflops += 2
                    ket_names[key] = nm
                    return nm

                for ic, c in enumerate(C_c):
                    for idd, d in enumerate(D_c):
                        nm = knode(c, d)
                        idx = ((ia * len(B_c) + ib) * len(C_c) + ic) * len(D_c) + idd
                        out_lines.append(f"    I[{idx}] = {nm};")
        self.hflops = hflops
        self.nacc = nacc
        self.vrr_flops = self.flops + nacc  # + accumulation adds
        self.consts_flops = ncon
        return vrr, consts, body, hr, out_lines


PRIM_SETUP_FLOPS = 0


def emit_class(la, lb, lc, ld):
    g = ClassGen(la, lb, lc, ld)
    vrr, consts, body, hr, out = g.gen("R")
    L = g.L
    name = f"{la}{lb}{lc}{ld}"
    nA, nB, nC, nD = ncart(la), ncart(lb), ncart(lc), ncart(ld)
    s = []
    s.append(f"// class ({'spd'[la]}{'spd'[lb]}|{'spd'[lc]}{'spd'[ld]}) -- generated by gen_eri.py, do not edit")
    s.append(f"template <> struct EriClass<{la}, {lb}, {lc}, {ld}> {{")
    s.append(f"  static constexpr int NACC = {g.nacc};")
    s.append(f"  static constexpr int N = {nA * nB * nC * nD};")
    s.append(f"  static constexpr int LTOT = {L};")
    s.append("  template <typename R>")
    s.append("  static __device__ __forceinline__ void prim(const PrimQuartet<R>& q, R* __restrict__ acc) {")
    s.append("    const R PAx = q.PA[0], PAy = q.PA[1], PAz = q.PA[2];")
    s.append("    const R QCx = q.QC[0], QCy = q.QC[1], QCz = q.QC[2];")
    s.append("    const R WPx = q.WP[0], WPy = q.WP[1], WPz = q.WP[2];")
    s.append("    const R WQx = q.WQ[0], WQy = q.WQ[1], WQz = q.WQ[2];")
    s.append("    const R oo2z = q.oo2z, oo2e = q.oo2e, oo2ze = q.oo2ze, roz = q.roz, roe = q.roe;")
    s.append("    (void)PAx; (void)PAy; (void)PAz; (void)QCx; (void)QCy; (void)QCz;")
    s.append("    (void)WPx; (void)WPy; (void)WPz; (void)WQx; (void)WQy; (void)WQz;")
    s.append("    (void)oo2z; (void)oo2e; (void)oo2ze; (void)roz; (void)roe;")
    for m in range(L + 1):
        s.append(f"    const R S{m} = q.S[{m}];")
    s.extend(consts)
    s.extend(vrr)
    for a, nm in body:
        s.append(f"    {a} += {nm};")
    s.append("  }")
    s.append("  template <typename R>")
    s.append("  static __device__ __forceinline__ void hrr(const R* __restrict__ acc, const R ABv[3], const R CDv[3], R* __restrict__ I) {")
    s.append("    (void)ABv; (void)CDv;")
    s.extend(hr)
    s.extend(out)
    s.append("  }")
    s.append("};")
    stats = dict(cls=name, L=L, N=nA * nB * nC * nD, nacc=g.nacc,
                 vrr_flops=g.vrr_flops + g.consts_flops, hrr_flops=g.hflops)
    return "\n".join(s) + "\n", stats


def classes():
    pcs = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    out = []
    for i, X in enumerate(pcs):
        for Y in pcs[:i + 1]:
            out.append((X[0], X[1], Y[0], Y[1]))
    return out


def main(outdir):
    os.makedirs(outdir, exist_ok=True)
    allstats = []
    for (la, lb, lc, ld) in classes():
        code, st = emit_class(la, lb, lc, ld)
        path = os.path.join(outdir, f"eri_{la}{lb}{lc}{ld}.cuh")
        old = open(path).read() if os.path.exists(path) else None
        if old != code:
            with open(path, "w") as fh:
                fh.write(code)
        allstats.append(st)
    js = json.dumps(allstats, indent=1)
    p = os.path.join(outdir, "eri_flops.json")
    if not os.path.exists(p) or open(p).read() != js:
        with open(p, "w") as fh:
            fh.write(js)
    return allstats


if __name__ == "__main__":
    for st in main(sys.argv[1]):
        print(st)
