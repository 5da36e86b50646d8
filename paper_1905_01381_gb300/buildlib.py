"""Build libcq.so for sm_103a: generate the per-class ERI code, compile every
translation unit with nvcc in parallel and link the shared library in-tree
(paper_1905_01381_gb300/_build/libcq.so)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
OBJ = os.path.join(BUILD, "obj")
SO = os.path.join(BUILD, "libcq.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                  "--expt-relaxed-constexpr", "-Xptxas=-warn-spills", "-I", CSRC, "-I", GEN,
                  "-I", os.path.join(os.path.dirname(HERE), "include")]
HAND_SOURCES = ["cq_basis.cu", "cq_fock.cu", "cq_peaks.cu", "cq_noalloc.cu", "cq_oneint.cu", "cq_drivers.cu",
                "cq_coop.cu", "cq_batch.cu", "cq_mlp.cu"]
LIBS = ["-lcublas", "-lcusolver"]

PCS = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]

# lanes per contracted quartet (G) for each class: classes with few quartets
# and expensive primitive quartets split the primitive loop over more lanes
LANES = {"2222": 32, "2221": 8, "2220": 4, "2211": 4, "2121": 4,
         "2120": 2, "2111": 2, "2210": 2, "1111": 2}


# classes without an axis-permutation kernel: their double-float tier runs
# the lane-group kernel, DF_LANES lanes per quartet (the double-float lists
# are short and their quartets deep: about 150 primitive quartets each;
# 8 lanes beat 4 and 2 on the 16-atom workload)
LANE_DF = ("0000", "1000", "1010", "1100", "1110", "2000", "2010", "2100")
DF_LANES = 8

# FP32 lane groups where they differ from LANES: the fastest of 1, 2, 4, 8
# per class on the 16-atom workload's FP32 lists (splitting a quartet's
# primitive quartets over lanes coalesces their loads and evens out the
# work of a warp; larger groups pay in reduction shuffles)
F32_LANES = {"0000": 8, "1000": 4, "1010": 4, "1100": 4, "1110": 2, "2000": 4, "2010": 2, "2011": 2,
             "2020": 2, "2100": 4, "2110": 2, "2200": 8, "1111": 4}

# axis-permutation kernels: lanes per frame splitting the primitive quartets
# (FP64 lists are the short, large-bound part of a mixed build)
SYM_H_F32, SYM_H_F64 = 1, 2

# lanes per shell pair in the Schwarz kernel, by la + lb: the (ab|ab)
# quartets of one pair have up to MAX_PRIM^4 primitive quartets
SCHWARZ_LANES = {0: 4, 1: 8, 2: 8, 3: 16, 4: 32}


def qclasses():
    out = []
    for i, X in enumerate(PCS):
        for Y in PCS[:i + 1]:
            out.append((X, Y))
    return out


def gen_sources():
    sys.path.insert(0, CSRC)
    import gen_eri  # noqa: E402
    stats = gen_eri.main(GEN)
    import gen_coop  # noqa: E402
    code, _ = gen_coop.emit(GEN, gen_eri.classes())
    path = os.path.join(GEN, "coop_tables.cuh")
    if not os.path.exists(path) or open(path).read() != code:
        with open(path, "w") as fh:
            fh.write(code)
    tus = []

    def write(path, lines):
        text = "\n".join(lines) + "\n"
        if not os.path.exists(path) or open(path).read() != text:
            with open(path, "w") as fh:
                fh.write(text)
        tus.append(path)

    for qc, (X, Y) in enumerate(qclasses()):
        la, lb, lc, ld = X[0], X[1], Y[0], Y[1]
        cls = f"{la}{lb}{lc}{ld}"
        head = [f"// generated by build.py: class ({cls})",
                '#include "cq_common.cuh"',
                "namespace cq {",
                f'#include "eri_{cls}.cuh"',
                "}",
                '#include "cq_jk.cuh"',
                "namespace cq {"]
        precs = [("double", "f64"), ("float", "f32")]
        if cls in LANE_DF:
            precs.append(("df", "df"))
        for R, tag in precs:
            G = DF_LANES if tag == "df" else F32_LANES.get(cls, LANES.get(cls, 1)) if tag == "f32" \
                else LANES.get(cls, 1)
            src = head + [
                f"void launch_jk_{cls}_{tag}(const JKArgs& a, cudaStream_t s)",
                "{",
                f"    const long long warps = (a.qmax + {32 // G} - 1) / {32 // G};",
                "    long long blocks = (warps * 32 + JK_THREADS - 1) / JK_THREADS;",
                "    if (blocks == 0) return;",
                "    const long long cap = jk_grid_cap();",
                "    if (blocks > cap) blocks = cap;",
                f"    jk_kernel<{la}, {lb}, {lc}, {ld}, {R}, {G}><<<(unsigned)blocks, JK_THREADS, 0, s>>>(a);",
                "}"]
            if X == Y and tag == "f64":
                src += [f"void launch_schwarz_{la}{lb}(const JKArgs& a, int begin, int end, float* Qf, double* Qd, cudaStream_t s)",
                        "{",
                        "    const int n = end - begin;",
                        "    if (n <= 0) return;",
                        f"    const int per = JK_THREADS / 32 * {32 // SCHWARZ_LANES[la + lb]};",
                        f"    schwarz_kernel<{la}, {lb}, {SCHWARZ_LANES[la + lb]}><<<(n + per - 1) / per, JK_THREADS, 0, s>>>(a, begin, end, Qf, Qd);",
                        "}"]
            src.append("}  // namespace cq")
            write(os.path.join(GEN, f"cls_{cls}_{tag}.cu"), src)
    # dispatch table
    d = ['#include "cq_internal.h"', "namespace cq {"]
    for (X, Y) in qclasses():
        c = f"{X[0]}{X[1]}{Y[0]}{Y[1]}"
        d.append(f"void launch_jk_{c}_f64(const JKArgs&, cudaStream_t);")
        d.append(f"void launch_jk_{c}_f32(const JKArgs&, cudaStream_t);")
        if c in LANE_DF:
            d.append(f"void launch_jk_{c}_df(const JKArgs&, cudaStream_t);")
        df_call = f"else if (prec == 2) launch_jk_{c}_df(a, s); " if c in LANE_DF else ""
        d.append(f"static void launch_jk_{c}(const JKArgs& a, int prec, cudaStream_t s) "
                 f"{{ if (prec == 1) launch_jk_{c}_f32(a, s); {df_call}else launch_jk_{c}_f64(a, s); }}")
    for X in PCS:
        d.append(f"void launch_schwarz_{X[0]}{X[1]}(const JKArgs&, int, int, float*, double*, cudaStream_t);")
    d.append("const LaunchJK JK_LAUNCH[NQC] = {" +
             ", ".join(f"launch_jk_{X[0]}{X[1]}{Y[0]}{Y[1]}" for X, Y in qclasses()) + "};")
    d.append("const int LANE_DF[NQC] = {" +
             ", ".join("1" if f"{X[0]}{X[1]}{Y[0]}{Y[1]}" in LANE_DF else "0" for X, Y in qclasses()) + "};")
    d.append("const LaunchSchwarz SCHWARZ_LAUNCH[NPC] = {" +
             ", ".join(f"launch_schwarz_{X[0]}{X[1]}" for X in PCS) + "};")
    d.append("}  // namespace cq")
    write(os.path.join(GEN, "cq_dispatch.cu"), d)
    # FP32 axis-permutation kernels of the high classes (gen_sym.py): one
    # translation unit per class, with the class's split recurrence and the
    # warp-cooperative HRR tables
    import gen_sym  # noqa: E402
    qc_of = {f"{X[0]}{X[1]}{Y[0]}{Y[1]}": qc for qc, (X, Y) in enumerate(qclasses())}
    sym = {}
    for (la, lb, lc, ld, G) in gen_sym.classes_for_sym():
        cls = f"{la}{lb}{lc}{ld}"
        code, _ = gen_sym.emit_class(la, lb, lc, ld, G)
        path = os.path.join(GEN, f"sym_{cls}.cuh")
        if not os.path.exists(path) or open(path).read() != code:
            with open(path, "w") as fh:
                fh.write(code)
        f64 = gen_sym.sym_fp64(la, lb, lc, ld)
        sym[cls] = (G, f64)
        lines = [
            f"// generated by build.py: class ({cls}), axis-permutation kernel",
            '#include "cq_internal.h"',
            '#include "cq_coop.cuh"',
            '#include "coop_tables.cuh"',
            '#include "cq_sym.cuh"',
            "namespace cq {",
            f'#include "sym_{cls}.cuh"',
            "template <typename R, int H>",
            f"static void launch_sym_{cls}_t(const JKArgs& a, cudaStream_t s)",
            "{",
            f"    constexpr int qc = {qc_of[cls]}, G = {G}, NGRP = 32 / (G * H), WARPS = SYM_THREADS / 32;",
            "    const int nslots = COOP_SIZES[qc].hslots;",
            "    const size_t bytes = (size_t)WARPS * sym_warp_bytes<R>(nslots);",
            f"    auto kern = jk_sym_kernel<{la}, {lb}, {lc}, {ld}, R, G, H>;",
            "    static int attr_done = 0;",
            "    if (!attr_done) {",
            "        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);",
            "        attr_done = 1;",
            "    }",
            "    const long long warps = (a.qmax + NGRP - 1) / NGRP;",
            "    long long blocks = (warps + WARPS - 1) / WARPS;",
            "    if (blocks == 0) return;",
            "    const long long cap = jk_grid_cap();",
            "    if (blocks > cap) blocks = cap;",
            "    kern<<<(unsigned)blocks, SYM_THREADS, bytes, s>>>(a, qc, nslots);",
            "}",
            f"void launch_sym_{cls}(const JKArgs& a, int fp32, cudaStream_t s)",
            "{",
            f"    if (fp32 == 1) launch_sym_{cls}_t<float, {SYM_H_F32}>(a, s);"]
        if f64:
            lines.append(f"    else if (fp32 == 2) launch_sym_{cls}_t<df, {SYM_H_F64}>(a, s);")
            lines.append(f"    else launch_sym_{cls}_t<double, {SYM_H_F64}>(a, s);")
        lines += ["}", "}  // namespace cq"]
        write(os.path.join(GEN, f"cls_{cls}_sym.cu"), lines)
    # dispatch table of the split kernels (NULL where a class has none)
    d = ['#include "cq_internal.h"', "namespace cq {"]
    for cls in sym:
        d.append(f"void launch_sym_{cls}(const JKArgs&, int, cudaStream_t);")
    entries = []
    for (X, Y) in qclasses():
        c = f"{X[0]}{X[1]}{Y[0]}{Y[1]}"
        entries.append(f"launch_sym_{c}" if c in sym else "nullptr")
    d.append("const LaunchJK SYM_LAUNCH[NQC] = {" + ", ".join(entries) + "};")
    f64s = []
    for (X, Y) in qclasses():
        c = f"{X[0]}{X[1]}{Y[0]}{Y[1]}"
        f64s.append("1" if c in sym and sym[c][1] else "0")
    d.append("const int SYM_F64[NQC] = {" + ", ".join(f64s) + "};")
    d.append("}  // namespace cq")
    write(os.path.join(GEN, "cq_dispatch_split.cu"), d)
    sys.path.remove(CSRC)
    return tus, stats


def _deps_mtime():
    m = 0.0
    for f in os.listdir(CSRC):
        if f.endswith((".cuh", ".h", ".py")):
            m = max(m, os.path.getmtime(os.path.join(CSRC, f)))
    m = max(m, os.path.getmtime(os.path.join(os.path.dirname(HERE), "include", "cq.h")))
    return m


def _compile(src, verbose=False):
    obj = os.path.join(OBJ, os.path.basename(src).replace(".cu", ".o"))
    dm = max(_deps_mtime(), os.path.getmtime(src))
    base = os.path.basename(src)
    is_sym = base.startswith("cls_") and base.endswith("_sym.cu")
    if base == "cq_coop.cu" or is_sym:
        dm = max(dm, os.path.getmtime(os.path.join(GEN, "coop_tables.cuh")))
    if is_sym:
        dm = max(dm, os.path.getmtime(os.path.join(GEN, "sym_" + os.path.basename(src)[4:8] + ".cuh")))
    if os.path.exists(obj) and os.path.getmtime(obj) >= dm:
        return obj, ""
    cmd = ["nvcc", "-c", src, "-o", obj + ".tmp"] + NVFLAGS
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, r.stderr


def build(jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(GEN, exist_ok=True)
    os.makedirs(OBJ, exist_ok=True)
    tus, _ = gen_sources()
    srcs = [os.path.join(CSRC, s) for s in HAND_SOURCES] + tus
    # heaviest TUs first so the parallel build finishes early
    def weight(s):
        if not os.path.basename(s).startswith("cls_"):
            return os.path.getsize(s)
        if s.endswith("_sym.cu"):
            return 3 * os.path.getsize(os.path.join(GEN, "sym_" + os.path.basename(s)[4:8] + ".cuh"))
        return (os.path.getsize(os.path.join(GEN, "eri_" + os.path.basename(s)[4:8] + ".cuh"))
                * (2 if s.endswith("_f64.cu") else 1))
    srcs.sort(key=lambda s: -weight(s))
    jobs = jobs or max(1, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(jobs) as ex:
        res = list(ex.map(lambda s: _compile(s, verbose), srcs))
    objs = [r[0] for r in res]
    if verbose:
        for o, err in res:
            if err.strip():
                print(os.path.basename(o), err.strip()[:2000])
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(SO) or os.path.getmtime(SO) < newest:
        tmp = SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["nvcc", "-shared", "-o", tmp] + ARCH + objs + LIBS)
        os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(verbose="-v" in sys.argv), f"{time.time() - t:.1f}s")
