"""Algorithmic operation counts of the Fock-build kernels (an FMA counts 2).

Per primitive quartet of class (la lb|lc ld), L = la+lb+lc+ld:
  * set-up of the quartet quantities (zeta+eta, 1/sqrt, T, prefactor, W-P,
    W-Q, 1/(2(zeta+eta)), [00|00]^(m) scaling): 25 + L;
  * Boys function by the tabulated Taylor step + downward recursion:
    25 (+ 16 + 3L when L > 0);
  * the generated vertical recurrence and primitive sum (counted by the
    generator).
Per contracted quartet:
  * the generated horizontal recurrence (counted by the generator);
  * digestion: 2 FMAs per integral for J and 4 FMAs per integral per K
    density, i.e. N (4 + 8 nk) with N the number of integrals in the block.
"""
from __future__ import annotations

import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
GEN_STATS = os.path.join(_HERE, "_build", "gen", "eri_flops.json")
PAIR_CLASSES = ["ss", "ps", "pp", "ds", "dp", "dd"]
_LS = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]


def _stats():
    with open(GEN_STATS) as fh:
        return {d["cls"]: d for d in json.load(fh)}


def class_name(X: int, Y: int) -> str:
    return f"({PAIR_CLASSES[X]}|{PAIR_CLASSES[Y]})"


def class_key(X: int, Y: int) -> str:
    return f"{_LS[X][0]}{_LS[X][1]}{_LS[Y][0]}{_LS[Y][1]}"


def per_prim(X: int, Y: int) -> int:
    st = _stats()[class_key(X, Y)]
    L = st["L"]
    boys = 25 + (16 + 3 * L if L > 0 else 0)
    return 25 + L + boys + st["vrr_flops"]


def per_quartet(X: int, Y: int, nk: int, want_j: bool = True) -> int:
    st = _stats()[class_key(X, Y)]
    N = st["N"]
    return st["hrr_flops"] + N * ((4 if want_j else 0) + 8 * nk)


def class_flops(X: int, Y: int, quartets: int, prims: int, nk: int) -> float:
    return float(prims) * per_prim(X, Y) + float(quartets) * per_quartet(X, Y, nk)
