"""The roofline numerator: the FLOP counts that flops.py takes from the ERI
generator equal the operations of the code it generates (an FMA counts 2,
a multiply or an add 1, a negated operand 0), counted here by parsing the
generated source.  CPU only."""
import ast
import os
import re
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(os.path.dirname(HERE), "paper_1905_01381_gb300", "csrc"))

import gen_eri  # noqa: E402


def _ops(expr: str) -> int:
    tree = ast.parse(expr.strip(), mode="eval")
    n = 0
    for node in ast.walk(tree):
        if isinstance(node, ast.Call) and getattr(node.func, "id", "") == "fma":
            n += 2
        elif isinstance(node, ast.BinOp) and isinstance(node.op, (ast.Add, ast.Sub, ast.Mult)):
            n += 1
    return n


def _count(lines):
    total = 0
    for ln in lines:
        ln = ln.strip()
        m = re.match(r"const R (\w+) = (.+);$", ln)
        if m and not ln.startswith("const R PAx") and "q." not in m.group(2):
            total += _ops(m.group(2))
            continue
        m = re.match(r"acc\[\d+\] \+= (\w+);$", ln)
        if m:
            total += 1
            continue
        m = re.match(r"I\[\d+\] = (.+);$", ln)
        if m:
            total += _ops(m.group(1))
    return total


def _section(code, start, stop):
    lines = code.splitlines()
    i = next(k for k, ln in enumerate(lines) if start in ln)
    out = []
    for ln in lines[i + 1:]:
        if ln.startswith(stop):
            break
        out.append(ln)
    return out


@pytest.mark.parametrize("cls", gen_eri.classes())
def test_generator_counts_match_generated_code(cls):
    code, st = gen_eri.emit_class(*cls)
    vrr = _count(_section(code, "void prim(", "  }"))
    hrr = _count(_section(code, "void hrr(", "  }"))
    assert vrr == st["vrr_flops"], (cls, vrr, st["vrr_flops"])
    assert hrr == st["hrr_flops"], (cls, hrr, st["hrr_flops"])
