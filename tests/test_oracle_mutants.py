"""The oracle's pins have teeth: each test plants one plausible mistake in a
text copy of oracle/oracle.c (a dropped carry, a flipped comparator, a
missing partial product, a missing remainder bound, a DPLL that never flips
a decision, a propagation that ignores units, a truncation one bit short, a
complement that leaves the high bits clear), builds that copy on the CPU,
and checks that the pins -- brute force over every input and the closed
forms -- reject it, while the unmodified source passes the same pins."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from closed_forms import bounds_algebra, partition_algebra
from workloads import queries
from workloads.ir import IR

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
CDCL_SRC = os.path.join(ROOT, "oracle", "cdcl.c")

MUTANTS = {
    "adder_drops_carry": (
        "carry = g_or(e, g_and(e, x, y), g_and(e, carry, xy));",
        "carry = g_and(e, x, y);"),
    "comparator_uses_le": (
        "int here = g_and(e, -xi, yi);",
        "int here = g_or(e, g_and(e, -xi, yi), i == 0 ? -g_xor(e, xi, yi) : BF);"),
    "multiplier_skips_last_row": (
        "for (int j = 0; j < b->w; j++) {",
        "for (int j = 0; j + 1 < b->w; j++) {"),
    "division_drops_remainder_bound": (
        "assert_bit(&e, w_ult(&e, &r, &kw));     /* r < k */",
        "/* r < k dropped */"),
    "dpll_never_flips": (
        "dflip[nd - 1] = 1;",
        "dflip[nd - 1] = 1; nd = 0; verdict = V_UNSAT; goto done;"),
    "propagation_ignores_units": (
        "if (nun == 1) {",
        "if (nun == 1 && 0) {"),
    "truncation_drops_top_bit": (
        "int w = wd[x].w < y ? wd[x].w : (int)y;",
        "int w = wd[x].w < y ? wd[x].w : (int)y - 1;"),
    "complement_misses_high_bits": (
        "for (int k = 0; k < y; k++) wd[i].b[k] = -w_bit(&wd[x], k);",
        "for (int k = 0; k < y; k++) wd[i].b[k] = k < wd[x].w ? -wd[x].b[k] : BF;"),
}


def _build(src_text: str, tag: str) -> ctypes.CDLL:
    d = tempfile.mkdtemp(prefix=f"oracle_{tag}_")
    c = os.path.join(d, "oracle.c")
    with open(c, "w") as f:
        f.write(src_text)
    so = os.path.join(d, "lib.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-w",
                           "-o", so, c, CDCL_SRC, "-lm"])
    L = ctypes.CDLL(so)
    P = ctypes.c_void_p
    L.oracle_solve_queries.restype = None
    L.oracle_solve_queries.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int64, P, P,
                                       P, ctypes.c_int, P, ctypes.c_int]
    L.oracle_brute_force.restype = ctypes.c_int
    L.oracle_brute_force.argtypes = [P, ctypes.c_int64, ctypes.c_int, P]
    return L


def _solve(L, irs):
    n = len(irs)
    offs = np.zeros(n + 1, np.int64)
    for i, a in enumerate(irs):
        offs[i + 1] = offs[i] + len(a)
    buf = np.ascontiguousarray(np.concatenate(irs), np.int64)
    v = np.zeros(n, np.uint8)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    L.oracle_solve_queries(n, p(buf), p(offs), 4, 200000, p(v), None, None, 0, None, 0)
    return v


def _pins_failed(L) -> int:
    """Number of pin violations for the library L."""
    fails = 0
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    # closed forms over both families at small widths
    b_params = [queries.config1_params(7000 + i, w=5) for i in range(48)]
    irs = [queries.bounds_query(**q).to_array() for q in b_params]
    v = _solve(L, irs)
    fails += int(sum(int(v[i]) != int(bounds_algebra(**q)) for i, q in enumerate(b_params)))
    p_params = [queries.config2_params(8000 + i, w=5) for i in range(48)]
    irs = [queries.partition_query(**q).to_array() for q in p_params]
    v = _solve(L, irs)
    fails += int(sum(int(v[i]) != int(partition_algebra(**q)) for i, q in enumerate(p_params)))
    # gadgets against brute force (the definition), 3-bit words
    gadget_irs = []
    for t in range(0, 50, 3):
        for op in ("add", "mul", "div3", "ult"):
            ir = IR()
            x, y = ir.free(3), ir.free(3)
            if op == "add":
                ir.assert_(ir.eq(ir.add(x, y), ir.const(t % 15)))
            elif op == "mul":
                ir.assert_(ir.eq(ir.mul(x, y), ir.const(t)))
            elif op == "div3":
                ir.assert_(ir.eq(ir.udiv(ir.mul(x, y), 3), ir.const(t % 17)))
            else:
                ir.assert_(ir.ult(ir.add(x, ir.const(t % 9)), y))
            gadget_irs.append(ir.to_array())
    v = _solve(L, gadget_irs)
    wit = np.zeros(64, np.uint64)
    for i, a in enumerate(gadget_irs):
        bf = L.oracle_brute_force(p(a), len(a), 12, p(wit))
        fails += int(bf != int(v[i]))
    # C's unsigned wrap-around, input by input against Python's modular arithmetic
    wrap_irs, want = [], []
    for xv in range(8):
        for yv in range(8):
            ir = IR()
            x, y = ir.free(3), ir.free(3)
            d = ir.trunc(ir.add(ir.add(x, ir.notw(y, 3)), ir.const(1)), 3)
            ir.assert_(ir.eq(x, ir.const(xv)))
            ir.assert_(ir.eq(y, ir.const(yv)))
            ir.assert_(ir.eq(d, ir.const((xv - yv) % 8)))
            ir.assert_(ir.eq(ir.notw(x, 5), ir.const(31 - xv)))
            wrap_irs.append(ir.to_array())
            want.append(1)
    v = _solve(L, wrap_irs)
    fails += int(sum(int(a) != b for a, b in zip(v, want)))
    return fails


def test_unmodified_source_passes_the_pins():
    L = _build(open(SRC).read(), "orig")
    assert _pins_failed(L) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    L = _build(src.replace(old, new), name)
    assert _pins_failed(L) > 0, f"the pins did not catch {name}"
