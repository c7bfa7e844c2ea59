"""Exact integer evaluation of a query IR with Python big integers.

Test-side checker (not part of the oracle or the product): used to re-verify
every SAT model against the original integer constraints (Sec. V-B: an OOB is
reported when all constraints hold simultaneously under some input).
"""
from __future__ import annotations

from workloads.ir import OP, decode


def evaluate(ir_array, inputs) -> bool:
    """True iff every asserted root holds when FREE node #i takes inputs[i]."""
    nodes, roots = decode(ir_array)
    val: list[int] = [0] * len(nodes)
    fi = 0
    for i, (op, x, y) in enumerate(nodes):
        if op == OP.FREE:
            v = int(inputs[fi])
            if not 0 <= v < (1 << x):
                raise ValueError("input out of its width")
            val[i] = v
            fi += 1
        elif op == OP.CONST:
            val[i] = x
        elif op == OP.ADD:
            val[i] = val[x] + val[y]
        elif op == OP.MUL:
            val[i] = val[x] * val[y]
        elif op == OP.UDIV:
            val[i] = val[x] // val[y]
        elif op == OP.UREM:
            val[i] = val[x] % val[y]
        elif op == OP.TRUNC:
            val[i] = val[x] % (1 << y)
        elif op == OP.NOTW:
            val[i] = (1 << y) - 1 - val[x] % (1 << y)
        elif op == OP.ULT:
            val[i] = int(val[x] < val[y])
        elif op == OP.ULE:
            val[i] = int(val[x] <= val[y])
        elif op == OP.EQ:
            val[i] = int(val[x] == val[y])
        elif op == OP.OR:
            val[i] = int(bool(val[x]) or bool(val[y]))
        elif op == OP.AND:
            val[i] = int(bool(val[x]) and bool(val[y]))
        elif op == OP.NOT:
            val[i] = int(not val[x])
        else:
            raise ValueError(op)
    return all(val[r] for r in roots)


def cnf_satisfied(clause_begin, lits, model) -> bool:
    """True iff the 0/1 model (index v-1) satisfies every clause."""
    for c in range(len(clause_begin) - 1):
        ok = False
        for k in range(int(clause_begin[c]), int(clause_begin[c + 1])):
            l = int(lits[k])
            b = int(model[abs(l) - 1])
            if (l > 0 and b == 1) or (l < 0 and b == 0):
                ok = True
                break
        if not ok:
            return False
    return True
