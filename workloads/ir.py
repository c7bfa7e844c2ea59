"""Query IR: the expression trees (ETs) and constraints of one memory access.

The paper builds one expression tree per program variable (Sec. V-A, Fig. 6):
leaves are constants or ``Unknown`` inputs, inner nodes are binary operators,
and a variable shared between trees is one node (an MLIR ``Value``). For each
memory instruction it then asserts three kinds of constraints (Sec. V-B):
thread/block ids below their dimensions, offset >= size, and equalities that
define offset, size, grid dimensions and asserts. This module is the data
format for such a query: a DAG of word nodes (unsigned integers of unbounded
precision) and Boolean nodes, plus the list of Boolean roots that must all hold.

Semantics (exact, non-wrapping): FREE nodes range over [0, 2^width); ADD and
MUL are exact integer operations; UDIV/UREM divide by a positive constant
(C floor division on non-negative values); ULT/ULE/EQ compare exactly.
TRUNC and NOTW take an immediate bit count k instead of a second node: the
low k bits of x, and their complement 2^k - 1 - (x mod 2^k). Together with
ADD and MUL they express C's unsigned k-bit arithmetic, which wraps modulo
2^k (x - y is TRUNC(x + NOTW(y) + 1)), for the wrap-around variant of the
queries.

Serialized layout (int64 array):
    [IR_MAGIC, IR_VERSION, N, R,  op_0, x_0, y_0, 0,  ...,  op_{N-1}, x, y, 0,
     root_0, ..., root_{R-1}]
Node operands refer to earlier node indices only (topological order).
"""
from __future__ import annotations

import numpy as np

IR_MAGIC = 0x53435542  # "SCUB"
IR_VERSION = 1


class OP:
    FREE = 1   # x = width (1..64), y = input-word ordinal
    CONST = 2  # x = value, 0 <= value < 2^62
    ADD = 3
    MUL = 4
    ULT = 5    # bool: x < y
    ULE = 6    # bool: x <= y
    EQ = 7     # bool: x == y
    OR = 8     # bool
    AND = 9    # bool
    NOT = 10   # bool: y unused
    UDIV = 11  # word: x // y, y a CONST node with value >= 1
    UREM = 12  # word: x % y, y a CONST node with value >= 1
    TRUNC = 13  # word: x mod 2^y, y = bit count (1..64), an immediate
    NOTW = 14   # word: 2^y - 1 - (x mod 2^y), y = bit count (1..64), an immediate

    WORD = {FREE, CONST, ADD, MUL, UDIV, UREM, TRUNC, NOTW}
    BOOL = {ULT, ULE, EQ, OR, AND, NOT}
    IMMEDIATE = {TRUNC, NOTW}
    NAMES = {
        "free": FREE, "const": CONST, "add": ADD, "mul": MUL, "ult": ULT,
        "ule": ULE, "eq": EQ, "or": OR, "and": AND, "not": NOT,
        "udiv": UDIV, "urem": UREM, "trunc": TRUNC, "notw": NOTW,
    }


class IR:
    """Builder for one query. Methods return node ids (ints)."""

    def __init__(self):
        self.nodes: list[tuple[int, int, int]] = []
        self.roots: list[int] = []
        self._consts: dict[int, int] = {}
        self.n_free = 0
        self.names: dict[int, str] = {}

    # -- leaves ---------------------------------------------------------
    def free(self, width: int, name: str | None = None) -> int:
        if not 1 <= width <= 64:
            raise ValueError("free width must be in [1, 64]")
        self.nodes.append((OP.FREE, width, self.n_free))
        self.n_free += 1
        nid = len(self.nodes) - 1
        if name:
            self.names[nid] = name
        return nid

    def const(self, value: int) -> int:
        value = int(value)
        if not 0 <= value < (1 << 62):
            raise ValueError("constant out of range")
        if value in self._consts:
            return self._consts[value]
        self.nodes.append((OP.CONST, value, 0))
        nid = len(self.nodes) - 1
        self._consts[value] = nid
        return nid

    # -- operators ------------------------------------------------------
    def _op(self, op: int, x: int, y: int = 0) -> int:
        n = len(self.nodes)
        if op in OP.IMMEDIATE:
            if not (0 <= x < n) or not self.is_word(x):
                raise ValueError("operand must be an existing word node")
            if not 1 <= y <= 64:
                raise ValueError("bit count must be in [1, 64]")
            self.nodes.append((op, x, y))
            return n
        if not (0 <= x < n) or (op != OP.NOT and not (0 <= y < n)):
            raise ValueError("operand must be an existing node")
        kinds = [self.is_word(x)] + ([] if op == OP.NOT else [self.is_word(y)])
        want_word = op in (OP.ADD, OP.MUL, OP.ULT, OP.ULE, OP.EQ, OP.UDIV, OP.UREM)
        if any(k != want_word for k in kinds):
            raise ValueError("operand kind mismatch")
        if op in (OP.UDIV, OP.UREM):
            if self.nodes[y][0] != OP.CONST or self.nodes[y][1] < 1:
                raise ValueError("divisor must be a positive constant node")
        self.nodes.append((op, x, y))
        return n

    def add(self, x, y):
        return self._op(OP.ADD, x, y)

    def mul(self, x, y):
        return self._op(OP.MUL, x, y)

    def udiv(self, x, k: int):
        return self._op(OP.UDIV, x, self.const(k))

    def urem(self, x, k: int):
        return self._op(OP.UREM, x, self.const(k))

    def trunc(self, x, bits: int):
        return self._op(OP.TRUNC, x, bits)

    def notw(self, x, bits: int):
        return self._op(OP.NOTW, x, bits)

    def ult(self, x, y):
        return self._op(OP.ULT, x, y)

    def ule(self, x, y):
        return self._op(OP.ULE, x, y)

    def eq(self, x, y):
        return self._op(OP.EQ, x, y)

    def or_(self, x, y):
        return self._op(OP.OR, x, y)

    def and_(self, x, y):
        return self._op(OP.AND, x, y)

    def not_(self, x):
        return self._op(OP.NOT, x, 0)

    def assert_(self, b: int) -> None:
        if self.is_word(b):
            raise ValueError("only Boolean nodes can be asserted")
        self.roots.append(b)

    def is_word(self, nid: int) -> bool:
        return self.nodes[nid][0] in OP.WORD

    # -- serialization ----------------------------------------------------
    def to_array(self) -> np.ndarray:
        n, r = len(self.nodes), len(self.roots)
        a = np.zeros(4 + 4 * n + r, dtype=np.int64)
        a[0], a[1], a[2], a[3] = IR_MAGIC, IR_VERSION, n, r
        if n:
            a[4:4 + 4 * n].reshape(n, 4)[:, :3] = np.asarray(self.nodes, dtype=np.int64)
        a[4 + 4 * n:] = np.asarray(self.roots, dtype=np.int64)
        return a

    def free_widths(self) -> list[int]:
        return [x for (op, x, _y) in self.nodes if op == OP.FREE]


def decode(a: np.ndarray) -> tuple[list[tuple[int, int, int]], list[int]]:
    """Parse a serialized IR back into (nodes, roots); validates the header."""
    a = np.asarray(a, dtype=np.int64)
    if len(a) < 4 or int(a[0]) != IR_MAGIC or int(a[1]) != IR_VERSION:
        raise ValueError("bad IR header")
    n, r = int(a[2]), int(a[3])
    if len(a) != 4 + 4 * n + r:
        raise ValueError("bad IR length")
    body = a[4:4 + 4 * n].reshape(n, 4)
    nodes = [(int(o), int(x), int(y)) for o, x, y, _ in body]
    roots = [int(v) for v in a[4 + 4 * n:]]
    return nodes, roots


def concat(irs: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """Pack several serialized queries into one buffer + int64 offsets[n+1]."""
    offs = np.zeros(len(irs) + 1, dtype=np.int64)
    for i, a in enumerate(irs):
        offs[i + 1] = offs[i] + len(a)
    buf = np.concatenate(irs) if irs else np.zeros(0, dtype=np.int64)
    return buf.astype(np.int64, copy=False), offs


def parse_text(text: str) -> tuple[IR, dict]:
    """Parse the small text form used by the golden fixtures.

    Lines: ``name = free W`` | ``name = const V`` | ``name = OP a b`` (a, b are
    names or integer literals; for trunc/notw b is the bit count) |
    ``name = not a`` | ``assert name`` |
    ``@key value`` (metadata). ``#`` starts a comment.
    """
    ir = IR()
    env: dict[str, int] = {}
    meta: dict[str, str] = {}

    def ref(tok: str) -> int:
        if tok in env:
            return env[tok]
        if tok.lstrip("-").isdigit():
            return ir.const(int(tok))
        raise ValueError(f"unknown name {tok!r}")

    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        if line.startswith("@"):
            key, _, val = line[1:].partition(" ")
            meta[key] = (meta[key] + " " + val.strip()) if key in meta else val.strip()
            continue
        if line.startswith("assert "):
            ir.assert_(ref(line.split()[1]))
            continue
        lhs, _, rhs = line.partition("=")
        name, toks = lhs.strip(), rhs.split()
        op = toks[0]
        if op == "free":
            env[name] = ir.free(int(toks[1]), name)
        elif op == "const":
            env[name] = ir.const(int(toks[1]))
        elif op == "not":
            env[name] = ir.not_(ref(toks[1]))
        elif op in ("udiv", "urem"):
            k = int(toks[2])
            env[name] = ir.udiv(ref(toks[1]), k) if op == "udiv" else ir.urem(ref(toks[1]), k)
        elif op in ("trunc", "notw"):  # the second operand is a bit count
            env[name] = ir._op(OP.NAMES[op], ref(toks[1]), int(toks[2]))
        elif op in OP.NAMES:
            env[name] = ir._op(OP.NAMES[op], ref(toks[1]), ref(toks[2]))
        else:
            raise ValueError(f"unknown op {op!r}")
    return ir, meta
