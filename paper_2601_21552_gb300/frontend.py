"""Front end: a small description of a CUDA program -> one satisfiability query
per memory instruction, and the use-after-free live-set pass.

The paper's front end reads the MLIR of the host and kernel code (Sec. V-A,
Fig. 7): from the host it collects the expression trees (ETs) of allocation
sizes, launch geometry, kernel arguments, the dynamic shared-memory size and
asserts; from the kernel the sizes of static (shared or local) allocations,
the logical partitions of dynamic shared memory and the offset of every
memory instruction. For each memory instruction it then asserts the three
kinds of constraints of Sec. V-B: ids below their dimensions; offset >= size
of the accessed data structure; and the equalities that define offset, size,
grid dimensions and asserts. A partition's size is the next partition's
offset minus its own, the last one's the dynamic shared-memory size minus its
offset (Fig. 7b). The UAF pass (Sec. V-C) keeps a set of live allocations
along the host and kernel code, intersecting the sets of the two branches of
a conditional, and reports every use of an allocation that is not live.

MLIR and CGeist are not available here, so programs are written in the small
line format below instead of being compiled; every construct maps to one of
the statements Fig. 7 tracks.

Host statements (outside ``kernel ... end``):
    input NAME WIDTH            a program input (a solver variable, WIDTH bits)
    let NAME = EXPR             a host value
    malloc PTR EXPR             cudaMalloc: PTR holds EXPR elements
    free PTR                    cudaFree
    assert BOOL                 host assert
    launch K grid(E[,E[,E]]|?) block(E[,E[,E]]) [shared E] args(A, ...)
    if BOOL / else / end        host conditionals (they matter to the UAF pass)
Kernel (``kernel K(P1, P2, ...)`` ... ``end``; parameters bind to the launch
arguments by position):
    let NAME = EXPR
    unknown NAME WIDTH          a value the analysis cannot see (read from memory)
    shared NAME[EXPR] | local NAME[EXPR]    static allocation
    extern shared NAME          base of the dynamic shared memory
    partition NAME = BASE + EXPR            logical partition of an allocation
                                (pointer arithmetic; the base is the first one)
    malloc NAME EXPR | free NAME            device-side allocation / release
    if BOOL / else / end        path condition of the accesses inside
    for VAR < EXPR / end        loop: VAR is any value below EXPR inside
    assert BOOL                 device assert (holds from here on)
    access PTR[EXPR]            a load, store or atomic (the same to the analysis)
Expressions: integers, names, threadIdx/blockIdx/blockDim/gridDim .x/.y/.z,
+ - * / % (divisor a positive constant), << and >> by a constant, & with a
constant low-bits mask 2^k - 1 (x % 2^k; '&' binds tighter than comparisons,
unlike C), min(a, b) and max(a, b) of non-negative values (a fresh value
with its defining constraint), parentheses; Booleans: < <= > >= == != && || ! over expressions. Values are exact integers (no wrap-around);
inputs are unsigned. A program whose first statement is ``wrap W`` takes C's
unsigned W-bit semantics instead: every value (inputs and constants too) is
taken modulo 2^W, + - * wrap modulo 2^W, / and % divide the wrapped values;
pointer arithmetic (partition offsets, the bounds check of an access) stays
exact, as a 64-bit address computation does. ``#`` starts a comment; ``@key value`` after a statement
(or on a line of its own) is metadata, e.g. ``access a[i] @expect SAT``.
"""
from __future__ import annotations

import re
from dataclasses import dataclass, field

import numpy as np

from workloads.ir import IR, OP

AXES = ("x", "y", "z")


class ProgramError(ValueError):
    pass


# ---------------------------------------------------------------------------
# Syntax
# ---------------------------------------------------------------------------

@dataclass
class Stmt:
    kind: str
    line: int
    args: dict
    meta: dict = field(default_factory=dict)
    body: list = field(default_factory=list)   # if / for / kernel
    orelse: list = field(default_factory=list)  # if


@dataclass
class Program:
    host: list
    kernels: dict  # name -> Stmt(kind="kernel")
    meta: dict
    wrap: int | None = None  # W of 'wrap W': unsigned W-bit arithmetic


_TOKEN = re.compile(r"\s*(?:(\d+)|([A-Za-z_][A-Za-z_0-9]*(?:\.[xyz])?)|"
                    r"(<<|>>|<=|>=|==|!=|&&|\|\||[-+*/%()<>!,\[\]&]))")


def _tokens(text: str, line: int) -> list:
    out, pos = [], 0
    text = text.rstrip()
    while pos < len(text):
        m = _TOKEN.match(text, pos)
        if not m or m.end() == pos:
            raise ProgramError(f"line {line}: cannot read {text[pos:]!r}")
        num, name, op = m.groups()
        out.append(("num", int(num)) if num else ("name", name) if name else ("op", op))
        pos = m.end()
    return out


class _Expr:
    """Recursive-descent parser over a token list -> a small expression tree
    of tuples: ('num', v) | ('name', s) | (op, a, b) | ('!', a)."""

    def __init__(self, toks, line):
        self.t, self.i, self.line = toks, 0, line

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else (None, None)

    def take(self, want=None):
        tok = self.peek()
        if tok[0] is None or (want is not None and tok[1] != want):
            raise ProgramError(f"line {self.line}: expected {want or 'more input'}")
        self.i += 1
        return tok

    def done(self):
        if self.i != len(self.t):
            raise ProgramError(f"line {self.line}: unexpected {self.t[self.i][1]!r}")

    def boolean(self):
        a = self.conj()
        while self.peek() == ("op", "||"):
            self.take()
            a = ("||", a, self.conj())
        return a

    def conj(self):
        a = self.neg()
        while self.peek() == ("op", "&&"):
            self.take()
            a = ("&&", a, self.neg())
        return a

    def neg(self):
        if self.peek() == ("op", "!"):
            self.take()
            return ("!", self.neg())
        if self.peek() == ("op", "("):  # a parenthesised Boolean or a word
            save = self.i
            self.take()
            try:
                b = self.boolean()
                self.take(")")
                if b[0] in ("<", "<=", ">", ">=", "==", "!=", "&&", "||", "!"):
                    return b
            except ProgramError:
                pass
            self.i = save
        a = self.word()
        tok = self.peek()
        if tok[0] == "op" and tok[1] in ("<", "<=", ">", ">=", "==", "!="):
            self.take()
            return (tok[1], a, self.word())
        raise ProgramError(f"line {self.line}: expected a comparison")

    def word(self):
        # '&' binds tighter than the comparisons here (unlike C), looser
        # than the shifts; shifts looser than + and -, as in C
        a = self.shift()
        while self.peek() == ("op", "&"):
            self.take()
            a = ("&", a, self.shift())
        return a

    def shift(self):
        a = self.additive()
        while self.peek() in (("op", "<<"), ("op", ">>")):
            op = self.take()[1]
            a = (op, a, self.additive())
        return a

    def additive(self):
        a = self.term()
        while self.peek() in (("op", "+"), ("op", "-")):
            op = self.take()[1]
            a = (op, a, self.term())
        return a

    def term(self):
        a = self.atom()
        while self.peek() in (("op", "*"), ("op", "/"), ("op", "%")):
            op = self.take()[1]
            a = (op, a, self.atom())
        return a

    def atom(self):
        kind, val = self.take()
        if kind == "num":
            return ("num", val)
        if kind == "name" and val in ("min", "max") and self.peek() == ("op", "("):
            self.take("(")
            a = self.word()
            self.take(",")
            c = self.word()
            self.take(")")
            return (val, a, c)
        if kind == "name":
            return ("name", val)
        if val == "(":
            a = self.word()
            self.take(")")
            return a
        raise ProgramError(f"line {self.line}: unexpected {val!r}")


def _split_meta(text: str):
    meta = {}
    if "@" in text:
        text, _, rest = text.partition("@")
        for part in ("@" + rest).split("@")[1:]:
            key, _, val = part.strip().partition(" ")
            meta[key] = val.strip()
    return text.strip(), meta


def _parse_word(text, line):
    p = _Expr(_tokens(text, line), line)
    e = p.word()
    p.done()
    return e


def _parse_bool(text, line):
    p = _Expr(_tokens(text, line), line)
    e = p.boolean()
    p.done()
    return e


def _dims(text, line):
    text = text.strip()
    if text == "?":
        return None
    parts, depth, cur = [], 0, ""
    for ch in text:
        if ch == "," and depth == 0:
            parts.append(cur)
            cur = ""
            continue
        depth += ch == "("
        depth -= ch == ")"
        cur += ch
    parts.append(cur)
    if not 1 <= len(parts) <= 3:
        raise ProgramError(f"line {line}: 1 to 3 dimensions")
    return [_parse_word(p, line) for p in parts]


_LAUNCH = re.compile(r"^launch\s+(\w+)\s+grid\((.*?)\)\s+block\((.*?)\)"
                     r"(?:\s+shared\s+(.*?))?\s+args\((.*)\)$")


def parse(text: str) -> Program:
    """Parse a program description (see the module docstring)."""
    host, kernels, meta = [], {}, {}
    stack = [("host", host, None)]  # (block kind, statement list, owning statement)
    last = None
    wrap = None
    for n, raw in enumerate(text.splitlines(), 1):
        line_text = raw.split("#", 1)[0].strip()
        if not line_text:
            continue
        line_text, m = _split_meta(line_text)
        if not line_text:  # metadata line
            (last.meta if last is not None else meta).update(m)
            continue
        words = line_text.split(None, 1)
        head, rest = words[0], words[1] if len(words) > 1 else ""
        where, block, owner = stack[-1]
        in_kernel = any(s[0] == "kernel" for s in stack)
        st = None
        if head == "end":
            if len(stack) == 1:
                raise ProgramError(f"line {n}: 'end' without a block")
            stack.pop()
            continue
        if head == "else":
            if where != "if":
                raise ProgramError(f"line {n}: 'else' outside 'if'")
            stack[-1] = ("else", owner.orelse, owner)
            continue
        if head == "kernel":
            mk = re.match(r"^(\w+)\s*\((.*)\)$", rest)
            if not mk or in_kernel or len(stack) != 1:
                raise ProgramError(f"line {n}: kernel NAME(P, ...) at the top level")
            params = [p.strip() for p in mk.group(2).split(",") if p.strip()]
            st = Stmt("kernel", n, {"name": mk.group(1), "params": params}, m)
            kernels[mk.group(1)] = st
            stack.append(("kernel", st.body, st))
            last = st
            continue
        if head == "wrap":
            if host or kernels or wrap is not None or not rest.strip().isdigit():
                raise ProgramError(f"line {n}: 'wrap W' must be the first statement")
            wrap = int(rest)
            if not 1 <= wrap <= 62:
                raise ProgramError(f"line {n}: wrap width in [1, 62]")
            continue
        if head == "input" or head == "unknown":
            name, width = rest.split()
            if head == "input" and in_kernel:
                raise ProgramError(f"line {n}: 'input' is a host statement; use 'unknown'")
            if head == "unknown" and not in_kernel:
                raise ProgramError(f"line {n}: 'unknown' is a kernel statement; use 'input'")
            w = int(width)
            if not 1 <= w <= 64:
                raise ProgramError(f"line {n}: width in [1, 64]")
            st = Stmt("input", n, {"name": name, "width": w}, m)
        elif head == "let":
            name, _, e = rest.partition("=")
            st = Stmt("let", n, {"name": name.strip(), "expr": _parse_word(e, n)}, m)
        elif head == "malloc":
            name, e = rest.split(None, 1)
            st = Stmt("malloc", n, {"name": name, "expr": _parse_word(e, n)}, m)
        elif head == "free":
            st = Stmt("free", n, {"name": rest.strip()}, m)
        elif head == "assert":
            st = Stmt("assert", n, {"cond": _parse_bool(rest, n)}, m)
        elif head == "if":
            st = Stmt("if", n, {"cond": _parse_bool(rest, n)}, m)
            block.append(st)
            stack.append(("if", st.body, st))
            last = st
            continue
        elif head == "launch" and not in_kernel:
            ml = _LAUNCH.match(line_text)
            if not ml:
                raise ProgramError(f"line {n}: launch K grid(..) block(..) [shared E] args(..)")
            args = [a.strip() for a in ml.group(5).split(",") if a.strip()]
            st = Stmt("launch", n, {"kernel": ml.group(1), "grid": _dims(ml.group(2), n),
                                    "block": _dims(ml.group(3), n),
                                    "shared": _parse_word(ml.group(4), n) if ml.group(4) else None,
                                    "args": args}, m)
        elif in_kernel and head in ("shared", "local"):
            if rest.startswith("extern"):
                raise ProgramError(f"line {n}: write 'extern shared NAME'")
            ma = re.match(r"^(\w+)\s*\[(.*)\]$", rest.strip())
            if not ma:
                raise ProgramError(f"line {n}: {head} NAME[SIZE]")
            st = Stmt("static", n, {"name": ma.group(1), "expr": _parse_word(ma.group(2), n)}, m)
        elif in_kernel and head == "extern":
            ms = re.match(r"^shared\s+(\w+)$", rest.strip())
            if not ms:
                raise ProgramError(f"line {n}: extern shared NAME")
            st = Stmt("dynshared", n, {"name": ms.group(1)}, m)
        elif in_kernel and head == "partition":
            mp = re.match(r"^(\w+)\s*=\s*(\w+)\s*\+\s*(.*)$", rest.strip())
            if not mp:
                raise ProgramError(f"line {n}: partition NAME = BASE + EXPR")
            st = Stmt("partition", n, {"name": mp.group(1), "base": mp.group(2),
                                       "expr": _parse_word(mp.group(3), n)}, m)
        elif in_kernel and head == "for":
            mf = re.match(r"^(\w+)\s*<\s*(.*)$", rest.strip())
            if not mf:
                raise ProgramError(f"line {n}: for VAR < EXPR")
            st = Stmt("for", n, {"var": mf.group(1), "bound": _parse_word(mf.group(2), n)}, m)
            block.append(st)
            stack.append(("for", st.body, st))
            last = st
            continue
        elif in_kernel and head == "access":
            ma = re.match(r"^(\w+)\s*\[(.*)\]$", rest.strip())
            if not ma:
                raise ProgramError(f"line {n}: access PTR[EXPR]")
            st = Stmt("access", n, {"ptr": ma.group(1), "expr": _parse_word(ma.group(2), n)}, m)
        else:
            raise ProgramError(f"line {n}: unknown statement {head!r}")
        block.append(st)
        last = st
    if len(stack) != 1:
        raise ProgramError("unterminated block (missing 'end')")
    return Program(host, kernels, meta, wrap)


# ---------------------------------------------------------------------------
# Values: exact integers as (positive part, negative part) of IR nodes
# ---------------------------------------------------------------------------

class _N:
    """An IR node (distinct from a folded Python integer or bool)."""
    __slots__ = ("i",)

    def __init__(self, i: int):
        self.i = i


class _Builder:
    """Builds one query. A word value is a pair (p, n) meaning p - n, each an
    IR node (_N) or a Python int (a folded constant); inputs are non-negative,
    so subtraction needs no wrap-around: comparisons move terms across.
    Booleans are _N nodes or folded Python bools.

    With wrap = W the program's own arithmetic (arith, constants, inputs) is
    unsigned W-bit: every value it makes is a pair (v, 0) with v < 2^W, and a
    result that may reach 2^W is truncated. The analysis' own arithmetic
    (partition sizes, the bounds check) keeps using add/sub/less, exactly."""

    def __init__(self, wrap: int | None = None):
        self.ir = IR()
        self.maxv = {}  # node id -> largest value it can take
        self.wrap = wrap

    def wrapv(self, v):
        """v modulo 2^W (no node when v cannot reach 2^W)."""
        if self.wrap is None:
            return v
        if not isinstance(v, _N):
            return v % (1 << self.wrap)
        if self.vmax(v) < (1 << self.wrap):
            return v
        r = _N(self.ir.trunc(v.i, self.wrap))
        self.maxv[r.i] = (1 << self.wrap) - 1
        return r

    def arith(self, kind, x, y):
        """The program's x + y, x - y or x * y."""
        if self.wrap is None:
            return {"+": self.add, "-": self.sub, "*": self.mul}[kind](x, y)
        a, c = x[0], y[0]  # wrapped values: no negative part
        if kind == "-":  # x - y = x + (2^W - y) = x + ~y + 1 (mod 2^W)
            if isinstance(c, _N):
                nc = _N(self.ir.notw(c.i, self.wrap))
                self.maxv[nc.i] = (1 << self.wrap) - 1
                r = self._bin("+", self._bin("+", a, nc), 1)
            else:
                r = self._bin("+", a, (-c) % (1 << self.wrap))
        else:
            r = self._bin(kind, a, c)
        return (self.wrapv(r), 0)

    def node(self, v) -> int:
        return v.i if isinstance(v, _N) else self.ir.const(v)

    def vmax(self, v) -> int:
        return self.maxv[v.i] if isinstance(v, _N) else v

    def _bin(self, op, a, b):
        if not isinstance(a, _N) and not isinstance(b, _N):
            return a + b if op == "+" else a * b
        if op == "+":
            if not isinstance(a, _N) and a == 0:
                return b
            if not isinstance(b, _N) and b == 0:
                return a
            r = _N(self.ir.add(self.node(a), self.node(b)))
            self.maxv[r.i] = self.vmax(a) + self.vmax(b)
        else:
            if (not isinstance(a, _N) and a == 0) or (not isinstance(b, _N) and b == 0):
                return 0
            if not isinstance(a, _N) and a == 1:
                return b
            if not isinstance(b, _N) and b == 1:
                return a
            r = _N(self.ir.mul(self.node(a), self.node(b)))
            self.maxv[r.i] = self.vmax(a) * self.vmax(b)
        return r

    def free(self, width, name):
        r = _N(self.ir.free(width, name))
        self.maxv[r.i] = (1 << width) - 1
        return self.wrapv(r)

    # word pairs
    def add(self, x, y):
        return (self._bin("+", x[0], y[0]), self._bin("+", x[1], y[1]))

    def sub(self, x, y):
        return (self._bin("+", x[0], y[1]), self._bin("+", x[1], y[0]))

    def mul(self, x, y):
        p = self._bin("+", self._bin("*", x[0], y[0]), self._bin("*", x[1], y[1]))
        n = self._bin("+", self._bin("*", x[0], y[1]), self._bin("*", x[1], y[0]))
        return (p, n)

    def divmod_(self, x, k, rem, line):
        if isinstance(x[1], _N) or x[1] != 0:
            raise ProgramError(f"line {line}: '/' and '%' need a non-negative dividend "
                               "(no subtraction inside)")
        if not isinstance(x[0], _N):
            return ((x[0] % k) if rem else (x[0] // k), 0)
        r = _N(self.ir.urem(x[0].i, k) if rem else self.ir.udiv(x[0].i, k))
        self.maxv[r.i] = min(self.vmax(x[0]), k - 1) if rem else self.vmax(x[0]) // k
        return (r, 0)

    def minmax(self, kind, x, y, line):
        """min(x, y) or max(x, y) as a fresh word r with its defining
        equality (r = x and x <= y) or (r = y and y < x) (max: the other
        way round) asserted: a kind 3 constraint of Sec. V-B."""
        for v in (x, y):
            if isinstance(v[1], _N) or v[1] != 0:
                raise ProgramError(f"line {line}: {kind} needs non-negative operands "
                                   "(no subtraction inside)")
        a, c = x[0], y[0]
        if not isinstance(a, _N) and not isinstance(c, _N):
            return (min(a, c) if kind == "min" else max(a, c), 0)
        hi = min(self.vmax(a), self.vmax(c)) if kind == "min" else max(self.vmax(a),
                                                                           self.vmax(c))
        r = (self.free(_bits(hi), f"{kind}@{line}"), 0)
        self.maxv[r[0].i] = hi
        first, second = (x, y) if kind == "min" else (y, x)
        self.require(self.bor(self.band(self.equal(r, x), self.less(first, second, strict=False)),
                              self.band(self.equal(r, y), self.less(second, first))))
        return r

    def _cmp(self, fold, make, x, y):
        a = self._bin("+", x[0], y[1])
        b = self._bin("+", y[0], x[1])
        if not isinstance(a, _N) and not isinstance(b, _N):
            return fold(a, b)
        return _N(make(self.node(a), self.node(b)))

    def less(self, x, y, strict=True):
        """x < y (or x <= y): x.p + y.n < y.p + x.n."""
        if strict:
            return self._cmp(lambda a, b: a < b, self.ir.ult, x, y)
        return self._cmp(lambda a, b: a <= b, self.ir.ule, x, y)

    def equal(self, x, y):
        return self._cmp(lambda a, b: a == b, self.ir.eq, x, y)

    def bnot(self, a):
        return (not a) if not isinstance(a, _N) else _N(self.ir.not_(a.i))

    def band(self, a, b):
        if not isinstance(a, _N):
            return b if a else False
        if not isinstance(b, _N):
            return a if b else False
        return _N(self.ir.and_(a.i, b.i))

    def bor(self, a, b):
        if not isinstance(a, _N):
            return True if a else b
        if not isinstance(b, _N):
            return True if b else a
        return _N(self.ir.or_(a.i, b.i))

    def require(self, b):
        """Assert a Boolean; a folded False makes the query trivially UNSAT."""
        if not isinstance(b, _N):
            if not b:
                zero = self.ir.const(0)
                self.ir.assert_(self.ir.ult(zero, zero))
            return
        self.ir.assert_(b.i)


def _bits(v: int) -> int:
    return max(1, int(v).bit_length())


def _is_const(x, c: int) -> bool:
    return not isinstance(x[0], _N) and not isinstance(x[1], _N) and x[0] - x[1] == c


# ---------------------------------------------------------------------------
# Queries (Sec. V-B)
# ---------------------------------------------------------------------------

@dataclass
class Access:
    kernel: str
    index: int          # position among the kernel's memory instructions
    line: int
    ptr: str
    meta: dict
    ir: np.ndarray      # the query: SAT iff this access can go out of bounds
    inputs: list        # names of the query's FREE words, in order


def _eval(b: _Builder, env: dict, e, line):
    kind = e[0]
    if kind == "num":
        return (b.wrapv(e[1]), 0)
    if kind == "name":
        if e[1] not in env:
            raise ProgramError(f"line {line}: unknown name {e[1]!r}")
        v = env[e[1]]
        if not isinstance(v, tuple):
            raise ProgramError(f"line {line}: {e[1]!r} is not a value")
        return v
    if kind in ("min", "max"):
        return b.minmax(kind, _eval(b, env, e[1], line), _eval(b, env, e[2], line), line)
    if kind == "&" and e[1][0] == "num" and e[2][0] != "num":
        e = ("&", e[2], e[1])  # the mask on the right
    x, y = _eval(b, env, e[1], line), None
    if kind in ("/", "%"):
        if e[2][0] != "num" or e[2][1] < 1:
            raise ProgramError(f"line {line}: divisor must be a positive constant")
        return b.divmod_(x, e[2][1], kind == "%", line)
    if kind in ("<<", ">>"):  # by a constant: * 2^k, or / 2^k
        if e[2][0] != "num" or e[2][1] > 62:
            raise ProgramError(f"line {line}: shift count must be a constant in [0, 62]")
        if kind == ">>":
            return b.divmod_(x, 1 << e[2][1], False, line)
        return b.arith("*", x, (b.wrapv(1 << e[2][1]), 0))
    if kind == "&":  # a low-bits mask 2^k - 1: % 2^k
        m = e[2][1] if e[2][0] == "num" else -1
        if m < 0 or (m + 1) & m:
            raise ProgramError(f"line {line}: '&' takes a constant mask 2^k - 1")
        return b.divmod_(x, m + 1, True, line)
    y = _eval(b, env, e[2], line)
    return b.arith(kind, x, y)


def _eval_bool(b: _Builder, env: dict, e, line):
    kind = e[0]
    if kind == "!":
        return b.bnot(_eval_bool(b, env, e[1], line))
    if kind in ("&&", "||"):
        x, y = _eval_bool(b, env, e[1], line), _eval_bool(b, env, e[2], line)
        return b.band(x, y) if kind == "&&" else b.bor(x, y)
    x, y = _eval(b, env, e[1], line), _eval(b, env, e[2], line)
    if kind == "<":
        return b.less(x, y)
    if kind == "<=":
        return b.less(x, y, strict=False)
    if kind == ">":
        return b.less(y, x)
    if kind == ">=":
        return b.less(y, x, strict=False)
    if kind == "==":
        return b.equal(x, y)
    return b.bnot(b.equal(x, y))  # !=


def _host_env(b: _Builder, prog: Program, launch_of: str, default_width: int):
    """Replays the host code up to the launch of kernel `launch_of`: inputs,
    values, allocation sizes, asserts (asserted into the query). Returns the
    environment and the launch statement."""
    env, allocs = {}, {}

    def walk(stmts):
        for st in stmts:
            if st.kind == "input":
                env[st.args["name"]] = (b.free(st.args["width"], st.args["name"]), 0)
            elif st.kind == "let":
                env[st.args["name"]] = _eval(b, env, st.args["expr"], st.line)
            elif st.kind == "malloc":
                allocs[st.args["name"]] = _eval(b, env, st.args["expr"], st.line)
                env.setdefault(st.args["name"] + ".size", allocs[st.args["name"]])
            elif st.kind == "assert":
                b.require(_eval_bool(b, env, st.args["cond"], st.line))
            elif st.kind == "launch" and st.args["kernel"] == launch_of:
                return st
            elif st.kind == "if":  # host conditionals: values on both paths are
                r = walk(st.body) or walk(st.orelse)  # taken as defined (no path constraint)
                if r:
                    return r
        return None

    launch = walk(prog.host)
    if launch is None:
        raise ProgramError(f"kernel {launch_of!r} is never launched")
    return env, allocs, launch


def _kernel_env(b: _Builder, env, allocs, launch, kern, bid_width):
    """Kind 1 constraints and the kernel's parameter bindings."""
    kenv = dict(env)
    block = launch.args["block"]
    grid = launch.args["grid"]
    for k, ax in enumerate(AXES):
        bd = _eval(b, env, block[k], launch.line) if k < len(block) else (1, 0)
        kenv[f"blockDim.{ax}"] = bd
        if _is_const(bd, 1):
            kenv[f"threadIdx.{ax}"] = (0, 0)
        else:
            t = (b.free(_bits(b.vmax(bd[0])), f"threadIdx.{ax}"), 0)
            b.require(b.less(t, bd))  # kind 1
            kenv[f"threadIdx.{ax}"] = t
        if grid is None:  # no grid dimension known: blockIdx bounded by its width only
            if k == 0:
                kenv["blockIdx.x"] = (b.free(bid_width, "blockIdx.x"), 0)
            else:
                kenv[f"blockIdx.{ax}"] = (0, 0)
            continue
        gd = _eval(b, env, grid[k], launch.line) if k < len(grid) else (1, 0)
        kenv[f"gridDim.{ax}"] = gd
        if _is_const(gd, 1):
            kenv[f"blockIdx.{ax}"] = (0, 0)
        else:
            g = (b.free(_bits(b.vmax(gd[0])), f"blockIdx.{ax}"), 0)
            b.require(b.less(g, gd))  # kind 1
            kenv[f"blockIdx.{ax}"] = g
    params = kern.args["params"]
    args = launch.args["args"]
    if len(params) != len(args):
        raise ProgramError(f"line {launch.line}: {len(args)} arguments for {len(params)} parameters")
    sizes = {}
    for p, a in zip(params, args):
        if a in allocs:  # a pointer to a host allocation: its size ET
            sizes[p] = allocs[a]
            kenv[p] = None
        else:
            kenv[p] = _eval(b, env, _parse_word(a, launch.line), launch.line)
    shared = _eval(b, env, launch.args["shared"], launch.line) if launch.args["shared"] else None
    return kenv, sizes, shared


def queries(prog: Program, bid_width: int = 16) -> list:
    """One query per memory instruction of every launched kernel (Sec. V-B)."""
    out = []
    for kname, kern in prog.kernels.items():
        # the memory instructions of the kernel, in program order
        accesses = []

        def collect(stmts):
            for st in stmts:
                if st.kind == "access":
                    accesses.append(st)
                collect(st.body)
                collect(st.orelse)
        collect(kern.body)
        if not any(st.kind == "launch" and st.args["kernel"] == kname for st in _flat(prog.host)):
            continue
        for idx, target in enumerate(accesses):
            b = _Builder(prog.wrap)
            env, allocs, launch = _host_env(b, prog, kname, bid_width)
            kenv, sizes, shared = _kernel_env(b, env, allocs, launch, kern, bid_width)
            state = {"parts": {}, "found": False}
            _kernel_path(b, kenv, sizes, shared, kern.body, target, state)
            if not state["found"]:
                raise ProgramError(f"line {target.line}: access not reached")
            names = [b.ir.names.get(i, f"free{k}") for k, i in
                     enumerate(j for j, nd in enumerate(b.ir.nodes) if nd[0] == OP.FREE)]
            out.append(Access(kname, idx, target.line, target.args["ptr"], target.meta,
                              b.ir.to_array(), names))
    return out


def _flat(stmts):
    for st in stmts:
        yield st
        yield from _flat(st.body)
        yield from _flat(st.orelse)


def _partition_sizes(b, chain, end, line):
    """Fig. 7b: a partition ends where the next one starts; the last one at
    the end of the allocation (for dynamic shared memory, the launch's
    dynamic size). The allocation's base is the first partition."""
    if end is None:
        raise ProgramError(f"line {line}: dynamic shared memory without a launch size")
    out = {}
    for k, (name, off) in enumerate(chain):
        out[name] = b.sub(chain[k + 1][1] if k + 1 < len(chain) else end, off)
    return out


def _kernel_path(b, kenv, sizes, shared, stmts, target, state):
    """Walks the kernel in program order, adding the path conditions and
    asserts that hold at `target`; at `target` adds kind 2 and stops.
    Returns True once the target was reached."""
    for st in stmts:
        a = st.args
        if st.kind == "let":
            kenv[a["name"]] = _eval(b, kenv, a["expr"], st.line)
        elif st.kind == "input":  # 'unknown' inside the kernel
            kenv[a["name"]] = (b.free(a["width"], a["name"]), 0)
        elif st.kind in ("static", "malloc"):
            sizes[a["name"]] = _eval(b, kenv, a["expr"], st.line)
            kenv[a["name"]] = None
        elif st.kind == "dynshared":
            state["parts"][a["name"]] = [(a["name"], (0, 0))]
            kenv[a["name"]] = None
        elif st.kind == "partition":
            base = a["base"]
            if base not in state["parts"]:
                if base not in sizes:
                    raise ProgramError(f"line {st.line}: partition of an unknown allocation")
                state["parts"][base] = [(base, (0, 0))]
            state["parts"][base].append((a["name"], _eval(b, kenv, a["expr"], st.line)))
            kenv[a["name"]] = None
        elif st.kind == "assert":
            b.require(_eval_bool(b, kenv, a["cond"], st.line))
        elif st.kind == "if":
            c = _eval_bool(b, kenv, a["cond"], st.line)
            if _contains(st.body, target):
                b.require(c)
                return _kernel_path(b, kenv, sizes, shared, st.body, target, state)
            if _contains(st.orelse, target):
                b.require(b.bnot(c))
                return _kernel_path(b, kenv, sizes, shared, st.orelse, target, state)
            # a branch not leading to the target: its definitions are not
            # visible after it (program values are SSA-like in this format)
        elif st.kind == "for":
            if _contains(st.body, target):
                bound = _eval(b, kenv, a["bound"], st.line)
                v = (b.free(_bits(b.vmax(bound[0])), a["var"]), 0)
                b.require(b.less(v, bound))
                kenv[a["var"]] = v
                return _kernel_path(b, kenv, sizes, shared, st.body, target, state)
        elif st.kind == "access" and st is target:
            ptr = a["ptr"]
            psize = {}
            for base, chain in state["parts"].items():
                end = shared if base not in sizes else sizes[base]
                psize.update(_partition_sizes(b, chain, end, st.line))
            if ptr in psize:
                size = psize[ptr]
            elif ptr in sizes:
                size = sizes[ptr]
            else:
                raise ProgramError(f"line {st.line}: {ptr!r} is not a known allocation")
            off = _eval(b, kenv, a["expr"], st.line)
            # kind 2: offset >= size, or below the base (a negative offset)
            oob = b.less(size, off, strict=False)
            if isinstance(off[1], _N) or off[1] != 0:
                oob = b.bor(oob, b.less(off, (0, 0)))
            b.require(oob)
            state["found"] = True
            return True
    return False


def _kernel_all(b, kenv, sizes, shared, stmts, conds, parts, out):
    """One walk over the kernel for the incremental form: every memory
    instruction gets the conjunction of the path conditions, loop bounds and
    asserts that hold at it, and its kind-2 constraint, as one Boolean
    (appended to out with the statement)."""
    kenv, sizes, parts = dict(kenv), dict(sizes), {k: list(v) for k, v in parts.items()}
    conds = list(conds)
    for st in stmts:
        a = st.args
        if st.kind == "let":
            kenv[a["name"]] = _eval(b, kenv, a["expr"], st.line)
        elif st.kind == "input":
            kenv[a["name"]] = (b.free(a["width"], a["name"]), 0)
        elif st.kind in ("static", "malloc"):
            sizes[a["name"]] = _eval(b, kenv, a["expr"], st.line)
            kenv[a["name"]] = None
        elif st.kind == "dynshared":
            parts[a["name"]] = [(a["name"], (0, 0))]
            kenv[a["name"]] = None
        elif st.kind == "partition":
            base = a["base"]
            if base not in parts:
                if base not in sizes:
                    raise ProgramError(f"line {st.line}: partition of an unknown allocation")
                parts[base] = [(base, (0, 0))]
            parts[base].append((a["name"], _eval(b, kenv, a["expr"], st.line)))
            kenv[a["name"]] = None
        elif st.kind == "assert":
            conds.append(_eval_bool(b, kenv, a["cond"], st.line))
        elif st.kind == "if":
            c = _eval_bool(b, kenv, a["cond"], st.line)
            _kernel_all(b, kenv, sizes, shared, st.body, conds + [c], parts, out)
            _kernel_all(b, kenv, sizes, shared, st.orelse, conds + [b.bnot(c)], parts, out)
        elif st.kind == "for":
            bound = _eval(b, kenv, a["bound"], st.line)
            v = (b.free(_bits(b.vmax(bound[0])), a["var"]), 0)
            inner = dict(kenv)
            inner[a["var"]] = v
            _kernel_all(b, inner, sizes, shared, st.body, conds + [b.less(v, bound)], parts, out)
        elif st.kind == "access":
            ptr = a["ptr"]
            psize = {}
            for base, chain in parts.items():
                end = shared if base not in sizes else sizes[base]
                psize.update(_partition_sizes(b, chain, end, st.line))
            size = psize.get(ptr, sizes.get(ptr))
            if size is None:
                raise ProgramError(f"line {st.line}: {ptr!r} is not a known allocation")
            off = _eval(b, kenv, a["expr"], st.line)
            oob = b.less(size, off, strict=False)
            if isinstance(off[1], _N) or off[1] != 0:
                oob = b.bor(oob, b.less(off, (0, 0)))
            for c in conds:
                oob = b.band(c, oob)
            out.append((st, oob))


@dataclass
class KernelQuery:
    """The incremental form of one kernel: one query holding the shared
    constraints (kinds 1 and 3 of Sec. V-B) and, per memory instruction, its
    own constraints guarded by a one-bit selector input (selector -> its
    constraints). Solving with selector k assumed true decides access k."""
    kernel: str
    ir: np.ndarray
    accesses: list       # Access entries (ir None): the instructions, in program order
    selectors: list      # FREE-word ordinal of each access's selector
    inputs: list         # names of the FREE words


def kernel_queries(prog: Program, bid_width: int = 16) -> list:
    out = []
    launched = {st.args["kernel"] for st in _flat(prog.host) if st.kind == "launch"}
    for kname, kern in prog.kernels.items():
        if kname not in launched:
            continue
        b = _Builder(prog.wrap)
        env, allocs, launch = _host_env(b, prog, kname, bid_width)
        kenv, sizes, shared = _kernel_env(b, env, allocs, launch, kern, bid_width)
        found = []
        _kernel_all(b, kenv, sizes, shared, kern.body, [], {}, found)
        sels = []
        for k, (st, cond) in enumerate(found):
            sel = b.free(1, f"@select{k}")
            b.require(b.bor(b.bnot(b.less((0, 0), (sel, 0))), cond))
            sels.append(sel)
        frees = [j for j, nd in enumerate(b.ir.nodes) if nd[0] == OP.FREE]
        names = [b.ir.names.get(j, f"free{k}") for k, j in enumerate(frees)]
        ordinals = [frees.index(sel.i) for sel in sels]
        accs = [Access(kname, k, st.line, st.args["ptr"], st.meta, None, names)
                for k, (st, _c) in enumerate(found)]
        out.append(KernelQuery(kname, b.ir.to_array(), accs, ordinals, names))
    return out


def _contains(stmts, target) -> bool:
    return any(st is target for st in _flat(stmts))


# ---------------------------------------------------------------------------
# Use after free (Sec. V-C)
# ---------------------------------------------------------------------------

@dataclass
class UAF:
    line: int
    what: str   # "access" or "launch"
    name: str
    where: str  # kernel or "host"


def use_after_free(prog: Program) -> list:
    """Live-set pass over the host code (launch arguments) and every launched
    kernel (memory instructions); a conditional's live set is the
    intersection of its two branches."""
    reports = []

    def kernel_pass(kern, live_in):
        def walk(stmts, live):
            live = set(live)
            for st in stmts:
                a = st.args
                if st.kind in ("static", "malloc", "dynshared", "partition"):
                    live.add(a["name"])
                elif st.kind == "free":
                    live.discard(a["name"])
                elif st.kind == "access" and a["ptr"] not in live:
                    reports.append(UAF(st.line, "access", a["ptr"], kern.args["name"]))
                elif st.kind == "if":
                    live = walk(st.body, live) & walk(st.orelse, live)
                elif st.kind == "for":
                    live = walk(st.body, live) & live  # zero or more iterations
            return live
        walk(kern.body, live_in)

    def host(stmts, live, allocs):
        live = set(live)
        for st in stmts:
            a = st.args
            if st.kind == "malloc":
                live.add(a["name"])
                allocs.add(a["name"])
            elif st.kind == "free":
                live.discard(a["name"])
            elif st.kind == "launch":
                kern = prog.kernels.get(a["kernel"])
                live_params = set()
                for k, arg in enumerate(a["args"]):
                    if arg in allocs:
                        if arg not in live:
                            reports.append(UAF(st.line, "launch", arg, "host"))
                        elif kern is not None and k < len(kern.args["params"]):
                            live_params.add(kern.args["params"][k])
                    elif kern is not None and k < len(kern.args["params"]):
                        live_params.add(kern.args["params"][k])  # scalars are always usable
                if kern is not None:
                    kernel_pass(kern, live_params)
            elif st.kind == "if":
                live = host(st.body, live, allocs) & host(st.orelse, live, allocs)
        return live

    host(prog.host, set(), set())
    return reports


# ---------------------------------------------------------------------------
# Whole-program analysis on the GPU
# ---------------------------------------------------------------------------

@dataclass
class Report:
    accesses: list   # Access with .verdict (0 UNSAT, 1 SAT = OOB possible, 2 UNKNOWN) and .witness
    uaf: list

    @property
    def oob(self):
        return [a for a in self.accesses if a.verdict == 1]


def _input_words(enc, model, verdicts) -> list:
    """The FREE words of every SAT query, decoded from its model through the
    encoder's input-bit map (least significant bit first)."""
    iib, widths, var = enc.inputs()
    vb = enc.inst_var_begin
    out, bit = [], 0
    for i in range(len(verdicts)):
        words = []
        for w in range(int(iib[i]), int(iib[i + 1])):
            x = 0
            for k in range(int(widths[w])):
                if verdicts[i] == 1 and model[vb[i] + var[bit] - 1]:
                    x |= 1 << k
                bit += 1
            words.append(x)
        out.append(words if verdicts[i] == 1 else None)
    return out


def analyze_programs(texts: list, device: str = "cuda", bid_width: int = 16,
                     **solve_opts) -> list:
    """Parse several programs, build every memory instruction's query, decide
    all of them in one GPU batch (scuba_solve_batch via api.solve_queries,
    every model re-verified on the host), and run the UAF pass on each. A SAT
    access carries a witness: the value of every input, unknown and id of its
    query. Returns one Report per program."""
    from . import api

    progs = [parse(t) for t in texts]
    per = [queries(p, bid_width=bid_width) for p in progs]
    flat = [a for accs in per for a in accs]
    if flat:
        res = api.solve_queries([a.ir for a in flat], device=device, **solve_opts)
        if res["status"] != 0 or res["fails"] != 0:
            raise RuntimeError(f"solve failed: status {res['status']}, {res['fails']} bad models")
        words = _input_words(res["enc"], res["model"], res["verdict"])
        for a, v, wd in zip(flat, res["verdict"], words):
            a.verdict = int(v)
            a.witness = dict(zip(a.inputs, wd)) if wd is not None else None
    return [Report(accs, use_after_free(p)) for p, accs in zip(progs, per)]


def analyze_incremental(texts: list, device: str = "cuda", bid_width: int = 16,
                        **solve_opts) -> list:
    """Like analyze_programs, but one query per kernel: its shared constraints
    are encoded and uploaded once, and every memory instruction is a unit of
    scuba_solve_units with its selector assumed true. Models are re-verified
    on the host, unit by unit."""
    import torch

    from . import api, binding as B

    progs = [parse(t) for t in texts]
    kqs = [kernel_queries(p, bid_width=bid_width) for p in progs]
    flat = [kq for ks in kqs for kq in ks]
    if flat:
        enc = B.scuba_encode_batch([kq.ir for kq in flat])
        db = api.DeviceBatch(enc, device)
        iib, widths, var = enc.inputs()
        bit0 = np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)
        unit_inst, asm = [], []
        for i, kq in enumerate(flat):
            for s in kq.selectors:
                unit_inst.append(i)
                asm.append(int(var[bit0[iib[i] + s]]))  # the selector's variable, true
        asm_begin = np.arange(len(asm) + 1, dtype=np.int64)
        v, m, mb = api.solve_units(db, unit_inst, asm_begin, np.array(asm, np.int32),
                                   **solve_opts)
        rc = api.status()
        if rc != 0:
            raise RuntimeError(f"solve failed: status {rc}")
        vh, mh, mbh = v.cpu().numpy(), m.cpu().numpy(), mb.cpu().numpy()
        nvs, vbs = enc.inst_num_vars, enc.inst_var_begin
        u = 0
        for i, kq in enumerate(flat):
            for a in kq.accesses:
                a.verdict = int(vh[u])
                a.witness = None
                if a.verdict == 1:
                    # this unit's model in the batch's layout, checked against the IR
                    full = np.zeros(max(int(vbs[-1]), 1), np.uint8)
                    full[vbs[i]:vbs[i] + nvs[i]] = mh[mbh[u]:mbh[u] + nvs[i]]
                    ver = np.full(len(flat), 2, np.uint8)
                    ver[i] = 1
                    fails, _ok = B.scuba_verify_batch(enc, ver, full)
                    if fails:
                        raise RuntimeError(f"unit {u}: the model fails the query")
                    words = _input_words(enc, full, ver)[i]
                    a.witness = {k: x for k, x in zip(kq.inputs, words)
                                 if not k.startswith("@select")}
                u += 1
        torch.cuda.synchronize()
    return [Report([a for kq in ks for a in kq.accesses], use_after_free(p))
            for p, ks in zip(progs, kqs)]


def analyze(text: str, device: str = "cuda", bid_width: int = 16, **solve_opts) -> Report:
    """analyze_programs for one program."""
    return analyze_programs([text], device=device, bid_width=bid_width, **solve_opts)[0]
