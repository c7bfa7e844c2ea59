"""Front end (program description -> per-access queries, UAF pass), on the
CPU with the oracle as the solver. Pins: the paper's worked examples written
as programs (tests/golden/programs, each access's expected verdict cited),
the closed forms of the bounds and partition families written as programs,
exact subtraction semantics, the use-after-free rule of Sec. V-C, and
malformed programs."""
import glob
import os

import numpy as np
import pytest

import oracle
from closed_forms import bounds_algebra, bounds_wrap, partition_algebra, partition_wrap
from ir_eval import evaluate
from paper_2601_21552_gb300 import frontend as F
from workloads import queries
from workloads.ir import OP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROGRAMS = sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "programs", "*.kp")))


def _solve(accs):
    r = oracle.solve_queries([a.ir for a in accs], max_words=16)
    return [int(v) for v in r["verdict"]], r["words"]


@pytest.mark.parametrize("path", PROGRAMS, ids=os.path.basename)
def test_worked_examples_as_programs(path):
    prog = F.parse(open(path).read())
    assert "cite" in prog.meta
    accs = F.queries(prog)
    assert accs and all(a.meta.get("expect") in ("SAT", "UNSAT") for a in accs)
    got, words = _solve(accs)
    assert got == [1 if a.meta["expect"] == "SAT" else 0 for a in accs]
    for a, v, wd in zip(accs, got, words):  # every witness satisfies its query
        if v == 1:
            assert evaluate(a.ir, [int(x) for x in wd[:len(a.inputs)]])
    want_uaf = prog.meta.get("uaf", "")
    want = sorted(tuple(x.strip().split(":")) for x in want_uaf.split(";") if x.strip())
    assert sorted((u.what, u.name) for u in F.use_after_free(prog)) == want


def bounds_program(w, k1, k0, a, c, guard):
    """The config-1 template as a program: one global allocation of k1*n + k0
    elements, blocks of bdim threads, an unknown number of blocks."""
    body = f"access b[{a} * idx + {c}]"
    if guard:
        body = f"if idx < m\n    {body}\n  end"
    return f"""input n {w}
input bdim {w}
malloc buf {k1} * n + {k0}
launch k grid(?) block(bdim) args(buf, n)
kernel k(b, m)
  let idx = blockIdx.x * blockDim.x + threadIdx.x
  {body}
end
"""


def partition_program(w, k1, k0, a, c, k, j, guard):
    """The config-2 template as a program: the allocation split at i*(n/k)
    (the base is partition 0), the access into partition j."""
    parts = "\n".join(f"  partition p{i} = b + {i} * (m)" for i in range(1, k))
    ptr = "b" if j == 0 else f"p{j}"
    body = f"access {ptr}[{a} * idx + {c}]"
    if guard:
        body = f"if idx < m\n    {body}\n  end"
    return f"""input n {w}
input bdim {w}
malloc buf {k1} * n + {k0}
launch k grid(?) block(bdim) args(buf, n)
kernel k(b, nn)
  let m = nn / {k}
{parts}
  let idx = blockIdx.x * blockDim.x + threadIdx.x
  {body}
end
"""


@pytest.mark.parametrize("w", [6, 8])
def test_families_as_programs_match_closed_forms(w):
    bp = [queries.config1_params(8100 + i, w=w) for i in range(40)]
    pp = [queries.config2_params(8200 + i, w=w) for i in range(40)]
    accs = []
    for p in bp:
        accs += F.queries(F.parse(bounds_program(**p)), bid_width=w)
    for p in pp:
        accs += F.queries(F.parse(partition_program(**p)), bid_width=w)
    got, _ = _solve(accs)
    want = [int(bounds_algebra(**p)) for p in bp] + [int(partition_algebra(**p)) for p in pp]
    assert got == want
    assert set(want) == {0, 1}


def test_program_query_equals_template_query():
    """Same verdicts as the hand-built templates on shared seeds (the
    templates are pinned by brute force at w <= 6)."""
    ps = [queries.config1_params(8300 + i, w=5) for i in range(24)]
    accs = [F.queries(F.parse(bounds_program(**p)), bid_width=5)[0] for p in ps]
    got, _ = _solve(accs)
    for p, g in zip(ps, got):
        bf, _ = oracle.brute_force(queries.bounds_query(**p).to_array(), max_bits=24)
        assert g == bf


def test_exact_subtraction():
    """Partition sizes and offsets are exact integers: a partition whose next
    one starts before it has a negative size, and an offset below the base is
    out of bounds, without wrap-around (b's own accesses would be checked
    against its first partition, [0, x), so the offset checks use f)."""
    text = """input n 6
input d 6
malloc buf 64
malloc flat 64
launch k grid(1) block(1) args(buf, flat, n, d)
kernel k(b, f, x, y)
  partition p1 = b + x
  partition p2 = b + y
  access p1[0]       @expect SAT
  access f[x - y]    @expect SAT
  if x < y
    access f[y - x - 1]   @expect UNSAT
  end
end
"""
    accs = F.queries(F.parse(text))
    got, words = _solve(accs)
    assert got == [1, 1, 0]
    n, d = int(words[0][0]), int(words[0][1])
    assert d <= n  # the witness of the first access: p1 has no room (y <= x)


def test_use_after_free_rules():
    text = """input n 8
malloc a n
malloc b n
if n < 4
  free a
else
  free b
end
launch k grid(1) block(1) args(a, b)
kernel k(x, y)
  shared s[4]
  access s[0]
  for i < 4
    malloc t 8
    free t
  end
  access x[0]
end
"""
    uaf = F.use_after_free(F.parse(text))
    # a and b are each freed on one branch: neither is live at the launch
    assert sorted((u.what, u.name) for u in uaf) == sorted([("launch", "a"), ("launch", "b"),
                                                             ("access", "x")])


@pytest.mark.parametrize("bad", [
    "input n 0\n",                                   # width out of range
    "input n 8\nlet m = n +\n",                      # incomplete expression
    "kernel k(\n",                                   # bad kernel header
    "input n 8\nif n < 2\n",                         # unterminated block
    "end\n",                                         # stray end
    "input n 8\nlaunch k grid(1) block(1) args(n)\nkernel k(x)\n  access q[0]\nend\n",
    "input n 8\nlaunch k grid(1) block(1) args(n)\nkernel k(x)\n  local l[4]\n  access l[x / (x)]\nend\n",
    "input n 8\nwrap 8\n",                         # wrap after another statement
    "wrap 0\n",                                     # wrap width out of range
    "wrap 63\n",
])
def test_malformed_programs_are_rejected(bad):
    with pytest.raises(F.ProgramError):
        F.queries(F.parse(bad))


# ---------------------------------------------------------------------------
# Incremental form: one query per kernel, a selector per memory instruction
# ---------------------------------------------------------------------------

def force_selector(ir_array, kq, k):
    """The kernel query with access k's selector asserted true (what the
    solver's assumption does), as a plain query for the oracle."""
    from workloads.ir import OP, decode
    nodes, roots = decode(ir_array)
    frees = [j for j, nd in enumerate(nodes) if nd[0] == OP.FREE]
    n = len(nodes)
    nodes = nodes + [(OP.CONST, 1, 0), (OP.EQ, frees[kq.selectors[k]], n)]
    roots = roots + [n + 1]
    a = np.zeros(4 + 4 * len(nodes) + len(roots), np.int64)
    a[:4] = ir_array[:4]
    a[2], a[3] = len(nodes), len(roots)
    a[4:4 + 4 * len(nodes)].reshape(-1, 4)[:, :3] = np.array(nodes, np.int64)
    a[4 + 4 * len(nodes):] = roots
    return a


def stencil_program(w=8, radius=3):
    """A kernel with many accesses sharing its ids, sizes and guards: a 1-D
    stencil reading idx-r .. idx+r of an allocation of n elements under
    the guard r <= idx < n - r, plus unguarded neighbours."""
    acc = "\n".join(f"    access a[idx + {d}]" if d >= 0 else f"    access a[idx - {-d}]"
                    for d in range(-radius, radius + 1))
    return f"""input n {w}
input bd {w}
malloc buf n
launch stencil grid((n + 63) / 64) block(bd) args(buf, n)
kernel stencil(a, m)
  let idx = blockIdx.x * blockDim.x + threadIdx.x
  if idx >= {radius} && idx + {radius} < m
{acc}
  end
  access a[idx + {radius}]
  if idx < m
    access a[idx]
    access a[m - idx - 1]
  end
end
"""


@pytest.mark.parametrize("path", PROGRAMS + ["stencil"], ids=lambda p: os.path.basename(p))
def test_incremental_form_matches_per_access(path):
    text = stencil_program() if path == "stencil" else open(path).read()
    prog = F.parse(text)
    per = F.queries(prog)
    want, _ = _solve(per)
    forced = [force_selector(kq.ir, kq, k) for kq in F.kernel_queries(prog)
              for k in range(len(kq.selectors))]
    got = [int(v) for v in oracle.solve_queries(forced)["verdict"]]
    assert got == want
    if path == "stencil":
        assert 0 in got and 1 in got
        # the shared constraints are encoded once instead of once per access
        one = sum(oracle.encode(kq.ir).nclauses for kq in F.kernel_queries(prog))
        each = sum(oracle.encode(a.ir).nclauses for a in per)
        assert one * 3 < each, (one, each)  # 10 accesses: 3,310 vs 12,732 clauses


# ---------------------------------------------------------------------------
# C wrap-around variant: unsigned W-bit program arithmetic
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("w,d", [(4, 1), (4, 2), (5, 1), (5, 2)])
def test_wrap_families_match_bruteforce(w, d):
    """The bounds and partition families as programs under 'wrap W' (W = w + d,
    inputs w-bit) against brute force over every input with explicit
    modulo-2^W arithmetic."""
    W = w + d
    bp = [queries.config1_params(8400 + i, w=w) for i in range(24)]
    pp = [queries.config2_params(8500 + i, w=w) for i in range(24)]
    accs = [F.queries(F.parse(f"wrap {W}\n" + bounds_program(**p)), bid_width=w)[0] for p in bp]
    accs += [F.queries(F.parse(f"wrap {W}\n" + partition_program(**p)), bid_width=w)[0]
             for p in pp]
    got, words = _solve(accs)
    want = [int(bounds_wrap(**p, W=W)) for p in bp] + [int(partition_wrap(**p, W=W)) for p in pp]
    assert got == want
    assert set(want) == {0, 1}
    exact = [int(bounds_algebra(**p)) for p in bp] + [int(partition_algebra(**p)) for p in pp]
    if d == 1:
        assert want != exact  # wrap-around changes verdicts of this sample
    for a, v, wd in zip(accs, got, words):
        if v == 1:
            assert evaluate(a.ir, [int(x) for x in wd[:len(a.inputs)]])


def test_wrap_program_against_exact_reading():
    """The wrap-around golden program read with exact arithmetic (its 'wrap'
    line removed) flips three of its four verdicts, as derived in its header."""
    path = os.path.join(ROOT, "tests", "golden", "programs", "wrap_matrix8.kp")
    text = open(path).read()
    assert F.parse(text).wrap == 8
    exact = F.parse(text.replace("wrap 8\n", ""))
    assert exact.wrap is None
    got, _ = _solve(F.queries(exact))
    assert got == [0, 0, 1, 0]


def test_wrap_truncates_only_what_can_wrap():
    """Values that cannot reach 2^W get no truncation node; a product that
    can gets one, and a subtraction of a node uses the W-bit complement."""
    from workloads.ir import decode
    text = """wrap 16
input n 8
input s 16
malloc buf 300
launch k grid(1) block(1) args(buf, n, s)
kernel k(b, x, y)
  access b[x + 3]
  access b[y * 2]
  access b[y - x]
end
"""
    ops = [[nd[0] for nd in decode(a.ir)[0]] for a in F.queries(F.parse(text))]
    assert OP.TRUNC not in ops[0] and OP.NOTW not in ops[0]
    assert OP.TRUNC in ops[1] and OP.NOTW not in ops[1]
    assert OP.TRUNC in ops[2] and OP.NOTW in ops[2]
    got, _ = _solve(F.queries(F.parse(text)))
    assert got == [0, 1, 1]  # 258 < 300; y*2 wraps to any even value; y - x wraps


def test_wrap_per_input_through_the_front_end():
    """Pinned inputs: division after an overflowing product, subtraction that
    underflows, and a guard computed in wrapped arithmetic, each against
    Python's modular arithmetic (SAT iff the wrapped offset >= size)."""
    cases = []
    for n in (0, 3, 5, 64, 100, 200, 255):
        for size in (1, 10, 40, 100):
            cases.append((n, size, "(m * 4) / 3", ((n * 4) % 256) // 3, True))
            cases.append((n, size, "m - 5", (n - 5) % 256, True))
            # the guard wraps too: (m * 8) % 256 < 16 is the path condition
            cases.append((n, size, "m + 7", (n + 7) % 256, (n * 8) % 256 < 16))
    texts, want = [], []
    for n, size, expr, off, guard_holds in cases:
        body = f"access b[{expr}]"
        if expr == "m + 7":
            body = f"if m * 8 < 16\n    {body}\n  end"
        texts.append(f"""wrap 8
input n 8
assert n == {n}
malloc buf {size}
launch k grid(1) block(1) args(buf, n)
kernel k(b, m)
  {body}
end
""")
        want.append(int(guard_holds and off >= size))
    accs = [F.queries(F.parse(t))[0] for t in texts]
    got, _ = _solve(accs)
    assert got == want
    assert set(want) == {0, 1}


def test_shifts_and_masks_per_input():
    """<< and >> by constants and & with a 2^k - 1 mask, exact and under
    'wrap 8', with pinned inputs, against Python's integer arithmetic."""
    exprs = {
        "(m << 3) >> 2": lambda n, M: ((n << 3) % M) >> 2,
        "m & 31": lambda n, M: n & 31,
        "(m << 4) & 255": lambda n, M: ((n << 4) % M) & 255,
        "31 & (m + 40)": lambda n, M: ((n + 40) % M) & 31,
        "m >> 3 << 1": lambda n, M: ((n >> 3) << 1) % M,
    }
    texts, want = [], []
    for wrap in (None, 8):
        M = (1 << 8) if wrap else (1 << 62)
        for expr, f in exprs.items():
            for n in (0, 7, 33, 100, 200, 255):
                for size in (8, 40, 300):
                    head = "wrap 8\n" if wrap else ""
                    texts.append(f"""{head}input n 8
assert n == {n}
malloc buf {size}
launch k grid(1) block(1) args(buf, n)
kernel k(b, m)
  access b[{expr}]
end
""")
                    want.append(int(f(n, M) >= size % M))  # the size literal wraps too
    got, _ = _solve([F.queries(F.parse(t))[0] for t in texts])
    assert got == want
    assert set(want) == {0, 1}


def test_lane_and_warp_ids_program():
    """Warp-level indexing (lane = tid & 31, warp = tid >> 5) into a shared
    array of one element per thread: in bounds for any block size that is a
    multiple of 32 up to 1024; a block of 33 threads with a 32-wide row per
    warp reads past the end."""
    def prog(bdim_expr, size_expr, guard=""):
        body = "access s[(threadIdx.x >> 5) * 32 + (threadIdx.x & 31)]"
        if guard:
            body = f"if {guard}\n    {body}\n  end"
        return f"""input w 5
launch k grid(1) block({bdim_expr}) args(w)
kernel k(q)
  shared s[{size_expr}]
  {body}
end
"""
    texts = [prog("(w + 1) * 32", "(q + 1) * 32"),       # whole warps: in bounds
             prog("(w + 1) * 32 + 1", "(q + 1) * 32"),   # one extra thread: OOB
             prog("(w + 1) * 32 + 1", "(q + 1) * 32", "threadIdx.x < (q + 1) * 32")]
    got, _ = _solve([F.queries(F.parse(t))[0] for t in texts])
    assert got == [0, 1, 0]


@pytest.mark.parametrize("bad", [
    "input n 8\nlaunch k grid(1) block(1) args(n)\nkernel k(x)\n  local l[4]\n  access l[x << x]\nend\n",
    "input n 8\nlaunch k grid(1) block(1) args(n)\nkernel k(x)\n  local l[4]\n  access l[x & 6]\nend\n",
    "input n 8\nlaunch k grid(1) block(1) args(n)\nkernel k(x)\n  local l[4]\n  access l[x >> 63]\nend\n",
])
def test_bad_shifts_and_masks_are_rejected(bad):
    with pytest.raises(F.ProgramError):
        F.queries(F.parse(bad))


def test_min_max_per_input_and_clamp():
    """min/max against Python's, with pinned inputs, exact and wrapped; a
    clamped index is in bounds exactly when the clamp is below the size."""
    exprs = {"min(m, 10)": lambda n: min(n, 10), "max(m, 50) - 40": lambda n: max(n, 50) - 40,
             "min(m * 3, 200) + max(7, m & 7)": lambda n: min(n * 3, 200) + max(7, n & 7)}
    texts, want = [], []
    for expr, f in exprs.items():
        for n in (0, 5, 33, 90, 255):
            for size in (9, 60, 300):
                texts.append(f"""input n 8
assert n == {n}
malloc buf {size}
launch k grid(1) block(1) args(buf, n)
kernel k(b, m)
  access b[{expr}]
end
""")
                want.append(int(f(n) >= size))
    got, _ = _solve([F.queries(F.parse(t))[0] for t in texts])
    assert got == want and set(want) == {0, 1}

    def clamp(bound, wrap=""):
        return f"""{wrap}input n 8
input bd 8
malloc buf 100
launch k grid(?) block(bd) args(buf, n)
kernel k(b, m)
  let idx = blockIdx.x * blockDim.x + threadIdx.x
  access b[min(idx, {bound})]
  if max(idx, m) < 100
    access b[idx]
  end
end
"""
    for wrap in ("", "wrap 16\n"):
        got, words = _solve(F.queries(F.parse(clamp(99, wrap)), bid_width=8) +
                            F.queries(F.parse(clamp(100, wrap)), bid_width=8))
        assert got == [0, 0, 1, 0], wrap
    # the incremental form agrees (the definitions are shared constraints)
    prog = F.parse(clamp(100))
    per, _ = _solve(F.queries(prog, bid_width=8))
    forced = [force_selector(kq.ir, kq, k) for kq in F.kernel_queries(prog, bid_width=8)
              for k in range(len(kq.selectors))]
    assert [int(v) for v in oracle.solve_queries(forced)["verdict"]] == per


def test_min_of_a_difference_is_rejected():
    bad = ("input n 8\nlaunch k grid(1) block(1) args(n)\nkernel k(x)\n  local l[4]\n"
           "  access l[min(x - 1, 3)]\nend\n")
    with pytest.raises(F.ProgramError):
        F.queries(F.parse(bad))
