"""Host-side product code on the CPU: the C ABI library loads and exports
every symbol of include/scuba.h, the 3-CNF encoder is equisatisfiable with the
integer semantics input by input, and the host re-verifier agrees with an
independent big-integer evaluator. No GPU calls."""
import itertools
import os
import re

import numpy as np
import pytest

from ir_eval import evaluate
from workloads import queries
from workloads.ir import IR, parse_text

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2601_21552_gb300 import build
    build.build()
    from paper_2601_21552_gb300 import binding
    return binding


def test_exports_every_header_symbol(B):
    hdr = open(os.path.join(ROOT, "include", "scuba.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(scuba_[a-z_]+)\s*\(", hdr))
    assert names, "no declarations found"
    for name in sorted(names):
        assert hasattr(B._lib, name), name
    assert set(B.EXPORTED) == names
    # the checked build (device bounds checks) exports the same ABI
    import ctypes
    from paper_2601_21552_gb300 import build
    chk = ctypes.CDLL(build.LIB_CHECKED)
    for name in sorted(names):
        assert hasattr(chk, name), name
    sizes = np.zeros(2, np.int64)
    chk.scuba_abi_sizes(sizes.ctypes.data_as(ctypes.c_void_p))
    ref = np.zeros(2, np.int64)
    B._lib.scuba_abi_sizes(ref.ctypes.data_as(ctypes.c_void_p))
    assert (sizes == ref).all()


def _unit_propagate(nv, clauses, assign):
    """Plain unit propagation; returns False on conflict."""
    changed = True
    while changed:
        changed = False
        for cl in clauses:
            open_l, sat = [], False
            for l in cl:
                v = assign.get(abs(l))
                if v is None:
                    if l not in open_l:
                        open_l.append(l)
                elif v == (l > 0):
                    sat = True
                    break
            if sat:
                continue
            if not open_l:
                return False
            if len(open_l) == 1:
                assign[abs(open_l[0])] = open_l[0] > 0
                changed = True
    return True


def _cnf_sat_under(nv, clauses, fixed):
    """Is the CNF satisfiable with the given variables fixed? Unit propagation,
    then brute force over what is left (tiny gadgets only)."""
    assign = dict(fixed)
    if not _unit_propagate(nv, clauses, assign):
        return False
    rest = [v for v in range(1, nv + 1) if v not in assign]
    assert len(rest) <= 14, "gadget too large for the exhaustive check"
    for bits in itertools.product([False, True], repeat=len(rest)):
        a = dict(assign)
        a.update(zip(rest, bits))
        if all(any(a[abs(l)] == (l > 0) for l in cl) for cl in clauses):
            return True
    return False


def _gadgets():
    out = []
    for op in ("add", "mul", "div3", "rem5", "div4", "ult", "ule", "eq", "orcmp",
               "wsub", "wmul", "wnot"):
        for t in range(0, 20, 3):
            ir = IR()
            x = ir.free(3)
            y = ir.free(3)
            if op == "add":
                ir.assert_(ir.eq(ir.add(x, y), ir.const(t)))
            elif op == "mul":
                ir.assert_(ir.ult(ir.mul(x, y), ir.const(t)))
            elif op == "div3":
                ir.assert_(ir.eq(ir.udiv(ir.add(x, y), 3), ir.const(t % 5)))
            elif op == "rem5":
                ir.assert_(ir.eq(ir.urem(ir.mul(x, y), 5), ir.const(t % 5)))
            elif op == "div4":
                ir.assert_(ir.ule(ir.udiv(ir.mul(x, y), 4), ir.const(t % 13)))
            elif op == "ult":
                ir.assert_(ir.ult(ir.add(x, ir.const(t % 7)), y))
            elif op == "ule":
                ir.assert_(ir.not_(ir.ule(ir.mul(x, ir.const(t % 5 + 1)), y)))
            elif op == "eq":
                ir.assert_(ir.or_(ir.eq(x, ir.const(t % 8)), ir.eq(ir.add(x, y), ir.const(t))))
            elif op == "wsub":  # (x - y) mod 8 in C's unsigned 3-bit arithmetic
                d = ir.trunc(ir.add(ir.add(x, ir.notw(y, 3)), ir.const(1)), 3)
                ir.assert_(ir.eq(d, ir.const(t % 8)))
            elif op == "wmul":
                ir.assert_(ir.ult(ir.trunc(ir.mul(x, y), 4), ir.const(t % 16)))
            elif op == "wnot":
                ir.assert_(ir.ule(ir.notw(ir.add(x, y), 2), ir.trunc(y, 2)))
            else:
                ir.assert_(ir.or_(ir.ult(x, y), ir.and_(ir.ule(y, x), ir.eq(y, ir.const(t % 8)))))
            out.append((op, t, ir))
    return out


@pytest.mark.parametrize("case", _gadgets(), ids=lambda c: f"{c[0]}-{c[1]}")
def test_encoder_equisatisfiable_per_input(B, case):
    op, t, ir = case
    a = ir.to_array()
    enc = B.scuba_encode_batch([a])
    cb, lits = enc.clause_begin, enc.lits
    clauses = [lits[cb[i]:cb[i + 1]].tolist() for i in range(enc.total_clauses)]
    assert all(len(c) <= 3 for c in clauses), "encoder must emit 3-CNF"
    iib, widths, var = enc.inputs()
    assert widths.tolist() == [3, 3]
    for xv in range(8):
        for yv in range(8):
            fixed = {}
            for k in range(3):
                fixed[int(var[k])] = bool((xv >> k) & 1)
                fixed[int(var[3 + k])] = bool((yv >> k) & 1)
            assert _cnf_sat_under(enc.total_vars, clauses, fixed) == evaluate(a, [xv, yv]), (xv, yv)


def test_input_bits_numbered_first_msb_first(B):
    ir = queries.bounds_query(8, 2, 3, 1, 2, True)
    enc = B.scuba_encode_batch([ir.to_array()])
    iib, widths, var = enc.inputs()
    assert widths.tolist() == [8, 8, 8, 8]
    # word 0 occupies variables 1..8 with its MSB = 1
    assert var[:8].tolist() == [8, 7, 6, 5, 4, 3, 2, 1]
    assert sorted(var.tolist()) == list(range(1, 33))


def test_verify_batch_against_big_int_evaluator(B):
    rng = np.random.default_rng(5)
    irs = []
    for i in range(40):
        p = queries.config1_params(1000 + i, w=6)
        irs.append(queries.bounds_query(**p).to_array())
    enc = B.scuba_encode_batch(irs)
    iib, widths, var = enc.inputs()
    for trial in range(3):
        model = rng.integers(0, 2, size=enc.total_vars, dtype=np.uint8)
        verdict = np.ones(enc.n, np.uint8)
        fails, ok = B.scuba_verify_batch(enc, verdict, model)
        vb = enc.inst_var_begin
        woff = np.concatenate([[0], np.cumsum(widths)])
        for i in range(enc.n):
            words = []
            for k in range(iib[i], iib[i + 1]):
                w = 0
                for j in range(widths[k]):
                    v = int(var[woff[k] + j])
                    w |= int(model[vb[i] + v - 1]) << j
                words.append(w)
            assert ok[i] == (1 if evaluate(irs[i], words) else 0)
        assert fails == int((ok == 0).sum())


def test_encoder_rejects_malformed_ir(B):
    a = queries.bounds_query(8, 1, 0, 1, 0, True).to_array()
    bad = a.copy()
    bad[0] = 7
    with pytest.raises(RuntimeError):
        B.scuba_encode_batch([bad])
    bad = a.copy()
    bad[4 + 4 * 5 + 1] = 99  # operand pointing forward
    with pytest.raises(RuntimeError):
        B.scuba_encode_batch([bad])


def test_worked_examples_encode_to_3cnf(B):
    import glob
    files = sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "*.sq")))
    irs = [parse_text(open(f).read())[0].to_array() for f in files]
    enc = B.scuba_encode_batch(irs)
    lens = np.diff(enc.clause_begin)
    assert lens.max() <= 3 and enc.n == len(files)


def test_wrap_evaluator_against_modular_arithmetic():
    """The test-side evaluator's truncation and complement against Python's
    modular arithmetic (the other wrap pins compare with this evaluator)."""
    for xv in range(8):
        for yv in range(8):
            ir = IR()
            x, y = ir.free(3), ir.free(3)
            d = ir.trunc(ir.add(ir.add(x, ir.notw(y, 3)), ir.const(1)), 3)
            ir.assert_(ir.eq(d, ir.const((xv - yv) % 8)))
            ir.assert_(ir.eq(ir.notw(ir.mul(x, y), 4), ir.const(15 - (xv * yv) % 16)))
            assert evaluate(ir.to_array(), [xv, yv])


def test_verify_wrap_ops_against_evaluator(B):
    """The host re-verifier's truncation and complement (any bit count up to
    64) against the test-side evaluator, on random models."""
    rng = np.random.default_rng(11)
    irs = []
    for k in (1, 7, 31, 32, 33, 63, 64):
        ir = IR()
        x, y = ir.free(40), ir.free(40)
        p = ir.mul(x, y)
        ir.assert_(ir.ult(ir.trunc(p, k), ir.notw(ir.add(p, y), k)))
        irs.append(ir.to_array())
    enc = B.scuba_encode_batch(irs)
    iib, widths, var = enc.inputs()
    woff = np.concatenate([[0], np.cumsum(widths)])
    for trial in range(4):
        model = rng.integers(0, 2, size=enc.total_vars, dtype=np.uint8)
        fails, ok = B.scuba_verify_batch(enc, np.ones(enc.n, np.uint8), model)
        vb = enc.inst_var_begin
        for i in range(enc.n):
            words = []
            for kk in range(iib[i], iib[i + 1]):
                wv = 0
                for j in range(widths[kk]):
                    wv |= int(model[vb[i] + int(var[woff[kk] + j]) - 1]) << j
                words.append(wv)
            assert ok[i] == (1 if evaluate(irs[i], words) else 0), (i, trial)


def test_wrap_queries_encode_equisatisfiably(B):
    """Front-end queries under 'wrap W': the product encoder's CNFs, decided
    by the oracle's CNF solver, give the verdicts the oracle reaches from its
    own encoding of the same queries."""
    import oracle
    from paper_2601_21552_gb300 import frontend as F
    from test_frontend import bounds_program, partition_program
    texts = [open(os.path.join(ROOT, "tests", "golden", "programs", "wrap_matrix8.kp")).read()]
    for d in (1, 2):
        texts += [f"wrap {8 + d}\n" + bounds_program(**queries.config1_params(8800 + i, w=8))
                  for i in range(16)]
        texts += [f"wrap {8 + d}\n" + partition_program(**queries.config2_params(8900 + i, w=8))
                  for i in range(16)]
    irs = [a.ir for t in texts for a in F.queries(F.parse(t), bid_width=8)]
    enc = B.scuba_encode_batch(irs)
    cb, lits, icb = enc.clause_begin, enc.lits, enc.inst_clause_begin
    cnfs = []
    for i in range(enc.n):
        c0, c1 = int(icb[i]), int(icb[i + 1])
        l0 = int(cb[c0])
        cnfs.append(oracle.CNF(int(enc.inst_num_vars[i]), cb[c0:c1 + 1] - l0,
                               lits[l0:int(cb[c1])]))
    got = oracle.solve_cnfs(cnfs)["verdict"]
    want = oracle.solve_queries(irs, max_words=16)["verdict"]
    assert got.tolist() == want.tolist()
    assert set(want.tolist()) == {0, 1}


def test_grown_queries_product_cnf_agrees_with_oracle_encoding(B):
    """The product encoder on the config-3 template family (2-D/3-D ids,
    row-major scalings, cubic size factors, partitions): the oracle's
    clause-learning solver decides the product's CNF and the oracle's own
    encoding of the same query, and the two verdicts agree wherever both
    are decided; every SAT model of the product CNF passes the host
    re-verification against the integer constraints."""
    import oracle
    irs, meta = queries.config3(400)
    enc = B.scuba_encode_batch(irs)
    nc = np.diff(enc.inst_clause_begin)
    sel = np.argsort(nc, kind="stable")[:48]          # the smallest, every width
    cnfs = []
    for i in sel:
        c0, c1 = enc.inst_clause_begin[i], enc.inst_clause_begin[i + 1]
        l0 = enc.clause_begin[c0]
        cnfs.append(oracle.CNF(int(enc.inst_num_vars[i]), enc.clause_begin[c0:c1 + 1] - l0,
                               enc.lits[l0:enc.clause_begin[c1]]))
    prod = oracle.solve_cnfs(cnfs, budget=20000, algo="cdcl")["verdict"]
    own = oracle.solve_queries([irs[i] for i in sel], budget=20000, algo="cdcl")["verdict"]
    both = (prod != 2) & (own != 2)
    assert both.sum() >= 40
    assert (prod[both] == own[both]).all()
    assert {0, 1} <= set(own[both].tolist())
    # models of the product CNF, decoded through its input map, satisfy the query
    verdict = np.full(enc.n, 2, np.uint8)
    model = np.zeros(enc.total_vars, np.uint8)
    for k, i in enumerate(sel):
        if prod[k] == 1:
            r = oracle.cdcl(cnfs[k])
            verdict[i] = 1
            vb = enc.inst_var_begin[i]
            model[vb:vb + enc.inst_num_vars[i]] = r["model"][:enc.inst_num_vars[i]]
    fails, ok = B.scuba_verify_batch(enc, verdict, model)
    assert fails == 0 and (ok[sel][prod == 1] == 1).all()
