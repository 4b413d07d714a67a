"""Pins of the oracle's logical-layout and scope check (section 3.4.1
scopes: module, function, block), independent of the oracle itself:

* hand-built modules, one per error kind, with the expected status and row
  worked out by hand;
* generated modules, which the generator writes in layout order, are clean;
* brute force against a second, independent statement of the same rules: a
  regular grammar over one letter per row. A row sequence is clean exactly
  when the grammar matches it whole, and the first error is at the end of
  the longest prefix that can still be extended to a match.
"""
import numpy as np
import pytest

import oracle
from paper_2305_09493_b300 import synth
from tests import spvhand as H

regex = pytest.importorskip("regex")

OpTypeVoid, OpTypeInt, OpTypeFloat, OpConstant = H.OpTypeVoid, H.OpTypeInt, H.OpTypeFloat, H.OpConstant
OpFunction, OpFunctionParameter, OpFunctionEnd = H.OpFunction, H.OpFunctionParameter, H.OpFunctionEnd
OpLabel, OpReturn, OpIAdd, OpVariable, OpBranch = H.OpLabel, H.OpReturn, H.OpIAdd, H.OpVariable, H.OpBranch
OpNop = H.OpNop


def lay(body, bound=40):
    m = H.module(body, bound=bound)
    st, er = oracle.layout(m, np.array([0, len(m)], np.int64))
    return oracle.LAYOUT_STATUS[int(st[0])], int(er[0])


def base():
    return H.minimal_body()     # rows 0..12: caps, memory model, entry point, types, constant, function


def test_clean_modules():
    assert lay(base()) == ("OK", -1)
    b = base()                                           # a declaration: OpFunction, OpFunctionEnd
    b[8:13] = [H.ins(OpFunction, 1, 5, 0, 3), H.ins(OpFunctionEnd)]
    assert lay(b) == ("OK", -1)
    b = base()                                           # a global variable among the types, a local one in a block
    b.insert(7, H.ins(OpVariable, 2, 20, 5))
    b.insert(11, H.ins(OpVariable, 2, 21, 7))
    assert lay(b) == ("OK", -1)
    b = base() + [H.ins(OpFunction, 1, 22, 0, 3), H.ins(OpLabel, 23), H.ins(OpReturn), H.ins(OpFunctionEnd)]
    assert lay(b) == ("OK", -1)                           # two functions
    b = base()
    b.insert(0, H.ins(OpNop)); b.insert(10, H.ins(OpNop))  # OpNop anywhere
    assert lay(b) == ("OK", -1)
    b = base()                                           # two blocks
    b[11:12] = [H.ins(OpBranch, 24), H.ins(OpLabel, 24), H.ins(OpReturn)]
    assert lay(b) == ("OK", -1)


@pytest.mark.parametrize("edit,want", [
    # a capability after the memory model (row 2 -> row 3 position)
    (lambda b: b[:1] + [b[2], b[1]] + b[3:], ("SECTION_ORDER", 2)),
    # a type after the function
    (lambda b: b + [H.ins(OpTypeFloat, 30, 32)], ("SECTION_ORDER", 13)),
    # an arithmetic instruction at module scope
    (lambda b: b[:7] + [H.ins(OpIAdd, 2, 30, 4, 4)] + b[7:], ("OUTSIDE_FUNCTION", 7)),
    # a type inside a block
    (lambda b: b[:10] + [H.ins(OpTypeInt, 30, 64, 0)] + b[10:], ("IN_FUNCTION", 10)),
    # a function opened inside a block
    (lambda b: b[:10] + [H.ins(OpFunction, 1, 30, 0, 3)] + b[10:], ("IN_FUNCTION", 10)),
    # a body instruction before the first label
    (lambda b: b[:9] + [H.ins(OpIAdd, 2, 30, 4, 4)] + b[9:], ("BLOCK", 9)),
    # no terminator: OpFunctionEnd in an open block
    (lambda b: b[:11] + b[12:], ("BLOCK", 11)),
    # an instruction after the terminator
    (lambda b: b[:12] + [H.ins(OpIAdd, 2, 30, 4, 4)] + b[12:], ("BLOCK", 12)),
    # a label in an open block
    (lambda b: b[:10] + [H.ins(OpLabel, 30)] + b[10:], ("BLOCK", 10)),
    # a parameter after the label
    (lambda b: b[:10] + [H.ins(OpFunctionParameter, 2, 30)] + b[10:], ("BLOCK", 10)),
    # a parameter at module scope
    (lambda b: b[:7] + [H.ins(OpFunctionParameter, 2, 30)] + b[7:], ("OUTSIDE_FUNCTION", 7)),
    # a function variable before the first label
    (lambda b: b[:9] + [H.ins(OpVariable, 2, 30, 7)] + b[9:], ("BLOCK", 9)),
    # the rows end inside the function (no OpFunctionEnd): row = the row count
    (lambda b: b[:12], ("UNCLOSED", 12)),
    # ... or inside a block
    (lambda b: b[:11], ("UNCLOSED", 11)),
])
def test_each_error_kind(edit, want):
    assert lay(edit(base())) == want


def test_generated_modules_are_clean():
    w, off = synth.module_batch(30, 7)
    st, er = oracle.layout(w, off)
    assert (st == 0).all() and (er == -1).all()
    w, off, _, _ = synth.large_module(3, n_instr=30_000, n_funcs=5)
    st, er = oracle.layout(w, off)
    assert int(st[0]) == 0


# ---------------------------------------------------------------------------
# brute force against an independent grammar
# ---------------------------------------------------------------------------
# one letter per row: '1'..'9' module sections, 'v' a variable (global at
# module scope, body in a function), 'F' OpFunction, 'P' parameter, 'E'
# OpFunctionEnd, 'L' label, 'T' terminator, 'B' body instruction
ROW = {
    "1": H.ins(H.OpCapability, H.CAP_KERNEL), "4": H.ins(H.OpMemoryModel, H.AM_PHYSICAL64, H.MM_OPENCL),
    "5": H.ins(H.OpEntryPoint, H.EXEC_KERNEL, 5, H.s("k")), "7": H.ins(H.OpName, 2, H.s("n")),
    "8": H.ins(H.OpDecorate, 2, 44, 4), "9": H.ins(OpTypeInt, 2, 32, 0), "v": H.ins(OpVariable, 2, 20, 7),
    "F": H.ins(OpFunction, 1, 5, 0, 3), "P": H.ins(OpFunctionParameter, 2, 21), "E": H.ins(OpFunctionEnd),
    "L": H.ins(OpLabel, 6), "T": H.ins(OpReturn), "B": H.ins(OpIAdd, 2, 7, 4, 4),
}
GRAMMAR = regex.compile(r"1*4*5*7*8*[9v]*(?:FP*(?:E|(?:L[Bv]*T)+E))*")


def expect(letters):
    if GRAMMAR.fullmatch(letters):
        return "OK", -1
    k = max(i for i in range(len(letters) + 1) if GRAMMAR.fullmatch(letters[:i], partial=True))
    return ("UNCLOSED" if k == len(letters) else "error"), k


def test_brute_force_against_the_grammar():
    rng = np.random.default_rng(5)
    alphabet = list(ROW)
    valid = "1145789v9FPLBvBTLBTEFE"
    cases = [valid]
    for n in range(1, 7):                               # short sequences of every mix
        for _ in range(300):
            cases.append("".join(rng.choice(alphabet, n)))
    for _ in range(600):                                # single edits of a valid module
        s = list(valid)
        i = int(rng.integers(0, len(s)))
        op = int(rng.integers(0, 3))
        if op == 0:
            del s[i]
        elif op == 1:
            s.insert(i, str(rng.choice(alphabet)))
        else:
            j = int(rng.integers(0, len(s)))
            s[i], s[j] = s[j], s[i]
        cases.append("".join(s))
    for letters in cases:
        want_kind, want_row = expect(letters)
        got, row = lay([ROW[c] for c in letters])
        if want_kind == "OK":
            assert (got, row) == ("OK", -1), letters
        elif want_kind == "UNCLOSED":
            assert (got, row) == ("UNCLOSED", len(letters)), letters
        else:
            assert got not in ("OK", "UNCLOSED") and row == want_row, (letters, got, row, want_row)
