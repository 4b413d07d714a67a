"""Pins of the oracle's builder (section 3.4.2, "Enabling Function
Composition": instructions added in order, each result taking the module's
next id), independent of the oracle:

* the paper's worked example: the capabilities listing built from five rows
  gives the hand-written words of tests/golden/listing8_capabilities.json,
  whose disassembly is the printed listing;
* the addition example and a branch with forward references to labels,
  words written out by hand;
* every error kind with its row;
* generated op lists (a JIT backend's rows for the batch recipe's modules):
  the built module is the generated module up to a renaming of ids, the
  renaming is one-to-one, and the decoded result ids run 1, 2, 3, ... in
  row order (the decoder and the id-word mask are independent of the
  builder).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2305_09493_b300 import synth
from tests import spvhand as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def oplist(rows):
    """rows: [(opcode, [operand, ...])], an operand int = literal, ("r", k) = a
    reference to row k of the module."""
    op, off, opd, ref = [], [0], [], []
    for o, ops in rows:
        op.append(o)
        for x in ops:
            if isinstance(x, tuple):
                opd.append(x[1]); ref.append(1)
            else:
                opd.append(x); ref.append(0)
        off.append(len(opd))
    return {"op": np.array(op, np.uint16), "opd_off": np.array(off, np.int64), "opd": np.array(opd, np.uint32),
            "opd_ref": np.array(ref, np.uint8), "row_off": np.array([0, len(op)], np.int64)}


def build(rows, **kw):
    w, woff, st, err, ids = oracle.build_batch(oplist(rows), **kw)
    return [int(x) for x in w], int(st[0]), int(err[0]), [int(x) for x in ids]


def R(k):
    return ("r", k)


def test_capabilities_listing():
    g = json.load(open(os.path.join(GOLDEN, "listing8_capabilities.json")))
    rows = [(H.OpCapability, [c]) for c in (H.CAP_ADDRESSES, H.CAP_LINKAGE, H.CAP_KERNEL, H.CAP_INT64, H.CAP_INT8)]
    w, st, err, _ = build(rows, version=0x00010200, generator=32)
    assert st == 0 and err == -1
    assert w == [int(x, 16) for x in g["words"]]
    text, _ = oracle.disassemble(np.array(w, np.uint32), np.array([0, len(w)], np.int64), True, False)
    assert text.decode() == g["text"]


def test_addition_example():
    # %1 = OpTypeInt 32 0; %2 = OpConstant %1 5; %3 = OpConstant %1 7;
    # %4 = OpIAdd %1 %2 %3 (result type first, then the new result id)
    rows = [(H.OpTypeInt, [32, 0]), (H.OpConstant, [R(0), 5]), (H.OpConstant, [R(0), 7]),
            (H.OpIAdd, [R(0), R(1), R(2)])]
    w, st, err, ids = build(rows)
    assert st == 0 and ids == [1, 2, 3, 4]
    want = H.module([H.ins(H.OpTypeInt, 1, 32, 0), H.ins(H.OpConstant, 1, 2, 5), H.ins(H.OpConstant, 1, 3, 7),
                     H.ins(H.OpIAdd, 1, 4, 2, 3)], bound=5, generator=0)
    assert w == list(want)


def test_forward_references_and_rows_without_results():
    # a conditional branch names both labels before they are added (the
    # paper's if-else composition); rows without a result take no id
    rows = [(H.OpCapability, [H.CAP_KERNEL]),          # 0
            (H.OpTypeBool, []),                          # 1 -> %1
            (41, [R(1)]),                                # 2 OpConstantTrue -> %2
            (250, [R(2), R(5), R(7)]),                   # 3 OpBranchConditional %2 %3 %4
            (H.OpNop, []),                               # 4
            (H.OpLabel, []),                             # 5 -> %3
            (H.OpReturn, []),                            # 6
            (H.OpLabel, []),                             # 7 -> %4
            (H.OpReturn, [])]                            # 8
    w, st, err, ids = build(rows)
    assert st == 0 and ids == [0, 1, 2, 0, 0, 3, 0, 4, 0]
    want = H.module([H.ins(H.OpCapability, H.CAP_KERNEL), H.ins(H.OpTypeBool, 1), H.ins(41, 1, 2),
                     H.ins(250, 2, 3, 4), H.ins(H.OpNop), H.ins(H.OpLabel, 3), H.ins(H.OpReturn),
                     H.ins(H.OpLabel, 4), H.ins(H.OpReturn)], bound=5, generator=0)
    assert w == list(want)


def test_unknown_opcodes_and_literals():
    # an opcode outside the table has no result id; its operands are copied
    rows = [(300, [1, 2, 3]), (H.OpTypeVoid, []), (301, [R(1), 9])]
    w, st, err, ids = build(rows, version=0x00010500, generator=7)
    assert st == 0 and ids == [0, 1, 0]
    assert w == [H.MAGIC, 0x00010500, 7, 2, 0, (4 << 16) | 300, 1, 2, 3, (2 << 16) | 19, 1, (3 << 16) | 301, 1, 9]


@pytest.mark.parametrize("rows,want", [
    ([(H.OpTypeVoid, []), (H.OpIAdd, [])], ("BAD_ROW", 1)),                          # no result type
    ([(H.OpTypeVoid, []), (H.OpName, [R(2), 0])], ("BAD_REF", 1)),                   # outside the module
    ([(H.OpCapability, [6]), (H.OpName, [R(0), 0])], ("BAD_REF", 1)),                # a row without result
    ([(H.OpTypeVoid, []), (H.OpName, [R(0), 0]), (H.OpIAdd, [])], ("BAD_ROW", 2)),   # first bad row wins
    ([(H.OpTypeVoid, []), (H.OpName, [R(5), 0]), (H.OpIAdd, [])], ("BAD_REF", 1)),
    ([(H.OpIAdd, [R(9), R(9)])], ("BAD_REF", 0)),                                    # the checks of one row
    ([(H.OpTypeVoid, []), (H.OpName, [R(0)] + [0] * 65533)], ("OK", -1)),           # 65535 words
    ([(H.OpTypeVoid, []), (H.OpName, [R(0)] + [0] * 65534)], ("BAD_ROW", 1)),       # 65536 words
])
def test_errors(rows, want):
    w, st, err, _ = build(rows)
    assert (oracle.BUILD_STATUS[st], err) == want
    if st:
        assert w == []


def test_generated_op_lists_build_the_modules_up_to_id_renaming():
    d = synth.oplist_module_batch(40, 21)
    w, woff, st, err, ids = oracle.build_batch(d, version=0x00010200, generator=32)
    assert (st == 0).all()
    assert np.array_equal(woff, d["mod_off"])
    orig, mask = d["words"], d["is_id"].astype(bool)
    for m in range(len(woff) - 1):
        a, b = woff[m], woff[m + 1]
        o, n, k = orig[a:b], w[a:b], mask[a:b]
        # the same words except ids; header words but the bound equal
        assert np.array_equal(o[~k][5:], n[~k][5:]) and np.array_equal(o[[0, 1, 2, 4]], n[[0, 1, 2, 4]])
        # the ids: a one-to-one renaming
        pairs = set(zip(o[k].tolist(), n[k].tolist()))
        assert len({p[0] for p in pairs}) == len(pairs) == len({p[1] for p in pairs})
        # the decoder's result ids run 1, 2, 3, ... in row order; bound = count + 1
        dec = oracle.decode(n, np.array([0, b - a], np.int64))
        rid = dec["rid"][:dec["n_rows"]]
        rid = rid[rid != 0]
        assert np.array_equal(rid, np.arange(1, len(rid) + 1)) and n[3] == len(rid) + 1


def test_several_modules_and_an_empty_one():
    d = synth.oplist_module_batch(5, 22)
    # an empty module (no rows) between others
    d2 = dict(d)
    d2["row_off"] = np.concatenate([d["row_off"][:3], d["row_off"][2:]])
    w, woff, st, err, ids = oracle.build_batch(d2)
    assert list(st) == [0] * 6
    assert woff[3] - woff[2] == 5                      # header only, bound 1
    assert list(w[woff[2]:woff[3]]) == [H.MAGIC, 0x00010200, 0, 1, 0]
