"""The batched GPU builder (spv_build_batch) against the oracle: words, word
offsets, statuses, first bad rows and each row's id, element by element, on
generated op lists (a JIT backend's rows for the batch recipe), hand-built
lists, lists with planted faults (references out of the module or to rows
without a result, result types missing, instructions too long), and the edge
cases (empty batch, empty modules, rows before the first module, bad offsets,
a word capacity below the total), and at the full batch size."""
import numpy as np
import pytest

import oracle
from paper_2305_09493_b300 import synth
from tests import spvhand as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    from paper_2305_09493_b300 import build, spvgpu
    build.build()
    spvgpu.load()
    return spvgpu


def _dev(ol):
    return (torch.from_numpy(np.ascontiguousarray(ol["op"], np.uint16).view(np.int16)).cuda(),
            torch.from_numpy(np.ascontiguousarray(ol["opd_off"], np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(ol["opd"], np.uint32).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(ol["opd_ref"], np.uint8)).cuda(),
            torch.from_numpy(np.ascontiguousarray(ol["row_off"], np.int64)).cuda())


def _run(gpu, ol, **kw):
    w, woff, st, err, ids = gpu.build_modules(*_dev(ol), **kw)
    torch.cuda.synchronize()
    return (w.cpu().numpy().view(np.uint32), woff.cpu().numpy(), st.cpu().numpy().view(np.uint32),
            err.cpu().numpy(), ids.cpu().numpy().view(np.uint32))


def _check(gpu, ol, version=0x00010200, generator=0):
    want = oracle.build_batch(ol, version, generator)
    got = _run(gpu, ol, version=version, generator=generator)
    for name, a, b in zip(("words", "word_off", "status", "err_row", "ids"), got, want):
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0][:8] if a.shape == b.shape else "shape"
            raise AssertionError(f"{name} differs at {bad}")
    return got


def _cat(lists):
    """Several op lists as one batch (operand and row offsets rebased)."""
    op, opd, ref = [], [], []
    flat_off, flat_roff = [np.array([0], np.int64)], [np.array([0], np.int64)]
    run_opd, run_rows = 0, 0
    for ol in lists:
        o0, o1 = int(ol["opd_off"][0]), int(ol["opd_off"][-1])
        op.append(ol["op"])
        opd.append(ol["opd"][o0:o1])
        ref.append(ol["opd_ref"][o0:o1])
        flat_off.append(ol["opd_off"][1:] - o0 + run_opd)
        flat_roff.append(ol["row_off"][1:] - ol["row_off"][0] + run_rows)
        run_opd += o1 - o0
        run_rows += int(ol["row_off"][-1] - ol["row_off"][0])
    return {"op": np.concatenate(op).astype(np.uint16), "opd_off": np.concatenate(flat_off),
            "opd": np.concatenate(opd).astype(np.uint32), "opd_ref": np.concatenate(ref).astype(np.uint8),
            "row_off": np.concatenate(flat_roff)}


def _rows(rows):
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


def R(k):
    return ("r", k)


def test_generated_op_lists(gpu):
    n_instr, n_k = synth.batch_shape(60, 31, median=700, lo=200, hi=6000)
    ol = synth.oplist_batch(n_instr, n_k, 31)
    w, woff, st, _, _ = _check(gpu, ol, 0x00010200, 32)
    assert (st == 0).all() and np.array_equal(woff, ol["mod_off"])


def test_hand_built_and_faulty_lists(gpu):
    cases = [
        [(H.OpCapability, [c]) for c in (4, 5, 6, 11, 39)],
        [(H.OpTypeInt, [32, 0]), (H.OpConstant, [R(0), 5]), (H.OpConstant, [R(0), 7]), (H.OpIAdd, [R(0), R(1), R(2)])],
        [(H.OpCapability, [6]), (H.OpTypeBool, []), (41, [R(1)]), (250, [R(2), R(5), R(7)]), (H.OpNop, []),
         (H.OpLabel, []), (H.OpReturn, []), (H.OpLabel, []), (H.OpReturn, [])],
        [(300, [1, 2, 3]), (H.OpTypeVoid, []), (301, [R(1), 9])],
        [],
        [(H.OpTypeVoid, []), (H.OpIAdd, [])],
        [(H.OpTypeVoid, []), (H.OpName, [R(2), 0])],
        [(H.OpCapability, [6]), (H.OpName, [R(0), 0])],
        [(H.OpTypeVoid, []), (H.OpName, [R(0), 0]), (H.OpIAdd, [])],
        [(H.OpTypeVoid, []), (H.OpName, [R(5), 0]), (H.OpIAdd, [])],
        [(H.OpIAdd, [R(9), R(9)])],
        [(H.OpTypeVoid, []), (H.OpName, [R(0)] + [0] * 65533)],
        [(H.OpTypeVoid, []), (H.OpName, [R(0)] + [0] * 65534)],
    ]
    ol = _cat([_rows(c) for c in cases])
    _, _, st, err, _ = _check(gpu, ol, 0x00010500, 7)
    assert list(st) == [0, 0, 0, 0, 0, 2, 1, 1, 2, 1, 1, 0, 2]


def test_planted_faults(gpu):
    rng = np.random.default_rng(5)
    n_instr, n_k = synth.batch_shape(80, 32, median=300, lo=100, hi=1500)
    ol = synth.oplist_batch(n_instr, n_k, 32)
    ol = {k: v.copy() for k, v in ol.items()}
    refs = np.nonzero(ol["opd_ref"])[0]
    for k in rng.choice(refs, 40, replace=False):              # references out of the module / to any row
        ol["opd"][k] = int(rng.integers(0, 3000))
    lits = np.nonzero(ol["opd_ref"] == 0)[0]
    for k in rng.choice(lits, 20, replace=False):              # literals turned into references
        ol["opd_ref"][k] = 1
        ol["opd"][k] = int(rng.integers(0, 50))
    _, _, st, _, _ = _check(gpu, ol)
    assert (st == 1).sum() >= 10 and (st == 0).sum() >= 10


def test_rows_before_the_first_module_and_capacity(gpu):
    n_instr, n_k = synth.batch_shape(8, 33, median=400, lo=200, hi=1000)
    ol = synth.oplist_batch(n_instr, n_k, 33)
    # the batch's modules start at row 7: rows 0..6 belong to no module
    first = int(ol["row_off"][1])
    ol2 = dict(ol)
    ol2["row_off"] = np.concatenate([[7], ol["row_off"][1:]]).astype(np.int64)
    want = oracle.build_batch(ol2)
    got = _run(gpu, ol2)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[2], want[2])
    assert np.array_equal(got[4][7:], want[4][7:])
    assert first > 7
    # a word capacity below the total: nothing written past it, offsets filled
    dev = _dev(ol)
    w_o, woff_o = oracle.build_batch(ol)[:2]
    for cap in (0, 3, len(w_o) // 2, len(w_o) - 1):
        out = torch.full((cap + 64,), -1, dtype=torch.int32, device="cuda")
        words, woff, _, _, _ = gpu.build_modules(*dev, words=out[:cap] if cap else out[:0], sync=False)
        torch.cuda.synchronize()
        assert np.array_equal(woff.cpu().numpy(), woff_o)
        o = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(o[:cap], w_o[:cap]) and (o[cap:] == 0xffffffff).all()


def test_empty_batch_and_bad_offsets(gpu):
    z = {"op": np.zeros(0, np.uint16), "opd_off": np.zeros(1, np.int64), "opd": np.zeros(0, np.uint32),
         "opd_ref": np.zeros(0, np.uint8), "row_off": np.zeros(1, np.int64)}
    w, woff, st, _, _ = _run(gpu, z)
    assert len(w) == 0 and list(woff) == [0]
    ol = _cat([_rows([(H.OpTypeVoid, []), (H.OpName, [R(0), 0])]), _rows([(H.OpCapability, [6])])])
    for bad in ({"row_off": np.array([0, 3, 2], np.int64)}, {"row_off": np.array([0, 2, 9], np.int64)},
                {"opd_off": np.array([0, 0, 2, 1], np.int64)}):
        b = dict(ol)
        b.update(bad)
        w, woff, st, _, _ = _run(gpu, b)
        assert (st == 3).all() and len(w) == 0


def test_full_batch(gpu):
    """The 10,000-module batch's op lists: every word, offset, status and id
    equal to the oracle's."""
    ol = synth.oplist_module_batch(10000, 0)
    _check(gpu, ol, 0x00010200, 32)
