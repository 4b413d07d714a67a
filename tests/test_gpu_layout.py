"""The layout and scope check on the GPU (spv_layout_batch) against the
oracle, module by module: generated batches (clean), hand-built modules with
every error kind, random instruction-level edits of real modules (moved,
deleted and duplicated instructions), framing faults, and a module of
hundreds of thousands of rows."""
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


def run_layout(gpu, words, offs):
    w = torch.from_numpy(np.ascontiguousarray(words, np.uint32).view(np.int32)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(offs, np.int64)).cuda()
    r = gpu.decode(w, o)
    st, er = gpu.layout(r["table"], len(offs) - 1)
    torch.cuda.synchronize()
    return st.cpu().numpy().view(np.uint32), er.cpu().numpy()


def check(gpu, words, offs):
    st, er = run_layout(gpu, words, offs)
    ost, oer = oracle.layout(words, offs)
    bad = np.nonzero((st != ost) | (er != oer))[0]
    assert len(bad) == 0, [(int(i), gpu.LAYOUT_STATUS[st[i]], int(er[i]), oracle.LAYOUT_STATUS[ost[i]], int(oer[i]))
                           for i in bad[:10]]
    return st


def instructions(words):
    out, p = [], 5
    while p < len(words):
        wc = int(words[p]) >> 16
        out.append(list(words[p:p + wc]))
        p += wc
    return out


def test_generated_batch_is_clean(gpu):
    w, off = synth.module_batch(200, 3)
    st = check(gpu, w, off)
    assert (st == 0).all()


def test_hand_built_error_kinds(gpu):
    b = H.minimal_body()
    mods = [H.module(b, bound=40),
            H.module(b[:1] + [b[2], b[1]] + b[3:], bound=40),
            H.module(b + [H.ins(H.OpTypeFloat, 30, 32)], bound=40),
            H.module(b[:7] + [H.ins(H.OpIAdd, 2, 30, 4, 4)] + b[7:], bound=40),
            H.module(b[:10] + [H.ins(H.OpTypeInt, 30, 64, 0)] + b[10:], bound=40),
            H.module(b[:10] + [H.ins(H.OpFunction, 1, 30, 0, 3)] + b[10:], bound=40),
            H.module(b[:9] + [H.ins(H.OpIAdd, 2, 30, 4, 4)] + b[9:], bound=40),
            H.module(b[:11] + b[12:], bound=40),
            H.module(b[:12] + [H.ins(H.OpIAdd, 2, 30, 4, 4)] + b[12:], bound=40),
            H.module(b[:10] + [H.ins(H.OpLabel, 30)] + b[10:], bound=40),
            H.module(b[:10] + [H.ins(H.OpFunctionParameter, 2, 30)] + b[10:], bound=40),
            H.module(b[:12], bound=40), H.module(b[:11], bound=40),
            H.module([], bound=1), H.module(b, bound=8)[:3]]
    words, offs = H.batch(mods)
    st = check(gpu, words, offs)
    assert sorted(set(int(x) for x in st)) == [0, 1, 2, 3, 4, 5]


def test_random_edits_of_real_modules(gpu):
    rng = np.random.default_rng(9)
    w, off = synth.module_batch(40, 11)
    mods = []
    for k in range(400):
        src = w[off[k % 40]:off[k % 40 + 1]]
        ins = instructions(src)
        for _ in range(int(rng.integers(1, 4))):
            kind = int(rng.integers(0, 3))
            i = int(rng.integers(0, len(ins)))
            if kind == 0 and len(ins) > 1:
                del ins[i]
            elif kind == 1:
                ins.insert(int(rng.integers(0, len(ins))), ins[i])
            else:
                j = int(rng.integers(0, len(ins)))
                ins.insert(j, ins.pop(i))
        mods.append(np.array(list(src[:5]) + [x for i_ in ins for x in i_], np.uint32))
    words, offs = H.batch(mods)
    st = check(gpu, words, offs)
    assert len(set(int(x) for x in st)) >= 4          # the edits reach several kinds


def test_framing_faults_and_empty_batch(gpu):
    w, off = synth.module_batch(20, 13)
    mods = [w[off[i]:off[i + 1]].copy() for i in range(20)]
    for i in range(0, 20, 3):
        mods[i] = mods[i][:len(mods[i]) // 2]          # cut mid-module: rows end inside a function
    for i in range(1, 20, 4):
        mods[i][5 + 3 * i] &= 0xffff                   # word count 0: decoding stops there
    words, offs = H.batch(mods)
    check(gpu, words, offs)
    st, er = run_layout(gpu, np.zeros(0, np.uint32), np.zeros(1, np.int64))
    assert len(st) == 0


def test_large_module(gpu):
    w, off, _, _ = synth.large_module(2, n_instr=400_000, n_funcs=50)
    st = check(gpu, w, off)
    assert int(st[0]) == 0


def test_segmented_modules(gpu):
    """Modules of more than 16,384 rows are checked in segments: errors in a
    middle segment, right at segment starts and ends, in the last segment,
    and a large module that ends inside a function, between small modules."""
    big, boff, _, _ = synth.large_module(5, n_instr=120_000, n_funcs=10)
    ins = instructions(big)
    small, soff = synth.module_batch(4, 17)
    smalls = [small[soff[i]:soff[i + 1]] for i in range(4)]

    def rebuild(rows):
        return H.module(rows, bound=int(big[3]), generator=int(big[2]))

    variants = [ins]
    for at in (16_384 - 1, 16_384, 32_768 + 7, 70_001, len(ins) - 3):
        v = list(ins)
        v.insert(at, H.ins(H.OpTypeVoid, 3))          # a type inside a function
        variants.append(v)
    v = list(ins)
    v.insert(16_384 * 3, H.ins(H.OpLabel, 3))         # a label in an open block, at a segment start
    variants.append(v)
    variants.append(list(ins)[:50_000])               # the rows end inside a function
    mods = []
    for k, rows in enumerate(variants):
        mods.append(smalls[k % 4])
        mods.append(rebuild(rows))
    words, offs = H.batch(mods)
    st = check(gpu, words, offs)
    assert (st[1::2] != 0).sum() == len(variants) - 1
