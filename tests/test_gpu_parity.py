"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and string work: every comparison is exact (tables, statuses, error
rows, encoded words, disassembly bytes)."""
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


def dev(words, mod_off):
    w = torch.from_numpy(np.ascontiguousarray(words, np.uint32).view(np.int32)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(mod_off, np.int64)).cuda()
    return w, o


def run(gpu, words, mod_off, cfg=None, validate=True, encode=True, **kw):
    w, o = dev(words, mod_off)
    r = gpu.process(w, o, validate=validate, encode=encode, cfg=cfg, **kw)
    torch.cuda.synchronize()
    m = len(mod_off) - 1
    out = {
        "table": r["table"].to_numpy(),
        "status": r["status"].cpu().numpy().view(np.uint32)[:m],
        "err_row": r["err_row"].cpu().numpy()[:m],
        "out": r["out"].cpu().numpy().view(np.uint32) if encode else None,
        "_r": r, "_w": w, "_o": o,
    }
    return out


def assert_table_equal(t, d, m):
    n = d["n_rows"]
    assert int(t["first_row"][m]) == n
    for k in ("op", "wc", "off", "rtype", "rid", "mod"):
        assert np.array_equal(t[k][:n], d[k]), k
    assert np.array_equal(t["first_row"][:m], d["first_row"])
    assert np.array_equal(t["n_instr"][:m], d["n_instr"])


def check(gpu, words, mod_off, cfg=None, dis=False):
    m = len(mod_off) - 1
    g = run(gpu, words, mod_off, cfg)
    d = oracle.decode(words, mod_off)
    assert_table_equal(g["table"], d, m)
    st, er = oracle.validate(words, mod_off)
    bad = np.nonzero((g["status"] != st) | (g["err_row"] != er))[0]
    assert len(bad) == 0, [(int(i), oracle.STATUS[st[i]], int(er[i]), gpu.STATUS[g["status"][i]], int(g["err_row"][i]))
                           for i in bad[:10]]
    assert np.array_equal(g["out"], oracle.encode(words, mod_off, d, True))
    # decode-only statuses (header / framing)
    g2 = run(gpu, words, mod_off, cfg, validate=False, encode=False)
    assert np.array_equal(g2["status"], d["status"])
    assert np.array_equal(g2["err_row"], d["err_row"])
    if dis:
        check_dis(gpu, words, mod_off, g)
    return g


def check_dis(gpu, words, mod_off, g, modes=((True, True), (False, False), (True, False))):
    for inline, header in modes:
        text, toff, dst = gpu.disassemble(g["_w"], g["_o"], g["_r"]["table"], inline_names=inline, header=header)
        torch.cuda.synchronize()
        want, woff = oracle.disassemble(words, mod_off, inline, header)
        got = text.cpu().numpy().tobytes()
        if got != want:
            i = next(k for k in range(min(len(got), len(want))) if got[k] != want[k]) if got[:len(want)] != want[:len(got)] else min(len(got), len(want))
            raise AssertionError(f"text differs at byte {i}: got {got[max(0,i-80):i+80]!r} want {want[max(0,i-80):i+80]!r}")
        assert np.array_equal(toff.cpu().numpy(), woff)


# ---------------------------------------------------------------------------
def test_single_modules(gpu):
    for seed in range(4):
        w, off, _, _ = synth.single_module(seed)
        check(gpu, w, off, dis=True)


def test_small_batch_ragged(gpu):
    n_instr, n_k = synth.batch_shape(300, 11, median=1500, lo=200, hi=20000)
    w, off = synth.batch(n_instr, n_k, 11)
    check(gpu, w, off, dis=True)


@pytest.mark.parametrize("tile,threads", [(4096, 256), (8192, 512), (2048, 256), (2048, 128), (1024, 128), (512, 64)])
def test_tile_configs(gpu, tile, threads):
    n_instr, n_k = synth.batch_shape(60, 3, median=3000, lo=200, hi=30000)
    w1, off1 = synth.batch(n_instr, n_k, 3)
    w2, off2, _, _ = synth.large_module(9, n_instr=150_000, n_funcs=20)
    words = np.concatenate([w1, w2])
    offs = np.concatenate([off1, off1[-1] + off2[1:]])
    check(gpu, words, offs, cfg=gpu.make_config(tile_words=tile, threads=threads), dis=(tile == 2048 and threads == 128))


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_word_buffer_off_a_16_byte_boundary(gpu, shift):
    """The word buffer starts 4, 8 or 12 bytes past a 16-byte boundary (a view
    into a larger allocation), so every module's tiles are staged with a
    different phase and the encoded words (in a buffer of another phase) are
    stored word by word; exact against the oracle."""
    n_instr, n_k = synth.batch_shape(30, 21, median=2000, lo=200, hi=20000)
    w, off = synth.batch(n_instr, n_k, 21)
    big = torch.zeros(len(w) + 8, dtype=torch.int32, device="cuda")
    wt = big[shift:shift + len(w)]
    wt.copy_(torch.from_numpy(w.view(np.int32)))
    assert wt.data_ptr() % 16 == 4 * shift
    o = torch.from_numpy(off).cuda()
    for cfg in (None, gpu.make_config(tile_words=2048, threads=128), gpu.make_config(tile_words=512, threads=64)):
        r = gpu.process(wt, o, validate=True, encode=True, cfg=cfg)
        torch.cuda.synchronize()
        d = oracle.decode(w, off)
        assert_table_equal(r["table"].to_numpy(), d, len(off) - 1)
        st, er = oracle.validate(w, off)
        assert np.array_equal(r["status"].cpu().numpy().view(np.uint32), st)
        assert np.array_equal(r["err_row"].cpu().numpy(), er)
        assert np.array_equal(r["out"].cpu().numpy().view(np.uint32), oracle.encode(w, off, d, True))


def test_entry_guesses_and_their_redo_match_the_oracle(gpu):
    """Tiles after a module's first take their first guessed instruction start
    as their entry and check it against the predecessor's exit afterwards; a
    framing error (a zero word count or an overrunning word count) early in a
    long module makes the later tiles' guesses wrong, and the call redoes the
    batch without guesses. Either way, and with guessing off, the results are
    the oracle's."""
    n_instr, n_k = synth.batch_shape(24, 31, median=8000, lo=2000, hi=40000)
    w, off = synth.batch(n_instr, n_k, 31)
    w = w.copy()
    rng = np.random.default_rng(8)
    for m in range(0, 24, 3):
        lo, hi = int(off[m]) + 5, int(off[m + 1])
        starts = oracle.decode(w[off[m]:off[m + 1]], np.array([0, hi - lo + 5], np.int64))["off"]
        p = int(off[m]) + int(starts[len(starts) // 8])
        w[p] = (w[p] & 0xffff) | ((0 if m % 2 else 0xfff0) << 16)    # zero word count / overrun
    for cfg in (None, gpu.make_config(no_speculation=1), gpu.make_config(tile_words=2048, threads=128)):
        check(gpu, w, off, cfg=cfg)
    n_instr, n_k = synth.batch_shape(30, 33, median=6000, lo=2000, hi=30000)
    w2, off2 = synth.batch(n_instr, n_k, 33)
    a = run(gpu, w2, off2)
    b = run(gpu, w2, off2, cfg=gpu.make_config(no_speculation=1))
    assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["out"], b["out"])
    for k in ("op", "wc", "off", "rtype", "rid", "mod", "first_row", "n_instr"):
        assert np.array_equal(a["table"][k], b["table"][k]), k


def _literal_module(pattern, n_pad, width=32):
    """The minimal module with n_pad 32-bit constants, then one constant whose
    literal words are `pattern` (of an integer type `width` bits wide), ahead
    of the function."""
    base = H.minimal_body()
    body = list(base[:8])
    ty = 2
    if width != 32:
        ty = 9
        body.append(H.ins(H.OpTypeInt, ty, width, 0))
    body += [H.ins(H.OpConstant, 2, 12 + i, 7) for i in range(n_pad)]
    body.append(H.ins(H.OpConstant, ty, 10, *pattern))
    body += base[8:]
    return H.module(body, bound=12 + n_pad)


def test_literals_that_read_as_instructions_in_a_first_tile(gpu):
    """A module's first tile whose constants hold words that read as
    instructions: a one-word OpReturn (its successor the next real start), a
    two-word OpBranch (its successor inside the next constant), an
    OpTypeStruct whose word count runs far past the tile, chains of two and
    of eight such words (a 64- and a 256-bit literal), at the start of the
    tile, inside it and at its end. The guessed starts are not a chain; the
    false ones are dropped (or, past a few rounds, the exact path runs) and
    every result is the oracle's."""
    RET = (1 << 16) | H.OpReturn
    BR = (2 << 16) | H.OpBranch
    FAR = (0xF000 << 16) | 30                       # OpTypeStruct, 61,440 words
    cases = [([RET], 32), ([BR], 32), ([FAR], 32), ([RET, RET], 64), ([RET] * 8, 256), ([BR, RET], 64),
             ([RET, BR], 64)]
    mods = []
    for pattern, width in cases:
        for n_pad in (0, 1, 120, 1018, 1019, 1020, 1021, 1022):
            mods.append(_literal_module(pattern, n_pad, width))
    # a false start in a later tile of a long module as well
    long_body = list(H.minimal_body()[:8]) + [H.ins(H.OpConstant, 2, 12 + i, RET if i % 700 == 699 else 7)
                                              for i in range(3000)] + list(H.minimal_body()[8:])
    mods.append(H.module(long_body, bound=3012))
    w, off = H.batch(mods)
    for cfg in (None, gpu.make_config(tile_words=2048, threads=128), gpu.make_config(tile_words=512, threads=64),
                gpu.make_config(no_speculation=1)):
        check(gpu, w, off, cfg=cfg)
    # the same modules one per batch (every one starts on a 16-byte boundary)
    for mm in mods[::5]:
        ww, oo = H.batch([mm])
        check(gpu, ww, oo)


def test_per_module_path_matches(gpu):
    n_instr, n_k = synth.batch_shape(40, 5, median=2000, lo=200, hi=20000)
    w, off = synth.batch(n_instr, n_k, 5)
    a = check(gpu, w, off, cfg=gpu.make_config(per_module=1))
    b = run(gpu, w, off)
    assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["out"], b["out"])


def test_large_module_with_strings(gpu):
    w, off, starts, bound = synth.large_module(2, n_instr=400_000, n_funcs=50)
    g = check(gpu, w, off, dis=True)
    assert np.array_equal(g["table"]["off"].astype(np.int64), starts)


# ---------------------------------------------------------------------------
# edge cases and corruptions
# ---------------------------------------------------------------------------
def hand_modules():
    base = H.minimal_body()
    mods = [H.module(base, bound=8), H.module(base, bound=0), H.module([], bound=1)]
    good = H.module(base, bound=8)
    for n in range(0, 6):
        mods.append(good[:n])
    mods.append(good[:-3])
    for i, v in [(0, 0x03022307), (1, 0x00020000), (4, 1), (1, 0x00010700)]:
        x = good.copy(); x[i] = v; mods.append(x)
    b = list(base); b[0] = H.ins(H.OpCapability, H.CAP_KERNEL); mods.append(H.module(b, bound=8))
    b = list(base); b.insert(11, H.ins(H.OpIAdd, 2, 7, 4, 4)); b.insert(12, H.ins(H.OpIAdd, 2, 7, 4, 4)); mods.append(H.module(b, bound=8))
    b = list(base); b.insert(4, [(1 << 16) | 9999]); mods.append(H.module(b, bound=8))
    b = list(base); b[3] = [(4 << 16) | H.OpEntryPoint, H.EXEC_KERNEL, 5, 0x6b6b6b6b]; mods.append(H.module(b, bound=8))
    b = list(base); b[10] = H.ins(H.OpIAdd, 2, 7, 4, 99); mods.append(H.module(b, bound=8))
    mods.append(H.module(base[:2] + base[3:], bound=8))
    mods.append(H.module(base[:3] + [base[2]] + base[3:], bound=8))
    mods.append(H.module(base[:3] + base[4:], bound=8))
    mods.append(H.module([i for i in base if i[0] & 0xffff != H.OpFunction], bound=8))
    mods.append(H.module([H.ins(H.OpTypeVoid, 1)], bound=8))
    b = list(base); b.insert(6, H.ins(H.OpTypeInt, 8, 64, 0)); mods.append(H.module(b, bound=9))
    b = list(base); b[0] = H.ins(H.OpCapability, H.CAP_GENERIC_POINTER); mods.append(H.module(b, bound=8))
    return mods


def test_edge_and_hand_built_modules(gpu):
    mods = hand_modules()
    w, off = H.batch(mods)
    check(gpu, w, off, dis=True)
    # the same modules as single-module batches, and an empty module between others
    for mm in mods[:8]:
        ww, oo = H.batch([mm])
        check(gpu, ww, oo)
    ww, oo = H.batch([mods[0], mods[0][:0], mods[0]])
    check(gpu, ww, oo, dis=True)


def test_empty_batch(gpu):
    w = torch.zeros(1, dtype=torch.int32, device="cuda")[:0]
    o = torch.zeros(1, dtype=torch.int64, device="cuda")
    r = gpu.process(w, o)
    torch.cuda.synchronize()
    assert r["status"].numel() == 0


def test_single_word_corruptions(gpu):
    base = H.module(H.minimal_body(), bound=8)
    values = [0, 1, 0xFFFFFFFF, 0x00010000, 0x00020000, 0x00050080, 0x7FFF0011, 0x00030011, 7, 8, 9999]
    mods = []
    for i in range(len(base)):
        for v in values:
            x = base.copy(); x[i] = v; mods.append(x)
    w, off = H.batch(mods)
    check(gpu, w, off, dis=True)


def corrupt(words, starts, bound, rng, kind):
    x = words.copy()
    r = int(rng.integers(0, len(starts)))
    p = int(starts[r])
    wc = int(x[p] >> 16)
    if kind == "opcode":
        x[p] = (x[p] & 0xFFFF0000) | int(rng.integers(256, 65536))
    elif kind == "wc":
        x[p] = (x[p] & 0xFFFF) | (int(rng.integers(0, 6)) << 16)
    elif kind == "operand" and wc > 1:
        x[p + int(rng.integers(1, wc))] = int(rng.choice([0, bound, bound + 7, 0xFFFFFFFF, int(rng.integers(1, bound))]))
    elif kind == "dup":
        q = int(starts[int(rng.integers(0, len(starts)))])
        if wc >= 3 and (x[q] >> 16) >= 3:
            x[p + 2] = x[q + 2]
    elif kind == "random":
        x[int(rng.integers(0, len(x)))] = int(rng.integers(0, 2**32))
    elif kind == "header":
        x[int(rng.integers(0, 5))] ^= 1 << int(rng.integers(0, 32))
    elif kind == "truncate":
        x = x[: int(rng.integers(5, len(x)))]
    return x


def test_random_corruptions(gpu):
    rng = np.random.default_rng(1234)
    mods = []
    for seed in range(8):
        w, off, starts, bound = synth.single_module(1000 + seed)
        for kind in ("opcode", "wc", "operand", "dup", "random", "header", "truncate"):
            for _ in range(6):
                mods.append(corrupt(w, starts, bound, rng, kind))
    words, offs = H.batch(mods)
    g = check(gpu, words, offs, dis=True)
    st = set(int(s) for s in g["status"])
    assert len(st) >= 8, st


def test_duplicates_across_chunks_and_missing_caps(gpu):
    w, off, starts, bound = synth.large_module(4, n_instr=60_000, n_funcs=6, string_permille=0)
    d = oracle.decode(w, off)
    rows = np.nonzero(d["rid"] > 0)[0]
    mods = []
    for a, b in [(rows[10], rows[5000]), (rows[3000], rows[3001]), (rows[100], rows[40000]), (rows[-1], rows[-2])]:
        x = w.copy()
        pb = int(d["off"][b]); pa = int(d["off"][a])
        x[pb + (2 if oracle.op_info(int(d["op"][b]))[1] else 1)] = x[pa + (2 if oracle.op_info(int(d["op"][a]))[1] else 1)]
        mods.append(x)
    x = w.copy()
    caps = np.nonzero(d["op"] == 17)[0]
    x[int(d["off"][caps[-1]]) + 1] = 39          # Int64 -> Int8: 64-bit int types now miss a capability
    mods.append(x)
    words, offs = H.batch(mods)
    check(gpu, words, offs)


# ---------------------------------------------------------------------------
# table-level entry points
# ---------------------------------------------------------------------------
def test_validate_from_table_and_encode_edited(gpu):
    n_instr, n_k = synth.batch_shape(50, 21, median=1500, lo=200, hi=10000)
    w, off = synth.batch(n_instr, n_k, 21)
    rng = np.random.default_rng(5)
    mods = []
    for m in range(50):
        x = w[off[m]:off[m + 1]].copy()
        if m % 3 == 0:
            x[int(rng.integers(5, len(x)))] = int(rng.integers(0, 2**32))
        mods.append(x)
    words, offs = H.batch(mods)
    g = run(gpu, words, offs)
    st, er = gpu.validate(g["_w"], g["_o"], g["_r"]["table"])
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy().view(np.uint32), g["status"])
    assert np.array_equal(er.cpu().numpy(), g["err_row"])
    # edit the table: rename result ids and swap opcodes, then encode
    t = g["_r"]["table"]
    d = oracle.decode(words, offs)
    n = d["n_rows"]
    sel = np.nonzero(d["rid"] > 0)[0][::7]
    d["rid"][sel] += 1000
    d["op"][sel[::2]] = np.where(d["op"][sel[::2]] == 128, 129, d["op"][sel[::2]])
    t.rid[:n] = torch.from_numpy(d["rid"].view(np.int32)).cuda()
    t.op[:n] = torch.from_numpy(d["op"].view(np.int16)).cuda()
    out = gpu.encode(g["_w"], g["_o"], t, recompute_bound=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.encode(words, offs, d, True))
    out2 = gpu.encode(g["_w"], g["_o"], t, recompute_bound=False)
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy().view(np.uint32), oracle.encode(words, offs, d, False))


def test_row_capacity(gpu):
    n_instr, n_k = synth.batch_shape(20, 8, median=1000, lo=200, hi=3000)
    w, off = synth.batch(n_instr, n_k, 8)
    d = oracle.decode(w, off)
    cap = int(d["first_row"][10]) + 7
    g = run(gpu, w, off, capacity_rows=cap)
    st, er = oracle.validate(w, off)
    full = [m for m in range(20) if d["first_row"][m] + d["n_instr"][m] <= cap]
    assert full == list(range(10))
    assert np.array_equal(g["status"][:10], st[:10])
    assert all(gpu.STATUS[s] == "CAPACITY" for s in g["status"][10:])
    for k in ("op", "wc", "off", "rid"):
        assert np.array_equal(g["table"][k][:cap], d[k][:cap])


def test_arena_capacity(gpu):
    n_instr, n_k = synth.batch_shape(20, 9, median=1000, lo=200, hi=3000)
    w, off = synth.batch(n_instr, n_k, 9)
    bounds = [int(w[off[m] + 3]) for m in range(20)]
    need = np.cumsum([(b + 31) // 32 for b in bounds])
    g = run(gpu, w, off, arena_words=int(need[4]))
    st, er = oracle.validate(w, off)
    assert np.array_equal(g["status"][:5], st[:5])
    assert all(gpu.STATUS[s] == "CAPACITY" for s in g["status"][5:])


def test_text_capacity_reports_size(gpu):
    w, off, _, _ = synth.single_module(3)
    g = run(gpu, w, off)
    text = torch.full((100,), 7, dtype=torch.uint8, device="cuda")
    t, toff, _ = gpu.disassemble(g["_w"], g["_o"], g["_r"]["table"], text=text, sync=False)
    torch.cuda.synchronize()
    want, woff = oracle.disassemble(w, off, True, True)
    assert int(toff[-1].item()) == len(want)
    assert bool((text == 7).all())


def test_text_buffer_at_any_alignment(gpu):
    """The tile copy-out stores 16-byte chunks when the text buffer is 16-byte
    aligned, 4-byte words when it is 4-byte aligned, else bytes: text written
    at every start offset 0..15 equals the oracle's, and the bytes around it
    stay untouched."""
    n_instr, n_k = synth.batch_shape(40, 19, median=1500, lo=200, hi=20000)
    w, off = synth.batch(n_instr, n_k, 19)
    g = run(gpu, w, off)
    want, woff = oracle.disassemble(w, off, True, True)
    big = torch.full((len(want) + 64,), 0xCD, dtype=torch.uint8, device="cuda")
    for shift in range(16):
        big.fill_(0xCD)
        view = big[shift:shift + len(want)]
        _, toff, _ = gpu.disassemble(g["_w"], g["_o"], g["_r"]["table"], text=view, sync=False)
        torch.cuda.synchronize()
        b = big.cpu().numpy()
        assert bytes(b[shift:shift + len(want)]) == want, shift
        assert (b[:shift] == 0xCD).all() and (b[shift + len(want):] == 0xCD).all(), shift
        assert np.array_equal(toff.cpu().numpy(), woff)


def test_thousands_of_tiny_modules(gpu):
    """Tiles that span thousands of modules: a batch of mostly 5-word (header
    only) and minimal modules, with truncated and bad-magic ones and a few
    normal ones mixed in, so that a disassembly tile of 2,048 items holds
    thousands of module headers and the per-tile module lookup runs at its
    maximum."""
    rng = np.random.default_rng(29)
    base = H.minimal_body()
    mods = []
    for i in range(7000):
        kind = int(rng.integers(0, 10))
        if kind < 5:
            mods.append(H.module([], bound=1))                  # header only
        elif kind < 8:
            mods.append(H.module(base, bound=8))
        elif kind == 8:
            mods.append(H.module(base, bound=8)[:int(rng.integers(0, 12))])  # truncated, possibly empty
        else:
            x = H.module(base, bound=8).copy(); x[0] = 0x12345678; mods.append(x)
    n_instr, n_k = synth.batch_shape(3, 5, median=1500, lo=200, hi=3000)
    w3, off3 = synth.batch(n_instr, n_k, 5)
    for i in range(3):
        mods.insert(1000 * (i + 1), w3[off3[i]:off3[i + 1]])
    words, offs = H.batch(mods)
    check(gpu, words, offs, dis=True)


def test_bounded_wait_times_out_without_hanging(gpu):
    w, off, _, _ = synth.large_module(6, n_instr=60_000, n_funcs=4)
    cfg = gpu.make_config(tile_words=1024, threads=128, max_spins=2000, test_stall_tile=5)
    g = run(gpu, w, off, cfg=cfg)
    assert gpu.STATUS[g["status"][0]] == "TIMEOUT"
    # the context is still usable and a normal call is exact
    check(gpu, w, off)


def test_map_entry_wait_times_out_without_hanging(gpu):
    """A tile that announces its tile map but never writes the entries (nor
    its exit or row count): the later tile that applies that map polls an
    entry that nothing writes, gives up after max_spins, and every module
    reports the timeout; the next call on the same context is exact."""
    w, off, _, _ = synth.large_module(6, n_instr=60_000, n_funcs=4)
    cfg = gpu.make_config(tile_words=1024, threads=128, max_spins=2000, test_stall_tile=-6)
    g = run(gpu, w, off, cfg=cfg)
    assert gpu.STATUS[g["status"][0]] == "TIMEOUT"
    check(gpu, w, off)


def test_text_lookback_times_out_without_hanging(gpu):
    """A text tile that never publishes its byte count (the test hook): the
    look-backs of the tiles after it give up after max_spins polls, every
    module reports TIMEOUT, and the next call on the same context is exact."""
    n_instr, n_k = synth.batch_shape(20, 41, median=1500, lo=1000, hi=3000)
    w, off = synth.batch(n_instr, n_k, 41)                  # about 30,000 rows: several text tiles
    g = run(gpu, w, off)
    _, _, dst = gpu.disassemble(g["_w"], g["_o"], g["_r"]["table"], sync=False, max_spins=2000, test_stall_tile=2)
    torch.cuda.synchronize()
    assert all(gpu.STATUS[int(x)] == "TIMEOUT" for x in dst.cpu().numpy())
    check_dis(gpu, w, off, g, modes=((True, True),))


# ---------------------------------------------------------------------------
# full-size workloads
# ---------------------------------------------------------------------------
def test_full_size_batch_10k_modules(gpu):
    """The benchmark's batch of 10,000 modules (122M words) at full size:
    table, statuses, encoded words, and the whole disassembly with inline
    names and header lines (about 830 MB of text) with its offsets, byte for
    byte against the oracle."""
    w, off = synth.module_batch(10_000, 0)
    g = run(gpu, w, off)
    d = oracle.decode(w, off)
    assert_table_equal(g["table"], d, 10_000)
    st, er = oracle.validate(w, off)
    assert np.array_equal(g["status"], st) and np.array_equal(g["err_row"], er)
    assert np.array_equal(g["out"], oracle.encode(w, off, d, True))
    del d
    check_dis(gpu, w, off, g, modes=((True, True),))


def test_full_size_large_module_and_text(gpu):
    w, off, starts, bound = synth.large_module(0)
    g = run(gpu, w, off)
    d = oracle.decode(w, off)
    assert_table_equal(g["table"], d, 1)
    st, er = oracle.validate(w, off)
    assert g["status"][0] == st[0] == 0
    assert np.array_equal(g["out"], w)
    check_dis(gpu, w, off, g, modes=((True, True),))


def test_every_opcode_word_counts_and_operands(gpu):
    """Every table opcode (and a few unknown ones) at word counts 1-8 with
    operand words in range, zero, at the bound and far above it, inserted
    into a valid module: the status and error row equal the oracle's."""
    base = H.minimal_body()
    ops = oracle.opcodes() + [2, 4, 9999]
    rng = np.random.default_rng(17)
    mods = []
    for op in ops:
        for wc in range(1, 9):
            for variant in range(3):
                vals = []
                for i in range(wc - 1):
                    pick = rng.integers(0, 6) if variant else 1
                    vals.append([3, 1, 0, 50, 0x41424344, int(rng.integers(1, 50))][int(pick)])
                b = list(base)
                b.insert(5, [(wc << 16) | op] + vals)
                mods.append(H.module(b, bound=50))
    words, offs = H.batch(mods)
    check(gpu, words, offs, dis=True)


def test_trailing_bit_enum_and_context_literal_operands(gpu):
    """Instructions ending in a bit-enum word (memory access of OpLoad and
    OpStore, loop and selection controls) with every mix of known and unknown
    bits and too few, exactly enough or too many parameter words, with the
    word absent, and OpConstant with no literal or several: statuses, error
    rows and text equal the oracle's."""
    base = H.minimal_body()
    fixed = {H.OpLoad: [2, 40, 4], H.OpStore: [4, 7], 246: [6, 6], 247: [6]}
    masks = [0, 1, 2, 3, 4, 5, 6, 7, 8, 0x10, 0x20, 0x3f, 0xff, 0x100, 0x80000000, 0x41424344, 0xffffffff]
    mods = []
    for op, ids in fixed.items():
        b = list(base)
        b.insert(5, [((len(ids) + 1) << 16) | op] + ids)            # the bit-enum word absent
        mods.append(H.module(b, bound=50))
        for mask in masks:
            for extra in range(5):
                b = list(base)
                b.insert(5, H.ins(op, ids, mask, [9] * extra))
                mods.append(H.module(b, bound=50))
    for n_lit in range(5):
        b = list(base)
        b.insert(8, H.ins(H.OpConstant, 2, 41, [5] * n_lit))
        mods.append(H.module(b, bound=50))
    words, offs = H.batch(mods)
    g = check(gpu, words, offs, dis=True)
    assert (g["status"] == 0).sum() >= 20 and (g["status"] != 0).sum() >= 20


def _long_instruction_module(seed, n):
    """A valid module whose instructions include many longer than 32 words
    (wide struct types, phis with many pairs, long strings and names, calls
    with many arguments), so that entries deep inside tiles and warp
    segments occur."""
    rng = np.random.default_rng(seed)
    base = H.minimal_body()
    head, tail = base[:7], base[7:]
    body = list(head)
    nid = 100
    for k in range(n):
        kind = int(rng.integers(0, 5))
        if kind == 0:
            body.append(H.ins(30, nid, [2] * int(rng.integers(1, 120))))                 # OpTypeStruct
        elif kind == 1:
            body.append(H.ins(H.OpString, nid, H.s("x" * int(rng.integers(1, 400)))))
        elif kind == 2:
            body.append(H.ins(H.OpName, 5, H.s("n" * int(rng.integers(1, 300)))))
        elif kind == 3:
            body.append(H.ins(H.OpTypeInt, nid, 32, 0))
        else:
            body.append(H.ins(44, 2, nid, [4] * int(rng.integers(1, 90))))               # OpConstantComposite
        nid += 1
    body.extend(tail)
    return H.module(body, bound=nid + 1)


@pytest.mark.parametrize("tile,threads", [(8192, 512), (4096, 256), (2048, 256), (2048, 128), (1024, 128)])
def test_long_instructions_cross_tiles(gpu, tile, threads):
    mods = [_long_instruction_module(s, 400) for s in range(3)]
    words, offs = H.batch(mods)
    st, er = oracle.validate(words, offs)
    assert (st == 0).all()
    check(gpu, words, offs, cfg=gpu.make_config(tile_words=tile, threads=threads), dis=(tile == 4096))


def _window_module(seed):
    """A module whose text lines are far longer than the disassembler's
    shared text window: ids with names of thousands of characters (printed
    at every use), a string of tens of thousands of bytes that need escapes,
    and many integer and float constants, so that lines cross window edges
    inside names, escapes, decimals and hex floats."""
    rng = np.random.default_rng(seed)
    base = H.minimal_body()
    head, tail = base[:7], base[7:]
    alphabet = np.frombuffer(b"abcXYZ019_-. +*/", np.uint8)
    def name(n):
        return bytes(alphabet[rng.integers(0, len(alphabet), n)]).decode()
    body = list(head)
    body.append(H.ins(H.OpTypeFloat, 50, 32))
    body.append(H.ins(H.OpTypeFloat, 51, 64))
    body.append(H.ins(H.OpName, 2, H.s(name(int(rng.integers(3000, 7000))))))
    body.append(H.ins(H.OpName, 50, H.s(name(int(rng.integers(15000, 25000))))))
    raw = bytes(int(x) for x in rng.choice([0x22, 0x5c, 0x01, 0x7f, 0x41, 0x61, 0xe9], size=int(rng.integers(30000, 45000))))
    sw = raw + b"\0" * (4 - len(raw) % 4)
    body.append(H.ins(H.OpString, 60, [int.from_bytes(sw[i:i + 4], "little") for i in range(0, len(sw), 4)]))
    nid = 100
    for k in range(int(rng.integers(300, 500))):
        kind = int(rng.integers(0, 4))
        if kind == 0:
            body.append(H.ins(H.OpConstant, 2, nid, int(rng.integers(0, 2 ** 32))))
        elif kind == 1:
            body.append(H.ins(H.OpConstant, 50, nid, int(rng.integers(0, 2 ** 32))))
        elif kind == 2:
            body.append(H.ins(H.OpConstant, 51, nid, int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 2 ** 32))))
        else:
            body.append(H.ins(H.OpDecorate, nid - 1, 44, int(rng.integers(1, 1 << 20))))    # Alignment
        nid += 1
    body.extend(tail)
    return H.module(body, bound=nid + 1)


def test_text_windows_and_lines_longer_than_a_window(gpu):
    mods = [_window_module(s) for s in range(3)] + [H.module(H.minimal_body(), bound=8)]
    words, offs = H.batch(mods)
    g = run(gpu, words, offs)
    check_dis(gpu, words, offs, g)


def test_big_tiles_on_generated_batch(gpu):
    n_instr, n_k = synth.batch_shape(80, 23, median=3000, lo=200, hi=40000)
    w, off = synth.batch(n_instr, n_k, 23)
    check(gpu, w, off, cfg=gpu.make_config(tile_words=8192, threads=512))


# ---------------------------------------------------------------------------
# autotuning and CUDA-graph replay
# ---------------------------------------------------------------------------
def test_autotune_returns_a_built_shape_with_exact_outputs(gpu):
    n_instr, n_k = synth.batch_shape(60, 77, median=2000, lo=200, hi=20000)
    w, off = synth.batch(n_instr, n_k, 77)
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    od = torch.from_numpy(off).cuda()
    cfg, ms, r = gpu.autotune(wd, od, reps=2)
    assert (cfg.tile_words, cfg.threads) in gpu.TILE_SHAPES and ms > 0
    d = oracle.decode(w, off)
    st, er = oracle.validate(w, off)
    assert_table_equal(r["table"].to_numpy(), d, len(off) - 1)
    assert np.array_equal(r["status"].cpu().numpy().view(np.uint32), st)
    assert np.array_equal(r["err_row"].cpu().numpy(), er)
    assert np.array_equal(r["out"].cpu().numpy().view(np.uint32), oracle.encode(w, off, d, True))


def test_step_captured_in_a_cuda_graph_replays_exactly(gpu):
    """decode + validate + encode + disassemble captured once into a CUDA
    graph and replayed: every replay reproduces the oracle's outputs (the
    persistent launches have no host synchronisation inside)."""
    n_instr, n_k = synth.batch_shape(40, 78, median=1500, lo=200, hi=10000)
    w, off = synth.batch(n_instr, n_k, 78)
    m = len(off) - 1
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    od = torch.from_numpy(off).cuda()
    want, woff = oracle.disassemble(w, off, True, True)
    table = gpu.Table(m, len(w), wd.device)
    ws = gpu.Workspace(m, len(w), wd.device)
    dws = gpu.DisWorkspace(m, len(w), len(w), wd.device)
    out = torch.empty_like(wd)
    text = torch.empty(len(want) + 16, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):                      # warm up outside the capture
        gpu.process(wd, od, encode=True, table=table, workspace=ws, out=out, stream=s)
        gpu.disassemble(wd, od, table, workspace=dws, text=text, sync=False, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        r = gpu.process(wd, od, encode=True, table=table, workspace=ws, out=out)
        _, toff, dst = gpu.disassemble(wd, od, table, workspace=dws, text=text, sync=False)
    d = oracle.decode(w, off)
    st, er = oracle.validate(w, off)
    for _ in range(3):
        out.zero_(); text.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(r["status"].cpu().numpy().view(np.uint32), st)
        assert np.array_equal(r["err_row"].cpu().numpy(), er)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.encode(w, off, d, True))
        assert bytes(text[:len(want)].cpu().numpy()) == want
        assert np.array_equal(toff.cpu().numpy(), woff)
