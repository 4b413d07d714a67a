"""The batched GPU assembler (spv_assemble_batch) against the oracle: words,
word offsets, statuses and first bad lines, element by element, on texts of
every kind the text form has: the disassembler's own output (with and without
inline names and header), hand-written lines, named ids, float constants in
every spelling (hexadecimal, shortest decimal, long and halfway decimals),
random mutations of valid texts, and the edge cases (empty batch, empty and
comment-only modules, tiny and huge modules, a text that starts at an
unaligned address or after a prefix, capacities too small, bad offsets).
At the full batch size the round trip assemble(disassemble(x)) == x is
checked for every module."""
import struct

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


def _texts_to_batch(texts, prefix=b""):
    off = [len(prefix)]
    for t in texts:
        off.append(off[-1] + len(t))
    return prefix + b"".join(texts), np.array(off, np.int64)


def _run(gpu, text, toff, shift=0, **kw):
    """Assemble on the GPU; shift > 0 places the text at an address that is
    shift bytes past a 256-byte boundary."""
    buf = torch.zeros(len(text) + shift + 16, dtype=torch.uint8)
    buf[shift:shift + len(text)] = torch.frombuffer(bytearray(text), dtype=torch.uint8) if text else buf[:0]
    d = buf.cuda()[shift:shift + len(text)]
    o = torch.from_numpy(np.asarray(toff, np.int64)).cuda()
    w, woff, st, err = gpu.assemble(d, o, **kw)
    torch.cuda.synchronize()
    return (w.cpu().numpy().view(np.uint32), woff.cpu().numpy(), st.cpu().numpy().astype(np.uint32),
            err.cpu().numpy())


def _check(gpu, text, toff, **kw):
    w_o, woff_o, st_o, err_o = oracle.assemble_batch(text, toff)
    w, woff, st, err = _run(gpu, text, toff, **kw)
    assert np.array_equal(st, st_o), (np.nonzero(st != st_o)[0][:10], st[st != st_o][:10], st_o[st != st_o][:10])
    assert np.array_equal(err, err_o), (np.nonzero(err != err_o)[0][:10], err[err != err_o][:10],
                                        err_o[err != err_o][:10])
    assert np.array_equal(woff, woff_o)
    if not np.array_equal(w, w_o):
        bad = np.nonzero(w != w_o)[0][:8]
        raise AssertionError(f"words differ at {bad}: {w[bad]} vs {w_o[bad]}")
    return w, woff, st, err


@pytest.mark.parametrize("inline,header", [(True, True), (False, True), (True, False), (False, False)])
def test_round_trip_of_disassembly(gpu, inline, header):
    n_instr, n_k = synth.batch_shape(60, 5, median=600, lo=200, hi=4000)
    w, off = synth.batch(n_instr, n_k, 5)
    text, toff = oracle.disassemble(w, off, inline, header)
    got, woff, st, _ = _check(gpu, text, toff)
    assert (st == 0).all()
    if header:                              # with the header the round trip is exact
        assert np.array_equal(got, w) and np.array_equal(woff, off)


def test_round_trip_of_the_gpu_disassembly(gpu):
    n_instr, n_k = synth.batch_shape(40, 6, median=800, lo=200, hi=4000)
    w, off = synth.batch(n_instr, n_k, 6)
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    od = torch.from_numpy(off).cuda()
    r = gpu.process(wd, od)
    text, toff, _ = gpu.disassemble(wd, od, r["table"])
    words, woff, st, err = gpu.assemble(text, toff)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    assert np.array_equal(words.cpu().numpy().view(np.uint32), w)
    assert np.array_equal(woff.cpu().numpy(), off)


HEAD = "; SPIR-V\n; Version: 1.2\n; Generator: 0x00000020\n; Bound: 100\n; Schema: 0\n"


def _hand_texts():
    t = []
    t.append("OpCapability Addresses\nOpCapability Kernel\nOpMemoryModel Physical64 OpenCL\n"
             'OpEntryPoint Kernel %main "k"\n%void = OpTypeVoid\n%fn = OpTypeFunction %void\n'
             "%main = OpFunction %void None %fn\n%entry = OpLabel\nOpReturn\nOpFunctionEnd\n")
    t.append("%7 = OpTypeVoid\n%a_7 = OpTypeVoid\n%_7 = OpTypeVoid\n%a7 = OpTypeVoid\n%_ = OpTypeVoid\n"
             "%7a = OpTypeVoid\n%a7 = OpTypeVoid\n%%5 = OpTypeVoid\n%a%_5 = OpTypeVoid\n%00012 = OpTypeVoid\n"
             "%_4294967296 = OpTypeVoid\n")
    t.append(HEAD + r'OpExtension "a\"b\\c\x41\x4a\xg1\q"' + "\nOpName %3 \"\"\nOpName %3 \"abcd\"\n")
    t.append("; Version: 1.5\n; Generator: 0xDEADbeef\n; Bound: 99\n; Schema: 3\nOpNop\n")
    t.append("; Version: 1.5 \n; Version:1.3\n; Bound: 4294967296\n; Bound: 9x\n; bound: 5\nOpNop\n")
    t.append(HEAD + "OpCapability 6\nOpDecorate %3 Alignment 16\nOpDecorate %3 1234 5 6\n"
             "%4 = OpFunction %1 Inline|Const %2\n%5 = OpFunction %1 None %2\n%6 = OpFunction %1 3 %2\n"
             "OpStore %7 %8 Aligned|Volatile 4\nOpDecorate %9 BuiltIn GlobalInvocationId\n")
    t.append(HEAD + "Op300 0x00000001 0xABCDEF01\nOpNop\nOpIAdd 0x00000002 0x00000003\nOp65535\n")
    t.append(HEAD + "%5 = OpConstant %2 1\n%2 = OpTypeInt 64 0\n%2 = OpTypeInt 32 0\n%6 = OpConstant %9 7\n")
    t.append("%4294967294 = OpTypeVoid\n%a = OpTypeVoid\n")
    t.append("%4294967295 = OpTypeVoid\nOpNop\n%a = OpTypeVoid\n")                 # fresh id overflow
    t.append("")                                                                     # empty module
    t.append("; only a comment\n\n\n")
    t.append("OpNop")                                                                # no final newline
    t.append("\n\nOpNop\n\n")
    t.append(HEAD + 'OpExtension "' + "a" * (65534 * 4 - 1) + '"\n')                # 65535 words
    t.append(HEAD + 'OpExtension "' + "a" * (65534 * 4) + '"\n')                    # one too many
    bad = ["OpFoo %1", "Op65536", "Op12x", "   ", "%1 = OpNop", "OpTypeVoid", "%1 = OpTypeInt 32",
           "%1 = OpTypeInt 32 0 1", "%1 = OpTypeInt 4294967296 0", "%1 = OpTypeInt x 0", "%1 = OpTypeVoid extra",
           'OpName % "a"', 'OpName %99999999999 "a"', 'OpName %1 "abc', 'OpName %1 "abc\\"', "OpName %1 abc",
           "%5 = OpConstant %2 1.5x", "%5 = OpConstant %2 0x", "%5 = OpConstant %2 1e",
           "%5 = OpConstant %2 1 4294967296", "%5 = OpConstant %2 Inf", "%5 = OpConstant %2", "OpCapability Kernels",
           "%4 = OpFunction %1 Inline| %2", "%4 = OpFunction %1 Inline||Const %2", "OpIAdd 0x00000002 3",
           "%3 = Op300 0x00000001"]
    for b in bad:
        t.append(HEAD + "OpNop\n\n; comment\n" + b + "\nOpNop\n")
    return [x.encode() for x in t]


def test_hand_written_lines(gpu):
    texts = _hand_texts()
    text, toff = _texts_to_batch(texts)
    _check(gpu, text, toff)


def _float_lines(vals, ty):
    lines = []
    for i, v in enumerate(vals):
        lines.append(f"%{100 + i} = OpConstant %2 {v}")
    return (HEAD + ty + "\n" + "\n".join(lines) + "\n").encode()


def test_float_constants(gpu):
    rng = np.random.default_rng(7)
    vals = list(rng.integers(0, 2 ** 64, 400, dtype=np.uint64).view(np.float64))
    vals += list(rng.standard_normal(200) * 10.0 ** rng.integers(-320, 300, 200))
    vals = [float(v) for v in vals if np.isfinite(v)]
    spell = []
    for v in vals:
        spell += [v.hex(), repr(v), f"{v:.25e}", f"{v:.3e}"]
    # hard decimal cases: halfway points, long digit strings, range edges
    spell += ["9007199254740993.0", "9007199254740993.0000000000000000001", "9007199254740995.0",
              "2.4703282292062327e-324", "2.4703282292062328e-324", "4.9406564584124654e-324",
              "1.7976931348623157e308", "1.7976931348623158e308", "1.7976931348623159e308",
              "2.2250738585072011e-308", "2.2250738585072012e-308", "0." + "0" * 400 + "1e400",
              "1" + "0" * 400 + "e-400", "3." + "1415926535" * 100, "0.1", "1e22", "1e23", "123456789012345678e-5",
              "-0.0", "0e999999999999", "1e-999999999999", "+inf", "-nan", "nan", "1e39", "3.4028235677973366e38",
              "1.00000005960464477539062499", "1.000000059604644775390625", "1.00000005960464477539062501",
              "0x1.000001p0", "0x1.00000100000008p0", "0x1p-1074", "0x1p-1075", "0x1.8p-1075", "0x.8p-1073",
              "0x1.fffffffffffff8p1023", "0X1P3", ".5", "5.", "0x0p0"]
    texts = [_float_lines(spell, "%2 = OpTypeFloat 64"), _float_lines(spell, "%2 = OpTypeFloat 32")]
    texts += [_float_lines(["1", "4294967296", "18446744073709551615", "18446744073709551616", "1 2 3", "7 8"],
                           ty) for ty in ("%2 = OpTypeInt 32 0", "%2 = OpTypeInt 64 0")]
    text, toff = _texts_to_batch(texts)
    w, woff, st, _ = _check(gpu, text, toff)
    assert (st == 0).all()
    # independent of the oracle: the 64-bit constants are Python's own parse
    k = woff[0] + 5 + 3
    for s in spell:
        n = w[k] >> 16
        try:
            v = float.fromhex(s) if "x" in s.lower() else float(s)
        except OverflowError:                       # Python raises where IEEE rounding gives infinity
            v = float("-inf") if s.startswith("-") else float("inf")
        want = struct.unpack("<2I", struct.pack("<d", v))
        assert tuple(int(x) for x in w[k + 3:k + n]) == want, s
        k += n


def _renamed(w, off, seed):
    """The texts of generated modules with a random half of their ids named."""
    import re
    text, toff = oracle.disassemble(w, off, False, True)
    idtok = re.compile(rb"%([0-9]+)(?=[ \n])")
    rng = np.random.default_rng(seed)
    out = []
    for m in range(len(off) - 1):
        t = re.sub(rb"(?m)^; Bound: .*\n", b"", text[toff[m]:toff[m + 1]])
        ids = sorted({int(x) for x in idtok.findall(t)})
        named = {i for i in ids if rng.random() < 0.5}
        out.append(idtok.sub(lambda mo: b"%%v%sx" % mo.group(1) if int(mo.group(1)) in named else mo.group(0), t))
    return out


def test_named_ids(gpu):
    n_instr, n_k = synth.batch_shape(50, 8, median=700, lo=200, hi=5000)
    w, off = synth.batch(n_instr, n_k, 8)
    texts = _renamed(w, off, 9)
    text, toff = _texts_to_batch(texts)
    _, _, st, _ = _check(gpu, text, toff)
    assert (st == 0).all()


def test_mutations(gpu):
    rng = np.random.default_rng(10)
    n_instr, n_k = synth.batch_shape(80, 11, median=300, lo=100, hi=1500)
    w, off = synth.batch(n_instr, n_k, 11)
    text, toff = oracle.disassemble(w, off, True, True)
    texts = [bytearray(text[toff[m]:toff[m + 1]]) for m in range(len(off) - 1)]
    alphabet = b" \n%=\"\\0123456789abxp.-|_OpNameIAdd;"
    for t in texts:
        for _ in range(int(rng.integers(0, 4))):
            i = int(rng.integers(0, len(t)))
            op = int(rng.integers(0, 3))
            c = alphabet[int(rng.integers(0, len(alphabet)))]
            if op == 0:
                t[i] = c
            elif op == 1:
                del t[i]
            else:
                t.insert(i, c)
    texts += _renamed(w[:off[10]], off[:11], 12)
    text, toff = _texts_to_batch([bytes(t) for t in texts])
    _, _, st, _ = _check(gpu, text, toff)
    assert (st == 1).sum() >= 10 and (st == 0).sum() >= 10


@pytest.mark.parametrize("shift", [1, 3, 7, 13])
def test_unaligned_text_and_prefix(gpu, shift):
    w, off = synth.module_batch(12, 13)
    text, toff = oracle.disassemble(w, off, True, True)
    texts = [text[toff[m]:toff[m + 1]] for m in range(len(off) - 1)]
    full, toff2 = _texts_to_batch(texts, prefix=b"x" * shift + b"\n")
    w_o, woff_o, st_o, err_o = oracle.assemble_batch(full, toff2)
    got = _run(gpu, full, toff2, shift=shift)
    assert np.array_equal(got[0], w_o) and np.array_equal(got[1], woff_o) and np.array_equal(got[2], st_o)


def test_many_tiny_and_one_huge(gpu):
    texts = [b"OpNop\n", b"", b"OpNop", b"\n"] * 1750                       # 7000 tiny modules
    big, boff, _, _ = synth.large_module(3, n_instr=150_000, n_funcs=20)
    bt, _ = oracle.disassemble(big, boff, True, True)
    texts.insert(3000, bt)
    text, toff = _texts_to_batch(texts)
    _check(gpu, text, toff)


def test_empty_batch(gpu):
    d = torch.zeros(1, dtype=torch.uint8, device="cuda")
    o = torch.zeros(1, dtype=torch.int64, device="cuda")
    w, woff, st, err = gpu.assemble(d[:0], o)
    assert w.numel() == 0 and woff.cpu().tolist() == [0]


def test_capacities(gpu):
    """Capacities too small: the modules past them get CAPACITY (and no
    words), the others are exact; the binding then sizes the workspace to
    what the call needed and every module is exact."""
    n_instr, n_k = synth.batch_shape(30, 14, median=500, lo=200, hi=2000)
    w, off = synth.batch(n_instr, n_k, 14)
    texts = _renamed(w, off, 15)
    text, toff = _texts_to_batch(texts)
    w_o, woff_o, st_o, err_o = oracle.assemble_batch(text, toff)
    d = torch.from_numpy(np.frombuffer(text, np.uint8).copy()).cuda()
    o = torch.from_numpy(toff).cuda()
    for lc, nc in ((2000, 0), (0, 3000)):
        ws = gpu.AsmWorkspace(len(texts), len(text), d.device, lc, nc)
        words, woff, st, err = gpu.assemble(d, o, workspace=ws, sync=False)
        torch.cuda.synchronize()
        st = st.cpu().numpy()
        woff = woff.cpu().numpy()
        words = words.cpu().numpy().view(np.uint32)
        assert (st == 2).any() and (st == 0).any()
        for m in np.nonzero(st == 0)[0]:
            assert np.array_equal(words[woff[m]:woff[m + 1]], w_o[woff_o[m]:woff_o[m + 1]])
        assert ((woff[1:] - woff[:-1])[st == 2] == 0).all()
        lines, names = gpu.spv_asm_required(gpu._ptr(ws.buf))
        assert lines == sum(t.count(b"\n") for t in texts) and names > 0
    _check(gpu, text, toff, line_capacity=500, name_capacity=500)


def test_word_capacity_below_total(gpu):
    w, off = synth.module_batch(10, 16)
    text, toff = oracle.disassemble(w, off, True, True)
    d = torch.from_numpy(np.frombuffer(text, np.uint8).copy()).cuda()
    o = torch.from_numpy(toff).cuda()
    for cap in (0, 1, 7, len(w) // 3, len(w) - 1):
        out = torch.full((cap + 64,), -1, dtype=torch.int32, device="cuda")
        words, woff, st, _ = gpu.assemble(d, o, words=out[:cap] if cap else out[:0], sync=False)
        torch.cuda.synchronize()
        assert np.array_equal(woff.cpu().numpy(), off)
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got[:cap], w[:cap])
        assert (got[cap:] == 0xffffffff).all()


def test_bad_offsets(gpu):
    w, off = synth.module_batch(4, 17)
    text, toff = oracle.disassemble(w, off, True, True)
    d = torch.from_numpy(np.frombuffer(text, np.uint8).copy()).cuda()
    for bad in (lambda t: np.concatenate([t[:2], [t[1] - 1], t[3:]]), lambda t: np.concatenate([t[:-1], [t[-1] + 9]])):
        o = torch.from_numpy(bad(toff.copy())).cuda()
        words, woff, st, err = gpu.assemble(d, o)
        assert (st.cpu().numpy() == 3).all() and words.numel() == 0


def test_full_batch_round_trip(gpu):
    """The 10,000-module batch: disassemble on the GPU, assemble on the GPU,
    every module's words equal the input (with header lines the round trip is
    exact)."""
    w, off = synth.module_batch(10000, 0)
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    od = torch.from_numpy(off).cuda()
    r = gpu.process(wd, od)
    text, toff, _ = gpu.disassemble(wd, od, r["table"])
    words, woff, st, err = gpu.assemble(text, toff)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    assert torch.equal(woff.cpu(), od.cpu())
    assert torch.equal(words, wd)
