"""Pins of the CPU oracle against things other than itself.

* the paper's own worked example (Listing 8's text, from Listing 7's
  capabilities) and hand-built modules written word by word from the public
  SPIR-V specification, with hand-written expected results;
* an independently written framing decoder (below), brute-forced over every
  short instruction stream of a small alphabet and every single-word
  corruption of a small module;
* the generator's own ground truth (where it wrote each instruction, which
  bound it wrote) and invariants: word counts sum to the module length minus
  the header, encode(decode(x)) == x, assemble(disassemble(x)) == x;
* hexadecimal float spellings worked out by hand from IEEE-754 bit fields.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import ST
from paper_2305_09493_b300 import synth
from tests import spvhand as H

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _one(words):
    return np.asarray(words, np.uint32), np.array([0, len(words)], np.int64)


def _golden(name):
    g = json.load(open(os.path.join(GOLD, name)))
    return np.array([int(x, 16) for x in g["words"]], np.uint32), g["text"]


# ----------------------------------------------------------------------------
# the paper's worked examples
# ----------------------------------------------------------------------------
def test_listing8_capability_text():
    """Listing 7 -> Listing 8 (section 3.4.3): five capabilities print as
    five 'OpCapability <name>' lines."""
    w, text = _golden("listing8_capabilities.json")
    got, off = oracle.disassemble(*_one(w), inline_names=True, header=False)
    assert got.decode() == text
    d = oracle.decode(*_one(w))
    assert list(d["op"]) == [17] * 5 and list(d["wc"]) == [2] * 5


def test_tiny_kernel_text_and_status():
    w, text = _golden("tiny_kernel.json")
    got, off = oracle.disassemble(*_one(w), inline_names=True, header=True)
    assert got.decode() == text
    st, er = oracle.validate(*_one(w))
    assert st[0] == ST["OK"] and er[0] == -1


def test_listing9_iadd_operand_order():
    """Listing 9: OpIAdd(result type, result id, operand 1, operand 2)."""
    w = H.module([H.ins(H.OpIAdd, 4, 7, 5, 6)], bound=8)
    d = oracle.decode(*_one(w))
    assert d["n_rows"] == 1
    assert (d["op"][0], d["wc"][0], d["off"][0], d["rtype"][0], d["rid"][0]) == (128, 5, 5, 4, 7)
    t, _ = oracle.disassemble(*_one(w), inline_names=False, header=False)
    assert t == b"%7 = OpIAdd %4 %5 %6\n"


def test_listing4_header_bound_recomputed_on_write():
    """Listing 4 builds the header with bound 0; the bound is recomputed
    (largest id + 1) when the module is written (section 3.4.1)."""
    body = H.minimal_body()
    w = H.module(body, bound=0)
    d = oracle.decode(*_one(w))
    out = oracle.encode(*_one(w), d, recompute_bound=True)
    assert out[3] == 8                      # ids used: 1..7
    assert np.array_equal(np.delete(out, 3), np.delete(w, 3))
    kept = oracle.encode(*_one(w), d, recompute_bound=False)
    assert np.array_equal(kept, w)
    # a module without result ids: bound becomes 1
    w2 = H.module([H.ins(H.OpCapability, 6)], bound=0)
    assert oracle.encode(*_one(w2), oracle.decode(*_one(w2)), True)[3] == 1


def test_header_fields_text():
    w = H.module([H.ins(H.OpCapability, 6)], bound=17, generator=0x00080001)
    t, _ = oracle.disassemble(*_one(w), header=True)
    assert t.decode().startswith("; SPIR-V\n; Version: 1.2\n; Generator: 0x00080001\n; Bound: 17\n; Schema: 0\n")


# ----------------------------------------------------------------------------
# validation rules (section 3.4.5 and the SSA rule of section 3.4.2)
# ----------------------------------------------------------------------------
def _status(body, bound=100):
    st, er = oracle.validate(*_one(H.module(body, bound=bound)))
    return oracle.STATUS[st[0]], int(er[0])


def test_minimal_module_valid():
    assert _status(H.minimal_body()) == ("OK", -1)


def test_rule_no_capability():
    body = [i for i in H.minimal_body() if i[0] & 0xffff != H.OpCapability]
    # without Addresses/Kernel the memory model row misses its capabilities;
    # the module-level rule shows when nothing requires a capability
    st = _status(body)
    assert st == ("MISSING_CAPABILITY", 0)
    plain = [H.ins(H.OpMemoryModel, H.AM_LOGICAL, 0)]
    assert _status(plain)[0] in ("MISSING_CAPABILITY", "NO_CAPABILITY")
    assert _status([H.ins(H.OpTypeVoid, 1)]) == ("NO_CAPABILITY", -1)


def test_rule_memory_model():
    body = H.minimal_body()
    assert _status(body[:2] + body[3:]) == ("NO_MEMORY_MODEL", -1)
    assert _status(body[:3] + [body[2]] + body[3:]) == ("MULTI_MEMORY_MODEL", -1)


def test_rule_entry_point_and_function():
    body = H.minimal_body()
    assert _status(body[:3] + body[4:]) == ("NO_ENTRY_POINT", -1)
    no_fn = [i for i in body if i[0] & 0xffff not in (H.OpFunction,)]
    assert _status(no_fn) == ("NO_FUNCTION", -1)


def test_rule_id_out_of_bound_and_zero_id():
    body = H.minimal_body()
    body[10] = H.ins(H.OpIAdd, 2, 7, 4, 99)
    assert _status(body, bound=8) == ("ID_OUT_OF_BOUND", 10)
    body[10] = H.ins(H.OpIAdd, 2, 7, 4, 0)
    assert _status(body, bound=8) == ("ID_OUT_OF_BOUND", 10)
    body = H.minimal_body()
    assert _status(body, bound=7) == ("ID_OUT_OF_BOUND", 10)   # result id 7 == bound


def test_rule_duplicate_result_id_reports_second_definition():
    body = H.minimal_body()
    body.insert(11, H.ins(H.OpIAdd, 2, 7, 4, 4))        # row 11 redefines 7
    body.insert(12, H.ins(H.OpIAdd, 2, 7, 4, 4))        # row 12 too
    assert _status(body) == ("DUP_RESULT_ID", 11)


def test_rule_unknown_opcode_and_bad_operands():
    body = H.minimal_body()
    body.insert(4, [(1 << 16) | 9999])
    assert _status(body) == ("UNKNOWN_OPCODE", 4)
    body = H.minimal_body()
    body[3] = [(4 << 16) | H.OpEntryPoint, H.EXEC_KERNEL, 5, 0x6b6b6b6b]   # string without NUL
    assert _status(body) == ("BAD_OPERANDS", 3)
    body = H.minimal_body()
    body[3] = H.ins(H.OpEntryPoint, H.EXEC_KERNEL, 5, [0x00ff006b])        # nonzero padding
    assert _status(body) == ("BAD_OPERANDS", 3)
    body = H.minimal_body()
    body[10] = H.ins(H.OpIAdd, 2, 7, 4)                                     # missing operand
    assert _status(body) == ("BAD_OPERANDS", 10)
    body[10] = H.ins(H.OpIAdd, 2, 7, 4, 4, 4)                               # extra operand
    assert _status(body) == ("BAD_OPERANDS", 10)


def test_rule_capability_requirement_and_dependency():
    body = H.minimal_body()
    body[0] = H.ins(H.OpCapability, H.CAP_KERNEL)       # Addresses missing: Physical64 needs it
    assert _status(body) == ("MISSING_CAPABILITY", 2)
    body[0] = H.ins(H.OpCapability, H.CAP_GENERIC_POINTER)   # GenericPointer implies Addresses
    assert _status(body) == ("OK", -1)
    body = H.minimal_body()
    body.insert(6, H.ins(H.OpTypeInt, 8, 64, 0))        # 64-bit int needs Int64
    assert _status(body) == ("MISSING_CAPABILITY", 6)
    body.insert(0, H.ins(H.OpCapability, H.CAP_INT64))
    assert _status(body) == ("OK", -1)


def test_first_error_wins_and_rank_within_row():
    body = H.minimal_body()
    body[7] = H.ins(H.OpConstant, 2, 4)                 # row 7: no value word -> BAD_OPERANDS
    body[10] = H.ins(H.OpIAdd, 2, 7, 4, 99)             # row 10: out of bound
    assert _status(body, bound=8) == ("BAD_OPERANDS", 7)
    body = H.minimal_body()
    body[0] = H.ins(H.OpCapability, H.CAP_KERNEL)
    body[2] = H.ins(H.OpMemoryModel, H.AM_PHYSICAL64, H.MM_OPENCL)
    body.insert(3, H.ins(H.OpTypeInt, 99, 64, 0))       # row 3: out of bound AND needs Int64
    assert _status(body, bound=50) == ("MISSING_CAPABILITY", 2)
    body[0] = H.ins(H.OpCapability, H.CAP_ADDRESSES)
    body.insert(1, H.ins(H.OpCapability, H.CAP_KERNEL))
    # row 2 is now fine; row 4 (the TypeInt) is out of bound before its capability check
    assert _status(body, bound=50) == ("ID_OUT_OF_BOUND", 4)


def test_framing_errors():
    body = H.minimal_body()
    w = H.module(body)
    assert _status(body) == ("OK", -1)
    bad = w.copy()
    bad[5 + 2 + 2] = 0x00000000 | H.OpMemoryModel       # word count 0 at row 2
    st, er = oracle.validate(*_one(bad))
    assert oracle.STATUS[st[0]] == "ZERO_WORDCOUNT" and er[0] == 2
    d = oracle.decode(*_one(bad))
    assert d["n_instr"][0] == 2 and d["status"][0] == ST["ZERO_WORDCOUNT"] and d["err_row"][0] == 2
    trunc = w[:-3]                  # drop OpFunctionEnd, OpReturn and the IAdd's last word
    st, er = oracle.validate(*_one(trunc))
    assert oracle.STATUS[st[0]] == "TRUNCATED" and er[0] == 10
    # an instruction-level error before the framing error wins
    body[1] = H.ins(9999)
    w2 = H.module(body)[:-3]
    st, er = oracle.validate(*_one(w2))
    assert oracle.STATUS[st[0]] == "UNKNOWN_OPCODE" and er[0] == 1


def test_header_errors():
    w = H.module(H.minimal_body())
    for i, val, want in [(0, 0x03022307, "BAD_MAGIC"), (1, 0x00020000, "BAD_HEADER"),
                         (1, 0x00010700, "BAD_HEADER"), (1, 0x01010200, "BAD_HEADER"),
                         (1, 0x00010201, "BAD_HEADER"), (4, 1, "BAD_HEADER")]:
        x = w.copy(); x[i] = val
        st, er = oracle.validate(*_one(x))
        assert oracle.STATUS[st[0]] == want and er[0] == -1
        d = oracle.decode(*_one(x))
        assert d["n_instr"][0] == 0 and oracle.STATUS[d["status"][0]] == want
    for n in range(5):
        st, er = oracle.validate(*_one(w[:n]))
        assert oracle.STATUS[st[0]] == "TRUNCATED"
    assert oracle.STATUS[oracle.validate(*_one(w[:5]))[0][0]] == "NO_CAPABILITY"


# ----------------------------------------------------------------------------
# brute force against an independently written framing decoder
# ----------------------------------------------------------------------------
def ref_framing(w):
    """Second framing decoder, written separately: returns (status, starts,
    error_row) with status one of OK / TRUNCATED / ZERO_WORDCOUNT /
    BAD_MAGIC / BAD_HEADER."""
    w = [int(x) for x in w]
    if len(w) < 5:
        return "TRUNCATED", [], -1
    if w[0] != 0x07230203:
        return "BAD_MAGIC", [], -1
    major, minor = (w[1] >> 16) & 255, (w[1] >> 8) & 255
    if w[1] & 0xFF0000FF or major != 1 or minor > 6 or w[4] != 0:
        return "BAD_HEADER", [], -1
    starts, i = [], 5
    while i < len(w):
        n = w[i] >> 16
        if n == 0:
            return "ZERO_WORDCOUNT", starts, len(starts)
        if i + n > len(w):
            return "TRUNCATED", starts, len(starts)
        starts.append(i)
        i += n
    return "OK", starts, -1


def _check_framing(words_list):
    words, off = H.batch(words_list)
    d = oracle.decode(words, off)
    for m, w in enumerate(words_list):
        st, starts, er = ref_framing(w)
        assert oracle.STATUS[d["status"][m]] == st
        assert int(d["err_row"][m]) == er
        fr, n = int(d["first_row"][m]), int(d["n_instr"][m])
        assert n == len(starts)
        assert [int(x) - int(off[m]) for x in d["off"][fr:fr + n]] == starts
        assert all(int(d["mod"][r]) == m for r in range(fr, fr + n))
        assert [int(x) for x in d["wc"][fr:fr + n]] == [int(w[p]) >> 16 for p in starts]


def test_bruteforce_short_streams():
    # alphabet: (opcode, word count) with filler operand words; some are
    # well-formed, some have the wrong word count for their opcode
    alphabet = [(17, 2), (128, 5), (248, 2), (253, 1), (5, 3), (9999, 1), (128, 3), (0, 4)]
    mods = []
    for k in range(0, 4):
        for combo in itertools.product(alphabet, repeat=k):
            body = []
            for op, wc in combo:
                body.append([(wc << 16) | op] + [7] * (wc - 1))
            w = H.module(body, bound=8)
            mods.append(w)
            mods.append(w[:-1])            # and the same stream cut one word short
    _check_framing(mods)
    # validation on all of them runs and gives a known status
    words, off = H.batch(mods)
    st, er = oracle.validate(words, off)
    assert st.max() < len(oracle.STATUS)


def test_bruteforce_single_word_corruptions():
    base = H.module(H.minimal_body(), bound=8)
    values = [0, 1, 0xFFFFFFFF, 0x00010000, 0x00020000, 0x00050080, 0x7FFF0011, 0x00030011]
    mods = []
    for i in range(len(base)):
        for v in values:
            x = base.copy(); x[i] = v
            mods.append(x)
    _check_framing(mods)
    words, off = H.batch(mods)
    st, er = oracle.validate(words, off)
    assert st.max() < len(oracle.STATUS)
    enc = oracle.encode(words, off, oracle.decode(words, off), recompute_bound=False)
    assert np.array_equal(enc, words)


# ----------------------------------------------------------------------------
# generator ground truth and invariants
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_generator_ground_truth(seed):
    w, off, starts, bound = synth.single_module(seed)
    d = oracle.decode(w, off)
    assert d["status"][0] == ST["OK"]
    assert np.array_equal(d["off"].astype(np.int64), starts)
    assert int(d["wc"].astype(np.int64).sum()) == len(w) - 5          # word counts fill the module
    assert int(d["rid"].max()) + 1 == bound == int(w[3])
    st, er = oracle.validate(w, off)
    assert st[0] == ST["OK"]
    assert np.array_equal(oracle.encode(w, off, d, True), w)
    assert np.array_equal(oracle.encode(w, off, d, False), w)


def test_generator_strings_module_ground_truth():
    w, off, starts, bound = synth.large_module(5, n_instr=20_000, n_funcs=4)
    d = oracle.decode(w, off)
    assert np.array_equal(d["off"].astype(np.int64), starts)
    assert (d["op"] == H.OpString).sum() > 500 and (d["op"] == H.OpName).sum() > 500
    assert oracle.validate(w, off)[0][0] == ST["OK"]
    assert int(d["rid"].max()) + 1 == bound


def test_batch_invariants():
    n_instr, n_k = synth.batch_shape(40, 7, median=300, lo=200, hi=2000)
    w, off = synth.batch(n_instr, n_k, 7)
    d = oracle.decode(w, off)
    assert (d["status"] == 0).all()
    for m in range(40):
        fr, n = d["first_row"][m], d["n_instr"][m]
        assert int(d["wc"][fr:fr + n].astype(np.int64).sum()) == off[m + 1] - off[m] - 5
    assert (oracle.validate(w, off)[0] == 0).all()
    assert np.array_equal(oracle.encode(w, off, d, True), w)


def test_encode_from_edited_table():
    w = H.module(H.minimal_body(), bound=8)
    d = oracle.decode(*_one(w))
    d["rid"][10] = 40                     # rename the IAdd result
    d["op"][10] = H.OpFAdd               # and turn it into an FAdd
    out = oracle.encode(*_one(w), d, recompute_bound=True)
    p = int(d["off"][10])
    assert out[p] == (5 << 16) | H.OpFAdd and out[p + 2] == 40
    assert out[3] == 41


@pytest.mark.parametrize("inline_names", [False, True])
def test_disassemble_assemble_round_trip(inline_names):
    for seed in (0, 1):
        w, off, _, _ = synth.single_module(seed)
        t, _ = oracle.disassemble(w, off, inline_names=inline_names, header=True)
        back = oracle.assemble(t)
        assert np.array_equal(back, w)
        t2, _ = oracle.disassemble(back, off, inline_names=inline_names, header=True)
        assert t2 == t
    w, off, _, _ = synth.large_module(3, n_instr=5000, n_funcs=2)
    t, _ = oracle.disassemble(w, off, inline_names=inline_names, header=True)
    assert np.array_equal(oracle.assemble(t), w)


# ----------------------------------------------------------------------------
# text details, worked out by hand
# ----------------------------------------------------------------------------
def _const_text(bits_words, width=32):
    body = [H.ins(H.OpTypeFloat, 1, width), H.ins(H.OpConstant, 1, 2, list(bits_words))]
    t, _ = oracle.disassemble(*_one(H.module(body, bound=3)), inline_names=False, header=False)
    return t.decode().splitlines()[1].split(" ", 4)[-1]


@pytest.mark.parametrize("bits,text", [
    (0x3FC00000, "0x1.8p+0"),        # 1.5 = 1.1b x 2^0
    (0x3DCCCCCD, "0x1.99999ap-4"),   # 0.1f: exponent 123-127=-4, fraction 0x4ccccd<<1
    (0x40490FDB, "0x1.921fb6p+1"),   # float pi
    (0x00000001, "0x1p-149"),        # smallest subnormal float, normal as a double
    (0x00000003, "0x1.8p-148"),      # 11b x 2^-149 = 1.1b x 2^-148
    (0x00000005, "0x1.4p-147"),      # 101b x 2^-149 = 1.01b x 2^-147
    (0x00400000, "0x1p-127"),        # 2^22 x 2^-149
    (0x007FFFFF, "0x1.fffffcp-127"), # largest subnormal: 1.(22 ones)b x 2^-127
    (0x00000000, "0x0p+0"),
    (0x80000000, "-0x0p+0"),
    (0xC1200000, "-0x1.4p+3"),       # -10
    (0x7F800000, "inf"),
    (0xFF800000, "-inf"),
    (0x7FC00000, "nan"),
])
def test_float_constant_spelling(bits, text):
    assert _const_text([bits]) == text


@pytest.mark.parametrize("bits,text", [
    (0x3FD5555555555555, "0x1.5555555555555p-2"),   # 1/3
    (0x0000000000000001, "0x0.0000000000001p-1022"), # smallest subnormal double
    (0x3FF0000000000000, "0x1p+0"),
])
def test_double_constant_spelling(bits, text):
    assert _const_text([bits & 0xFFFFFFFF, bits >> 32], width=64) == text


def test_integer_constants_and_escapes_and_names():
    body = [H.ins(H.OpTypeInt, 1, 64, 0), H.ins(H.OpConstant, 1, 2, [0xFFFFFFFF, 0x1]),
            H.ins(H.OpTypeInt, 3, 32, 0), H.ins(H.OpConstant, 3, 4, [4000000000]),
            H.ins(H.OpString, 5, [0x5c226261, 0x7f0a6363, 0x00000080]),   # a b " \ c c \n 0x7f 0x80
            H.ins(H.OpName, 4, H.s("a b-c")), H.ins(H.OpName, 4, H.s("second"))]
    t, _ = oracle.disassemble(*_one(H.module(body, bound=6)), inline_names=True, header=False)
    lines = t.decode().splitlines()
    assert lines[1] == "%2 = OpConstant %1 8589934591"
    assert lines[3] == "%a_b_c_4 = OpConstant %3 4000000000"
    assert lines[4] == '%5 = OpString "ab\\"\\\\cc\\x0a\\x7f\\x80"'
    assert lines[5] == 'OpName %a_b_c_4 "a b-c"'


def test_unparsed_rows_print_raw_words():
    body = [H.ins(H.OpIAdd, 1, 2, 3), [(2 << 16) | 4321, 0xdeadbeef]]
    t, _ = oracle.disassemble(*_one(H.module(body, bound=9)), inline_names=False, header=False)
    assert t == b"OpIAdd 0x00000001 0x00000002 0x00000003\nOp4321 0xdeadbeef\n"
    assert np.array_equal(oracle.assemble(b"; Bound: 9\n" + t), H.module(body, bound=9, generator=0))


def test_enum_spellings():
    body = [H.ins(H.OpLoad, 1, 2, 3, 0x3, 16),                 # Volatile|Aligned 16
            H.ins(H.OpStore, 3, 2, 0),                          # None
            H.ins(H.OpStore, 3, 2, 0x10),                       # unknown bit -> decimal
            H.ins(H.OpDecorate, 3, 11, 28),                     # BuiltIn GlobalInvocationId
            H.ins(H.OpDecorate, 3, 999, 1, 2),                  # unknown decoration, literal tail
            H.ins(H.OpExecutionMode, 4, 17, 8, 1, 1)]
    t, _ = oracle.disassemble(*_one(H.module(body, bound=9)), inline_names=False, header=False)
    assert t.decode().splitlines() == [
        "%2 = OpLoad %1 %3 Volatile|Aligned 16", "OpStore %3 %2 None", "OpStore %3 %2 16",
        "OpDecorate %3 BuiltIn GlobalInvocationId", "OpDecorate %3 999 1 2",
        "OpExecutionMode %4 LocalSize 8 1 1"]


def test_empty_and_header_error_modules_have_no_text():
    good = H.module(H.minimal_body())
    bad = good.copy(); bad[0] = 0
    words, off = H.batch([good[:0], bad, good])
    t, toff = oracle.disassemble(words, off, True, True)
    assert toff[0] == toff[1] == toff[2] == 0 and toff[3] == len(t) > 0
