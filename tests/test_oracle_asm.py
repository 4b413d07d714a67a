"""Pins of the oracle's assembler (section 3.4.4, Dis/Assembler: text back to
words, with the paper's map from id names to ids), independent of the oracle:

* hand-written texts whose words are built by hand from the SPIR-V numbering
  (tests/spvhand.py), with named ids numbered by first appearance above the
  largest explicit id, worked out by hand;
* float constants against bit patterns fixed by IEEE 754 (worked examples, and
  Python's own correctly rounded float parser on random values in both the
  hexadecimal and the shortest decimal spelling), including the rounding of a
  32-bit constant through double;
* every kind of bad line, with its line number;
* the named-id rule against a second statement of it: renaming every named
  token to the id the rule gives, in Python, must give the same words.
"""
import re
import struct

import numpy as np
import pytest

import oracle
from paper_2305_09493_b300 import synth
from tests import spvhand as H

HEAD = ("; SPIR-V\n; Version: 1.2\n; Generator: 0x00000020\n; Bound: 100\n; Schema: 0\n")


def sb(b: bytes):
    b = b + b"\0"
    b += b"\0" * (-len(b) % 4)
    return [int.from_bytes(b[i:i + 4], "little") for i in range(0, len(b), 4)]


def asm(text: str):
    return oracle.assemble_one(text.encode())


def words_of(text: str):
    w, line = asm(text)
    assert w is not None, f"line {line}"
    return [int(x) for x in w]


def test_named_ids_by_first_appearance():
    text = (
        "OpCapability Addresses\n"
        "OpCapability Kernel\n"
        "OpMemoryModel Physical64 OpenCL\n"
        'OpEntryPoint Kernel %main "k"\n'
        "%void = OpTypeVoid\n"
        "%fn = OpTypeFunction %void\n"
        "%main = OpFunction %void None %fn\n"
        "%entry = OpLabel\n"
        "OpReturn\n"
        "OpFunctionEnd\n")
    # no explicit id: main 1, void 2, fn 3, entry 4 (first appearances in
    # that order); bound 5
    body = [H.ins(H.OpCapability, H.CAP_ADDRESSES), H.ins(H.OpCapability, H.CAP_KERNEL),
            H.ins(H.OpMemoryModel, H.AM_PHYSICAL64, H.MM_OPENCL), H.ins(H.OpEntryPoint, H.EXEC_KERNEL, 1, H.s("k")),
            H.ins(H.OpTypeVoid, 2), H.ins(H.OpTypeFunction, 3, 2), H.ins(H.OpFunction, 2, 1, 0, 3),
            H.ins(H.OpLabel, 4), H.ins(H.OpReturn), H.ins(H.OpFunctionEnd)]
    assert words_of(text) == list(H.module(body, bound=5, generator=0))
    # an explicit id anywhere in the module moves every named id above it
    text2 = text.replace("%fn = OpTypeFunction %void\n", "%fn = OpTypeFunction %void\n%x_7 = OpTypeInt 32 0\n")
    body2 = [H.ins(H.OpCapability, H.CAP_ADDRESSES), H.ins(H.OpCapability, H.CAP_KERNEL),
             H.ins(H.OpMemoryModel, H.AM_PHYSICAL64, H.MM_OPENCL), H.ins(H.OpEntryPoint, H.EXEC_KERNEL, 8, H.s("k")),
             H.ins(H.OpTypeVoid, 9), H.ins(H.OpTypeFunction, 10, 9), H.ins(H.OpTypeInt, 7, 32, 0),
             H.ins(H.OpFunction, 9, 8, 0, 10), H.ins(H.OpLabel, 11), H.ins(H.OpReturn), H.ins(H.OpFunctionEnd)]
    assert words_of(text2) == list(H.module(body2, bound=12, generator=0))


def test_more_id_forms():
    # %%5 is a name (the digits follow a '%' that is not the first byte);
    # %a%_5 is id 5; %00012 is id 12
    w = words_of("%%5 = OpTypeVoid\n%a%_5 = OpTypeVoid\n%00012 = OpTypeVoid\n")
    assert w[5:] == [H.ins(H.OpTypeVoid, i)[k] for i in (13, 5, 12) for k in (0, 1)]
    assert asm("%_4294967296 = OpTypeVoid\n") == (None, 1)


def test_explicit_id_forms():
    # %7, %a_7 and %_7 are all id 7; %a7, %_ and %7a are names
    w = words_of("%7 = OpTypeVoid\n%a_7 = OpTypeVoid\n%_7 = OpTypeVoid\n%a7 = OpTypeVoid\n%_ = OpTypeVoid\n"
                 "%7a = OpTypeVoid\n%a7 = OpTypeVoid\n")
    assert w[5:] == [H.ins(H.OpTypeVoid, i)[k] for i in (7, 7, 7, 8, 9, 10, 8) for k in (0, 1)]
    assert w[3] == 11                                    # bound: largest id + 1


def _const_module(type_line, value):
    return HEAD + type_line + "\n%5 = OpConstant %2 " + value + "\n"


def const_words(type_line, value):
    return words_of(_const_module(type_line, value))[5 + (3 if "Float" in type_line else 4):][3:]


F32, F64 = "%2 = OpTypeFloat 32", "%2 = OpTypeFloat 64"
I32, I64 = "%2 = OpTypeInt 32 0", "%2 = OpTypeInt 64 0"


@pytest.mark.parametrize("ty,value,want", [
    (F32, "0x1.8p+0", [0x3fc00000]),                      # 1.5
    (F32, "-0x1.8p+1", [0xc0400000]),                     # -3
    (F32, "0.1", [0x3dcccccd]),
    (F64, "0.1", [0x9999999a, 0x3fb99999]),
    (F32, "inf", [0x7f800000]), (F32, "-inf", [0xff800000]),
    (F32, "nan", [0x7fc00000]), (F32, "-nan", [0xffc00000]),
    (F64, "nan", [0x00000000, 0x7ff80000]),
    (F32, "0x1p-149", [0x00000001]),                      # smallest subnormal float
    (F64, "0x1.fffffffffffffp+1023", [0xffffffff, 0x7fefffff]),
    (F64, "0x0.0000000000001p-1022", [0x00000001, 0x00000000]),
    (F32, "1e39", [0x7f800000]),                          # overflows float
    (F32, "0x1.000001p0", [0x3f800000]),                  # halfway: to even
    (F32, "0x1.0000010000001p0", [0x3f800001]),           # above halfway: up
    # 1 + 2^-24 + 2^-53 rounds to double 1 + 2^-24 (a tie, to even), then to
    # float 1.0 (a tie again): double rounding, as defined
    (F32, "0x1.00000100000008p0", [0x3f800000]),
    (F32, "-0", [0x80000000]), (F32, "0.", [0x00000000]), (F32, ".5", [0x3f000000]),
    (F32, "+2.5e-1", [0x3e800000]), (F32, "0X1P3", [0x41000000]),
    (I32, "7", [7]), (I32, "4294967296", [0, 1]),         # a 32-bit type, 33-bit value: two words
    (I64, "5", [5, 0]), (I64, "18446744073709551615", [0xffffffff, 0xffffffff]),
    (I32, "1.0", [0x3f800000]),                           # a float literal is a float
    (I32, "18446744073709551616", [0x5f800000]),          # so is an integer beyond 64 bits: 2^64
    (I32, "1 2 3", [1, 2, 3]),                            # several tokens: one word each
])
def test_constant_values(ty, value, want):
    w = words_of(_const_module(ty, value))
    # header 5, type line (3 or 4 words), then OpConstant: word 0, type, id, value
    k = 5 + len(H.ins(0, *([0] * (2 if "Float" in ty else 3))))
    assert w[k] == ((3 + len(want)) << 16) | H.OpConstant
    assert w[k + 3:] == want


def test_constant_width_from_first_declaration_anywhere():
    # the type is declared after the constant, then again with another width
    t = HEAD + "%5 = OpConstant %2 1\n%2 = OpTypeInt 64 0\n%2 = OpTypeInt 32 0\n"
    w = words_of(t)
    assert w[5:10] == H.ins(H.OpConstant, 2, 5, 1, 0)
    t = HEAD + "%5 = OpConstant %9 1\n"                     # no declaration: 32-bit integer
    assert words_of(t)[5:] == H.ins(H.OpConstant, 9, 5, 1)


def _bits64(x: float):
    return struct.unpack("<2I", struct.pack("<d", x))


def _bits32(x: float):
    with np.errstate(over="ignore"):
        return [int(np.array([x], np.float64).astype(np.float32).view(np.uint32)[0])]


def test_float_constants_against_python_parser():
    rng = np.random.default_rng(3)
    vals = list(rng.integers(0, 2 ** 64, 300, dtype=np.uint64).view(np.float64))
    vals += list(rng.standard_normal(100) * 10.0 ** rng.integers(-40, 40, 100))
    vals = [v for v in vals if np.isfinite(v)]
    lines64, lines32, want64, want32 = [], [], [], []
    for i, v in enumerate(vals):
        v = float(v)
        for spelling in (v.hex(), repr(v)):
            lines64.append(f"%{100 + len(lines64)} = OpConstant %2 {spelling}")
            want64.append(list(_bits64(v)))
            lines32.append(f"%{100 + len(lines32)} = OpConstant %2 {spelling}")
            want32.append(_bits32(v))
    for ty, lines, want in ((F64, lines64, want64), (F32, lines32, want32)):
        w = words_of(HEAD + ty + "\n" + "\n".join(lines) + "\n")
        k = 5 + len(H.ins(0, 0, 0))
        for i, exp in enumerate(want):
            n = w[k] >> 16
            assert w[k + 3:k + n] == exp, (lines[i], [hex(x) for x in w[k + 3:k + n]], [hex(x) for x in exp])
            k += n


def test_strings_and_escapes():
    t = HEAD + r'OpExtension "a\"b\\c\x41\x4a\xg1\q"' + "\n" + 'OpName %3 ""\n' + 'OpName %3 "abcd"\n'
    w = words_of(t)
    want = H.ins(10, sb(b'a"b\\cAJxg1q')) + H.ins(H.OpName, 3, sb(b"")) + H.ins(H.OpName, 3, sb(b"abcd"))
    assert w[5:] == want


def test_header_lines():
    def hdr(t):
        return words_of(t + "OpNop\n")[:5]
    assert hdr("") == [H.MAGIC, 0x00010200, 0, 1, 0]        # defaults; no id: bound 1
    assert hdr("; Version: 1.5\n; Generator: 0xDEADbeef\n; Bound: 99\n; Schema: 3\n") == \
        [H.MAGIC, 0x00010500, 0xdeadbeef, 99, 3]
    # other spellings are plain comments; the last header line wins
    assert hdr("; Version: 1.5 \n; Version:1.3\n; Bound: 4294967296\n; Bound: 9x\n; bound: 5\n") == \
        [H.MAGIC, 0x00010200, 0, 1, 0]
    assert hdr("; Version: 1.256\n; Version: 1.0\n; Version: 1.4\n; Bound: 7\n; Bound: 8\n") == \
        [H.MAGIC, 0x00010400, 0, 8, 0]


def test_enumerants():
    t = HEAD + ("OpCapability 6\nOpDecorate %3 Alignment 16\nOpDecorate %3 1234 5 6\n"
                "%4 = OpFunction %1 Inline|Const %2\n%5 = OpFunction %1 None %2\n%6 = OpFunction %1 3 %2\n"
                "OpStore %7 %8 Aligned|Volatile 4\n")
    w = words_of(t)
    want = (H.ins(H.OpCapability, 6) + H.ins(H.OpDecorate, 3, 44, 16) + H.ins(H.OpDecorate, 3, 1234, 5, 6)
            + H.ins(H.OpFunction, 1, 4, 9, 2) + H.ins(H.OpFunction, 1, 5, 0, 2) + H.ins(H.OpFunction, 1, 6, 3, 2)
            + H.ins(H.OpStore, 7, 8, 3, 4))
    assert w[5:] == want


def test_raw_lines():
    t = HEAD + "Op300 0x00000001 0xABCDEF01\nOpNop\nOpIAdd 0x00000002 0x00000003\nOp65535\n"
    w = words_of(t)
    assert w[5:] == [(3 << 16) | 300, 1, 0xabcdef01, H.OpNop | (1 << 16), (3 << 16) | H.OpIAdd, 2, 3,
                     (1 << 16) | 65535]


@pytest.mark.parametrize("line", [
    "OpFoo %1",                       # unknown name
    "Op65536",                        # opcode beyond 16 bits
    "Op12x",
    "   ",                            # spaces only
    "%1 = OpNop",                     # a result id on an instruction without one
    "OpTypeVoid",                     # a result id missing
    "%1 = OpTypeInt 32",              # an operand missing
    "%1 = OpTypeInt 32 0 1",          # one too many
    "%1 = OpTypeInt 4294967296 0",    # literal beyond 32 bits
    "%1 = OpTypeInt x 0",
    "%1 = OpTypeVoid extra",
    "OpName % \"a\"",                 # an id without a name
    "OpName %99999999999 \"a\"",      # an explicit id beyond 32 bits
    "OpName %1 \"abc",                # an unclosed string
    "OpName %1 \"abc\\\"",            # the closing quote escaped
    "OpName %1 abc",                  # not a string
    "%5 = OpConstant %2 1.5x",        # not a float literal
    "%5 = OpConstant %2 0x",
    "%5 = OpConstant %2 1e",
    "%5 = OpConstant %2 1 4294967296",
    "%5 = OpConstant %2 Inf",
    "%5 = OpConstant %2",
    "OpCapability Kernels",
    "%4 = OpFunction %1 Inline| %2",  # an empty bit name
    "%4 = OpFunction %1 Inline||Const %2",
    "OpIAdd 0x00000002 3",            # a raw line with a non-raw word
    "%3 = Op300 0x00000001",          # a raw line with a result id
])
def test_bad_lines(line):
    t = HEAD + "OpNop\n\n; comment\n" + line + "\nOpNop\n"
    w, err = asm(t)
    assert w is None and err == 9, (line, err)


def test_word_limit():
    ok = HEAD + 'OpExtension "' + "a" * (65534 * 4 - 1) + '"\n'
    assert len(words_of(ok)) == 5 + 65535
    bad = HEAD + 'OpExtension "' + "a" * (65534 * 4) + '"\n'
    assert asm(bad) == (None, 6)


def test_fresh_id_overflow():
    t = "%4294967295 = OpTypeVoid\nOpNop\n%a = OpTypeVoid\n"
    assert asm(t) == (None, 3)
    assert words_of("%4294967294 = OpTypeVoid\n%a = OpTypeVoid\n")[7:] == [(2 << 16) | 19, 0xffffffff]


def test_named_rule_against_a_renaming():
    """Give a random half of the ids of generated modules a name ("%v<id>x"),
    and assemble: the words must be those of the text with each name replaced
    by M + 1 + its rank of first appearance (M = the largest id left
    explicit), worked out here."""
    w, off = synth.module_batch(6, 11)
    text, toff = oracle.disassemble(w, off, False, True)
    idtok = re.compile(rb"%([0-9]+)(?=[ \n])")
    rng = np.random.default_rng(4)
    for m in range(len(off) - 1):
        t = re.sub(rb"(?m)^; Bound: .*\n", b"", text[toff[m]:toff[m + 1]])
        ids = sorted({int(x) for x in idtok.findall(t)})
        named = {i for i in ids if rng.random() < 0.5}
        kept = [i for i in ids if i not in named]
        base = max(kept) if kept else 0
        order = []
        for mo in idtok.finditer(t):
            i = int(mo.group(1))
            if i in named and i not in order:
                order.append(i)
        rank = {i: base + 1 + k for k, i in enumerate(order)}
        as_names = idtok.sub(lambda mo: b"%%v%sx" % mo.group(1) if int(mo.group(1)) in named else mo.group(0), t)
        as_ids = idtok.sub(lambda mo: b"%%%d" % rank.get(int(mo.group(1)), int(mo.group(1))), t)
        got, line = oracle.assemble_one(as_names)
        want, line2 = oracle.assemble_one(as_ids)
        assert got is not None and want is not None, (line, line2)
        assert np.array_equal(got, want)
        assert got[3] == max(kept + list(rank.values())) + 1


def test_batch_wrapper():
    w, off = synth.module_batch(5, 2)
    text, toff = oracle.disassemble(w, off, True, True)
    bad = text[:toff[2]] + b"OpBogus\n" + text[toff[2]:]
    toff2 = toff.copy()
    toff2[3:] += len(b"OpBogus\n")
    words, woff, st, err = oracle.assemble_batch(bad, toff2)
    assert list(st) == [0, 0, 1, 0, 0]
    assert err[2] == 1 and (err[[0, 1, 3, 4]] == -1).all()
    assert woff[3] == woff[2]
    for m in (0, 1, 3, 4):
        assert np.array_equal(words[woff[m]:woff[m + 1]], w[off[m]:off[m + 1]])
