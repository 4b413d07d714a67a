"""CPU oracle for the batched SPIR-V hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package. The product path (the CUDA library in
``paper_2305_09493_b300``) never imports it and shares no code with it.

The oracle itself is plain sequential C (``spv_oracle.c``); this module only
builds it with gcc and marshals numpy arrays through ctypes. What each
function computes, and which passage of arXiv 2305.09493 it follows, is
documented at the C definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spv_oracle.c")
_LIB = os.path.join(_HERE, "libspv_oracle.so")

# Module status codes, in the order of the C definition.
STATUS = [
    "OK", "BAD_MAGIC", "BAD_HEADER", "TRUNCATED", "ZERO_WORDCOUNT", "UNKNOWN_OPCODE",
    "BAD_OPERANDS", "ID_OUT_OF_BOUND", "DUP_RESULT_ID", "NO_CAPABILITY", "NO_MEMORY_MODEL",
    "MULTI_MEMORY_MODEL", "NO_ENTRY_POINT", "NO_FUNCTION", "MISSING_CAPABILITY",
]
ST = {name: i for i, name in enumerate(STATUS)}


def build_library(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vectorisation tricks)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build_library()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.orc_decode.restype = ctypes.c_int64
        lib.orc_decode.argtypes = [P, P, ctypes.c_int32] + [P] * 10 + [ctypes.c_int64]
        lib.orc_validate.restype = None
        lib.orc_validate.argtypes = [P, P, ctypes.c_int32, P, P]
        lib.orc_encode.restype = None
        lib.orc_encode.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64] + [P] * 7 + [P, ctypes.c_int]
        lib.orc_disassemble.restype = ctypes.c_int64
        lib.orc_disassemble.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, ctypes.c_int, P,
                                        ctypes.c_int64, P]
        lib.orc_build.restype = ctypes.c_int64
        lib.orc_build.argtypes = [P, P, P, P, P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, P,
                                  ctypes.c_int64, P, P, P, P]
        lib.orc_assemble.restype = ctypes.c_int64
        lib.orc_assemble.argtypes = [ctypes.c_char_p, ctypes.c_int64, P, ctypes.c_int64]
        lib.orc_op_info.restype = ctypes.c_int
        lib.orc_op_info.argtypes = [ctypes.c_uint32, P, P, P, P]
        lib.orc_enum_name.restype = ctypes.c_int
        lib.orc_enum_name.argtypes = [ctypes.c_char_p, ctypes.c_uint32, P, P]
        lib.orc_num_ops.restype = ctypes.c_int
        lib.orc_op_at.restype = ctypes.c_uint32
        lib.orc_op_at.argtypes = [ctypes.c_int]
        lib.orc_layout.restype = None
        lib.orc_layout.argtypes = [P, P, P, ctypes.c_int32, P, P]
        lib.orc_layout_class.restype = ctypes.c_int
        lib.orc_layout_class.argtypes = [ctypes.c_uint32, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(words, mod_off):
    words = np.ascontiguousarray(words, dtype=np.uint32)
    mod_off = np.ascontiguousarray(mod_off, dtype=np.int64)
    return words, mod_off


def decode(words, mod_off) -> dict:
    """Decode a batch into the row table (see orc_decode)."""
    words, mod_off = _prep(words, mod_off)
    m = len(mod_off) - 1
    cap = max(1, int(len(words)))
    t = {
        "op": np.zeros(cap, np.uint16), "wc": np.zeros(cap, np.uint16),
        "off": np.zeros(cap, np.uint64), "rtype": np.zeros(cap, np.uint32),
        "rid": np.zeros(cap, np.uint32), "mod": np.zeros(cap, np.uint32),
        "first_row": np.zeros(m, np.int64), "n_instr": np.zeros(m, np.uint32),
        "status": np.zeros(m, np.uint32), "err_row": np.zeros(m, np.int64),
    }
    n = _L().orc_decode(_p(words), _p(mod_off), m, _p(t["op"]), _p(t["wc"]), _p(t["off"]),
                        _p(t["rtype"]), _p(t["rid"]), _p(t["mod"]), _p(t["first_row"]),
                        _p(t["n_instr"]), _p(t["status"]), _p(t["err_row"]), cap)
    assert n >= 0
    for k in ("op", "wc", "off", "rtype", "rid", "mod"):
        t[k] = t[k][:n]
    t["n_rows"] = int(n)
    return t


LAYOUT_STATUS = ["OK", "SECTION_ORDER", "OUTSIDE_FUNCTION", "IN_FUNCTION", "BLOCK", "UNCLOSED"]


def layout(words, mod_off):
    """Logical layout and scopes of every module's decoded rows (see
    orc_layout); returns (status[M] uint32, err_row[M] int64)."""
    words, mod_off = _prep(words, mod_off)
    d = decode(words, mod_off)
    m = len(mod_off) - 1
    status = np.zeros(m, np.uint32)
    err_row = np.zeros(m, np.int64)
    op = d["op"] if len(d["op"]) else np.zeros(1, np.uint16)
    _L().orc_layout(_p(np.ascontiguousarray(op)), _p(d["first_row"]), _p(d["n_instr"]), m, _p(status), _p(err_row))
    return status, err_row


def layout_class(op: int):
    """(class, section) of an opcode for the layout check (see orc_layout_class)."""
    sec = ctypes.c_int()
    c = _L().orc_layout_class(op, ctypes.byref(sec))
    return int(c), int(sec.value)


def validate(words, mod_off):
    """Full validation; returns (status[M] uint32, err_row[M] int64)."""
    words, mod_off = _prep(words, mod_off)
    m = len(mod_off) - 1
    status = np.zeros(m, np.uint32)
    err_row = np.zeros(m, np.int64)
    _L().orc_validate(_p(words), _p(mod_off), m, _p(status), _p(err_row))
    return status, err_row


def encode(words, mod_off, table: dict, recompute_bound: bool = True) -> np.ndarray:
    """Re-encode a (possibly edited) row table over the source words."""
    words, mod_off = _prep(words, mod_off)
    m = len(mod_off) - 1
    out = np.zeros(len(words), np.uint32)
    cols = [np.ascontiguousarray(table[k], dtype=dt) for k, dt in
            (("op", np.uint16), ("wc", np.uint16), ("off", np.uint64), ("rtype", np.uint32),
             ("rid", np.uint32), ("first_row", np.int64), ("n_instr", np.uint32))]
    _L().orc_encode(_p(words), _p(mod_off), m, len(words), *[_p(c) for c in cols], _p(out),
                    1 if recompute_bound else 0)
    return out


def disassemble(words, mod_off, inline_names: bool = True, header: bool = True):
    """Disassembly text of every module; returns (bytes, text_off[M+1] int64)."""
    words, mod_off = _prep(words, mod_off)
    m = len(mod_off) - 1
    text_off = np.zeros(m + 1, np.int64)
    n = _L().orc_disassemble(_p(words), _p(mod_off), m, int(inline_names), int(header), None, 0,
                             _p(text_off))
    buf = ctypes.create_string_buffer(max(1, n))
    _L().orc_disassemble(_p(words), _p(mod_off), m, int(inline_names), int(header), buf, n,
                         _p(text_off))
    return buf.raw[:n], text_off


def assemble_one(text: bytes):
    """Assemble one module's text. Returns (words, 0) or (None, line): the
    1-based number of the first line that does not parse."""
    text = bytes(text)
    cap = len(text) + 64
    while True:
        out = np.zeros(cap, np.uint32)
        n = _L().orc_assemble(text, len(text), _p(out), cap)
        if n < 0:
            return None, int(-n)
        if n <= cap:
            return out[:n].copy(), 0
        cap = int(n)


def assemble(text: bytes) -> np.ndarray:
    """Assemble one module from text (inverse of disassemble with header)."""
    words, line = assemble_one(text)
    if words is None:
        raise ValueError(f"assemble: parse error at line {line}")
    return words


# Assembler module status codes.
ASM_STATUS = ["OK", "SYNTAX"]


def assemble_batch(text: bytes, text_off):
    """Assemble every module of a batch: module m's text is
    text[text_off[m]:text_off[m+1]]. Returns (words, word_off, status,
    err_line): a module that does not parse gets no words, status SYNTAX and
    the number of its first bad line (-1 when OK)."""
    text = bytes(text)
    text_off = np.asarray(text_off, np.int64)
    n = len(text_off) - 1
    parts, word_off = [], np.zeros(n + 1, np.int64)
    status = np.zeros(n, np.uint32)
    err = np.full(n, -1, np.int64)
    for m in range(n):
        w, line = assemble_one(text[text_off[m]:text_off[m + 1]])
        if w is None:
            status[m], err[m] = 1, line
            w = np.zeros(0, np.uint32)
        parts.append(w)
        word_off[m + 1] = word_off[m] + len(w)
    words = np.concatenate(parts) if parts else np.zeros(0, np.uint32)
    return words.astype(np.uint32), word_off, status, err


# Builder module status codes.
BUILD_STATUS = ["OK", "BAD_REF", "BAD_ROW"]


def build_batch(ol, version: int = 0x00010200, generator: int = 0):
    """Modules from op lists (a dict with op, opd_off, opd, opd_ref, row_off).
    Returns (words, word_off, status, err_row, ids): ids[r] is the id given to
    row r (0 if its opcode has no result id)."""
    op = np.ascontiguousarray(ol["op"], np.uint16)
    opd_off = np.ascontiguousarray(ol["opd_off"], np.int64)
    opd = np.ascontiguousarray(ol["opd"], np.uint32)
    opd_ref = np.ascontiguousarray(ol["opd_ref"], np.uint8)
    row_off = np.ascontiguousarray(ol["row_off"], np.int64)
    m = len(row_off) - 1
    word_off = np.zeros(m + 1, np.int64)
    status = np.zeros(max(1, m), np.uint32)
    err = np.zeros(max(1, m), np.int64)
    ids = np.zeros(max(1, len(op)), np.uint32)
    n = _L().orc_build(_p(op), _p(opd_off), _p(opd), _p(opd_ref), _p(row_off), m, version, generator, None, 0,
                       _p(word_off), _p(status), _p(err), _p(ids))
    out = np.zeros(max(1, n), np.uint32)
    _L().orc_build(_p(op), _p(opd_off), _p(opd), _p(opd_ref), _p(row_off), m, version, generator, _p(out), n,
                   _p(word_off), _p(status), _p(err), _p(ids))
    return out[:n], word_off, status[:m], err[:m], ids[:len(op)]


def op_info(op: int):
    """(name, has_rtype, has_rid, capability) of an opcode, or None."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    name = ctypes.c_char_p()
    if _L().orc_op_info(op, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(name)):
        return None
    return name.value.decode(), a.value, b.value, c.value


def enum_name(kind: str, value: int):
    """(name, capability) of an enumerant, or None."""
    name = ctypes.c_char_p()
    cap = ctypes.c_int()
    if _L().orc_enum_name(kind.encode(), value, ctypes.byref(name), ctypes.byref(cap)):
        return None
    return name.value.decode(), cap.value


def opcodes():
    lib = _L()
    return [lib.orc_op_at(i) for i in range(lib.orc_num_ops())]
