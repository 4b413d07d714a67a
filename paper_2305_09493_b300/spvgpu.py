"""Python binding of the C ABI in include/spv.h (libspvgpu.so).

Argument marshalling only: every step of decode / validate / encode /
disassemble runs in the library's CUDA kernels. PyTorch provides device
memory (tensors) and streams. There is no CPU fallback: if the library is
missing or cannot be loaded, every call raises.

Two layers:
  * ``spv_*`` functions with the C names and raw pointer arguments;
  * ``process`` / ``decode`` / ``validate`` / ``encode`` / ``disassemble``,
    which take torch tensors, allocate outputs and workspace with torch and
    return tensors (uint32 / uint16 data are held in int32 / int16 tensors).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspvgpu.so")

STATUS = [
    "OK", "BAD_MAGIC", "BAD_HEADER", "TRUNCATED", "ZERO_WORDCOUNT", "UNKNOWN_OPCODE", "BAD_OPERANDS",
    "ID_OUT_OF_BOUND", "DUP_RESULT_ID", "NO_CAPABILITY", "NO_MEMORY_MODEL", "MULTI_MEMORY_MODEL",
    "NO_ENTRY_POINT", "NO_FUNCTION", "MISSING_CAPABILITY", "TIMEOUT", "CAPACITY",
]
SPV_SUCCESS, SPV_E_ARG, SPV_E_WORKSPACE, SPV_E_CUDA, SPV_E_UNSUPPORTED = 0, -1, -2, -3, -4

P = ctypes.c_void_p


class SpvBatch(ctypes.Structure):
    _fields_ = [("words", P), ("mod_off", P), ("n_modules", ctypes.c_int32), ("n_words", ctypes.c_int64)]


class SpvTable(ctypes.Structure):
    _fields_ = [("op", P), ("wc", P), ("off", P), ("rtype", P), ("rid", P), ("mod", P),
                ("mod_first_row", P), ("mod_n_instr", P), ("capacity_rows", ctypes.c_int64)]


class SpvConfig(ctypes.Structure):
    _fields_ = [("tile_words", ctypes.c_int32), ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("per_module", ctypes.c_int32), ("max_spins", ctypes.c_int64), ("test_stall_tile", ctypes.c_int64),
                ("no_speculation", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SpvOplist(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("opd_off", ctypes.c_void_p), ("opd", ctypes.c_void_p),
                ("opd_ref", ctypes.c_void_p), ("row_off", ctypes.c_void_p), ("n_modules", ctypes.c_int32),
                ("n_rows", ctypes.c_int64)]


class SpvDisOpts(ctypes.Structure):
    _fields_ = [("inline_names", ctypes.c_int32), ("header", ctypes.c_int32), ("max_spins", ctypes.c_int64),
                ("test_stall_tile", ctypes.c_int64)]


class SpvError(RuntimeError):
    pass


_lib = None


def load():
    """Load libspvgpu.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libspvgpu.so not built ({LIB_PATH}); run paper_2305_09493_b300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    BP, TP, CP, DOP = (ctypes.POINTER(SpvBatch), ctypes.POINTER(SpvTable), ctypes.POINTER(SpvConfig),
                       ctypes.POINTER(SpvDisOpts))
    i32, i64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.spv_workspace_bytes.restype = sz
    lib.spv_workspace_bytes.argtypes = [i32, i64, i64, CP]
    lib.spv_process_batch.restype = ctypes.c_int
    lib.spv_process_batch.argtypes = [BP, TP, P, P, ctypes.c_int, P, ctypes.c_int, P, sz, i64, CP, P]
    lib.spv_decode_batch.restype = ctypes.c_int
    lib.spv_decode_batch.argtypes = [BP, TP, P, P, P, sz, CP, P]
    lib.spv_validate_batch.restype = ctypes.c_int
    lib.spv_validate_batch.argtypes = [BP, TP, P, P, P, sz, i64, P]
    lib.spv_encode_batch.restype = ctypes.c_int
    lib.spv_encode_batch.argtypes = [BP, TP, P, ctypes.c_int, P]
    lib.spv_dis_workspace_bytes.restype = sz
    lib.spv_dis_workspace_bytes.argtypes = [i32, i64, i64, i64]
    lib.spv_disassemble_batch.restype = ctypes.c_int
    lib.spv_disassemble_batch.argtypes = [BP, TP, DOP, P, ctypes.c_uint64, P, P, P, sz, i64, P]
    lib.spv_op_info.restype = ctypes.c_int
    lib.spv_op_info.argtypes = [ctypes.c_uint32, P, P, P, P]
    lib.spv_enum_info.restype = ctypes.c_int
    lib.spv_enum_info.argtypes = [ctypes.c_char_p, ctypes.c_uint32, P, P]
    lib.spv_version.restype = ctypes.c_char_p
    lib.spv_process_batch_noalloc.restype = ctypes.c_int
    lib.spv_process_batch_noalloc.argtypes = [BP, TP, P, P, ctypes.c_int, P, ctypes.c_int, CP, P]
    lib.spv_layout_batch.restype = ctypes.c_int
    lib.spv_layout_batch.argtypes = [TP, i32, P, P, P, sz, P]
    lib.spv_layout_workspace_bytes.restype = sz
    lib.spv_layout_workspace_bytes.argtypes = [i32, i64]
    lib.spv_op_layout.restype = ctypes.c_int
    lib.spv_op_layout.argtypes = [ctypes.c_uint32, P, P]
    lib.spv_autotune_batch.restype = ctypes.c_int
    lib.spv_autotune_batch.argtypes = [BP, TP, P, P, ctypes.c_int, P, P, sz, ctypes.c_int, CP,
                                       ctypes.POINTER(ctypes.c_float), P]
    lib.spv_asm_workspace_bytes.restype = sz
    lib.spv_asm_workspace_bytes.argtypes = [i32, ctypes.c_uint64, i64, i64]
    lib.spv_assemble_batch.restype = ctypes.c_int
    lib.spv_assemble_batch.argtypes = [P, ctypes.c_uint64, P, i32, P, i64, P, P, P, P, sz, i64, i64, P]
    lib.spv_build_workspace_bytes.restype = sz
    lib.spv_build_workspace_bytes.argtypes = [i32, i64]
    lib.spv_build_batch.restype = ctypes.c_int
    lib.spv_build_batch.argtypes = [ctypes.POINTER(SpvOplist), ctypes.c_uint32, ctypes.c_uint32, P, i64, P, P, P, P,
                                    P, sz, P]
    lib.spv_query_sizes.restype = ctypes.c_int
    lib.spv_query_sizes.argtypes = [BP, DOP, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_uint64), P]
    lib.spv_asm_required.restype = ctypes.c_int
    lib.spv_asm_required.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# raw C-named layer
# ---------------------------------------------------------------------------
def spv_workspace_bytes(n_modules, n_words, arena_words=0, cfg=None):
    return load().spv_workspace_bytes(n_modules, n_words, arena_words, ctypes.byref(cfg) if cfg else None)


def spv_dis_workspace_bytes(n_modules, n_words, n_rows_capacity, arena_words=0):
    return load().spv_dis_workspace_bytes(n_modules, n_words, n_rows_capacity, arena_words)


def spv_process_batch(batch, table, status, err_row, validate, out_words, recompute_bound, workspace, ws_bytes,
                      arena_words, cfg, stream):
    return load().spv_process_batch(ctypes.byref(batch), ctypes.byref(table), status, err_row, validate,
                                    out_words, recompute_bound, workspace, ws_bytes, arena_words,
                                    ctypes.byref(cfg) if cfg else None, stream)


def spv_process_batch_noalloc(batch, table, status, err_row, validate, out_words, recompute_bound, cfg, stream):
    """spv_process_batch without a workspace: the library's fixed device
    scratch (SPV_NOALLOC_SCRATCH_BYTES) is used instead, for callers that
    cannot allocate device memory."""
    return load().spv_process_batch_noalloc(ctypes.byref(batch), ctypes.byref(table), status, err_row, validate,
                                            out_words, recompute_bound, ctypes.byref(cfg) if cfg else None, stream)


SPV_NOALLOC_SCRATCH_BYTES = 32 << 20


def spv_decode_batch(batch, table, status, err_row, workspace, ws_bytes, cfg, stream):
    return load().spv_decode_batch(ctypes.byref(batch), ctypes.byref(table), status, err_row, workspace,
                                   ws_bytes, ctypes.byref(cfg) if cfg else None, stream)


def spv_validate_batch(batch, table, status, err_row, workspace, ws_bytes, arena_words, stream):
    return load().spv_validate_batch(ctypes.byref(batch), ctypes.byref(table), status, err_row, workspace,
                                     ws_bytes, arena_words, stream)


def spv_encode_batch(batch, table, out_words, recompute_bound, stream):
    return load().spv_encode_batch(ctypes.byref(batch), ctypes.byref(table), out_words, recompute_bound, stream)


def spv_disassemble_batch(batch, table, opts, text, text_capacity, text_off, dis_status, workspace, ws_bytes,
                          arena_words, stream):
    return load().spv_disassemble_batch(ctypes.byref(batch), ctypes.byref(table), ctypes.byref(opts), text,
                                        text_capacity, text_off, dis_status, workspace, ws_bytes, arena_words,
                                        stream)


def spv_op_info(op):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    name = ctypes.c_char_p()
    if load().spv_op_info(op, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(name)):
        return None
    return name.value.decode(), a.value, b.value, c.value


def spv_enum_info(kind, value):
    name = ctypes.c_char_p()
    cap = ctypes.c_int()
    if load().spv_enum_info(kind.encode(), value, ctypes.byref(name), ctypes.byref(cap)):
        return None
    return name.value.decode(), cap.value


def spv_version():
    return load().spv_version().decode()


# ---------------------------------------------------------------------------
# torch layer
# ---------------------------------------------------------------------------
def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc, what):
    if rc != SPV_SUCCESS:
        raise SpvError(f"{what} failed with code {rc}")


def make_config(tile_words=0, threads=0, ctas_per_sm=0, per_module=0, max_spins=0, test_stall_tile=0,
                no_speculation=0):
    return SpvConfig(tile_words, threads, ctas_per_sm, per_module, max_spins, test_stall_tile, no_speculation, 0)


class Table:
    """Device columns of the structure-of-arrays instruction table."""

    def __init__(self, n_modules, capacity_rows, device):
        e = lambda n, dt: torch.empty(max(1, n), dtype=dt, device=device)
        self.op = e(capacity_rows, torch.int16)
        self.wc = e(capacity_rows, torch.int16)
        self.off = e(capacity_rows, torch.int64)
        self.rtype = e(capacity_rows, torch.int32)
        self.rid = e(capacity_rows, torch.int32)
        self.mod = e(capacity_rows, torch.int32)
        self.mod_first_row = e(n_modules + 1, torch.int64)
        self.mod_n_instr = e(n_modules, torch.int32)
        self.capacity_rows = capacity_rows

    def c(self):
        return SpvTable(self.op.data_ptr(), self.wc.data_ptr(), self.off.data_ptr(), self.rtype.data_ptr(),
                        self.rid.data_ptr(), self.mod.data_ptr(), self.mod_first_row.data_ptr(),
                        self.mod_n_instr.data_ptr(), self.capacity_rows)

    def to_numpy(self, n_rows=None):
        """Host copy with the table's own unsigned dtypes."""
        if n_rows is None:
            n_rows = int(self.mod_first_row[-1].item())
        n = min(n_rows, self.capacity_rows)
        cpu = lambda t, k: t[:k].cpu().numpy()
        return {
            "op": cpu(self.op, n).view(np.uint16), "wc": cpu(self.wc, n).view(np.uint16),
            "off": cpu(self.off, n).view(np.uint64), "rtype": cpu(self.rtype, n).view(np.uint32),
            "rid": cpu(self.rid, n).view(np.uint32), "mod": cpu(self.mod, n).view(np.uint32),
            "first_row": self.mod_first_row.cpu().numpy(), "n_instr": self.mod_n_instr.cpu().numpy().view(np.uint32),
        }


def batch_of(words, mod_off):
    return SpvBatch(words.data_ptr(), mod_off.data_ptr(), mod_off.numel() - 1, words.numel())


class Workspace:
    """Caller-owned workspace reused across calls of the same batch shape."""

    def __init__(self, n_modules, n_words, device, arena_words=0, cfg=None):
        self.bytes = spv_workspace_bytes(n_modules, n_words, arena_words, cfg)
        if self.bytes == 0 and (n_modules or n_words):
            raise SpvError("invalid configuration for workspace")
        self.buf = torch.empty(max(1, self.bytes), dtype=torch.uint8, device=device)
        self.arena_words = arena_words


def process(words, mod_off, *, validate=True, encode=False, recompute_bound=True, cfg=None, table=None,
            workspace=None, out=None, stream=None, capacity_rows=None, arena_words=0):
    """Decode (+ validate) (+ encode) a batch on its device in one persistent
    launch. words: int32 device tensor (the uint32 words); mod_off: int64
    device tensor of n_modules + 1 offsets. Returns a dict of tensors."""
    m = mod_off.numel() - 1
    dev = words.device
    cap = capacity_rows if capacity_rows is not None else max(1, words.numel())
    if table is None:
        table = Table(m, cap, dev)
    if workspace is None:
        workspace = Workspace(m, words.numel(), dev, arena_words, cfg)
    status = torch.empty(max(1, m), dtype=torch.int32, device=dev)
    err_row = torch.empty(max(1, m), dtype=torch.int64, device=dev)
    if encode and out is None:
        out = torch.empty_like(words)
    b, t = batch_of(words, mod_off), table.c()
    rc = spv_process_batch(b, t, _ptr(status), _ptr(err_row), 1 if validate else 0, _ptr(out) if encode else None,
                           1 if recompute_bound else 0, _ptr(workspace.buf), workspace.bytes,
                           workspace.arena_words, cfg, _stream(stream))
    _check(rc, "spv_process_batch")
    return {"table": table, "status": status[:m], "err_row": err_row[:m], "out": out if encode else None,
            "workspace": workspace}


# the tile shapes the library's autotuner tries
TILE_SHAPES = ((4096, 256), (8192, 512), (2048, 256), (2048, 128), (1024, 128), (512, 64))


def autotune_workspace_bytes(n_modules, n_words, arena_words=0):
    """Workspace bytes that fit spv_process_batch for every tile shape."""
    return max(spv_workspace_bytes(n_modules, n_words, arena_words, make_config(t, n)) for t, n in TILE_SHAPES)


def autotune(words, mod_off, *, validate=True, encode=True, table=None, workspace=None, out=None, reps=3, stream=None):
    """spv_autotune_batch: the fastest tile shape of spv_process_batch for
    this batch. Returns (SpvConfig, mean ms of one call, process outputs of
    that shape)."""
    m = mod_off.numel() - 1
    dev = words.device
    if table is None:
        table = Table(m, max(1, words.numel()), dev)
    if workspace is None:
        workspace = Workspace.__new__(Workspace)
        workspace.bytes = autotune_workspace_bytes(m, words.numel())
        workspace.buf = torch.empty(max(1, workspace.bytes), dtype=torch.uint8, device=dev)
        workspace.arena_words = 0
    status = torch.empty(max(1, m), dtype=torch.int32, device=dev)
    err_row = torch.empty(max(1, m), dtype=torch.int64, device=dev)
    if encode and out is None:
        out = torch.empty_like(words)
    best = SpvConfig()
    ms = ctypes.c_float(0)
    rc = load().spv_autotune_batch(ctypes.byref(batch_of(words, mod_off)), ctypes.byref(table.c()), _ptr(status),
                                   _ptr(err_row), 1 if validate else 0, _ptr(out) if encode else None,
                                   _ptr(workspace.buf), workspace.bytes, reps, ctypes.byref(best), ctypes.byref(ms),
                                   _stream(stream))
    _check(rc, "spv_autotune_batch")
    return best, ms.value, {"table": table, "status": status[:m], "err_row": err_row[:m],
                            "out": out if encode else None, "workspace": workspace}


LAYOUT_STATUS = ["OK", "SECTION_ORDER", "OUTSIDE_FUNCTION", "IN_FUNCTION", "BLOCK", "UNCLOSED"]


def layout(table, n_modules, *, stream=None, workspace=None):
    """spv_layout_batch over a decoded table: (layout_status[M] int32,
    layout_err_row[M] int64) device tensors. workspace: a uint8 device tensor
    of at least spv_layout_workspace_bytes bytes (allocated when None)."""
    dev = table.op.device
    status = torch.empty(max(1, n_modules), dtype=torch.int32, device=dev)
    err_row = torch.empty(max(1, n_modules), dtype=torch.int64, device=dev)
    need = load().spv_layout_workspace_bytes(n_modules, table.capacity_rows)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
    rc = load().spv_layout_batch(ctypes.byref(table.c()), n_modules, _ptr(status), _ptr(err_row),
                                 _ptr(workspace), workspace.numel(), _stream(stream))
    _check(rc, "spv_layout_batch")
    return status[:n_modules], err_row[:n_modules]


def op_layout(op):
    """(layout class, module section) of an opcode in the library's table."""
    c, sec = ctypes.c_int(), ctypes.c_int()
    load().spv_op_layout(op, ctypes.byref(c), ctypes.byref(sec))
    return c.value, sec.value


def decode(words, mod_off, **kw):
    return process(words, mod_off, validate=False, encode=False, **kw)


def validate(words, mod_off, table, *, workspace=None, stream=None, arena_words=0):
    """Validate from an existing decoded table."""
    m = mod_off.numel() - 1
    dev = words.device
    if workspace is None:
        workspace = Workspace(m, words.numel(), dev, arena_words)
    status = torch.empty(max(1, m), dtype=torch.int32, device=dev)
    err_row = torch.empty(max(1, m), dtype=torch.int64, device=dev)
    rc = spv_validate_batch(batch_of(words, mod_off), table.c(), _ptr(status), _ptr(err_row), _ptr(workspace.buf),
                            workspace.bytes, workspace.arena_words, _stream(stream))
    _check(rc, "spv_validate_batch")
    return status[:m], err_row[:m]


def encode(words, mod_off, table, *, recompute_bound=True, out=None, stream=None):
    """Re-encode from a (possibly edited) table."""
    if out is None:
        out = torch.empty_like(words)
    rc = spv_encode_batch(batch_of(words, mod_off), table.c(), _ptr(out), 1 if recompute_bound else 0,
                          _stream(stream))
    _check(rc, "spv_encode_batch")
    return out


def query_sizes(words, mod_off, *, inline_names=True, header=True, stream=None):
    """(rows_upper, text_bytes) of a batch: a shape bound on the decoded rows
    and the exact text size of disassemble() with these options (waits)."""
    rows, text = ctypes.c_int64(0), ctypes.c_uint64(0)
    opts = SpvDisOpts(1 if inline_names else 0, 1 if header else 0, 0, 0)
    rc = load().spv_query_sizes(ctypes.byref(batch_of(words, mod_off)), ctypes.byref(opts), ctypes.byref(rows),
                                ctypes.byref(text), _stream(stream))
    _check(rc, "spv_query_sizes")
    return int(rows.value), int(text.value)


class DisWorkspace:
    def __init__(self, n_modules, n_words, capacity_rows, device, arena_words=0):
        self.bytes = spv_dis_workspace_bytes(n_modules, n_words, capacity_rows, arena_words)
        self.buf = torch.empty(max(1, self.bytes), dtype=torch.uint8, device=device)
        self.arena_words = arena_words


def disassemble(words, mod_off, table, *, inline_names=True, header=True, text=None, workspace=None, stream=None,
                arena_words=0, sync=True, max_spins=0, test_stall_tile=0):
    """Text of every module. With sync (default) the call waits for the
    stream, grows the text buffer if needed, and returns
    (text uint8 tensor trimmed to its size, text_off int64 tensor, dis_status)."""
    m = mod_off.numel() - 1
    dev = words.device
    if workspace is None:
        workspace = DisWorkspace(m, words.numel(), table.capacity_rows, dev, arena_words)
    text_off = torch.empty(m + 1, dtype=torch.int64, device=dev)
    dis_status = torch.empty(max(1, m), dtype=torch.int32, device=dev)
    if text is None:
        text = torch.empty(max(1, 8 * words.numel()), dtype=torch.uint8, device=dev)
    opts = SpvDisOpts(1 if inline_names else 0, 1 if header else 0, max_spins, test_stall_tile)
    for _ in range(2):
        rc = spv_disassemble_batch(batch_of(words, mod_off), table.c(), opts, _ptr(text), text.numel(),
                                   _ptr(text_off), _ptr(dis_status), _ptr(workspace.buf), workspace.bytes,
                                   workspace.arena_words, _stream(stream))
        _check(rc, "spv_disassemble_batch")
        if not sync:
            return text, text_off, dis_status[:m]
        total = int(text_off[-1].item())
        if total <= text.numel():
            return text[:total], text_off, dis_status[:m]
        text = torch.empty(total, dtype=torch.uint8, device=dev)
    raise SpvError("text buffer sizing failed")


# ---------------------------------------------------------------------------
# assembler
# ---------------------------------------------------------------------------
ASM_STATUS = ["OK", "SYNTAX", "CAPACITY", "BAD_OFFSETS"]


def spv_asm_workspace_bytes(n_modules, text_bytes, line_capacity=0, name_capacity=0):
    return load().spv_asm_workspace_bytes(n_modules, text_bytes, line_capacity, name_capacity)


def spv_assemble_batch(text, text_bytes, text_off, n_modules, words, words_capacity, word_off, asm_status,
                       asm_err_line, workspace, ws_bytes, line_capacity, name_capacity, stream):
    return load().spv_assemble_batch(text, text_bytes, text_off, n_modules, words, words_capacity, word_off,
                                     asm_status, asm_err_line, workspace, ws_bytes, line_capacity, name_capacity,
                                     stream)


def spv_asm_required(workspace):
    lines, names = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().spv_asm_required(workspace, ctypes.byref(lines), ctypes.byref(names)), "spv_asm_required")
    return int(lines.value), int(names.value)


class AsmWorkspace:
    def __init__(self, n_modules, text_bytes, device, line_capacity=0, name_capacity=0):
        self.bytes = spv_asm_workspace_bytes(n_modules, text_bytes, line_capacity, name_capacity)
        self.buf = torch.empty(max(1, self.bytes), dtype=torch.uint8, device=device)
        self.line_capacity, self.name_capacity = line_capacity, name_capacity


def assemble(text, text_off, *, words=None, workspace=None, stream=None, line_capacity=0, name_capacity=0,
             sync=True):
    """Words of every module's text (device uint8 text, device int64
    text_off of n + 1 entries). With sync (default) the call waits for the
    stream, grows the word buffer and the workspace capacities when needed,
    and returns (words int32 tensor trimmed to its size, word_off int64,
    asm_status int32, asm_err_line int64)."""
    m = text_off.numel() - 1
    dev = text.device
    if words is None:
        words = torch.empty(max(16, text.numel() // 2 + 8 * m), dtype=torch.int32, device=dev)
    word_off = torch.empty(m + 1, dtype=torch.int64, device=dev)
    status = torch.empty(max(1, m), dtype=torch.int32, device=dev)
    err = torch.empty(max(1, m), dtype=torch.int64, device=dev)
    for _ in range(4):
        if workspace is None:
            workspace = AsmWorkspace(m, text.numel(), dev, line_capacity, name_capacity)
        rc = spv_assemble_batch(_ptr(text), text.numel(), _ptr(text_off), m, _ptr(words), words.numel(),
                                _ptr(word_off), _ptr(status), _ptr(err), _ptr(workspace.buf), workspace.bytes,
                                workspace.line_capacity, workspace.name_capacity, _stream(stream))
        _check(rc, "spv_assemble_batch")
        if not sync:
            return words, word_off, status[:m], err[:m]
        if m and bool((status[:m] == 2).any()):           # CAPACITY: size the workspace to what was needed
            lines, names = spv_asm_required(_ptr(workspace.buf))
            line_capacity, name_capacity = lines + 1, names + 1
            workspace = None
            continue
        total = int(word_off[-1].item())
        if total <= words.numel():
            return words[:total], word_off, status[:m], err[:m]
        words = torch.empty(total, dtype=torch.int32, device=dev)
    raise SpvError("assembler buffer sizing failed")


# ---------------------------------------------------------------------------
# builder
# ---------------------------------------------------------------------------
BUILD_STATUS = ["OK", "BAD_REF", "BAD_ROW", "BAD_OFFSETS"]


def spv_build_workspace_bytes(n_modules, n_rows):
    return load().spv_build_workspace_bytes(n_modules, n_rows)


def spv_build_batch(ol, version, generator, words, words_capacity, word_off, ids, status, err_row, workspace,
                    ws_bytes, stream):
    return load().spv_build_batch(ctypes.byref(ol), version, generator, words, words_capacity, word_off, ids,
                                  status, err_row, workspace, ws_bytes, stream)


class BuildWorkspace:
    def __init__(self, n_modules, n_rows, device):
        self.bytes = spv_build_workspace_bytes(n_modules, n_rows)
        self.buf = torch.empty(max(1, self.bytes), dtype=torch.uint8, device=device)


def build_modules(op, opd_off, opd, opd_ref, row_off, *, version=0x00010200, generator=0, words=None,
                  workspace=None, stream=None, sync=True, want_ids=True):
    """Modules from op lists (device tensors: op int16 (the uint16 opcodes),
    opd_off int64, opd int32 (the uint32 operand values), opd_ref uint8,
    row_off int64). With sync (default) the call waits, grows the word buffer
    if needed and returns (words int32 trimmed, word_off int64, status int32,
    err_row int64, ids int32 or None)."""
    m = row_off.numel() - 1
    n_rows = op.numel()
    dev = row_off.device
    if workspace is None:
        workspace = BuildWorkspace(m, n_rows, dev)
    if words is None:
        words = torch.empty(max(16, opd.numel() + 2 * n_rows + 5 * m), dtype=torch.int32, device=dev)
    word_off = torch.empty(m + 1, dtype=torch.int64, device=dev)
    status = torch.empty(max(1, m), dtype=torch.int32, device=dev)
    err = torch.empty(max(1, m), dtype=torch.int64, device=dev)
    ids = torch.empty(max(1, n_rows), dtype=torch.int32, device=dev) if want_ids else None
    ol = SpvOplist(_ptr(op), _ptr(opd_off), _ptr(opd), _ptr(opd_ref), _ptr(row_off), m, n_rows)
    for _ in range(2):
        rc = spv_build_batch(ol, version, generator, _ptr(words), words.numel(), _ptr(word_off), _ptr(ids),
                             _ptr(status), _ptr(err), _ptr(workspace.buf), workspace.bytes, _stream(stream))
        _check(rc, "spv_build_batch")
        if not sync:
            return words, word_off, status[:m], err[:m], (ids[:n_rows] if ids is not None else None)
        total = int(word_off[-1].item())
        if total <= words.numel():
            return words[:total], word_off, status[:m], err[:m], (ids[:n_rows] if ids is not None else None)
        words = torch.empty(total, dtype=torch.int32, device=dev)
    raise SpvError("builder buffer sizing failed")


# ---------------------------------------------------------------------------
# per-kernel timing of the library's launches
# ---------------------------------------------------------------------------
def profile_enable(on=True):
    lib = load()
    lib.spv_profile_enable.restype = ctypes.c_int
    lib.spv_profile_enable.argtypes = [ctypes.c_int]
    return lib.spv_profile_enable(1 if on else 0)


def profile_read(max_kernels=64):
    """{kernel name: (launches, total ms)} of the launches recorded since
    profile_enable(True)."""
    lib = load()
    lib.spv_profile_read.restype = ctypes.c_int
    lib.spv_profile_read.argtypes = [ctypes.c_int, P, P, P]
    names = (ctypes.c_char_p * max_kernels)()
    launches = (ctypes.c_int64 * max_kernels)()
    ms = (ctypes.c_double * max_kernels)()
    n = lib.spv_profile_read(max_kernels, names, launches, ms)
    if n < 0:
        raise SpvError(f"spv_profile_read failed with code {n}")
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(n, max_kernels))}


# ---------------------------------------------------------------------------
# serving handle
# ---------------------------------------------------------------------------
SPV_E_BUSY = -5


class SpvServeCfg(ctypes.Structure):
    _fields_ = [("hbm_cap_bytes", ctypes.c_uint64), ("max_batch_words", ctypes.c_int64),
                ("max_batch_modules", ctypes.c_int32), ("inline_names", ctypes.c_int32),
                ("header", ctypes.c_int32), ("device", ctypes.c_int32)]


class SpvResult(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("status", ctypes.c_uint32), ("err_row", ctypes.c_int64),
                ("n_instr", ctypes.c_uint32), ("text", ctypes.c_void_p), ("text_len", ctypes.c_uint64),
                ("op", P), ("wc", P), ("rtype", P), ("rid", P), ("off", P), ("words_base", P),
                ("submit_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64), ("batch_modules", ctypes.c_uint32)]


def _serve_lib():
    lib = load()
    if not getattr(lib, "_serve_ready", False):
        lib.spv_serve_create.restype = ctypes.c_void_p
        lib.spv_serve_create.argtypes = [ctypes.POINTER(SpvServeCfg)]
        lib.spv_serve_submit.restype = ctypes.c_int
        lib.spv_serve_submit.argtypes = [P, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
        lib.spv_serve_poll.restype = ctypes.c_int
        lib.spv_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(SpvResult)]
        lib.spv_serve_wait.restype = ctypes.c_int
        lib.spv_serve_wait.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(SpvResult), ctypes.c_int64]
        lib.spv_serve_release.restype = ctypes.c_int
        lib.spv_serve_release.argtypes = [P, ctypes.c_uint64]
        lib.spv_serve_destroy.restype = None
        lib.spv_serve_destroy.argtypes = [P]
        lib.spv_serve_replay.restype = ctypes.c_int
        lib.spv_serve_replay.argtypes = [P, ctypes.c_int32, P, P, P, P, P, P, P]
        lib._serve_ready = True
    return lib


def spv_serve_create(cfg):
    return _serve_lib().spv_serve_create(ctypes.byref(cfg))


def spv_serve_submit(server, host_words_ptr, n_words, ticket):
    return _serve_lib().spv_serve_submit(server, host_words_ptr, n_words, ctypes.byref(ticket))


def spv_serve_poll(server, ticket, result):
    return _serve_lib().spv_serve_poll(server, ticket, ctypes.byref(result))


def spv_serve_wait(server, ticket, result, timeout_us):
    return _serve_lib().spv_serve_wait(server, ticket, ctypes.byref(result), timeout_us)


def spv_serve_release(server, ticket):
    return _serve_lib().spv_serve_release(server, ticket)


def spv_serve_destroy(server):
    _serve_lib().spv_serve_destroy(server)


class Server:
    """Continuous-batching server (thin wrapper over spv_serve_*)."""

    def __init__(self, hbm_cap_bytes=0, max_batch_words=0, max_batch_modules=0, inline_names=True, header=True,
                 device=0):
        cfg = SpvServeCfg(hbm_cap_bytes, max_batch_words, max_batch_modules, 1 if inline_names else 0,
                          1 if header else 0, device)
        self.h = spv_serve_create(cfg)
        if not self.h:
            raise SpvError("spv_serve_create failed")

    def submit(self, words):
        """words: contiguous uint32 numpy array. Returns a ticket, or None when busy."""
        t = ctypes.c_uint64()
        rc = spv_serve_submit(self.h, words.ctypes.data_as(ctypes.c_void_p), len(words), t)
        if rc == SPV_E_BUSY:
            return None
        _check(rc, "spv_serve_submit")
        return t.value

    def poll(self, ticket):
        r = SpvResult()
        rc = spv_serve_poll(self.h, ticket, r)
        if rc < 0:
            raise SpvError(f"spv_serve_poll failed with code {rc}")
        return r if rc == 1 else None

    def wait(self, ticket, timeout_us=10_000_000):
        r = SpvResult()
        rc = spv_serve_wait(self.h, ticket, r, timeout_us)
        if rc < 0:
            raise SpvError(f"spv_serve_wait failed with code {rc}")
        return r if rc == 1 else None

    def replay(self, modules, arrive_ns):
        """Submit modules[i] (contiguous uint32 numpy arrays) arrive_ns[i]
        nanoseconds after the start from a native thread and collect them in
        order. Returns (latency_ns from arrival, server_ns from submission,
        batch_modules, busy_retries)."""
        n = len(modules)
        ptrs = (ctypes.c_void_p * max(1, n))(*[m.ctypes.data for m in modules])
        nw = np.array([len(m) for m in modules], np.int64)
        arr = np.ascontiguousarray(arrive_ns, np.int64)
        lat = np.zeros(n, np.int64)
        srv_ns = np.zeros(n, np.int64)
        bm = np.zeros(n, np.uint32)
        busy = ctypes.c_int64(0)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        rc = _serve_lib().spv_serve_replay(self.h, n, ctypes.cast(ptrs, ctypes.c_void_p), p(nw), p(arr), p(lat),
                                           p(srv_ns), p(bm), ctypes.byref(busy))
        _check(rc, "spv_serve_replay")
        return lat, srv_ns, bm, busy.value

    @staticmethod
    def text_of(r):
        return ctypes.string_at(r.text, r.text_len) if r.text_len else b""

    def release(self, ticket):
        _check(spv_serve_release(self.h, ticket), "spv_serve_release")

    def close(self):
        if self.h:
            spv_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# host-resident batches with overlapped transfers
# ---------------------------------------------------------------------------
class SpvPipeCfg(ctypes.Structure):
    _fields_ = [("chunk_words", ctypes.c_int64), ("depth", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("encode", ctypes.c_int32), ("inline_names", ctypes.c_int32), ("header", ctypes.c_int32)]


def _pipe_lib():
    lib = load()
    if not getattr(lib, "_pipe_ready", False):
        lib.spv_pipe_create.restype = ctypes.c_void_p
        lib.spv_pipe_create.argtypes = [ctypes.POINTER(SpvPipeCfg)]
        lib.spv_pipe_run.restype = ctypes.c_int
        lib.spv_pipe_run.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int32, P, P, P, P, ctypes.c_uint64, P, P]
        lib.spv_pipe_destroy.restype = None
        lib.spv_pipe_destroy.argtypes = [P]
        lib._pipe_ready = True
    return lib


def spv_pipe_create(cfg):
    return _pipe_lib().spv_pipe_create(ctypes.byref(cfg))


def spv_pipe_run(pipe, h_words, n_words, h_mod_off, n_modules, h_status, h_err_row, h_text_off, h_text,
                 text_capacity, h_out_words, h_dis_status):
    return _pipe_lib().spv_pipe_run(pipe, h_words, n_words, h_mod_off, n_modules, h_status, h_err_row, h_text_off,
                                    h_text, text_capacity, h_out_words, h_dis_status)


def spv_pipe_destroy(pipe):
    _pipe_lib().spv_pipe_destroy(pipe)


def _host_ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        assert a.device.type == "cpu" and a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


class Pipe:
    """A batch in host memory through spv_pipe_run (thin wrapper). Arrays are
    numpy arrays or CPU torch tensors (pinned ones let the copies overlap)."""

    def __init__(self, chunk_words=0, depth=0, validate=True, encode=True, inline_names=True, header=True):
        self.h = spv_pipe_create(SpvPipeCfg(chunk_words, depth, 1 if validate else 0, 1 if encode else 0,
                                            1 if inline_names else 0, 1 if header else 0))
        if not self.h:
            raise SpvError("spv_pipe_create failed")

    def run(self, words, mod_off, status, err_row, text_off, text, out_words=None, dis_status=None):
        """Fills the output arrays in place; returns the total text size
        (text_off[-1]); text holds min(size, len(text)) bytes."""
        n_mod = len(mod_off) - 1
        cap = text.numel() if isinstance(text, torch.Tensor) else len(text)
        rc = spv_pipe_run(self.h, _host_ptr(words), len(words), _host_ptr(mod_off), n_mod, _host_ptr(status),
                          _host_ptr(err_row), _host_ptr(text_off), _host_ptr(text), cap, _host_ptr(out_words),
                          _host_ptr(dis_status))
        _check(rc, "spv_pipe_run")
        return int(text_off[n_mod])

    def close(self):
        if self.h:
            spv_pipe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
