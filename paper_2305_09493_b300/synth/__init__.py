"""Seeded synthetic SPIR-V compute modules (input generation only).

Both the CUDA path and the CPU oracle consume these inputs; this package
contains none of the method's arithmetic (it writes modules, it never decodes,
validates or prints them). The generator itself is C (``spv_synth.c``).

Named workloads (sizes of the benchmark configurations):
  * ``single_module``  one ~10k-word kernel module: 3 capabilities, OpenCL.std
    import, 1 entry point + LocalSize, 50 OpDecorate, 40 type/constant
    definitions, one function of ~2,000 instructions in 40 basic blocks.
  * ``module_batch``   10,000 such modules, instruction counts lognormal
    (median 1,500, sigma 1.0, clipped to [200, 50,000]), 1-8 kernels each,
    module m generated from seed m.
  * ``large_module``   one module of 4M instructions, 500 functions, 10% of
    the instructions OpString / OpName with printable ASCII strings of 1-64
    bytes (~20M words).
  * ``size_bins``      1,000 modules each of 200 / 2k / 20k / 50k instructions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spv_synth.c")
_LIB = os.path.join(_HERE, "libspv_synth.so")
_lib = None


def build_library(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build_library()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.synth_module.restype = ctypes.c_int64
        lib.synth_module.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     P, ctypes.c_int64, P, ctypes.c_int64, P, P]
        lib.synth_batch_shape.restype = None
        lib.synth_batch_shape.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int32, P, P]
        lib.synth_oplist_batch.restype = ctypes.c_int64
        lib.synth_oplist_batch.argtypes = [ctypes.c_int32, ctypes.c_uint64, P, P, ctypes.c_int32] + [P] * 8 + \
            [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        lib.synth_batch.restype = ctypes.c_int64
        lib.synth_batch.argtypes = [ctypes.c_int32, ctypes.c_uint64, P, P, ctypes.c_int32, P,
                                    ctypes.c_int64, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def module(seed: int, func_instr: int, n_kernels: int = 1, n_funcs: int = 1, block_len: int = 50,
           n_decorations: int = 50, n_consts: int = 26, string_permille: int = 0):
    """One module. Returns (words uint32, starts int64, bound): starts are the
    module-relative word offsets at which the generator wrote instructions."""
    lib = _L()
    ni = ctypes.c_int64()
    b = ctypes.c_uint32()
    args = (seed, func_instr, n_kernels, n_funcs, block_len, n_decorations, n_consts, string_permille)
    n = lib.synth_module(*args, None, 0, None, 0, ctypes.byref(ni), ctypes.byref(b))
    words = np.zeros(n, np.uint32)
    starts = np.zeros(ni.value, np.int64)
    lib.synth_module(*args, _p(words), n, _p(starts), ni.value, ctypes.byref(ni), ctypes.byref(b))
    return words, starts, int(b.value)


def batch_shape(n_mod: int, seed0: int = 0, median: float = 1500.0, sigma: float = 1.0,
                lo: int = 200, hi: int = 50_000, max_kernels: int = 8):
    n_instr = np.zeros(n_mod, np.int64)
    n_kernels = np.zeros(n_mod, np.int32)
    _L().synth_batch_shape(n_mod, seed0, median, sigma, lo, hi, max_kernels, _p(n_instr),
                           _p(n_kernels))
    return n_instr, n_kernels


def batch(n_instr, n_kernels, seed0: int = 0, string_permille: int = 0):
    """Pack len(n_instr) modules into one word buffer; returns (words, mod_off)."""
    n_instr = np.ascontiguousarray(n_instr, np.int64)
    n_kernels = np.ascontiguousarray(n_kernels, np.int32)
    m = len(n_instr)
    mod_off = np.zeros(m + 1, np.int64)
    lib = _L()
    total = lib.synth_batch(m, seed0, _p(n_instr), _p(n_kernels), string_permille, None, 0,
                            _p(mod_off))
    words = np.zeros(total, np.uint32)
    lib.synth_batch(m, seed0, _p(n_instr), _p(n_kernels), string_permille, _p(words), total,
                    _p(mod_off))
    return words, mod_off


def single_module(seed: int = 0):
    """~10k-word kernel module; returns (words, mod_off, starts, bound)."""
    w, starts, bound = module(seed, 2000, 1, 1, 50, 50, 26, 0)
    return w, np.array([0, len(w)], np.int64), starts, bound


def module_batch(n_mod: int = 10_000, seed0: int = 0, median: float = 1500.0):
    n_instr, n_kernels = batch_shape(n_mod, seed0, median)
    return batch(n_instr, n_kernels, seed0)


def large_module(seed: int = 0, n_instr: int = 4_000_000, n_funcs: int = 500, string_permille: int = 100):
    """One large module with strings and names; returns (words, mod_off, starts, bound)."""
    module_level = 3 + 2 + 3 + 1 + 50 + 40
    func_instr = int((n_instr - module_level) * (1000 - string_permille) / 1000)
    w, starts, bound = module(seed, func_instr, 1, n_funcs, 50, 50, 26, string_permille)
    return w, np.array([0, len(w)], np.int64), starts, bound


def size_bins(per_bin: int = 1000, bins=(200, 2000, 20_000, 50_000), seed0: int = 0):
    """Modules binned by size; returns [(bin_instr, words, mod_off)]."""
    out = []
    for b, size in enumerate(bins):
        n_instr = np.full(per_bin, size, np.int64)
        rng = np.random.default_rng(seed0 + b)
        n_kernels = rng.integers(1, 9, per_bin).astype(np.int32)
        w, off = batch(n_instr, n_kernels, seed0 + 1_000_000 * (b + 1))
        out.append((size, w, off))
    return out


def oplist_batch(n_instr, n_kernels, seed0: int = 0, string_permille: int = 0):
    """The batch of batch() as op lists, what a JIT backend hands a builder:
    one row per instruction, its operands without the result id, id operands
    as references to the defining row of the module. Returns a dict: words,
    mod_off (the batch itself), is_id (1 for its id words), op, opd_off, opd,
    opd_ref, row_off."""
    n_instr = np.ascontiguousarray(n_instr, np.int64)
    n_kernels = np.ascontiguousarray(n_kernels, np.int32)
    m = len(n_instr)
    lib = _L()
    nr, no = ctypes.c_int64(0), ctypes.c_int64(0)
    total = lib.synth_oplist_batch(m, seed0, _p(n_instr), _p(n_kernels), string_permille, *([None] * 8),
                                   ctypes.byref(nr), ctypes.byref(no))
    d = {"words": np.zeros(total, np.uint32), "mod_off": np.zeros(m + 1, np.int64),
         "is_id": np.zeros(total, np.uint8), "op": np.zeros(nr.value, np.uint16),
         "opd_off": np.zeros(nr.value + 1, np.int64), "opd": np.zeros(no.value, np.uint32),
         "opd_ref": np.zeros(no.value, np.uint8), "row_off": np.zeros(m + 1, np.int64)}
    lib.synth_oplist_batch(m, seed0, _p(n_instr), _p(n_kernels), string_permille, _p(d["words"]), _p(d["mod_off"]),
                           _p(d["is_id"]), _p(d["op"]), _p(d["opd_off"]), _p(d["opd"]), _p(d["opd_ref"]),
                           _p(d["row_off"]), ctypes.byref(nr), ctypes.byref(no))
    return d


def oplist_module_batch(n_mod: int = 10_000, seed0: int = 0, median: float = 1500.0):
    n_instr, n_kernels = batch_shape(n_mod, seed0, median)
    return oplist_batch(n_instr, n_kernels, seed0)
