"""Hand-building of small SPIR-V modules for tests.

Words are written from the public SPIR-V specification's numbering: an
instruction's first word is (word count << 16) | opcode; a literal string is
its UTF-8 bytes, little-endian four to a word, NUL-terminated and zero-padded.
The numbers used below are spelled out where they are used.
"""
import numpy as np

MAGIC = 0x07230203
V12 = 0x00010200

# opcodes (SPIR-V 1.2)
OpNop, OpSource, OpName, OpString, OpExtInstImport, OpExtInst = 0, 3, 5, 7, 11, 12
OpMemoryModel, OpEntryPoint, OpExecutionMode, OpCapability = 14, 15, 16, 17
OpTypeVoid, OpTypeBool, OpTypeInt, OpTypeFloat, OpTypePointer, OpTypeFunction = 19, 20, 21, 22, 32, 33
OpConstant, OpFunction, OpFunctionParameter, OpFunctionEnd = 43, 54, 55, 56
OpVariable, OpLoad, OpStore, OpPtrAccessChain, OpDecorate = 59, 61, 62, 67, 71
OpIAdd, OpFAdd, OpPhi, OpLabel, OpBranch, OpReturn = 128, 129, 245, 248, 249, 253
# enumerants
CAP_ADDRESSES, CAP_LINKAGE, CAP_KERNEL, CAP_INT64, CAP_INT8, CAP_GENERIC_POINTER = 4, 5, 6, 11, 39, 38
AM_LOGICAL, AM_PHYSICAL64, MM_OPENCL = 0, 2, 2
EXEC_KERNEL = 6


def s(text: str):
    b = text.encode() + b"\0"
    b += b"\0" * (-len(b) % 4)
    return [int.from_bytes(b[i:i + 4], "little") for i in range(0, len(b), 4)]


def ins(op, *operands):
    flat = []
    for x in operands:
        if isinstance(x, (list, tuple)):
            flat.extend(x)
        else:
            flat.append(x)
    return [((len(flat) + 1) << 16) | op] + flat


def module(body, bound=100, version=V12, generator=32, schema=0, magic=MAGIC):
    words = [magic, version, generator, bound, schema]
    for i in body:
        words.extend(i)
    return np.array(words, dtype=np.uint32)


def batch(modules):
    offs = [0]
    for m in modules:
        offs.append(offs[-1] + len(m))
    words = np.concatenate([np.asarray(m, np.uint32) for m in modules]) if modules else np.zeros(0, np.uint32)
    return words, np.array(offs, np.int64)


def minimal_body():
    """A valid minimal kernel module body (rows 0..9): capabilities Addresses
    and Kernel, memory model Physical64 OpenCL, entry point, void function
    with one block that adds two constants."""
    return [
        ins(OpCapability, CAP_ADDRESSES),                 # row 0
        ins(OpCapability, CAP_KERNEL),                    # row 1
        ins(OpMemoryModel, AM_PHYSICAL64, MM_OPENCL),     # row 2
        ins(OpEntryPoint, EXEC_KERNEL, 5, s("k")),        # row 3
        ins(OpTypeVoid, 1),                               # row 4
        ins(OpTypeInt, 2, 32, 0),                         # row 5
        ins(OpTypeFunction, 3, 1),                        # row 6
        ins(OpConstant, 2, 4, 7),                         # row 7
        ins(OpFunction, 1, 5, 0, 3),                      # row 8
        ins(OpLabel, 6),                                  # row 9
        ins(OpIAdd, 2, 7, 4, 4),                          # row 10
        ins(OpReturn),                                    # row 11
        ins(OpFunctionEnd),                               # row 12
    ]
