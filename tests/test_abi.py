"""C-ABI library checks that need no GPU: it builds, loads, exports every
function include/*.h declares, and its opcode / enumerant tables agree entry
by entry with the oracle's separately typed tables."""
import ctypes
import glob
import os
import re

import pytest

import oracle
from paper_2305_09493_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(spv_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("spv_process_batch", "spv_decode_batch", "spv_validate_batch", "spv_encode_batch",
                 "spv_disassemble_batch", "spv_workspace_bytes", "spv_dis_workspace_bytes"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_workspace_queries(lib):
    from paper_2305_09493_b300 import spvgpu
    assert "sm_103a" in spvgpu.spv_version()
    assert spvgpu.spv_workspace_bytes(10, 10000) > 0
    assert spvgpu.spv_workspace_bytes(10, 10000, 0, spvgpu.make_config(tile_words=1000)) == 0  # invalid tile
    assert spvgpu.spv_dis_workspace_bytes(10, 10000, 10000) > 0


def test_opcode_tables_agree():
    from paper_2305_09493_b300 import spvgpu
    ops = set(oracle.opcodes())
    for op in range(0, 300):
        a, b = oracle.op_info(op), spvgpu.spv_op_info(op)
        assert (a is None) == (b is None), op
        if a:
            assert a == b, (op, a, b)
    assert len(ops) > 100


@pytest.mark.parametrize("kind", ["SourceLanguage", "AddressingModel", "MemoryModel", "ExecutionModel",
                                  "ExecutionMode", "Capability", "StorageClass", "Decoration", "BuiltIn",
                                  "FuncParamAttr", "LinkageType"])
def test_value_enum_tables_agree(kind):
    from paper_2305_09493_b300 import spvgpu
    for v in range(0, 64):
        assert oracle.enum_name(kind, v) == spvgpu.spv_enum_info(kind, v), (kind, v)


@pytest.mark.parametrize("kind", ["FunctionControl", "MemoryAccess", "SelectionControl", "LoopControl"])
def test_bit_enum_tables_agree(kind):
    from paper_2305_09493_b300 import spvgpu
    for b in range(32):
        assert oracle.enum_name(kind, 1 << b) == spvgpu.spv_enum_info(kind, 1 << b), (kind, b)


def test_layout_classes_agree():
    from paper_2305_09493_b300 import spvgpu
    for op in range(0, 300):
        assert oracle.layout_class(op) == spvgpu.op_layout(op), op
