"""The grammar-driven table generator (the paper's generator of instruction
and operand-kind classes from the Khronos grammar, section 3.3):

* the tables as a grammar in the Khronos schema and back give the same model;
* the generated source lists, put in place of the hand-written ones, compile
  to byte-identical dense tables (host compile of the tables header);
* what the dense tables cannot hold (opcodes from 256, enumerants from 64,
  bit enumerants of several bits, operand kinds the kernels do not model,
  more than five operand codes) is reported and left out;
* capabilities without a named constant are written as numbers.
"""
import copy
import json
import os
import re
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2305_09493_b300 import grammar as G  # noqa: E402


def test_round_trip_through_the_schema():
    m = G.read_tables()
    assert len(m["ops"]) > 100 and len(m["value"]["Capability"]) > 50 and m["cap_deps"]
    g = json.loads(json.dumps(G.to_grammar(m)))      # through JSON text
    assert g["magic_number"] == "0x07230203"
    load = next(i for i in g["instructions"] if i["opname"] == "OpLoad")
    assert [o["kind"] for o in load["operands"]][:3] == ["IdResultType", "IdResult", "IdRef"]
    assert load["operands"][3] == {"kind": "MemoryAccess", "quantifier": "?"}
    text, dropped = G.from_grammar(g)
    assert dropped == []
    m2 = G.read_tables(text)
    for key in ("ops", "value", "bits", "cap_deps"):
        assert m2[key] == m[key], key


def _replace_lists(src, gen):
    """The tables file with each generated list in place of the written one."""
    for m in re.finditer(r"constexpr (\w+) (\w+)\[\] = \{.*?\n?\};", gen, re.S):
        name = m.group(2)
        pat = re.compile(r"constexpr \w+ " + re.escape(name) + r"\[\] = \{.*?\n?\};", re.S)
        assert pat.search(src), name
        src = pat.sub(lambda _: m.group(0), src, count=1)
    return src


_MAIN = r"""
#define __device__
#define __forceinline__ inline
#include "spv_tables.cuh"
#include <cstdio>
int main() {
    static constexpr spvt::Tables T = spvt::build_tables();
    const unsigned char *p = reinterpret_cast<const unsigned char *>(&T);
    unsigned long long h = 1469598103934665603ull;
    for (size_t i = 0; i < sizeof(T); i++) { h ^= p[i]; h *= 1099511628211ull; }
    std::printf("%zu %llx\n", sizeof(T), h);
}
"""


def _compile_and_hash(header_text, tmp):
    d = tempfile.mkdtemp(dir=tmp)
    with open(os.path.join(d, "spv_tables.cuh"), "w") as f:
        f.write(header_text)
    with open(os.path.join(d, "main.cpp"), "w") as f:
        f.write(_MAIN)
    exe = os.path.join(d, "t")
    subprocess.run(["g++", "-std=c++17", "-O0", "-fconstexpr-ops-limit=1000000000", "-I", d,
                    os.path.join(d, "main.cpp"), "-o", exe], check=True, capture_output=True)
    return subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip()


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_generated_lists_compile_to_the_same_tables(tmp_path):
    src = open(G.TABLES).read()
    gen, dropped = G.from_grammar(G.to_grammar(G.read_tables()))
    assert dropped == []
    swapped = _replace_lists(src, gen)
    assert swapped != src                                    # the lists were replaced (formatting differs)
    assert _compile_and_hash(swapped, str(tmp_path)) == _compile_and_hash(src, str(tmp_path))


def test_what_the_dense_tables_cannot_hold_is_reported():
    g = G.to_grammar(G.read_tables())
    g = copy.deepcopy(g)
    g["instructions"] += [
        {"opname": "OpWide", "opcode": 300, "operands": [{"kind": "IdRef"}]},
        {"opname": "OpImageThing", "opcode": 99, "operands": [{"kind": "IdRef"}, {"kind": "ImageOperands", "quantifier": "?"}]},
        {"opname": "OpSixOperands", "opcode": 98, "operands": [{"kind": "IdRef"}] * 6},
        {"opname": "OpNeedsRare", "opcode": 97, "operands": [{"kind": "IdRef"}], "capabilities": ["Pipes"]},
    ]
    sc = next(k for k in g["operand_kinds"] if k["kind"] == "StorageClass")
    sc["enumerants"].append({"enumerant": "FarAway", "value": 70})
    ma = next(k for k in g["operand_kinds"] if k["kind"] == "MemoryAccess")
    ma["enumerants"].append({"enumerant": "TwoBits", "value": "0x0030"})
    text, dropped = G.from_grammar(g)
    assert set(dropped) == {"OpWide", "OpImageThing", "OpSixOperands", "StorageClass.FarAway", "MemoryAccess.TwoBits"}
    m = G.read_tables(text.replace("(int8_t)17", "C_PIPES_AS_NUMBER"))
    rare = next(o for o in m["ops"] if o["opname"] == "OpNeedsRare")
    assert rare["cap"] == "C_PIPES_AS_NUMBER"                # Pipes (17) has no named constant: written as a number


def test_command_line_dump():
    out = subprocess.run([sys.executable, "-m", "paper_2305_09493_b300.grammar", "--dump"], cwd=ROOT,
                         check=True, capture_output=True, text=True).stdout
    g = json.loads(out)
    assert len(g["instructions"]) == len(G.read_tables()["ops"])
    assert {k["kind"] for k in g["operand_kinds"]} == set(G.VALUE_KINDS + G.BIT_KINDS)
