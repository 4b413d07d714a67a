"""Grammar-driven opcode and enumerant tables (the paper's generator, section
3.3: the library's instruction and operand-kind classes are generated from the
Khronos machine-readable grammar).

The kernels index compact tables (`csrc/spv_tables.cuh`): per opcode a result
type / result id flag, a required capability and an operand program of at most
five codes; per value-enum and bit-enum kind its enumerants with capability and
parameters. This module converts between those tables and a grammar in the
Khronos JSON schema ("instructions" with "opname", "opcode", "operands" of
{"kind", "quantifier"}; "operand_kinds" with "category", "kind" and
"enumerants" of {"enumerant", "value", "capabilities", "parameters"}):

* `read_tables(text)` parses the source lists of `spv_tables.cuh`;
* `to_grammar(model)` writes them as a grammar in that schema;
* `from_grammar(grammar)` turns a grammar back into the source lists, keeping
  what the dense tables can hold (opcodes below 256, value enumerants below
  64, bit enumerants of one bit below 32, five operand codes) and reporting
  the rest.

Run as `python -m paper_2305_09493_b300.grammar --dump` to print the current
tables as a grammar, or `python -m paper_2305_09493_b300.grammar FILE.json` to
print the source lists a grammar file gives.
"""
import json
import os
import re
import sys

TABLES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "spv_tables.cuh")

# the kinds the kernels know, in the order of their enum constants
VALUE_KINDS = ["SourceLanguage", "AddressingModel", "MemoryModel", "ExecutionModel", "ExecutionMode",
               "Capability", "StorageClass", "Decoration", "BuiltIn", "FuncParamAttr", "LinkageType"]
BIT_KINDS = ["FunctionControl", "MemoryAccess", "SelectionControl", "LoopControl"]

# operand codes of the tables <-> grammar operands
_SIMPLE = {"I": ("IdRef", None), "L": ("LiteralInteger", None), "S": ("LiteralString", None),
           "A_CTX": ("LiteralContextDependentNumber", None), "A_IDS": ("IdRef", "*"),
           "A_LITS": ("LiteralInteger", "*"), "LT": ("LiteralInteger", "*"),
           "A_IDPAIRS": ("PairIdRefIdRef", "*")}
# grammar operand kinds that the tables read as one <id> or one literal word
_ID_KINDS = {"IdRef", "IdScope", "IdMemorySemantics"}
_LIT_KINDS = {"LiteralInteger", "LiteralExtInstInteger", "LiteralSpecConstantOpInteger"}


def _split_codes(body):
    """'I, OPT(E(K_x)), A_IDS' -> ['I', 'OPT(E(K_x))', 'A_IDS'] (top-level commas only)."""
    out, depth, cur = [], 0, ""
    for ch in body:
        if ch == "," and depth == 0:
            if cur.strip():
                out.append(cur.strip())
            cur = ""
            continue
        depth += ch == "("
        depth -= ch == ")"
        cur += ch
    if cur.strip():
        out.append(cur.strip())
    return out


def _code_to_operand(code):
    opt = code.startswith("OPT(")
    if opt:
        code = code[4:-1]
    if code in _SIMPLE:
        kind, q = _SIMPLE[code]
    elif code.startswith("E(K_"):
        kind, q = code[4:-1], None
    elif code.startswith("BI(B_"):
        kind, q = code[5:-1], None
    else:
        raise ValueError(f"unknown operand code {code}")
    if opt:
        q = "?"
    o = {"kind": kind}
    if q:
        o["quantifier"] = q
    return o


def _block(text, name):
    m = re.search(r"constexpr \w+ " + re.escape(name) + r"\[\] = \{(.*?)\n?\};", text, re.S)
    if not m:
        raise ValueError(f"no list {name}")
    return m.group(1)


def read_tables(text=None):
    """The source lists of the tables file as a model: {"caps": {C_ name: number},
    "ops": [...], "value": {kind: [...]}, "bits": {kind: [...]}, "cap_deps": [(a, b)]}."""
    if text is None:
        text = open(TABLES).read()
    caps = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(C_\w+) = (-?\d+)", text)}
    ops = []
    for m in re.finditer(r'\{(\d+), "(\w+)", (\d), (\d), (C_\w+), \{([^{}]*(?:\([^{}]*\)[^{}]*)*)\}\}',
                         _block(text, "OP_LIST")):
        ops.append({"opcode": int(m.group(1)), "opname": m.group(2), "rt": int(m.group(3)),
                    "rid": int(m.group(4)), "cap": m.group(5), "codes": _split_codes(m.group(6))})
    def enumerants(name):
        out = []
        for m in re.finditer(r'\{(0x[0-9a-fA-F]+|\d+), "(\w+)", (C_\w+), \{([^{}]*)\}\}', _block(text, name)):
            out.append({"value": int(m.group(1), 0), "name": m.group(2), "cap": m.group(3),
                        "params": _split_codes(m.group(4))})
        return out
    value = {k: enumerants("EN_" + k) for k in VALUE_KINDS}
    bits = {k: enumerants("BN_" + k) for k in BIT_KINDS}
    deps = [(int(a), int(b)) for a, b in re.findall(r"\{(\d+), (\d+)\}", _block(text, "CAP_DEPS"))]
    return {"caps": caps, "ops": ops, "value": value, "bits": bits, "cap_deps": deps}


def to_grammar(model):
    """The model as a grammar in the Khronos JSON schema."""
    cap_name = {v: k for k, v in ((e["name"], e["value"]) for e in model["value"]["Capability"])}
    def caps_of(c):
        n = model["caps"][c]
        return [] if n < 0 else [cap_name[n]]
    instrs = []
    for o in model["ops"]:
        operands = ([{"kind": "IdResultType"}] if o["rt"] else []) + ([{"kind": "IdResult"}] if o["rid"] else [])
        operands += [_code_to_operand(c) for c in o["codes"]]
        instrs.append({"opname": o["opname"], "opcode": o["opcode"], "operands": operands,
                       "capabilities": caps_of(o["cap"])})
    deps = {}
    for a, b in model["cap_deps"]:
        deps.setdefault(a, []).append(cap_name[b])
    kinds = []
    for k in VALUE_KINDS:
        ens = []
        for e in model["value"][k]:
            d = {"enumerant": e["name"], "value": e["value"],
                 "capabilities": deps.get(e["value"], []) if k == "Capability" else caps_of(e["cap"])}
            if e["params"]:
                d["parameters"] = [_code_to_operand(p) for p in e["params"]]
            ens.append(d)
        kinds.append({"category": "ValueEnum", "kind": k, "enumerants": ens})
    for k in BIT_KINDS:
        ens = [{"enumerant": "None", "value": "0x0000"}]
        for e in model["bits"][k]:
            d = {"enumerant": e["name"], "value": f"0x{e['value']:04x}", "capabilities": caps_of(e["cap"])}
            if e["params"]:
                d["parameters"] = [_code_to_operand(p) for p in e["params"]]
            ens.append(d)
        kinds.append({"category": "BitEnum", "kind": k, "enumerants": ens})
    return {"magic_number": "0x07230203", "major_version": 1, "minor_version": 2,
            "instructions": instrs, "operand_kinds": kinds}


def _operand_to_code(o, in_enum=False):
    """A grammar operand as a table code, or None when the tables cannot hold it."""
    kind, q = o.get("kind"), o.get("quantifier")
    if kind in _ID_KINDS:
        base, many = "I", "A_IDS"
    elif kind in _LIT_KINDS:
        base, many = "L", ("LT" if in_enum else "A_LITS")
    elif kind == "LiteralString":
        base, many = "S", None
    elif kind == "LiteralContextDependentNumber":
        return "A_CTX" if q is None else None
    elif kind == "PairIdRefIdRef":
        return "A_IDPAIRS" if q == "*" else None
    elif kind in VALUE_KINDS:
        base, many = f"E(K_{kind})", None
    elif kind in BIT_KINDS:
        base, many = f"BI(B_{kind})", None
    else:
        return None
    if q is None:
        return base
    if q == "?":
        return f"OPT({base})"
    return many


def from_grammar(grammar, cap_consts=None):
    """Source lists for the tables file from a grammar in the Khronos schema.
    Returns (text, dropped): dropped names what the dense tables cannot hold."""
    if cap_consts is None:
        cap_consts = read_tables()["caps"]
    kinds = {k["kind"]: k for k in grammar.get("operand_kinds", [])}
    cap_value = {e["enumerant"]: int(e["value"]) for e in kinds.get("Capability", {}).get("enumerants", [])}
    def cap_code(names):
        if not names:
            return "C_NONE"
        n = names[0]
        return f"C_{n}" if f"C_{n}" in cap_consts else f"(int8_t){cap_value[n]}"
    dropped, lines = [], ["constexpr OpSrc OP_LIST[] = {"]
    for ins in sorted(grammar.get("instructions", []), key=lambda i: i["opcode"]):
        ops = list(ins.get("operands", []))
        rt = int(bool(ops) and ops[0]["kind"] == "IdResultType")
        ops = ops[rt:]
        rid = int(bool(ops) and ops[0]["kind"] == "IdResult")
        ops = ops[rid:]
        codes = [_operand_to_code(o) for o in ops]
        if ins["opcode"] >= 256 or None in codes or len(codes) > 5:
            dropped.append(ins["opname"])
            continue
        lines.append(f'    {{{ins["opcode"]}, "{ins["opname"]}", {rt}, {rid}, {cap_code(ins.get("capabilities"))}, '
                     f'{{{", ".join(codes)}}}}},')
    lines.append("};")
    deps = []
    for kind in VALUE_KINDS + BIT_KINDS:
        bit = kind in BIT_KINDS
        lines.append(f"constexpr EnSrc {'BN' if bit else 'EN'}_{kind}[] = {{")
        for e in kinds.get(kind, {}).get("enumerants", []):
            v = int(e["value"], 0) if isinstance(e["value"], str) else int(e["value"])
            params = [_operand_to_code(p, in_enum=True) for p in e.get("parameters", [])]
            fits = (v and not (v & (v - 1)) and v < (1 << 32)) if bit else v < 64
            if not fits or None in params or len(params) > 3:
                if not (bit and v == 0):
                    dropped.append(f"{kind}.{e['enumerant']}")
                continue
            if kind == "Capability":
                deps += [(v, cap_value[d]) for d in e.get("capabilities", [])]
                cap = "C_NONE"
            else:
                cap = cap_code(e.get("capabilities"))
            val = f"0x{v:x}" if bit else str(v)
            lines.append(f'    {{{val}, "{e["enumerant"]}", {cap}, {{{", ".join(params)}}}}},')
        lines.append("};")
    lines.append("constexpr CapDep CAP_DEPS[] = {")
    lines += [f"    {{{a}, {b}}}," for a, b in deps]
    lines.append("};")
    return "\n".join(lines) + "\n", dropped


def main(argv):
    if argv[1:2] == ["--dump"]:
        print(json.dumps(to_grammar(read_tables()), indent=1))
        return 0
    if len(argv) != 2:
        print("usage: python -m paper_2305_09493_b300.grammar (--dump | GRAMMAR.json)", file=sys.stderr)
        return 2
    text, dropped = from_grammar(json.load(open(argv[1])))
    sys.stdout.write(text)
    if dropped:
        print(f"not representable in the dense tables ({len(dropped)}): {' '.join(dropped)}", file=sys.stderr)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
