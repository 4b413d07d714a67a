// spv_info.cu -- host-side queries of the compiled opcode / enumerant tables
// (the same compile-time tables the kernels read).
#include <string.h>
#include "../../include/spv.h"
#include "spv_tables.cuh"

namespace {
thread_local char g_name[128];

const char *copy_name(uint16_t off, uint8_t len)
{
    memcpy(g_name, SPV_TABLES_HOST.names + off, len);
    g_name[len] = 0;
    return g_name;
}

int kind_index(const char *kind, bool *bits)
{
    static const char *vk[] = {"SourceLanguage", "AddressingModel", "MemoryModel", "ExecutionModel",
                               "ExecutionMode", "Capability", "StorageClass", "Decoration", "BuiltIn",
                               "FuncParamAttr", "LinkageType"};
    static const char *bk[] = {"FunctionControl", "MemoryAccess", "SelectionControl", "LoopControl"};
    for (int i = 0; i < 11; i++) if (!strcmp(kind, vk[i])) { *bits = false; return i; }
    for (int i = 0; i < 4; i++) if (!strcmp(kind, bk[i])) { *bits = true; return i; }
    return -1;
}
}  // namespace

extern "C" int spv_op_info(uint32_t opcode, int *has_rtype, int *has_rid, int *cap, const char **name)
{
    if (opcode >= 256) return -1;
    const spvt::OpDesc &d = SPV_TABLES_HOST.ops[opcode];
    if (!(d.flags & 1)) return -1;
    if (has_rtype) *has_rtype = (d.flags >> 1) & 1;
    if (has_rid) *has_rid = (d.flags >> 2) & 1;
    if (cap) *cap = d.cap;
    if (name) *name = copy_name(d.name_off, d.name_len);
    return 0;
}

extern "C" int spv_enum_info(const char *kind, uint32_t value, const char **name, int *cap)
{
    bool bits = false;
    int k = kind ? kind_index(kind, &bits) : -1;
    if (k < 0) return -1;
    const spvt::EnDesc *e = nullptr;
    if (bits) {
        if (value == 0 || (value & (value - 1))) return -1;
        int b = __builtin_ctz(value);
        e = &SPV_TABLES_HOST.benum[k][b];
    } else {
        if (value >= 64) return -1;
        e = &SPV_TABLES_HOST.venum[k][value];
    }
    if (!e->known) return -1;
    if (name) *name = copy_name((uint16_t)((e->name_hi << 8) | e->name_lo), e->name_len);
    if (cap) *cap = e->cap;
    return 0;
}

extern "C" const char *spv_version(void) { return "spvgpu 0.1 (sm_103a)"; }
