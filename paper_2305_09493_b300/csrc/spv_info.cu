// spv_info.cu -- host-side queries of the compiled opcode / enumerant tables
// (the same compile-time tables the kernels read), and the sizes of a
// batch's outputs.
#include <cuda_runtime.h>
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

// Sizes of a batch's outputs: rows_upper from the shape alone; text_bytes
// exactly, by a decode and a disassembly with no text buffer (the measuring
// half of spv_disassemble_batch) on the stream, with scratch allocated and
// freed here; the call waits for the stream.
extern "C" int spv_query_sizes(const spv_batch *batch, const spv_dis_opts *opts, int64_t *rows_upper,
                               uint64_t *text_bytes, spv_stream_t stream)
{
    if (!batch || batch->n_modules < 0 || batch->n_words < 0) return SPV_E_ARG;
    const int64_t M = batch->n_modules, W = batch->n_words;
    if (rows_upper) *rows_upper = W > 5 * M ? W - 5 * M : 0;
    if (!text_bytes) return SPV_SUCCESS;
    *text_bytes = 0;
    if (M == 0) return SPV_SUCCESS;
    if (!batch->words || !batch->mod_off) return SPV_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t R = W > 0 ? W : 1;
    const size_t ws = spv_workspace_bytes((int32_t)M, W, 0, nullptr);
    const size_t dws = spv_dis_workspace_bytes((int32_t)M, W, R, 0);
    const size_t table_bytes = (size_t)R * (2 + 2 + 8 + 4 + 4 + 4) + (size_t)(M + 1) * 8 + (size_t)M * 4;
    const size_t per_mod = (size_t)M * (4 + 8 + 4) + (size_t)(M + 1) * 8;
    const size_t total = ws + dws + table_bytes + per_mod + 64 * 16;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, total, st) != cudaSuccess) return SPV_E_CUDA;
    size_t o = 0;
    auto take = [&](size_t n) { char *p = buf + o; o += (n + 255) & ~(size_t)255; return p; };
    spv_table t{};
    t.op = (uint16_t *)take((size_t)R * 2);
    t.wc = (uint16_t *)take((size_t)R * 2);
    t.off = (uint64_t *)take((size_t)R * 8);
    t.rtype = (uint32_t *)take((size_t)R * 4);
    t.rid = (uint32_t *)take((size_t)R * 4);
    t.mod = (uint32_t *)take((size_t)R * 4);
    t.mod_first_row = (int64_t *)take((size_t)(M + 1) * 8);
    t.mod_n_instr = (uint32_t *)take((size_t)M * 4);
    t.capacity_rows = R;
    uint32_t *status = (uint32_t *)take((size_t)M * 4);
    int64_t *err = (int64_t *)take((size_t)M * 8);
    uint32_t *dst = (uint32_t *)take((size_t)M * 4);
    uint64_t *toff = (uint64_t *)take((size_t)(M + 1) * 8);
    void *w1 = take(ws), *w2 = take(dws);
    int rc = spv_decode_batch(batch, &t, status, err, w1, ws, nullptr, stream);
    if (rc == SPV_SUCCESS)
        rc = spv_disassemble_batch(batch, &t, opts, nullptr, 0, toff, dst, w2, dws, 0, stream);
    uint64_t total_text = 0;
    if (rc == SPV_SUCCESS &&
        cudaMemcpyAsync(&total_text, toff + M, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = SPV_E_CUDA;
    cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == SPV_SUCCESS) rc = SPV_E_CUDA;
    if (rc == SPV_SUCCESS) *text_bytes = total_text;
    return rc;
}
