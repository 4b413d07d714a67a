// spv_build.cu -- batched builder: modules from op lists (section 3.4.2,
// "Enabling Function Composition"). In the paper an instruction is added to
// its scope in order, and every instruction with a result first asks the
// module for the next id (getNextId). Here a JIT backend hands over a whole
// batch of op lists at once: each row is an opcode and its operands, the
// result id left out, and an operand is a literal word or a reference to
// another row of the module. getNextId becomes a scan: the rows whose opcode
// has a result id take ids 1, 2, ... of their module in row order.
//
// Kernels, all on the caller's stream:
//   k_bld_mod_init   offsets checked, module records cleared
//   k_bld_rmod       each row's module (one warp per module)
//   k_bld_rows       per row: result id or not, word count, and the checks
//                    (result type present, at most 65535 words, references
//                    inside the module and to a row with a result id); the
//                    first bad row of a module wins
//   scans            of the result flags (ids) and of the word counts
//   k_bld_mod        module status, words, and the module scan of the words
//   k_bld_write      each row's words: word 0, the result type, the new
//                    result id, the operands with references resolved
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spv.h"
#include "spv_prof.h"
#include "spv_scan.cuh"
#include "spv_tables.cuh"

namespace {

struct BldCtrl {
    long long n_rows;          // rows of the modules: [row_off[0], row_off[n_modules])
    long long r_first;
    long long n_mod;
    unsigned int bad_offsets;
    unsigned int pad;
};

struct BP {
    const uint16_t *op;
    const int64_t *opd_off;
    const uint32_t *opd;
    const uint8_t *opd_ref;
    const int64_t *row_off;
    int n_mod;
    long long n_rows_total;
    uint32_t version, generator;
    BldCtrl *ctrl;
    unsigned long long *err;           // per module: row << 8 | status, ~0 none
    int32_t *rmod;                     // per row (from r_first)
    uint32_t *res, *rw;                // per row: has a result id; words
    unsigned long long *rsc, *wsc;     // their exclusive scans (n_rows + 1)
    unsigned long long *msize;         // per module: words (then scanned into word_off)
    uint32_t *words;
    long long words_cap;
    int64_t *word_off;
    uint32_t *ids;
    uint32_t *status;
    int64_t *err_row;
};

__device__ __forceinline__ uint32_t op_flags(uint32_t op)
{
    return op < 256 ? g_spv_tables.ops[op].flags : 0u;     // bit0 known, bit1 result type, bit2 result id
}

__global__ void k_bld_mod_init(BP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        P.err[m] = ~0ull;
        if (P.row_off[m] > P.row_off[m + 1]) atomicOr(&P.ctrl->bad_offsets, 1u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long a = P.row_off[0], b = P.row_off[P.n_mod];
        if (a < 0 || b > P.n_rows_total || a > b) atomicOr(&P.ctrl->bad_offsets, 1u);
        P.ctrl->r_first = a;
        P.ctrl->n_rows = a <= b ? b - a : 0;
        P.ctrl->n_mod = P.n_mod;
    }
}

// operand offsets must not decrease over the modules' rows
__global__ void k_bld_check_opd(BP P)
{
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c.n_rows;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = c.r_first + i;
        if (P.opd_off[r] > P.opd_off[r + 1] || P.opd_off[r] < 0) atomicOr(&P.ctrl->bad_offsets, 1u);
    }
}

__global__ void k_bld_rmod(BP P)
{
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    const int lane = threadIdx.x & 31, warps = (gridDim.x * blockDim.x) >> 5;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < P.n_mod; m += warps)
        for (long long r = P.row_off[m] + lane; r < P.row_off[m + 1]; r += 32) P.rmod[r - c.r_first] = m;
}

__global__ void __launch_bounds__(256) k_bld_rows(BP P)
{
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c.n_rows;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = c.r_first + i;
        const int m = P.rmod[i];
        const long long r0 = P.row_off[m], nrows = P.row_off[m + 1] - r0;
        const uint32_t f = op_flags(P.op[r]);
        const long long a = P.opd_off[r], nopd = P.opd_off[r + 1] - a;
        const bool rid = f & 4;
        const long long wc = 1 + nopd + (rid ? 1 : 0);
        uint32_t st = SPV_BUILD_OK;
        if (((f & 2) && nopd == 0) || wc > 65535) {
            st = SPV_BUILD_BAD_ROW;
        } else {
            for (long long k = a; k < a + nopd; k++) {
                if (!P.opd_ref[k]) continue;
                const uint32_t t = P.opd[k];
                if ((long long)t >= nrows || !(op_flags(P.op[r0 + t]) & 4)) { st = SPV_BUILD_BAD_REF; break; }
            }
        }
        if (st) atomicMin(&P.err[m], ((unsigned long long)(r - r0) << 8) | st);
        P.res[i] = rid ? 1u : 0u;
        P.rw[i] = wc <= 65535 ? (uint32_t)wc : 0u;
    }
}

__global__ void k_bld_mod(BP P)
{
    const BldCtrl &c = *P.ctrl;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        uint32_t st = SPV_BUILD_OK;
        long long bad = -1;
        unsigned long long nw = 0;
        if (c.bad_offsets) {
            st = SPV_BUILD_BAD_OFFSETS;
        } else if (P.err[m] != ~0ull) {
            st = (uint32_t)(P.err[m] & 255u);
            bad = (long long)(P.err[m] >> 8);
        } else {
            const long long i0 = P.row_off[m] - c.r_first, i1 = P.row_off[m + 1] - c.r_first;
            nw = 5 + (P.wsc[i1] - P.wsc[i0]);
        }
        P.status[m] = st;
        if (P.err_row) P.err_row[m] = bad;
        P.msize[m] = nw;
    }
}

__global__ void k_bld_head(BP P)
{
    const BldCtrl &c = *P.ctrl;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        if (P.status[m] != SPV_BUILD_OK) continue;
        const long long i0 = P.row_off[m] - c.r_first, i1 = P.row_off[m + 1] - c.r_first;
        const uint32_t h[5] = {0x07230203u, P.version, P.generator, (uint32_t)(1 + P.rsc[i1] - P.rsc[i0]), 0u};
        const long long at = P.word_off[m];
        for (int k = 0; k < 5; k++)
            if (at + k < P.words_cap) P.words[at + k] = h[k];
    }
}

__global__ void __launch_bounds__(256) k_bld_write(BP P)
{
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c.n_rows;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = c.r_first + i;
        const int m = P.rmod[i];
        const long long r0 = P.row_off[m], i0 = r0 - c.r_first;
        const unsigned long long id0 = P.rsc[i0];
        const uint32_t id = P.res[i] ? (uint32_t)(1 + P.rsc[i] - id0) : 0u;
        if (P.ids) P.ids[r] = id;
        if (P.status[m] != SPV_BUILD_OK) continue;
        const uint32_t op = P.op[r];
        const uint32_t f = op_flags(op);
        const long long a = P.opd_off[r], nopd = P.opd_off[r + 1] - a;
        const int at_rid = (f & 2) ? 1 : 0;            // the result id's place among the operands
        long long o = P.word_off[m] + 5 + (long long)(P.wsc[i] - P.wsc[i0]);
        const long long cap = P.words_cap;
        if (o < cap) P.words[o] = (P.rw[i] << 16) | op;
        o++;
        for (long long j = 0; j <= nopd; j++) {
            if (id && j == at_rid) {
                if (o < cap) P.words[o] = id;
                o++;
            }
            if (j == nopd) break;
            const long long k = a + j;
            uint32_t v = P.opd[k];
            if (P.opd_ref[k]) v = (uint32_t)(1 + P.rsc[i0 + v] - id0);
            if (o < cap) P.words[o] = v;
            o++;
        }
    }
}

struct BLayout {
    size_t ctrl, err, rmod, res, rw, rsc, wsc, msize, sums, total;
    long long sums_cap;
};

BLayout blayout(int32_t n_mod, int64_t n_rows)
{
    BLayout L{};
    long long mx = n_rows + 1 > n_mod + 1 ? n_rows + 1 : n_mod + 1;
    L.sums_cap = mx / SC_TILE + 2;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const size_t R = (size_t)(n_rows > 0 ? n_rows : 1), M = (size_t)(n_mod > 0 ? n_mod : 1);
    L.ctrl = take(sizeof(BldCtrl));
    L.err = take(8 * M);
    L.rmod = take(4 * R);
    L.res = take(4 * R);
    L.rw = take(4 * R);
    L.rsc = take(8 * (R + 1));
    L.wsc = take(8 * (R + 1));
    L.msize = take(8 * (M + 1));
    L.sums = take(8 * (size_t)(L.sums_cap + 1));
    L.total = o;
    return L;
}

}  // namespace

extern "C" size_t spv_build_workspace_bytes(int32_t n_modules, int64_t n_rows)
{
    if (n_modules < 0 || n_rows < 0) return 0;
    return blayout(n_modules, n_rows).total;
}

extern "C" int spv_build_batch(const spv_oplist *ol, uint32_t version, uint32_t generator, uint32_t *words,
                               int64_t words_capacity, int64_t *word_off, uint32_t *ids, uint32_t *status,
                               int64_t *err_row, void *workspace, size_t workspace_bytes, spv_stream_t stream)
{
    if (!ol || ol->n_modules < 0 || ol->n_rows < 0 || !ol->row_off || !word_off || words_capacity < 0 ||
        (words_capacity && !words) || (ol->n_modules && !status) ||
        (ol->n_rows && (!ol->op || !ol->opd_off || !ol->opd || !ol->opd_ref)))
        return SPV_E_ARG;
    const BLayout L = blayout(ol->n_modules, ol->n_rows);
    if (!workspace || workspace_bytes < L.total) return SPV_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (ol->n_modules == 0) return cudaMemsetAsync(word_off, 0, 8, st) == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
    char *w = (char *)workspace;
    BP P{};
    P.op = ol->op; P.opd_off = ol->opd_off; P.opd = ol->opd; P.opd_ref = ol->opd_ref; P.row_off = ol->row_off;
    P.n_mod = ol->n_modules; P.n_rows_total = ol->n_rows; P.version = version; P.generator = generator;
    P.ctrl = (BldCtrl *)(w + L.ctrl);
    P.err = (unsigned long long *)(w + L.err);
    P.rmod = (int32_t *)(w + L.rmod);
    P.res = (uint32_t *)(w + L.res);
    P.rw = (uint32_t *)(w + L.rw);
    P.rsc = (unsigned long long *)(w + L.rsc);
    P.wsc = (unsigned long long *)(w + L.wsc);
    P.msize = (unsigned long long *)(w + L.msize);
    P.words = words; P.words_cap = words_capacity; P.word_off = word_off; P.ids = ids;
    P.status = status; P.err_row = err_row;
    unsigned long long *sums = (unsigned long long *)(w + L.sums);
    BldCtrl *c = P.ctrl;
    if (cudaMemsetAsync(c, 0, sizeof(BldCtrl), st) != cudaSuccess) return SPV_E_CUDA;
    const int gm = grid_for(ol->n_modules, 256);
    const int gr = grid_for(ol->n_rows, 256);
    SPV_LAUNCH("k_bld_mod_init", st, k_bld_mod_init<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_check_opd", st, k_bld_check_opd<<<gr, 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_rmod", st, k_bld_rmod<<<grid_for(32ll * ol->n_modules, 256), 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_rows", st, k_bld_rows<<<gr, 256, 0, st>>>(P));
    scan(P.res, &c->n_rows, ol->n_rows, sums, P.rsc, nullptr, st);
    scan(P.rw, &c->n_rows, ol->n_rows, sums, P.wsc, nullptr, st);
    SPV_LAUNCH("k_bld_mod", st, k_bld_mod<<<gm, 256, 0, st>>>(P));
    scan(P.msize, &c->n_mod, ol->n_modules, sums, (unsigned long long *)word_off, nullptr, st);
    SPV_LAUNCH("k_bld_head", st, k_bld_head<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_write", st, k_bld_write<<<gr, 256, 0, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}
