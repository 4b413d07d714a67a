// spv_build.cu -- batched builder: modules from op lists (section 3.4.2,
// "Enabling Function Composition"). In the paper an instruction is added to
// its scope in order, and every instruction with a result first asks the
// module for the next id (getNextId). Here a JIT backend hands over a whole
// batch of op lists at once: each row is an opcode and its operands, the
// result id left out, and an operand is a literal word or a reference to
// another row of the module. getNextId becomes a scan: the rows whose opcode
// has a result id take ids 1, 2, ... of their module in row order.
//
// Kernels, all on the caller's stream, over tiles of 2,048 consecutive rows
// (row k * 256 + thread of a tile, so that a warp reads consecutive rows):
//   k_bld_mod_init   offsets checked, module records cleared
//   k_bld_tilemod    each tile's first and last modules (binary searches)
//   k_bld_rows       per row: result id or not, word count, and the checks
//                    (result type present, at most 65535 words, references
//                    inside the module and to a row with a result id; the
//                    first bad row of a module wins); a tile scan of result
//                    flags and word counts gives the tile's sums and the
//                    prefixes at the first rows of its modules
//   k_bld_tscan      one block: exclusive scans of the tile sums
//   k_bld_mstart     each module's prefixes at its first row
//   k_bld_mod        module totals (the next module's first-row prefix less
//                    its own), status and words; the module scan of the
//                    words gives the word offsets
//   k_bld_ids        per tile: each row's id from the tile scan of result
//                    flags (getNextId in row order)
//   k_bld_write      per tile: each row's place from the tile scan of word
//                    counts; word 0, the result type, the new result id, the
//                    operands with references resolved through the ids
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spv.h"
#include "spv_prof.h"
#include "spv_scan.cuh"
#include "spv_tables.cuh"

namespace {

constexpr int BT = 256, BPT = 8, BTILE = BT * BPT;      // rows per tile

struct BldCtrl {
    long long n_rows;          // rows of the modules: [row_off[0], row_off[n_modules])
    long long r_first;
    long long n_mod;
    long long n_tiles;
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
    unsigned long long *mres;          // per module: result rows (the bound less one)
    uint32_t *fres, *frw;              // per module: the prefix within the tile at its first row
    unsigned long long *sres, *srw;    // per module: the prefix at its first row
    unsigned long long *tres, *trw;    // per tile: sums, then their exclusive scans (n_tiles + 1)
    int32_t *tm;                       // per tile: the modules of its first and last rows
    unsigned long long *msize;         // per module: words (then scanned into word_off)
    long long tile_cap;
    uint32_t *words;
    long long words_cap;
    int64_t *word_off;
    uint32_t *ids;                     // per row (the caller's array, or workspace)
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
        P.ctrl->n_tiles = a <= b ? (b - a + BTILE - 1) / BTILE : 0;
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

// the module of row r: the last m in [lo, hi] with row_off[m] <= r
__device__ __forceinline__ int module_of(const int64_t *row_off, int lo, int hi, long long r)
{
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// per tile, the modules of its first and last rows (one thread per tile)
__global__ void k_bld_tilemod(BP P)
{
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < c.n_tiles;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r0 = c.r_first + t * BTILE;
        const long long r1 = r0 + BTILE < c.r_first + c.n_rows ? r0 + BTILE : c.r_first + c.n_rows;
        const int m0 = module_of(P.row_off, 0, P.n_mod - 1, r0);
        P.tm[2 * t] = m0;
        P.tm[2 * t + 1] = module_of(P.row_off, m0, P.n_mod - 1, r1 - 1);
    }
}

// the tile's rows [r0, r1) (absolute) and the modules of its first and last rows
__device__ __forceinline__ void tile_rows(const BP &P, const BldCtrl &c, long long t, long long &r0, long long &r1,
                                          int &m0, int &m1)
{
    r0 = c.r_first + t * BTILE;
    r1 = r0 + BTILE < c.r_first + c.n_rows ? r0 + BTILE : c.r_first + c.n_rows;
    m0 = P.tm[2 * t];
    m1 = P.tm[2 * t + 1];
}


// Exclusive scan, in tile row order, of two values per row held in shared
// memory (BTILE rows): each thread scans BPT consecutive rows, then a block
// scan of the thread sums; the prefixes replace the values. Returns the
// tile's totals.
__device__ __forceinline__ void tile_exscan2(uint32_t *va, uint32_t *vb, unsigned long long &ta, unsigned long long &tb)
{
    __shared__ unsigned long long s_a[BT / 32], s_b[BT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t la[BPT], lb[BPT];
    unsigned long long sa = 0, sb = 0;
    #pragma unroll
    for (int k = 0; k < BPT; k++) {
        la[k] = va[threadIdx.x * BPT + k];
        lb[k] = vb[threadIdx.x * BPT + k];
        sa += la[k]; sb += lb[k];
    }
    unsigned long long x = sa, y = sb;
    #pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, x, d), v = __shfl_up_sync(0xffffffffu, y, d);
        if (lane >= d) { x += u; y += v; }
    }
    if (lane == 31) { s_a[wid] = x; s_b[wid] = y; }
    __syncthreads();
    unsigned long long pa = 0, pb = 0;
    ta = 0; tb = 0;
    #pragma unroll
    for (int w = 0; w < BT / 32; w++) {
        if (w < wid) { pa += s_a[w]; pb += s_b[w]; }
        ta += s_a[w]; tb += s_b[w];
    }
    pa += x - sa;
    pb += y - sb;
    #pragma unroll
    for (int k = 0; k < BPT; k++) {
        va[threadIdx.x * BPT + k] = (uint32_t)pa;
        vb[threadIdx.x * BPT + k] = (uint32_t)pb;
        pa += la[k]; pb += lb[k];
    }
    __syncthreads();
}

// row k * BT + threadIdx.x of the tile: a warp takes consecutive rows
__global__ void __launch_bounds__(BT) k_bld_rows(BP P)
{
    __shared__ uint32_t s_res[BTILE], s_rw[BTILE];
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (long long t = blockIdx.x; t < c.n_tiles; t += gridDim.x) {
        long long r0, r1;
        int m0, m1;
        tile_rows(P, c, t, r0, r1, m0, m1);
        int m = m0;
        #pragma unroll 2
        for (int k = 0; k < BPT; k++) {
            const int i = k * BT + threadIdx.x;
            const long long r = r0 + i;
            uint32_t res = 0, rw = 0;
            if (r < r1) {
                if (P.row_off[m + 1] <= r) m = module_of(P.row_off, m, m1, r);
                const long long mr0 = P.row_off[m], nrows = P.row_off[m + 1] - mr0;
                const uint32_t f = op_flags(P.op[r]);
                const long long a = P.opd_off[r], nopd = P.opd_off[r + 1] - a;
                const bool rid = f & 4;
                const long long wc = 1 + nopd + (rid ? 1 : 0);
                uint32_t st = SPV_BUILD_OK;
                if (((f & 2) && nopd == 0) || wc > 65535) {
                    st = SPV_BUILD_BAD_ROW;
                } else {
                    for (long long q = a; q < a + nopd; q++) {
                        if (!P.opd_ref[q]) continue;
                        const uint32_t tr = P.opd[q];
                        if ((long long)tr >= nrows || !(op_flags(P.op[mr0 + tr]) & 4)) { st = SPV_BUILD_BAD_REF; break; }
                    }
                }
                if (st) atomicMin(&P.err[m], ((unsigned long long)(r - mr0) << 8) | st);
                res = rid ? 1u : 0u;
                rw = wc <= 65535 ? (uint32_t)wc : 0u;
            }
            s_res[i] = res;
            s_rw[i] = rw;
        }
        __syncthreads();
        unsigned long long ta, tb;
        tile_exscan2(s_res, s_rw, ta, tb);
        if (threadIdx.x == 0) { P.tres[t] = ta; P.trw[t] = tb; }
        // the first rows of modules: their prefixes in the tile
        m = m0;
        for (int k = 0; k < BPT; k++) {
            const int i = k * BT + threadIdx.x;
            const long long r = r0 + i;
            if (r >= r1) break;
            if (P.row_off[m + 1] <= r) m = module_of(P.row_off, m, m1, r);
            if (P.row_off[m] == r) { P.fres[m] = s_res[i]; P.frw[m] = s_rw[i]; }
        }
        __syncthreads();
    }
}

// one block: exclusive scans of the tile sums, in place (n_tiles + 1 entries)
__global__ void __launch_bounds__(1024) k_bld_tscan(BP P)
{
    const long long n = P.ctrl->bad_offsets ? 0 : P.ctrl->n_tiles;
    __shared__ unsigned long long s_a[32], s_b[32], s_ca, s_cb;
    if (threadIdx.x == 0) { s_ca = 0; s_cb = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long base = 0; base < n; base += 1024) {
        const long long i = base + threadIdx.x;
        const unsigned long long va = i < n ? P.tres[i] : 0, vb = i < n ? P.trw[i] : 0;
        unsigned long long x = va, y = vb;
        #pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, x, d), v = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) { x += u; y += v; }
        }
        if (lane == 31) { s_a[wid] = x; s_b[wid] = y; }
        __syncthreads();
        if (wid == 0) {
            unsigned long long u = s_a[lane], v = s_b[lane];
            #pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long uu = __shfl_up_sync(0xffffffffu, u, d), vv = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) { u += uu; v += vv; }
            }
            s_a[lane] = u; s_b[lane] = v;
        }
        __syncthreads();
        const unsigned long long ca = s_ca, cb = s_cb;
        if (i < n) {
            P.tres[i] = ca + (wid ? s_a[wid - 1] : 0) + x - va;
            P.trw[i] = cb + (wid ? s_b[wid - 1] : 0) + y - vb;
        }
        __syncthreads();
        if (threadIdx.x == 0) { s_ca = ca + s_a[31]; s_cb = cb + s_b[31]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { P.tres[n] = s_ca; P.trw[n] = s_cb; }
}

// the prefixes at each module's first row (modules with rows)
__global__ void k_bld_mstart(BP P)
{
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        const long long x = P.row_off[m];
        if (x < P.row_off[m + 1]) {
            const long long t = (x - c.r_first) / BTILE;
            P.sres[m] = P.tres[t] + P.fres[m];
            P.srw[m] = P.trw[t] + P.frw[m];
        }
    }
}

// module totals (the prefix where the next module with rows starts, or the
// grand total, less the prefix at its own first row), status and words
__global__ void k_bld_mod(BP P)
{
    const BldCtrl &c = *P.ctrl;
    const long long rend = c.r_first + c.n_rows;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        uint32_t st = SPV_BUILD_OK;
        long long bad = -1;
        unsigned long long nw = 0, nres = 0, nrw = 0;
        if (c.bad_offsets) {
            st = SPV_BUILD_BAD_OFFSETS;
        } else {
            const long long x = P.row_off[m], y = P.row_off[m + 1];
            if (x < y) {
                unsigned long long er, ew;
                if (y >= rend) { er = P.tres[c.n_tiles]; ew = P.trw[c.n_tiles]; }
                else {
                    const int mn = module_of(P.row_off, m + 1, P.n_mod - 1, y);     // the module that starts at y
                    er = P.sres[mn]; ew = P.srw[mn];
                }
                nres = er - P.sres[m];
                nrw = ew - P.srw[m];
            }
            if (P.err[m] != ~0ull) {
                st = (uint32_t)(P.err[m] & 255u);
                bad = (long long)(P.err[m] >> 8);
            } else {
                nw = 5 + nrw;
            }
        }
        P.mres[m] = nres;
        P.status[m] = st;
        if (P.err_row) P.err_row[m] = bad;
        P.msize[m] = nw;
    }
}

__global__ void k_bld_head(BP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        if (P.status[m] != SPV_BUILD_OK) continue;
        const uint32_t h[5] = {0x07230203u, P.version, P.generator, (uint32_t)(1 + P.mres[m]), 0u};
        const long long at = P.word_off[m];
        for (int k = 0; k < 5; k++)
            if (at + k < P.words_cap) P.words[at + k] = h[k];
    }
}

// PASS 0: each row's id; PASS 1: each row's words. Row k * BT + threadIdx.x
// of the tile: a warp takes consecutive rows.
template <int PASS>
__global__ void __launch_bounds__(BT) k_bld_tile(BP P)
{
    __shared__ uint32_t s_res[BTILE], s_rw[BTILE];
    const BldCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (long long t = blockIdx.x; t < c.n_tiles; t += gridDim.x) {
        long long r0, r1;
        int m0, m1;
        tile_rows(P, c, t, r0, r1, m0, m1);
        #pragma unroll 4
        for (int k = 0; k < BPT; k++) {
            const int i = k * BT + threadIdx.x;
            const long long r = r0 + i;
            uint32_t res = 0, rw = 0;
            if (r < r1) {
                res = (op_flags(P.op[r]) & 4) ? 1u : 0u;
                if (PASS) rw = (uint32_t)(1 + P.opd_off[r + 1] - P.opd_off[r] + res);
            }
            s_res[i] = res;
            s_rw[i] = rw;
        }
        __syncthreads();
        unsigned long long ta, tb;
        tile_exscan2(s_res, s_rw, ta, tb);
        const unsigned long long bres = P.tres[t], brw = P.trw[t];
        int m = m0;
        for (int k = 0; k < BPT; k++) {
            const int i = k * BT + threadIdx.x;
            const long long r = r0 + i;
            if (r >= r1) break;
            if (P.row_off[m + 1] <= r) m = module_of(P.row_off, m, m1, r);
            const uint32_t f = op_flags(P.op[r]);
            const bool rid = f & 4;
            if (PASS == 0) {
                P.ids[r] = rid ? (uint32_t)(1 + bres + s_res[i] - P.sres[m]) : 0u;
            } else if (P.status[m] == SPV_BUILD_OK) {
                const long long mr0 = P.row_off[m];
                const uint32_t op = P.op[r];
                const uint32_t id = rid ? P.ids[r] : 0u;
                const long long a = P.opd_off[r], nopd = P.opd_off[r + 1] - a;
                const int at_rid = (f & 2) ? 1 : 0;     // the result id's place among the operands
                long long o = P.word_off[m] + 5 + (long long)(brw + s_rw[i] - P.srw[m]);
                const long long cap = P.words_cap;
                if (o < cap) P.words[o] = ((uint32_t)(1 + nopd + (rid ? 1 : 0)) << 16) | op;
                o++;
                for (long long j = 0; j <= nopd; j++) {
                    if (rid && j == at_rid) {
                        if (o < cap) P.words[o] = id;
                        o++;
                    }
                    if (j == nopd) break;
                    const long long q = a + j;
                    uint32_t v = P.opd[q];
                    if (P.opd_ref[q]) v = P.ids[mr0 + v];
                    if (o < cap) P.words[o] = v;
                    o++;
                }
            }
        }
        __syncthreads();
    }
}

struct BLayout {
    size_t ctrl, err, mres, fres, frw, sres, srw, tres, trw, tm, msize, msums, ids, total;
    long long tile_cap;
};

BLayout blayout(int32_t n_mod, int64_t n_rows)
{
    BLayout L{};
    L.tile_cap = n_rows / BTILE + 2;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const size_t R = (size_t)(n_rows > 0 ? n_rows : 1), M = (size_t)(n_mod > 0 ? n_mod : 1);
    L.ctrl = take(sizeof(BldCtrl));
    L.err = take(8 * M);
    L.mres = take(8 * M);
    L.fres = take(4 * M);
    L.frw = take(4 * M);
    L.sres = take(8 * M);
    L.srw = take(8 * M);
    L.tres = take(8 * (size_t)(L.tile_cap + 1));
    L.trw = take(8 * (size_t)(L.tile_cap + 1));
    L.tm = take(8 * (size_t)L.tile_cap);
    L.msize = take(8 * (M + 1));
    L.msums = take(8 * (M / SC_TILE + 3));      // the module scan's tile sums
    L.ids = take(4 * R);                 // the ids when the caller wants none
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
    P.mres = (unsigned long long *)(w + L.mres);
    P.fres = (uint32_t *)(w + L.fres);
    P.frw = (uint32_t *)(w + L.frw);
    P.sres = (unsigned long long *)(w + L.sres);
    P.srw = (unsigned long long *)(w + L.srw);
    P.tres = (unsigned long long *)(w + L.tres);
    P.trw = (unsigned long long *)(w + L.trw);
    P.tm = (int32_t *)(w + L.tm);
    P.msize = (unsigned long long *)(w + L.msize);
    P.tile_cap = L.tile_cap;
    P.words = words; P.words_cap = words_capacity; P.word_off = word_off;
    P.ids = ids ? ids : (uint32_t *)(w + L.ids);
    P.status = status; P.err_row = err_row;
    BldCtrl *c = P.ctrl;
    if (cudaMemsetAsync(c, 0, sizeof(BldCtrl), st) != cudaSuccess) return SPV_E_CUDA;
    const int gm = grid_for(ol->n_modules, 256);
    const int gr = grid_for(ol->n_rows, 256);
    const int gt = grid_for((ol->n_rows + BTILE - 1) / BTILE * BT, BT);
    SPV_LAUNCH("k_bld_mod_init", st, k_bld_mod_init<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_check_opd", st, k_bld_check_opd<<<gr, 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_tilemod", st, k_bld_tilemod<<<grid_for((ol->n_rows + BTILE - 1) / BTILE, 256), 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_rows", st, k_bld_rows<<<gt, BT, 0, st>>>(P));
    SPV_LAUNCH("k_bld_tscan", st, k_bld_tscan<<<1, 1024, 0, st>>>(P));
    SPV_LAUNCH("k_bld_mstart", st, k_bld_mstart<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_mod", st, k_bld_mod<<<gm, 256, 0, st>>>(P));
    scan(P.msize, &c->n_mod, ol->n_modules, (unsigned long long *)(w + L.msums), (unsigned long long *)word_off,
         nullptr, st);
    SPV_LAUNCH("k_bld_head", st, k_bld_head<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_bld_ids", st, k_bld_tile<0><<<gt, BT, 0, st>>>(P));
    SPV_LAUNCH("k_bld_write", st, k_bld_tile<1><<<gt, BT, 0, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}
