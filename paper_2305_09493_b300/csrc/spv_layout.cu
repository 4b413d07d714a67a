// spv_layout.cu -- logical layout and scopes of decoded modules.
//
// Section 3.4.1 (scopes): the module scope holds the global declarations
// (capabilities, memory model, entry points, debug names, decorations,
// types, constants, global variables) and the functions; a function holds
// its parameters and its body; a body is a sequence of basic blocks, each
// opened by a label. Checked over the decoded table: module-scope rows come
// in the specification's section order, and functions and blocks nest as
// the scopes say (the status codes and their rows are spv_layout_status in
// the header).
//
// One CTA per module. Each row's effect on the scope state (module,
// function head, in a block, after a terminator) is a map of four states.
// Each thread summarises a contiguous slice of the module's rows for every
// entry state (the composed map, and the highest module section met at
// module scope); a block scan of the summaries gives every slice its true
// entry state and incoming section maximum; each thread then walks its slice
// again from there and the earliest error of the block is the module's.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spv.h"
#include "spv_prof.h"
#include "spv_tables.cuh"

namespace {

enum : uint32_t { S_MODULE = 0, S_HEAD = 1, S_BLOCK = 2, S_AFTER = 3 };

// The effect of one row of layout class cls: next state per state (2 bits
// each) and error per state (3 bits each, spv_layout_status; 0 = none).
// Section-order errors are found separately.
__device__ __forceinline__ void transition(uint32_t cls, uint32_t &next, uint32_t &err)
{
    auto n4 = [](uint32_t a, uint32_t b, uint32_t c, uint32_t d) { return a | (b << 2) | (c << 4) | (d << 6); };
    auto e4 = [](uint32_t a, uint32_t b, uint32_t c, uint32_t d) { return a | (b << 3) | (c << 6) | (d << 9); };
    const uint32_t O = SPV_LAYOUT_OUTSIDE_FUNCTION, I = SPV_LAYOUT_IN_FUNCTION, B = SPV_LAYOUT_BLOCK;
    switch (cls) {
    case spvt::LCL_SECTION:  next = n4(S_MODULE, S_HEAD, S_BLOCK, S_AFTER); err = e4(0, I, I, I); break;
    case spvt::LCL_MIXED:    next = n4(S_MODULE, S_HEAD, S_BLOCK, S_AFTER); err = e4(0, B, 0, B); break;
    case spvt::LCL_FUNCTION: next = n4(S_HEAD, S_HEAD, S_BLOCK, S_AFTER); err = e4(0, I, I, I); break;
    case spvt::LCL_PARAM:    next = n4(S_MODULE, S_HEAD, S_BLOCK, S_AFTER); err = e4(O, 0, B, B); break;
    case spvt::LCL_LABEL:    next = n4(S_MODULE, S_BLOCK, S_BLOCK, S_BLOCK); err = e4(O, 0, B, 0); break;
    case spvt::LCL_BODY:     next = n4(S_MODULE, S_HEAD, S_BLOCK, S_AFTER); err = e4(O, B, 0, B); break;
    case spvt::LCL_TERM:     next = n4(S_MODULE, S_HEAD, S_AFTER, S_AFTER); err = e4(O, B, 0, B); break;
    case spvt::LCL_FUNCEND:  next = n4(S_MODULE, S_MODULE, S_BLOCK, S_MODULE); err = e4(O, 0, B, 0); break;
    default:                 next = n4(S_MODULE, S_HEAD, S_BLOCK, S_AFTER); err = 0; break;    // neutral
    }
}

// b after a: (b o a)[s] = b[a[s]]
__device__ __forceinline__ uint32_t compose(uint32_t b, uint32_t a)
{
    uint32_t r = 0;
    #pragma unroll
    for (int s = 0; s < 4; s++) r |= ((b >> (2 * ((a >> (2 * s)) & 3u))) & 3u) << (2 * s);
    return r;
}

// A slice of rows summarised for every entry state: the exit state (map,
// 2 bits per entry state) and the highest module section met at module scope
// (4 bits per entry state).
struct Summary { uint32_t map, maxs; };
__device__ __forceinline__ Summary identity_summary() { return {0u | (1u << 2) | (2u << 4) | (3u << 6), 0u}; }
// a followed by b
__device__ __forceinline__ Summary combine(Summary a, Summary b)
{
    Summary r;
    r.map = compose(b.map, a.map);
    r.maxs = 0;
    #pragma unroll
    for (int s = 0; s < 4; s++) {
        const uint32_t ma = (a.maxs >> (4 * s)) & 15u, mid = (a.map >> (2 * s)) & 3u;
        const uint32_t mb = (b.maxs >> (4 * mid)) & 15u;
        r.maxs |= (ma > mb ? ma : mb) << (4 * s);
    }
    return r;
}

__device__ __forceinline__ bool section_class(uint32_t cls)
{
    return cls == spvt::LCL_SECTION || cls == spvt::LCL_MIXED || cls == spvt::LCL_FUNCTION;
}

__device__ __forceinline__ uint32_t row_code(const uint16_t *op, long long r)
{
    const uint32_t o = op[r];
    return o < 256 ? g_spv_tables.layout[o] : 0u;
}

constexpr int LNT = 256;

// One CTA per module (grid-stride): each thread takes a contiguous slice of
// the module's rows, summarises it for every entry state, a block scan gives
// every slice its true entry state and incoming section maximum, and each
// thread walks its slice again to find its first error.
__global__ void __launch_bounds__(LNT) k_layout(const uint16_t *op, const int64_t *first_row, int n_mod,
                                               long long cap_rows, uint32_t *status, int64_t *err_row)
{
    __shared__ Summary s_warp[LNT / 32];
    __shared__ unsigned long long s_best;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int m = blockIdx.x; m < n_mod; m += gridDim.x) {
        const long long r0 = first_row[m];
        long long r1 = first_row[m + 1];
        if (r1 > cap_rows) r1 = cap_rows;
        const long long n = r1 > r0 ? r1 - r0 : 0;
        const long long per = (n + LNT - 1) / LNT;
        const long long lo = tid * per < n ? tid * per : n, hi = lo + per < n ? lo + per : n;
        // pass 1: this slice for every entry state
        uint32_t cur = identity_summary().map, mx = 0;
        for (long long i = lo; i < hi; i++) {
            const uint32_t code = row_code(op, r0 + i), cls = code & 15u, sec = code >> 4;
            uint32_t next, err;
            transition(cls, next, err);
            #pragma unroll
            for (int s = 0; s < 4; s++) {
                const uint32_t st = (cur >> (2 * s)) & 3u;
                if (st == S_MODULE && section_class(cls)) {
                    const uint32_t m0 = (mx >> (4 * s)) & 15u;
                    if (sec > m0) mx = (mx & ~(15u << (4 * s))) | (sec << (4 * s));
                }
                cur = (cur & ~(3u << (2 * s))) | (((next >> (2 * st)) & 3u) << (2 * s));
            }
        }
        // exclusive block scan of the slice summaries (in slice order)
        Summary mine{cur, mx}, incl = mine;
        #pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            Summary o{__shfl_up_sync(0xffffffffu, incl.map, d), __shfl_up_sync(0xffffffffu, incl.maxs, d)};
            if (lane >= d) incl = combine(o, incl);
        }
        if (lane == 31) s_warp[wid] = incl;
        if (tid == 0) s_best = ~0ull;
        __syncthreads();
        Summary pre = identity_summary();
        for (int w = 0; w < wid; w++) pre = combine(pre, s_warp[w]);
        Summary lane_ex{__shfl_up_sync(0xffffffffu, incl.map, 1), __shfl_up_sync(0xffffffffu, incl.maxs, 1)};
        if (lane == 0) lane_ex = identity_summary();
        const Summary ex = combine(pre, lane_ex);
        uint32_t state = ex.map & 3u;                  // entry state from S_MODULE
        uint32_t maxsec = ex.maxs & 15u;
        // pass 2: the slice again from its true entry, first error
        for (long long i = lo; i < hi; i++) {
            const uint32_t code = row_code(op, r0 + i), cls = code & 15u, sec = code >> 4;
            uint32_t next, err;
            transition(cls, next, err);
            uint32_t e = (err >> (3 * state)) & 7u;
            if (e == 0 && state == S_MODULE && section_class(cls)) {
                if (sec < maxsec) e = SPV_LAYOUT_SECTION_ORDER;
                else maxsec = sec;
            }
            if (e) {
                atomicMin(&s_best, ((unsigned long long)i << 8) | e);
                break;
            }
            state = (next >> (2 * state)) & 3u;
        }
        __syncthreads();
        if (tid == LNT - 1) {
            // the whole module from S_MODULE: the last slice's entry, then the slice
            const uint32_t final_state = (combine(ex, mine).map) & 3u;
            unsigned long long best = s_best;
            uint32_t st = SPV_LAYOUT_OK;
            long long row = -1;
            if (best != ~0ull) { st = (uint32_t)(best & 255u); row = (long long)(best >> 8); }
            else if (final_state != S_MODULE) { st = SPV_LAYOUT_UNCLOSED; row = n; }
            status[m] = st;
            err_row[m] = row;
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" int spv_layout_batch(const spv_table *table, int32_t n_modules, uint32_t *layout_status,
                                int64_t *layout_err_row, spv_stream_t stream)
{
    if (!table || n_modules < 0 || (n_modules && (!layout_status || !layout_err_row || !table->op ||
                                                  !table->mod_first_row)))
        return SPV_E_ARG;
    if (n_modules == 0) return SPV_SUCCESS;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    int blocks = n_modules < nsm * 32 ? n_modules : nsm * 32;
    SPV_LAUNCH("k_layout", st, k_layout<<<blocks, LNT, 0, st>>>(table->op, table->mod_first_row, n_modules,
                                                               table->capacity_rows, layout_status,
                                                               layout_err_row));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}

extern "C" int spv_op_layout(uint32_t opcode, int *layout_class, int *section)
{
    const uint8_t v = opcode < 256 ? SPV_TABLES_HOST.layout[opcode] : 0;
    if (layout_class) *layout_class = v & 15;
    if (section) *section = v >> 4;
    return 0;
}
