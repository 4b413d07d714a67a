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
// A module of more than SEG rows is split into segments of SEG rows, one CTA
// each: the segments' summaries, scanned in order per module, give each
// segment its entry state, and each segment is then walked like a module.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spv.h"
#include "spv_prof.h"
#include "spv_scan.cuh"
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
constexpr long long SEG = 16384;       // rows per segment of a large module

// Summarise rows [a, b) (absolute) in a CTA: each thread a contiguous slice.
// Returns the thread's slice summary in mine and the exclusive prefix of the
// slices before it in ex (in slice order); total (the whole range) in every
// thread. lo / hi receive the thread's slice.
__device__ __forceinline__ void range_scan(const uint16_t *op, long long a, long long b, Summary &mine, Summary &ex,
                                           Summary &total, long long &lo, long long &hi)
{
    __shared__ Summary s_warp[LNT / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = b > a ? b - a : 0;
    const long long per = (n + LNT - 1) / LNT;
    lo = a + (tid * per < n ? tid * per : n);
    hi = lo + per < a + n ? lo + per : a + n;
    uint32_t cur = identity_summary().map, mx = 0;
    for (long long i = lo; i < hi; i++) {
        const uint32_t code = row_code(op, i), cls = code & 15u, sec = code >> 4;
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
    mine = Summary{cur, mx};
    Summary incl = mine;
    #pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        Summary o{__shfl_up_sync(0xffffffffu, incl.map, d), __shfl_up_sync(0xffffffffu, incl.maxs, d)};
        if (lane >= d) incl = combine(o, incl);
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    Summary pre = identity_summary();
    for (int w = 0; w < wid; w++) pre = combine(pre, s_warp[w]);
    total = identity_summary();
    for (int w = 0; w < LNT / 32; w++) total = combine(total, s_warp[w]);
    Summary lane_ex{__shfl_up_sync(0xffffffffu, incl.map, 1), __shfl_up_sync(0xffffffffu, incl.maxs, 1)};
    if (lane == 0) lane_ex = identity_summary();
    ex = combine(pre, lane_ex);
    __syncthreads();
}

// Walk rows [lo, hi) from state / maxsec; the first error as row - r0 << 8 |
// code into *best (shared); returns the state after the slice.
__device__ __forceinline__ uint32_t range_walk(const uint16_t *op, long long lo, long long hi, long long r0,
                                               uint32_t state, uint32_t maxsec, unsigned long long *best)
{
    for (long long i = lo; i < hi; i++) {
        const uint32_t code = row_code(op, i), cls = code & 15u, sec = code >> 4;
        uint32_t next, err;
        transition(cls, next, err);
        uint32_t e = (err >> (3 * state)) & 7u;
        if (e == 0 && state == S_MODULE && section_class(cls)) {
            if (sec < maxsec) e = SPV_LAYOUT_SECTION_ORDER;
            else maxsec = sec;
        }
        if (e) {
            atomicMin(best, ((unsigned long long)(i - r0) << 8) | e);
            return 0xffu;
        }
        state = (next >> (2 * state)) & 3u;
    }
    return state;
}

// One CTA per module of at most SEG rows (grid-stride); larger modules go
// to the segment kernels.
__global__ void __launch_bounds__(LNT) k_layout(const uint16_t *op, const int64_t *first_row, int n_mod,
                                               long long cap_rows, uint32_t *status, int64_t *err_row)
{
    __shared__ unsigned long long s_best;
    const int tid = threadIdx.x;
    for (int m = blockIdx.x; m < n_mod; m += gridDim.x) {
        const long long r0 = first_row[m];
        long long r1 = first_row[m + 1];
        if (r1 > cap_rows) r1 = cap_rows;
        const long long n = r1 > r0 ? r1 - r0 : 0;
        if (n > SEG) continue;
        if (tid == 0) s_best = ~0ull;
        Summary mine, ex, total;
        long long lo, hi;
        range_scan(op, r0, r0 + n, mine, ex, total, lo, hi);
        range_walk(op, lo, hi, r0, ex.map & 3u, ex.maxs & 15u, &s_best);
        __syncthreads();
        if (tid == 0) {
            const uint32_t final_state = total.map & 3u;          // the whole module from S_MODULE
            const unsigned long long best = s_best;
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

struct SegP {
    const uint16_t *op;
    const int64_t *first_row;
    int n_mod;
    long long cap_rows;
    unsigned long long *mseg;          // per module: segments (then their exclusive scan, n_mod + 1)
    unsigned long long *mbest;         // per module: first error, row << 8 | code
    uint32_t *mfinal;                  // per module: the state after its last row
    Summary *seg_sum;                  // per segment: its summary, then its entry (map, maxs at S_MODULE)
    uint32_t *status;
    int64_t *err_row;
    long long seg_cap;
    long long *n_dev;                  // the module count, for the scan
};

__device__ __forceinline__ long long mod_rows(const SegP &P, int m, long long &r0)
{
    r0 = P.first_row[m];
    long long r1 = P.first_row[m + 1];
    if (r1 > P.cap_rows) r1 = P.cap_rows;
    return r1 > r0 ? r1 - r0 : 0;
}

__global__ void k_layout_seg_count(SegP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        long long r0;
        const long long n = mod_rows(P, m, r0);
        P.mseg[m] = n > SEG ? (unsigned long long)((n + SEG - 1) / SEG) : 0ull;
        P.mbest[m] = ~0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.n_dev = P.n_mod;
}

// the module of segment s: the last m with mseg[m] <= s
__device__ __forceinline__ int seg_module(const SegP &P, long long s)
{
    int lo = 0, hi = P.n_mod - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)P.mseg[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// PASS 0: each segment's summary; PASS 1: each segment walked from its entry
template <int PASS>
__global__ void __launch_bounds__(LNT) k_layout_seg(SegP P)
{
    __shared__ int s_m;
    __shared__ unsigned long long s_best;
    const long long nseg = (long long)P.mseg[P.n_mod] < P.seg_cap ? (long long)P.mseg[P.n_mod] : P.seg_cap;
    for (long long sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        if (threadIdx.x == 0) { s_m = seg_module(P, sg); s_best = ~0ull; }
        __syncthreads();
        const int m = s_m;
        long long r0;
        const long long n = mod_rows(P, m, r0);
        const long long k = sg - (long long)P.mseg[m];
        const long long a = r0 + k * SEG, b = a + SEG < r0 + n ? a + SEG : r0 + n;
        Summary mine, ex, total;
        long long lo, hi;
        range_scan(P.op, a, b, mine, ex, total, lo, hi);
        if (PASS == 0) {
            if (threadIdx.x == 0) P.seg_sum[sg] = total;
        } else {
            const Summary in = P.seg_sum[sg];                 // entry: map value and maxs at S_MODULE
            const uint32_t st0 = in.map & 3u, mx0 = in.maxs & 15u;
            const uint32_t st = (ex.map >> (2 * st0)) & 3u;
            const uint32_t exm = (ex.maxs >> (4 * st0)) & 15u;
            range_walk(P.op, lo, hi, r0, st, mx0 > exm ? mx0 : exm, &s_best);
            __syncthreads();
            if (threadIdx.x == 0 && s_best != ~0ull) atomicMin(&P.mbest[m], s_best);
            if (b == r0 + n && threadIdx.x == 0) P.mfinal[m] = (total.map >> (2 * st0)) & 3u;   // the last segment
        }
        __syncthreads();
    }
}

// per large module: the segments' entries, in order (one thread per module)
__global__ void k_layout_seg_scan(SegP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        const long long s0 = (long long)P.mseg[m], s1 = (long long)P.mseg[m + 1];
        Summary acc = identity_summary();
        for (long long s = s0; s < s1; s++) {
            const Summary t = P.seg_sum[s];
            P.seg_sum[s] = Summary{acc.map & 3u, acc.maxs & 15u};
            acc = combine(acc, t);
        }
    }
}

__global__ void k_layout_seg_fin(SegP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        const long long s0 = (long long)P.mseg[m], s1 = (long long)P.mseg[m + 1];
        if (s1 == s0) continue;
        long long r0;
        const long long n = mod_rows(P, m, r0);
        uint32_t st = SPV_LAYOUT_OK;
        long long row = -1;
        if (P.mbest[m] != ~0ull) {
            st = (uint32_t)(P.mbest[m] & 255u);
            row = (long long)(P.mbest[m] >> 8);
        } else if (P.mfinal[m] != S_MODULE) {
            st = SPV_LAYOUT_UNCLOSED;
            row = n;
        }
        P.status[m] = st;
        P.err_row[m] = row;
    }
}

}  // namespace

namespace {
struct LLayout { size_t mseg, mbest, mfinal, seg, sums, total; long long seg_cap; };
LLayout llayout(int32_t n_mod, int64_t cap_rows)
{
    LLayout L{};
    L.seg_cap = 2 * (cap_rows / SEG) + 2;      // a large module has more than SEG rows
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += (bytes + 255) & ~(size_t)255; return at; };
    const size_t M = (size_t)(n_mod > 0 ? n_mod : 1);
    L.mseg = take(8 * (M + 1));
    L.mbest = take(8 * M);
    L.mfinal = take(4 * M);
    L.seg = take(sizeof(Summary) * (size_t)L.seg_cap);
    L.sums = take(8 * (M / SC_TILE + 3));
    L.total = o + 256;                         // + the module count for the scan
    return L;
}
}  // namespace

extern "C" size_t spv_layout_workspace_bytes(int32_t n_modules, int64_t capacity_rows)
{
    if (n_modules < 0 || capacity_rows < 0) return 0;
    return llayout(n_modules, capacity_rows).total;
}

extern "C" int spv_layout_batch(const spv_table *table, int32_t n_modules, uint32_t *layout_status,
                                int64_t *layout_err_row, void *workspace, size_t workspace_bytes,
                                spv_stream_t stream)
{
    if (!table || n_modules < 0 || (n_modules && (!layout_status || !layout_err_row || !table->op ||
                                                  !table->mod_first_row)))
        return SPV_E_ARG;
    if (n_modules == 0) return SPV_SUCCESS;
    const LLayout L = llayout(n_modules, table->capacity_rows);
    if (!workspace || workspace_bytes < L.total) return SPV_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    char *w = (char *)workspace;
    SegP P{};
    P.op = table->op; P.first_row = table->mod_first_row; P.n_mod = n_modules; P.cap_rows = table->capacity_rows;
    P.mseg = (unsigned long long *)(w + L.mseg);
    P.mbest = (unsigned long long *)(w + L.mbest);
    P.mfinal = (uint32_t *)(w + L.mfinal);
    P.seg_sum = (Summary *)(w + L.seg);
    P.seg_cap = L.seg_cap;
    P.status = layout_status; P.err_row = layout_err_row;
    P.n_dev = (long long *)(w + L.total - 256);
    const int gm = (n_modules + 255) / 256 < nsm * 8 ? (n_modules + 255) / 256 : nsm * 8;
    int blocks = n_modules < nsm * 32 ? n_modules : nsm * 32;
    SPV_LAUNCH("k_layout", st, k_layout<<<blocks, LNT, 0, st>>>(table->op, table->mod_first_row, n_modules,
                                                               table->capacity_rows, layout_status,
                                                               layout_err_row));
    SPV_LAUNCH("k_layout_seg_count", st, k_layout_seg_count<<<gm, 256, 0, st>>>(P));
    scan(P.mseg, P.n_dev, n_modules, (unsigned long long *)(w + L.sums), P.mseg, nullptr, st);
    const int gs = nsm * 8;
    SPV_LAUNCH("k_layout_seg", st, k_layout_seg<0><<<gs, LNT, 0, st>>>(P));
    SPV_LAUNCH("k_layout_seg_scan", st, k_layout_seg_scan<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_layout_seg", st, k_layout_seg<1><<<gs, LNT, 0, st>>>(P));
    SPV_LAUNCH("k_layout_seg_fin", st, k_layout_seg_fin<<<gm, 256, 0, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}

extern "C" int spv_op_layout(uint32_t opcode, int *layout_class, int *section)
{
    const uint8_t v = opcode < 256 ? SPV_TABLES_HOST.layout[opcode] : 0;
    if (layout_class) *layout_class = v & 15;
    if (section) *section = v >> 4;
    return 0;
}
