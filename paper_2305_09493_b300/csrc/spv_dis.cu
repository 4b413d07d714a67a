// spv_dis.cu -- batched disassembly of decoded SPIR-V modules (section 3.4.4:
// mapper classes turn opcode integers and operands into text; Listing 10's
// "inline names" and "header" options; one line per instruction as in
// Listing 8).
//
// Two passes over the table's rows with one formatter, templated on its
// output: pass 1 counts each row's bytes, scans the counts (block scan +
// decoupled look-back) into 64-bit positions; pass 2 writes the bytes. Before
// them, each module gets two id tables in a workspace arena: the row of the
// first OpName naming each id (for inline names) and the row of the first
// instruction defining each id (whether an OpConstant's type is a float).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spv.h"
#include "spv_device.cuh"
#include "spv_prof.h"

using namespace spvd;

namespace {

constexpr uint32_t NOROW = 0xFFFFFFFFu;
constexpr int DNT = 256;             // threads per CTA in the row passes
constexpr int DPT = 8;               // rows per thread in the scan pass
constexpr int DROWS = DNT * DPT;     // rows per scan tile
constexpr unsigned long long F_AGG = 1ull << 62, F_INC = 2ull << 62, F_MSK = 3ull << 62;

struct DisCtrl {
    unsigned int next_tile;
    unsigned int timeout;
    unsigned long long arena_used;
    unsigned long long n_rows;
};

struct DisMod {
    uint32_t ok;             // header valid and tables fit
    uint32_t bound;
    long long arena_off;     // the module's id tables (see IdTab)
    uint32_t slots;          // 0: direct tables indexed by id; else hash map of this many ids
    uint32_t header_len;     // bytes of the header comment lines
    uint32_t status;         // S_OK / header status / S_CAPACITY
    unsigned long long hincl; // inclusive scan of header_len over modules
};

struct DP {
    const uint32_t *words;
    const int64_t *mod_off;
    int n_mod;
    const uint16_t *op; const uint16_t *wc; const uint64_t *off; const uint32_t *rid; const uint32_t *mod;
    const int64_t *first_row; const uint32_t *n_instr;
    long long cap_rows;
    int inline_names, header;
    char *text; unsigned long long text_cap; uint64_t *text_off; uint32_t *dis_status;
    DisCtrl *ctrl; DisMod *dm; uint32_t *arena; long long arena_words;
    unsigned long long *tstate; uint64_t *rowpos;
    long long max_spins;
};

__device__ __forceinline__ int dec_len(unsigned long long v) { int n = 1; while (v >= 10) { v /= 10; n++; } return n; }

// header comment lines: "; SPIR-V\n; Version: M.m\n; Generator: 0x%08x\n; Bound: B\n; Schema: S\n"
__device__ uint32_t header_len(const uint32_t *w)
{
    return 9 + (11 + dec_len((w[1] >> 16) & 0xff) + 1 + dec_len((w[1] >> 8) & 0xff) + 1) + (13 + 10 + 1) +
           (9 + dec_len(w[3]) + 1) + (10 + dec_len(w[4]) + 1);
}

// Per-module id tables: for every id the module-local row of its first
// OpName and of its first definition. Direct tables of 2 * bound words when
// bound <= 2 * len + 64; otherwise a hash map of len + 64 ids (keys, then
// name rows, then definition rows; empty key 0xFFFFFFFF). A module of len
// words names or defines fewer than len ids, so the map never fills.
__host__ __device__ inline bool idtab_dense(uint32_t bound, long long len)
{
    return (unsigned long long)bound <= 2ull * (unsigned long long)len + 64;
}
__host__ __device__ inline unsigned long long idtab_words(uint32_t bound, long long len)
{
    return idtab_dense(bound, len) ? 2ull * bound : 3ull * ((unsigned long long)len + 64);
}
__device__ __forceinline__ uint32_t idtab_hash(uint32_t id, uint32_t slots) { return (uint32_t)(((unsigned long long)id * 2654435761ull) % slots); }
// slot of id (id < bound), or -1 when absent (create = false)
__device__ __forceinline__ long long idtab_slot(uint32_t *base, uint32_t bound, uint32_t slots, uint32_t id, bool create)
{
    if (!slots) return id < bound ? (long long)id : -1;
    uint32_t h = idtab_hash(id, slots);
    for (;;) {
        uint32_t k = create ? atomicCAS(&base[h], NOROW, id) : base[h];
        if (k == id || (create && k == NOROW)) return h;
        if (k == NOROW) return -1;
        h = h + 1 == slots ? 0 : h + 1;
    }
}
__device__ __forceinline__ uint32_t *idtab_names(uint32_t *base, uint32_t bound, uint32_t slots) { return slots ? base + slots : base; }
__device__ __forceinline__ uint32_t *idtab_defs(uint32_t *base, uint32_t bound, uint32_t slots) { return slots ? base + 2ull * slots : base + bound; }

// ---------------------------------------------------------------------------
// sinks
// ---------------------------------------------------------------------------
struct CountSink {
    unsigned long long n = 0;
    __device__ void put(char) { n++; }
    __device__ void puts(const char *s, int len) { n += len; }
};
struct WriteSink {
    char *p;
    __device__ void put(char c) { *p++ = c; }
    __device__ void puts(const char *s, int len) { for (int i = 0; i < len; i++) p[i] = s[i]; p += len; }
};

template <class Sink> __device__ void put_lit(Sink &k, const char *s)
{
    int n = 0;
    while (s[n]) n++;
    k.puts(s, n);
}
template <class Sink> __device__ void put_dec(Sink &k, unsigned long long v)
{
    char b[20];
    int n = 0;
    do { b[n++] = (char)('0' + v % 10); v /= 10; } while (v);
    while (n) k.put(b[--n]);
}
template <class Sink> __device__ void put_hex_digits(Sink &k, unsigned long long v, int digits)
{
    for (int i = digits - 1; i >= 0; i--) {
        unsigned d = (unsigned)((v >> (4 * i)) & 15);
        k.put((char)(d < 10 ? '0' + d : 'a' + d - 10));
    }
}
template <class Sink> __device__ void put_hex8(Sink &k, uint32_t v) { k.put('0'); k.put('x'); put_hex_digits(k, v, 8); }
template <class Sink> __device__ void put_name(Sink &k, uint16_t off, uint8_t len)
{
    k.puts(g_spv_tables.names + off, len);
}

// C99 "%a" spelling of a double as glibc prints it: [-]0x1.<hex>p<+|-><dec>
// for normal numbers (trailing zero digits dropped, no point when none are
// left), [-]0x0.<hex>p-1022 for subnormals, [-]0x0p+0 for zero, [-]inf and
// [-]nan.
template <class Sink> __device__ void put_hexfloat64(Sink &k, unsigned long long b)
{
    bool neg = b >> 63;
    unsigned e = (unsigned)((b >> 52) & 0x7ff);
    unsigned long long m = b & ((1ull << 52) - 1);
    if (e == 0x7ff) { if (neg) k.put('-'); put_lit(k, m ? "nan" : "inf"); return; }
    if (neg) k.put('-');
    if (e == 0 && m == 0) { put_lit(k, "0x0p+0"); return; }
    k.put('0'); k.put('x'); k.put(e == 0 ? '0' : '1');
    if (m) {
        int digits = 13;
        while (!(m & 15)) { m >>= 4; digits--; }
        k.put('.');
        put_hex_digits(k, m, digits);
    }
    k.put('p');
    int ex = e == 0 ? -1022 : (int)e - 1023;
    if (ex < 0) { k.put('-'); ex = -ex; } else k.put('+');
    put_dec(k, (unsigned long long)ex);
}

// a 32-bit float widened exactly to double bits
__device__ unsigned long long f32_to_f64_bits(uint32_t f)
{
    unsigned long long s = (unsigned long long)(f >> 31) << 63;
    uint32_t e = (f >> 23) & 0xff, m = f & 0x7fffff;
    if (e == 0xff) return s | (0x7ffull << 52) | ((unsigned long long)m << 29);
    if (e == 0) {
        if (m == 0) return s;
        int lz = __clz(m) - 8;              // leading zeros within the 23-bit field (1..23)
        m = (m << (lz + 1)) & 0x7fffff;      // normalise: drop the leading one
        unsigned long long ex = (unsigned long long)(1023 - 126 - (lz + 1));
        return s | (ex << 52) | ((unsigned long long)m << 29);
    }
    return s | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)m << 29);
}

// ---------------------------------------------------------------------------
// per-row formatting
// ---------------------------------------------------------------------------
struct RowCtx {
    const uint32_t *iw;          // the instruction's words
    uint32_t wc, op;
    const DisMod *md;
    uint32_t *tab;               // module's id tables
    bool names;                  // inline names on
    const DP *P;
    int64_t first;               // module's first row
};

template <class Sink> __device__ void put_id(Sink &k, const RowCtx &c, uint32_t id)
{
    k.put('%');
    if (c.names && id < c.md->bound) {
        long long sl = idtab_slot(c.tab, c.md->bound, c.md->slots, id, false);
        uint32_t nr = sl < 0 ? NOROW : idtab_names(c.tab, c.md->bound, c.md->slots)[sl];
        if (nr != NOROW) {
            int64_t row = c.first + nr;
            const uint32_t *nw = c.P->words + c.P->off[row];
            uint32_t nwc = c.P->wc[row];
            bool stop = false;
            for (uint32_t i = 2; i < nwc && !stop; i++) {
                uint32_t v = __ldg(nw + i);
                for (int b = 0; b < 4; b++) {
                    unsigned ch = (v >> (8 * b)) & 0xffu;
                    if (!ch) { stop = true; break; }
                    bool keep = (ch >= '0' && ch <= '9') || (ch >= 'A' && ch <= 'Z') || (ch >= 'a' && ch <= 'z') || ch == '_';
                    k.put(keep ? (char)ch : '_');
                }
            }
            k.put('_');
        }
    }
    put_dec(k, id);
}

template <class Sink> __device__ void put_string(Sink &k, const uint32_t *iw, uint32_t pos, uint32_t n)
{
    k.put('"');
    for (uint32_t i = 0; i < n; i++) {
        uint32_t v = __ldg(iw + pos + i);
        for (int b = 0; b < 4; b++) {
            unsigned ch = (v >> (8 * b)) & 0xffu;
            if (!ch) { k.put('"'); return; }
            if (ch == '"' || ch == '\\') { k.put('\\'); k.put((char)ch); }
            else if (ch < 0x20 || ch > 0x7e) { k.put('\\'); k.put('x'); put_hex_digits(k, ch, 2); }
            else k.put((char)ch);
        }
    }
    k.put('"');
}

template <class Sink> __device__ void put_venum(Sink &k, int kind, uint32_t v)
{
    if (v < 64 && g_spv_tables.venum[kind][v].known) {
        const spvt::EnDesc &e = g_spv_tables.venum[kind][v];
        put_name(k, (uint16_t)((e.name_hi << 8) | e.name_lo), e.name_len);
    } else put_dec(k, v);
}

template <class Sink> __device__ void put_benum(Sink &k, int kind, uint32_t v)
{
    if (v == 0) { put_lit(k, "None"); return; }
    uint32_t known = 0;
    for (int b = 0; b < 32; b++) if (g_spv_tables.benum[kind][b].known) known |= 1u << b;
    if (v & ~known) { put_dec(k, v); return; }
    bool first = true;
    uint32_t x = v;
    while (x) {
        int b = __ffs(x) - 1;
        x &= x - 1;
        if (!first) k.put('|');
        const spvt::EnDesc &e = g_spv_tables.benum[kind][b];
        put_name(k, (uint16_t)((e.name_hi << 8) | e.name_lo), e.name_len);
        first = false;
    }
}

template <class Sink> __device__ void put_raw_tail(Sink &k, const RowCtx &c)
{
    for (uint32_t i = 1; i < c.wc; i++) { k.put(' '); put_hex8(k, __ldg(c.iw + i)); }
}

// one operand of a parameter list (no optional / repeat forms except A_LITS)
template <class Sink> __device__ void put_param(Sink &k, const RowCtx &c, uint8_t pc, uint32_t &pos)
{
    auto word = [&](uint32_t i) -> uint32_t { return __ldg(c.iw + i); };
    if (pc == spvt::A_LITS) { for (; pos < c.wc; pos++) { k.put(' '); put_dec(k, word(pos)); } return; }
    k.put(' ');
    if (pc == spvt::A_ID) { put_id(k, c, word(pos)); pos++; }
    else if (pc == spvt::A_LIT) { put_dec(k, word(pos)); pos++; }
    else if (pc == spvt::A_STR) { uint32_t n = string_words(word, pos, c.wc); put_string(k, c.iw, pos, n); pos += n; }
    else { put_venum(k, pc - spvt::A_ENUM, word(pos)); pos++; }
}

template <class Sink> __device__ void format_row(Sink &k, const RowCtx &c)
{
    const spvt::Tables &T = g_spv_tables;
    auto word = [&](uint32_t i) -> uint32_t { return __ldg(c.iw + i); };
    if (c.op >= 256 || !(T.ops[c.op].flags & 1)) {
        k.put('O'); k.put('p'); put_dec(k, c.op);
        put_raw_tail(k, c); k.put('\n');
        return;
    }
    const spvt::OpDesc &d = T.ops[c.op];
    Walk wk = walk_instruction(word, c.wc, d, 0xffffffffu);
    if (!wk.ok) {
        put_name(k, d.name_off, d.name_len);
        put_raw_tail(k, c); k.put('\n');
        return;
    }
    uint32_t pos = 1;
    uint32_t rt = 0;
    if (d.flags & 2) { rt = word(1); pos++; }
    if (d.flags & 4) { put_id(k, c, word(pos)); put_lit(k, " = "); pos++; }
    put_name(k, d.name_off, d.name_len);
    if (d.flags & 2) { k.put(' '); put_id(k, c, rt); }
    for (int q = 0; q < d.nprog; q++) {
        uint8_t code = d.prog[q];
        bool opt = (code & spvt::A_OPT) != 0;
        code &= 0x7f;
        if (code == spvt::A_IDS || code == spvt::A_IDPAIRS) { for (; pos < c.wc; pos++) { k.put(' '); put_id(k, c, word(pos)); } continue; }
        if (code == spvt::A_LITS) { for (; pos < c.wc; pos++) { k.put(' '); put_dec(k, word(pos)); } continue; }
        if (pos >= c.wc) { if (opt) continue; break; }
        if (code == spvt::A_ID) { k.put(' '); put_id(k, c, word(pos)); pos++; }
        else if (code == spvt::A_LIT) { k.put(' '); put_dec(k, word(pos)); pos++; }
        else if (code == spvt::A_STR) {
            uint32_t n = string_words(word, pos, c.wc);
            k.put(' '); put_string(k, c.iw, pos, n); pos += n;
        } else if (code == spvt::A_CTX) {
            uint32_t n = c.wc - pos;
            bool is_float = false;
            if (rt < c.md->bound) {
                long long sl = idtab_slot(c.tab, c.md->bound, c.md->slots, rt, false);
                uint32_t dr = sl < 0 ? NOROW : idtab_defs(c.tab, c.md->bound, c.md->slots)[sl];
                if (dr != NOROW && c.P->op[c.first + dr] == 22) is_float = true;
            }
            k.put(' ');
            if (is_float && n == 1) put_hexfloat64(k, f32_to_f64_bits(word(pos)));
            else if (is_float && n == 2) put_hexfloat64(k, (unsigned long long)word(pos) | ((unsigned long long)word(pos + 1) << 32));
            else if (n == 1) put_dec(k, word(pos));
            else if (n == 2) put_dec(k, (unsigned long long)word(pos) | ((unsigned long long)word(pos + 1) << 32));
            else for (uint32_t i = 0; i < n; i++) { if (i) k.put(' '); put_dec(k, word(pos + i)); }
            pos = c.wc;
        } else if (code >= spvt::A_ENUM && code < spvt::A_ENUM + spvt::NUM_VKINDS) {
            int kind = code - spvt::A_ENUM;
            uint32_t v = word(pos++);
            k.put(' ');
            put_venum(k, kind, v);
            if (v < 64 && T.venum[kind][v].known) {
                const spvt::EnDesc &e = T.venum[kind][v];
                for (int p = 0; p < e.nparam; p++) put_param(k, c, e.param[p], pos);
            } else if (T.vunknown[kind]) {
                put_param(k, c, T.vunknown[kind], pos);
            }
        } else {
            int kind = code - spvt::A_BITS;
            uint32_t v = word(pos++);
            k.put(' ');
            put_benum(k, kind, v);
            uint32_t x = v;
            while (x) {
                int b = __ffs(x) - 1;
                x &= x - 1;
                const spvt::EnDesc &e = T.benum[kind][b];
                if (!e.known) continue;
                for (int p = 0; p < e.nparam; p++) { k.put(' '); put_dec(k, word(pos)); pos++; }
            }
        }
    }
    k.put('\n');
}

__device__ __forceinline__ bool make_ctx(const DP &P, long long row, RowCtx &c)
{
    uint32_t m = P.mod[row];
    const DisMod &md = P.dm[m];
    if (!md.ok) return false;
    c.iw = P.words + P.off[row];
    c.wc = P.wc[row];
    c.op = P.op[row];
    c.md = &md;
    c.tab = P.arena + md.arena_off;
    c.names = P.inline_names != 0;
    c.P = &P;
    c.first = P.first_row[m];
    return true;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// chunked block-wide exclusive scan over modules (1024 threads): calls
// f(m, excl) for every module with the exclusive prefix of val(m)
template <class Val, class F>
__device__ unsigned long long block_scan_modules(int n_mod, Val val, F f)
{
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_base;
    int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int base = 0; base < n_mod; base += 1024) {
        int m = base + tid;
        unsigned long long v = m < n_mod ? val(m) : 0;
        unsigned long long incl = v;
        for (int d = 1; d < 32; d <<= 1) { unsigned long long a = __shfl_up_sync(0xffffffffu, incl, d); if (lane >= d) incl += a; }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned long long a = s_w[lane];
            for (int d = 1; d < 32; d <<= 1) { unsigned long long x = __shfl_up_sync(0xffffffffu, a, d); if (lane >= d) a += x; }
            s_w[lane] = a;
        }
        __syncthreads();
        unsigned long long excl = s_base + (wid ? s_w[wid - 1] : 0) + incl - v;
        if (m < n_mod) f(m, excl, v);
        __syncthreads();
        if (tid == 1023) s_base = excl + v;
        __syncthreads();
    }
    return s_base;
}

__global__ void __launch_bounds__(1024) k_dis_prepass(DP P)
{
    // pass A: header status, bound, id-table arena layout
    unsigned long long used = block_scan_modules(P.n_mod,
        [&](int m) -> unsigned long long {
            long long o = P.mod_off[m], len = P.mod_off[m + 1] - o;
            uint32_t st = (len < 0 || len > 0x7fffffffLL) ? S_CAPACITY : header_status(P.words + o, len);
            return st == S_OK ? idtab_words(P.words[o + 3], len) : 0ull;
        },
        [&](int m, unsigned long long excl, unsigned long long na) {
            long long o = P.mod_off[m], len = P.mod_off[m + 1] - o;
            uint32_t st = (len < 0 || len > 0x7fffffffLL) ? S_CAPACITY : header_status(P.words + o, len);
            DisMod d;
            d.bound = st == S_OK ? P.words[o + 3] : 0;
            d.slots = (st == S_OK && !idtab_dense(d.bound, len)) ? (uint32_t)(len + 64) : 0;
            d.arena_off = (long long)excl;
            d.ok = st == S_OK && (long long)(excl + na) <= P.arena_words;
            d.status = st != S_OK ? st : (d.ok ? S_OK : S_CAPACITY);
            d.header_len = (d.ok && P.header) ? header_len(P.words + o) : 0;
            d.hincl = 0;
            P.dm[m] = d;
        });
    // pass B: inclusive scan of the header bytes of the modules that print
    block_scan_modules(P.n_mod,
        [&](int m) -> unsigned long long { return P.dm[m].header_len; },
        [&](int m, unsigned long long excl, unsigned long long nh) { P.dm[m].hincl = excl + nh; });
    if (threadIdx.x == 0) {
        P.ctrl->arena_used = used < (unsigned long long)P.arena_words ? used : (unsigned long long)P.arena_words;
        long long nr = P.first_row[P.n_mod];
        P.ctrl->n_rows = (unsigned long long)(nr < P.cap_rows ? nr : P.cap_rows);
        P.ctrl->next_tile = 0;
        P.ctrl->timeout = 0;
    }
}

__global__ void k_dis_clear(DP P)
{
    unsigned long long n = P.ctrl->arena_used;
    unsigned long long nt = P.ctrl->n_rows / DROWS + 1;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n; i += stride) P.arena[i] = NOROW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nt; i += stride) P.tstate[i] = 0;
}

// first OpName per id and first definition per id (module-local rows)
__global__ void k_dis_ids(DP P)
{
    const spvt::Tables &T = g_spv_tables;
    long long n = (long long)P.ctrl->n_rows;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < n; row += stride) {
        uint32_t m = P.mod[row];
        const DisMod &md = P.dm[m];
        if (!md.ok) continue;
        uint32_t op = P.op[row], wc = P.wc[row];
        uint32_t local = (uint32_t)(row - P.first_row[m]);
        uint32_t *tab = P.arena + md.arena_off;
        if (op == 5 && wc >= 2 && P.inline_names) {
            uint32_t target = __ldg(P.words + P.off[row] + 1);
            if (target < md.bound) {
                long long sl = idtab_slot(tab, md.bound, md.slots, target, true);
                atomicMin(&idtab_names(tab, md.bound, md.slots)[sl], local);
            }
        }
        if (op < 256 && (T.ops[op].flags & 4)) {
            uint32_t q = 1 + ((T.ops[op].flags >> 1) & 1);
            if (q < wc) {
                uint32_t id = P.rid[row];
                if (id < md.bound) {
                    long long sl = idtab_slot(tab, md.bound, md.slots, id, true);
                    atomicMin(&idtab_defs(tab, md.bound, md.slots)[sl], local);
                }
            }
        }
    }
}

// pass 1: byte count per row, scanned into 64-bit positions
__global__ void __launch_bounds__(DNT) k_dis_len(DP P)
{
    __shared__ unsigned long long s_w[DNT / 32];
    __shared__ unsigned long long s_base;
    __shared__ long long s_tile;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = (long long)P.ctrl->n_rows;
    const long long ntiles = n / DROWS + 1;
    for (;;) {
        if (tid == 0) s_tile = (long long)atomicAdd(&P.ctrl->next_tile, 1u);
        __syncthreads();
        long long t = s_tile;
        if (t >= ntiles) break;
        unsigned long long len[DPT];
        unsigned long long mine = 0;
        #pragma unroll
        for (int i = 0; i < DPT; i++) {
            long long row = t * DROWS + (long long)tid * DPT + i;
            len[i] = 0;
            if (row < n) {
                RowCtx c;
                if (make_ctx(P, row, c)) { CountSink k; format_row(k, c); len[i] = k.n; }
            }
            mine += len[i];
        }
        unsigned long long incl = mine;
        #pragma unroll
        for (int d = 1; d < 32; d <<= 1) { unsigned long long v = __shfl_up_sync(0xffffffffu, incl, d); if (lane >= d) incl += v; }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned long long v = lane < DNT / 32 ? s_w[lane] : 0;
            #pragma unroll
            for (int d = 1; d < 32; d <<= 1) { unsigned long long u = __shfl_up_sync(0xffffffffu, v, d); if (lane >= d) v += u; }
            if (lane < DNT / 32) s_w[lane] = v;
            unsigned long long total = __shfl_sync(0xffffffffu, v, DNT / 32 - 1);
            unsigned long long excl = 0;
            if (t == 0) {
                if (lane == 0) st_release(&P.tstate[0], F_INC | total);
            } else {
                if (lane == 0) st_release(&P.tstate[t], F_AGG | total);
                long long hi = t - 1, spins = 0;
                bool gave_up = false;
                for (;;) {
                    long long j = hi - lane;
                    unsigned long long st = j >= 0 ? ld_acquire(&P.tstate[j]) : F_INC;
                    unsigned long long f = st & F_MSK;
                    unsigned incm = __ballot_sync(0xffffffffu, f == F_INC);
                    unsigned nonem = __ballot_sync(0xffffffffu, f == 0);
                    int le = incm ? __ffs(incm) - 1 : 32;
                    unsigned below = le == 32 ? 0xffffffffu : ((1u << le) - 1u);
                    if (nonem & below) {
                        if (++spins > P.max_spins) { gave_up = true; break; }
                        spin_pause();
                        continue;
                    }
                    unsigned long long v2 = (lane <= le && j >= 0) ? (st & ~F_MSK) : 0ull;
                    #pragma unroll
                    for (int d = 16; d > 0; d >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, d);
                    excl += v2;
                    if (incm) break;
                    hi -= 32;
                }
                if (gave_up && lane == 0) atomicExch(&P.ctrl->timeout, 1u);
                if (lane == 0) st_release(&P.tstate[t], F_INC | (excl + total));
            }
            if (lane == 0) s_base = excl;
        }
        __syncthreads();
        unsigned long long pos = s_base + (wid ? s_w[wid - 1] : 0) + incl - mine;
        #pragma unroll
        for (int i = 0; i < DPT; i++) {
            long long row = t * DROWS + (long long)tid * DPT + i;
            if (row <= n) P.rowpos[row] = pos;      // rowpos[n] = total bytes of all rows
            pos += len[i];
        }
        __syncthreads();
    }
}

// module offsets, status and the capacity decision
__global__ void k_dis_offsets(DP P)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)P.ctrl->n_rows;
    if (m < P.n_mod) {
        const DisMod &md = P.dm[m];
        long long fr = P.first_row[m];
        if (fr > n) fr = n;
        unsigned long long hexcl = md.hincl - md.header_len;
        P.text_off[m] = P.rowpos[fr] + hexcl;
        if (P.dis_status) P.dis_status[m] = P.ctrl->timeout ? S_TIMEOUT : md.status;
    }
    if (m == P.n_mod) {
        unsigned long long h = P.n_mod ? P.dm[P.n_mod - 1].hincl : 0;
        P.text_off[P.n_mod] = P.rowpos[n] + h;
    }
}

// pass 2: write rows
__global__ void k_dis_write_rows(DP P)
{
    // nothing is written when the text does not fit or a wait gave up (offsets void)
    if (P.text_off[P.n_mod] > P.text_cap || P.ctrl->timeout) return;
    long long n = (long long)P.ctrl->n_rows;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < n; row += stride) {
        RowCtx c;
        if (!make_ctx(P, row, c)) continue;
        WriteSink k{P.text + P.rowpos[row] + P.dm[P.mod[row]].hincl};
        format_row(k, c);
    }
}

// header lines
__global__ void k_dis_write_headers(DP P)
{
    if (P.text_off[P.n_mod] > P.text_cap || P.ctrl->timeout) return;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= P.n_mod) return;
    const DisMod &md = P.dm[m];
    if (!md.ok || !P.header) return;
    const uint32_t *w = P.words + P.mod_off[m];
    WriteSink k{P.text + P.text_off[m]};
    put_lit(k, "; SPIR-V\n; Version: ");
    put_dec(k, (w[1] >> 16) & 0xff); k.put('.'); put_dec(k, (w[1] >> 8) & 0xff);
    put_lit(k, "\n; Generator: "); put_hex8(k, w[2]);
    put_lit(k, "\n; Bound: "); put_dec(k, w[3]);
    put_lit(k, "\n; Schema: "); put_dec(k, w[4]); k.put('\n');
}

struct DLayout { size_t ctrl, dm, tstate, rowpos, arena, total; long long arena_words; };
size_t dal(size_t x) { return (x + 255) & ~size_t(255); }
DLayout dlayout(int n_mod, long long n_words, long long rows_cap, long long arena_words)
{
    DLayout L{};
    L.arena_words = arena_words > 0 ? arena_words : 4 * n_words + 192LL * n_mod + 64;
    size_t o = 0;
    L.ctrl = o; o = dal(o + sizeof(DisCtrl));
    L.dm = o; o = dal(o + sizeof(DisMod) * (size_t)n_mod);
    L.tstate = o; o = dal(o + 8 * (size_t)(rows_cap / DROWS + 2));
    L.rowpos = o; o = dal(o + 8 * (size_t)(rows_cap + 1));
    L.arena = o; o = dal(o + 4 * (size_t)L.arena_words);
    L.total = o;
    return L;
}

}  // namespace

extern "C" size_t spv_dis_workspace_bytes(int32_t n_modules, int64_t n_words, int64_t n_rows_capacity,
                                          int64_t arena_words)
{
    if (n_modules < 0 || n_words < 0 || n_rows_capacity < 0) return 0;
    return dlayout(n_modules, n_words, n_rows_capacity, arena_words).total;
}

extern "C" int spv_disassemble_batch(const spv_batch *batch, const spv_table *table, const spv_dis_opts *opts,
                                     char *text, uint64_t text_capacity, uint64_t *text_off, uint32_t *dis_status,
                                     void *workspace, size_t workspace_bytes, int64_t arena_words,
                                     spv_stream_t stream)
{
    if (!batch || !table || !text_off || batch->n_modules < 0 || !batch->mod_off ||
        (batch->n_words && !batch->words) || !table->op || !table->wc || !table->off || !table->rid ||
        !table->mod || !table->mod_first_row || table->capacity_rows < 0)
        return SPV_E_ARG;
    if (text_capacity && !text) return SPV_E_ARG;
    DLayout L = dlayout(batch->n_modules, batch->n_words, table->capacity_rows, arena_words);
    if (!workspace || workspace_bytes < L.total) return SPV_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (batch->n_modules == 0) {
        return cudaMemsetAsync(text_off, 0, 8, st) == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
    }
    char *w = (char *)workspace;
    DP P{};
    P.words = batch->words; P.mod_off = batch->mod_off; P.n_mod = batch->n_modules;
    P.op = table->op; P.wc = table->wc; P.off = table->off; P.rid = table->rid; P.mod = table->mod;
    P.first_row = table->mod_first_row; P.n_instr = table->mod_n_instr; P.cap_rows = table->capacity_rows;
    P.inline_names = opts ? opts->inline_names : 1;
    P.header = opts ? opts->header : 1;
    P.text = text; P.text_cap = text_capacity; P.text_off = text_off; P.dis_status = dis_status;
    P.ctrl = (DisCtrl *)(w + L.ctrl); P.dm = (DisMod *)(w + L.dm);
    P.tstate = (unsigned long long *)(w + L.tstate); P.rowpos = (uint64_t *)(w + L.rowpos);
    P.arena = (uint32_t *)(w + L.arena); P.arena_words = L.arena_words;
    P.max_spins = 1LL << 20;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    int nb = (batch->n_modules + 1 + 255) / 256;
    SPV_LAUNCH("k_dis_prepass", st, k_dis_prepass<<<1, 1024, 0, st>>>(P));
    SPV_LAUNCH("k_dis_clear", st, k_dis_clear<<<nsm * 4, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_ids", st, k_dis_ids<<<nsm * 8, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_len", st, k_dis_len<<<nsm * 4, DNT, 0, st>>>(P));
    SPV_LAUNCH("k_dis_offsets", st, k_dis_offsets<<<nb, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_write_rows", st, k_dis_write_rows<<<nsm * 8, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_write_headers", st, k_dis_write_headers<<<nb, 256, 0, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}
