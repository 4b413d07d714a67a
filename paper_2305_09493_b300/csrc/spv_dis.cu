// spv_dis.cu -- batched disassembly of decoded SPIR-V modules (section 3.4.4:
// mapper classes turn opcode integers and operands into text; Listing 10's
// "inline names" and "header" options; one line per instruction as in
// Listing 8).
//
// The text of a batch is a sequence of items: for each module its header
// lines (possibly empty), then one line per row of the module. Item i of
// module m is its header when i == first_row[m] + m, else row
// first_row[m] + (i - first_row[m] - m - 1). One persistent kernel takes
// tiles of 512 items; per tile it
//   1. measures every item (an arithmetic count of the formatter's output),
//   2. scans the lengths in the block and gets the tile's 64-bit text base
//      from a decoupled look-back over the predecessors' totals,
//   3. formats every item once into shared memory and copies the tile's text
//      out with 4-byte coalesced stores (tiles whose text exceeds the shared
//      buffer format straight into global memory).
// Before it, each module gets a per-id table in a workspace arena: the row
// and name length of the first OpName naming the id (inline names) and the
// row of the first instruction defining it (whether an OpConstant's type is
// a float).
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/spv.h"
#include "spv_device.cuh"
#include "spv_prof.h"

using namespace spvd;

namespace {

constexpr uint32_t NOROW = 0xFFFFFFFFu;
#ifndef SPV_DIS_NT
#define SPV_DIS_NT 768
#endif
#ifndef SPV_DIS_IPT
#define SPV_DIS_IPT 3
#endif
#ifndef SPV_DIS_TEXT_KB
#define SPV_DIS_TEXT_KB 88
#endif
#ifndef SPV_DIS_MIN_BLOCKS
#define SPV_DIS_MIN_BLOCKS 1
#endif
constexpr int DNT = SPV_DIS_NT;                   // threads per CTA
constexpr int IPT = SPV_DIS_IPT;                  // items per thread
constexpr int ITEMS = DNT * IPT;                  // items per tile
constexpr int TEXT_SMEM = SPV_DIS_TEXT_KB * 1024; // shared text buffer per tile
#ifndef SPV_DIS_STAGE_WORDS
#define SPV_DIS_STAGE_WORDS 12288
#endif
constexpr int STAGE_WORDS = SPV_DIS_STAGE_WORDS;  // a tile's instruction words staged in shared memory
constexpr uint32_t NOSTAGE = 0xFFFFFFFFu;
constexpr unsigned long long F_AGG = 1ull << 62, F_INC = 2ull << 62, F_MSK = 3ull << 62;

struct DisCtrl {
    unsigned int next_tile;
    unsigned int timeout;
    unsigned long long arena_used;
    unsigned long long n_rows;
    unsigned long long n_items;
};

struct DisMod {
    uint32_t ok;             // header valid and id table fits
    uint32_t bound;
    long long arena_off;     // the module's id table
    uint32_t slots;          // 0: direct table by id (3 words per id); else hash map (4 words per slot)
    uint32_t header_len;     // bytes of the header comment lines (0 when not printed)
    uint32_t status;         // S_OK / header status / S_CAPACITY
    uint32_t named;          // 1 when some OpName names an id of the module
    long long item_base;     // index of the module's header item
    unsigned long long bloom;// bit name_hash(id) set for every named id (a superset test)
};

// one of 64 bits per id for the modules' named-id filters
__device__ __forceinline__ uint32_t name_hash(uint32_t id) { return (id * 0x9E3779B1u) >> 26; }

struct DP {
    const uint32_t *words;
    const int64_t *mod_off;
    int n_mod;
    const uint16_t *op; const uint16_t *wc; const uint64_t *off; const uint32_t *rid; const uint32_t *mod;
    const int64_t *first_row;
    long long cap_rows;
    int inline_names, header;
    char *text; unsigned long long text_cap; uint64_t *text_off; uint32_t *dis_status;
    DisCtrl *ctrl; DisMod *dm; uint32_t *arena; long long arena_words;
    unsigned long long *tstate;
    int *tile_m0;            // per tile of k_dis_main: the module holding its first item
    long long max_spins;
    long long stall_tile;    // test hook: this tile never publishes its look-back state (-1: none)
};

// ---------------------------------------------------------------------------
// per-module id tables
// ---------------------------------------------------------------------------
// Direct table of 3 words per id [name row, name length, definition row]
// when bound <= len + 64; otherwise a hash map of len + 64 slots of 4 words
// [id, name row, name length, definition row] (empty id 0xFFFFFFFF). A
// module of len words names or defines fewer than len ids, so the map never
// fills, and a huge bound in a header costs nothing.
__host__ __device__ inline bool idtab_dense(uint32_t bound, long long len)
{
    return (unsigned long long)bound <= (unsigned long long)len + 64;
}
__host__ __device__ inline unsigned long long idtab_words(uint32_t bound, long long len)
{
    // dense: the table, then a bitmap with one bit per id, cleared when the id is named
    return idtab_dense(bound, len) ? 3ull * bound + ((unsigned long long)bound + 31) / 32
                                   : 4ull * ((unsigned long long)len + 64);
}
// the id's [name row, name length, def row] triple, or null when absent
__device__ __forceinline__ uint32_t *idtab_entry(uint32_t *base, uint32_t bound, uint32_t slots, uint32_t id,
                                                 bool create)
{
    if (!slots) return id < bound ? base + 3ull * id : nullptr;
    uint32_t h = (uint32_t)(((unsigned long long)id * 2654435761ull) % slots);
    for (;;) {
        uint32_t *e = base + 4ull * h;
        uint32_t k = create ? atomicCAS(e, NOROW, id) : e[0];
        if (k == id || (create && k == NOROW)) return e + 1;
        if (k == NOROW) return nullptr;
        h = h + 1 == slots ? 0 : h + 1;
    }
}

// header comment lines: "; SPIR-V\n; Version: M.m\n; Generator: 0x%08x\n; Bound: B\n; Schema: S\n"
static __device__ const uint32_t c_pow10[10] = {1u, 10u, 100u, 1000u, 10000u, 100000u, 1000000u, 10000000u,
                                                 100000000u, 1000000000u};
// decimal digits of v: with b its bit length, t = floor(b * 1233 / 4096)
// (1233 / 4096 just below log10(2)) makes the count t + 1 when v >= 10^t, else t
__device__ __forceinline__ uint32_t dec_len32(uint32_t v)
{
    uint32_t u = v | 1u;                               // 0 prints like 1: one digit
    uint32_t t = ((32u - __clz(u)) * 1233u) >> 12;
    return t + 1u - (u < c_pow10[t] ? 1u : 0u);
}
__device__ __forceinline__ uint32_t dec_len64(unsigned long long v)
{
    if (!(v >> 32)) return dec_len32((uint32_t)v);
    uint32_t n = 10;
    unsigned long long t = 10000000000ull;
    while (n < 20 && v >= t) { n++; t *= 10; }
    return n;
}
__device__ uint32_t header_len(const uint32_t *w)
{
    return 9 + (11 + dec_len32((w[1] >> 16) & 0xff) + 1 + dec_len32((w[1] >> 8) & 0xff) + 1) + (13 + 10 + 1) +
           (9 + dec_len32(w[3]) + 1) + (10 + dec_len32(w[4]) + 1);
}

// ---------------------------------------------------------------------------
// sinks: the formatter below runs once counting, once writing
// ---------------------------------------------------------------------------
struct CountSink {
    static constexpr bool counting = true, clipping = false;
    uint32_t n = 0;
    __device__ __forceinline__ void put(char) { n++; }
    __device__ __forceinline__ void puts(const char *, int len) { n += len; }
};
// k_dis_main's dynamic shared memory; its text buffer starts at byte 0. The
// writing sinks hold byte offsets into it rather than pointers, so every
// text store is a shared-memory store, also inside the out-of-line helpers
// that take and return a sink (a pointer passed through them would lose its
// address space and turn every later store generic).
extern __shared__ __align__(16) unsigned char smem_raw[];
__device__ __forceinline__ char *stext() { return reinterpret_cast<char *>(smem_raw); }

struct WriteSink {
    static constexpr bool counting = false, clipping = false;
    uint32_t p;                  // byte offset in the shared text buffer
    __device__ __forceinline__ void put(char c) { stext()[p++] = c; }
    __device__ __forceinline__ void puts(const char *s, int len)
    {
        for (int i = 0; i < len; i++) stext()[p + i] = s[i];
        p += len;
    }
};
// writes only the bytes of a window [0, lim) of positions of the shared text
// buffer; p starts at the line's position relative to the window (possibly
// negative)
struct ClipSink {
    static constexpr bool counting = false, clipping = true;
    long long p, lim;
    __device__ __forceinline__ void put(char c)
    {
        if ((unsigned long long)p < (unsigned long long)lim) stext()[p] = c;
        p++;
    }
    __device__ __forceinline__ void puts(const char *s, int len) { for (int i = 0; i < len; i++) put(s[i]); }
};

// a string literal, its length known at compile time
template <class Sink, int N> __device__ __forceinline__ void put_lit(Sink &k, const char (&s)[N])
{
    #pragma unroll
    for (int i = 0; i < N - 1; i++) k.put(s[i]);
}
template <class Sink> __device__ __forceinline__ void put_dec(Sink &k, uint32_t v)
{
    if constexpr (Sink::counting) {
        k.n += dec_len32(v);
    } else if constexpr (Sink::clipping) {
        for (int i = (int)dec_len32(v) - 1; i >= 0; i--) k.put((char)('0' + (v / c_pow10[i]) % 10u));
    } else {
        uint32_t n = dec_len32(v);
        uint32_t e = k.p + n;
        do { stext()[--e] = (char)('0' + v % 10u); v /= 10u; } while (v);
        k.p += n;
    }
}
template <class Sink> __device__ __forceinline__ void put_dec(Sink &k, unsigned long long v)
{
    if constexpr (Sink::counting) {
        k.n += dec_len64(v);
    } else if constexpr (Sink::clipping) {
        unsigned long long pw = 1;
        for (uint32_t i = 1; i < dec_len64(v); i++) pw *= 10;
        for (; pw; pw /= 10) k.put((char)('0' + (v / pw) % 10));
    } else {
        // digits written backwards into place: no local buffer
        uint32_t n = dec_len64(v);
        uint32_t e = k.p + n;
        if (!(v >> 32)) {
            uint32_t x = (uint32_t)v;
            do { stext()[--e] = (char)('0' + x % 10u); x /= 10u; } while (x);
        } else {
            do { stext()[--e] = (char)('0' + v % 10); v /= 10; } while (v);
        }
        k.p += n;
    }
}
template <class Sink> __device__ __forceinline__ void put_hex_digits(Sink &k, unsigned long long v, int digits)
{
    if constexpr (Sink::counting) {
        k.n += digits;
    } else {
        for (int i = digits - 1; i >= 0; i--) {
            unsigned d = (unsigned)((v >> (4 * i)) & 15);
            k.put((char)(d < 10 ? '0' + d : 'a' + d - 10));
        }
    }
}
template <class Sink> __device__ __forceinline__ void put_hex8(Sink &k, uint32_t v)
{
    k.put('0'); k.put('x'); put_hex_digits(k, v, 8);
}
template <class Sink> __device__ __forceinline__ void put_name(Sink &k, uint16_t off, uint8_t len)
{
    k.puts(g_spv_tables.names + off, len);
}

// C99 "%a" spelling of a double as glibc prints it: [-]0x1.<hex>p<+|-><dec>
// for normal numbers (trailing zero digits dropped, no point when none are
// left), [-]0x0.<hex>p-1022 for subnormals, [-]0x0p+0 for zero, [-]inf and
// [-]nan.
template <class Sink> __device__ __noinline__ Sink put_hexfloat64(Sink k, unsigned long long b)
{
    bool neg = b >> 63;
    unsigned e = (unsigned)((b >> 52) & 0x7ff);
    unsigned long long m = b & ((1ull << 52) - 1);
    if (e == 0x7ff) { if (neg) k.put('-'); if (m) put_lit(k, "nan"); else put_lit(k, "inf"); return k; }
    if (neg) k.put('-');
    if (e == 0 && m == 0) { put_lit(k, "0x0p+0"); return k; }
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
    return k;
}

// a 32-bit float widened exactly to double bits
__device__ unsigned long long f32_to_f64_bits(uint32_t f)
{
    unsigned long long s = (unsigned long long)(f >> 31) << 63;
    uint32_t e = (f >> 23) & 0xff, m = f & 0x7fffff;
    if (e == 0xff) return s | (0x7ffull << 52) | ((unsigned long long)m << 29);
    if (e == 0) {
        if (m == 0) return s;
        // value m * 2^-149 with the leading one of m at bit 31 - clz(m):
        // shifting by lz = clz(m) - 8 (1..23) moves it to bit 23, where the
        // mask drops it, and the value is 1.f * 2^(-126 - lz)
        int lz = __clz(m) - 8;
        m = (m << lz) & 0x7fffff;
        unsigned long long ex = (unsigned long long)(1023 - 126 - lz);
        return s | (ex << 52) | ((unsigned long long)m << 29);
    }
    return s | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)m << 29);
}

// ---------------------------------------------------------------------------
// per-row formatting
// ---------------------------------------------------------------------------
struct RowCtx {
    const uint32_t *iw;          // the instruction's words (shared or global memory)
    uint32_t wc, op;
    uint32_t bound, slots;       // the module's bound and id-table form (values:
    bool named;                  // byte stores through a sink cannot alias them)
    uint32_t *tab;               // the module's id table
    const uint32_t *words;       // the batch's words and table columns (values,
    const uint64_t *off;         // not a pointer to the kernel's parameters,
    const uint16_t *opcol;       // which would copy them to local memory)
    bool inline_names;
    int64_t first;               // module's first row
    bool walk_ok;
};

// "<name>_" of a named id (nothing when the id has no name); kept out of
// line: most ids have no name, and an inlined copy at every id operand of
// both formatter passes bloats the kernel's code
template <class Sink> __device__ __noinline__ Sink put_id_name(Sink k, RowCtx c, uint32_t id)
{
    const uint32_t *e = idtab_entry(c.tab, c.bound, c.slots, id, false);
    uint32_t nr = e ? e[0] : NOROW;
    if (nr == NOROW) return k;
    if constexpr (Sink::counting) {
        k.n += e[1] + 1;
    } else {
        int64_t row = c.first + nr;
        const uint32_t *nw = c.words + c.off[row];
        uint32_t left = e[1];
        for (uint32_t i = 2; left; i++) {
            uint32_t v = __ldg(nw + i);
            for (int b = 0; b < 4 && left; b++, left--) {
                unsigned ch = (v >> (8 * b)) & 0xffu;
                bool keep = (ch >= '0' && ch <= '9') || (ch >= 'A' && ch <= 'Z') || (ch >= 'a' && ch <= 'z') || ch == '_';
                k.put(keep ? (char)ch : '_');
            }
        }
        k.put('_');
    }
    return k;
}

template <class Sink> __device__ __forceinline__ void put_id(Sink &k, const RowCtx &c, uint32_t id)
{
    k.put('%');
    // dense tables keep a bitmap after the table whose bit is cleared for a
    // named id: most ids have no name and cost one cached bit test
    if (c.named && id < c.bound &&
        (c.slots || !((c.tab[3ull * c.bound + (id >> 5)] >> (id & 31)) & 1u)))
        k = put_id_name(k, c, id);
    put_dec(k, id);
}

template <class Sink> __device__ __noinline__ Sink put_string(Sink k, const uint32_t *iw, uint32_t pos, uint32_t n)
{
    k.put('"');
    for (uint32_t i = 0; i < n; i++) {
        uint32_t v = iw[pos + i];
        for (int b = 0; b < 4; b++) {
            unsigned ch = (v >> (8 * b)) & 0xffu;
            if (!ch) { k.put('"'); return k; }
            if (ch == '"' || ch == '\\') { k.put('\\'); k.put((char)ch); }
            else if (ch < 0x20 || ch > 0x7e) { k.put('\\'); k.put('x'); put_hex_digits(k, ch, 2); }
            else k.put((char)ch);
        }
    }
    k.put('"');
    return k;
}

template <class Sink> __device__ __forceinline__ void put_venum(Sink &k, int kind, uint32_t v)
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

template <class Sink> __device__ __noinline__ Sink put_raw_tail(Sink k, const uint32_t *iw, uint32_t wc)
{
    if constexpr (Sink::counting) {
        k.n += 11 * (wc - 1);
    } else {
        for (uint32_t i = 1; i < wc; i++) { k.put(' '); put_hex8(k, iw[i]); }
    }
    return k;
}

// one operand of a parameter list (no optional / repeat forms except A_LITS)
template <class Sink> __device__ void put_param(Sink &k, const RowCtx &c, uint8_t pc, uint32_t &pos)
{
    auto word = [&](uint32_t i) -> uint32_t { return c.iw[i]; };
    if (pc == spvt::A_LITS) { for (; pos < c.wc; pos++) { k.put(' '); put_dec(k, word(pos)); } return; }
    k.put(' ');
    if (pc == spvt::A_ID) { put_id(k, c, word(pos)); pos++; }
    else if (pc == spvt::A_LIT) { put_dec(k, word(pos)); pos++; }
    else if (pc == spvt::A_STR) { uint32_t n = string_words(word, pos, c.wc); k = put_string(k, c.iw, pos, n); pos += n; }
    else { put_venum(k, pc - spvt::A_ENUM, word(pos)); pos++; }
}

template <class Sink> __device__ __noinline__ Sink put_ctx_literal(Sink k, RowCtx c, uint32_t rt, uint32_t pos)
{
    auto word = [&](uint32_t i) -> uint32_t { return c.iw[i]; };
    uint32_t n = c.wc - pos;
    bool is_float = false;
    if (rt < c.bound) {
        const uint32_t *e = idtab_entry(c.tab, c.bound, c.slots, rt, false);
        uint32_t dr = e ? e[2] : NOROW;
        if (dr != NOROW && c.opcol[c.first + dr] == 22) is_float = true;
    }
    k.put(' ');
    if (is_float && n == 1) k = put_hexfloat64(k, f32_to_f64_bits(word(pos)));
    else if (is_float && n == 2) k = put_hexfloat64(k, (unsigned long long)word(pos) | ((unsigned long long)word(pos + 1) << 32));
    else if (n == 1) put_dec(k, word(pos));
    else if (n == 2) put_dec(k, (unsigned long long)word(pos) | ((unsigned long long)word(pos + 1) << 32));
    else for (uint32_t i = 0; i < n; i++) { if (i) k.put(' '); put_dec(k, word(pos + i)); }
    return k;
}

template <class Sink> __device__ void format_row(Sink &k, const RowCtx &c)
{
    const spvt::Tables &T = g_spv_tables;
    auto word = [&](uint32_t i) -> uint32_t { return c.iw[i]; };
    if (c.op >= 256 || !(T.ops[c.op].flags & 1)) {
        k.put('O'); k.put('p'); put_dec(k, c.op);
        k = put_raw_tail(k, c.iw, c.wc); k.put('\n');
        return;
    }
    const spvt::OpDesc &d = T.ops[c.op];
    if (!c.walk_ok) {
        put_name(k, d.name_off, d.name_len);
        k = put_raw_tail(k, c.iw, c.wc); k.put('\n');
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
            k.put(' '); k = put_string(k, c.iw, pos, n); pos += n;
        } else if (code == spvt::A_CTX) {
            k = put_ctx_literal(k, c, rt, pos);
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

template <class Sink> __device__ void format_header(Sink &k, const uint32_t *w)
{
    put_lit(k, "; SPIR-V\n; Version: ");
    put_dec(k, (w[1] >> 16) & 0xff); k.put('.'); put_dec(k, (w[1] >> 8) & 0xff);
    put_lit(k, "\n; Generator: "); put_hex8(k, w[2]);
    put_lit(k, "\n; Bound: "); put_dec(k, w[3]);
    put_lit(k, "\n; Schema: "); put_dec(k, w[4]); k.put('\n');
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// chunked block-wide exclusive scan over modules (1024 threads): calls
// f(m, excl, v) for every module with the exclusive prefix of val(m)
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

// per module (many CTAs): header status, id-table form and size (parked in
// arena_off until the scan), header bytes, first item
__global__ void k_dis_premod(DP P)
{
    long long n_rows = P.first_row[P.n_mod];
    if (n_rows > P.cap_rows) n_rows = P.cap_rows;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long mm = blockIdx.x * (long long)blockDim.x + threadIdx.x; mm < P.n_mod; mm += stride) {
        const int m = (int)mm;
        long long o = P.mod_off[m], len = P.mod_off[m + 1] - o;
        uint32_t st = (len < 0 || len > 0x7fffffffLL) ? S_CAPACITY : header_status(P.words + o, len);
        DisMod d;
        d.bound = st == S_OK ? P.words[o + 3] : 0;
        d.slots = (st == S_OK && !idtab_dense(d.bound, len)) ? (uint32_t)(len + 64) : 0;
        d.arena_off = st == S_OK ? (long long)idtab_words(d.bound, len) : 0;
        d.ok = st == S_OK;
        d.status = st;
        d.header_len = (st == S_OK && P.header) ? header_len(P.words + o) : 0;
        d.named = 0;
        d.bloom = 0;
        long long fr = P.first_row[m];
        d.item_base = (fr < n_rows ? fr : n_rows) + m;
        P.dm[m] = d;
    }
}

// one CTA: id-table offsets (exclusive prefix of the sizes); a module whose
// table does not fit the arena gets no table and SPV_CAPACITY
__global__ void __launch_bounds__(1024) k_dis_prescan(DP P)
{
    long long n_rows = P.first_row[P.n_mod];
    if (n_rows > P.cap_rows) n_rows = P.cap_rows;
    unsigned long long used = block_scan_modules(P.n_mod,
        [&](int m) -> unsigned long long { return (unsigned long long)P.dm[m].arena_off; },
        [&](int m, unsigned long long excl, unsigned long long na) {
            DisMod &d = P.dm[m];
            d.arena_off = (long long)excl;
            if (d.ok && (long long)(excl + na) > P.arena_words) {
                d.ok = 0;
                d.status = S_CAPACITY;
                d.header_len = 0;
            }
        });
    if (threadIdx.x == 0) {
        P.ctrl->arena_used = used < (unsigned long long)P.arena_words ? used : (unsigned long long)P.arena_words;
        P.ctrl->n_rows = (unsigned long long)n_rows;
        P.ctrl->n_items = (unsigned long long)n_rows + P.n_mod;
        P.ctrl->next_tile = 0;
        P.ctrl->timeout = 0;
    }
}

// id tables to NOROW (dense bitmaps to all ones: nothing named), look-back
// states to zero, and the tile -> first module map: every module owns the
// tiles whose first item falls in its item range
__global__ void k_dis_clear(DP P)
{
    unsigned long long n = P.ctrl->arena_used;
    const long long n_items = (long long)P.ctrl->n_items;
    unsigned long long nt = n_items / ITEMS + 1;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long i = g; i < (long long)n; i += stride) P.arena[i] = NOROW;
    for (long long i = g; i < (long long)nt; i += stride) P.tstate[i] = 0;
    for (long long m = g; m < P.n_mod; m += stride) {
        long long b = P.dm[m].item_base, e = m + 1 < P.n_mod ? P.dm[m + 1].item_base : n_items;
        for (long long t = (b + ITEMS - 1) / ITEMS; t * ITEMS < e; t++) P.tile_m0[t] = (int)m;
    }
}

// first OpName per id and first definition per id (module-local rows)
__global__ void k_dis_ids(DP P)
{
    // four rows per thread and step, all their loads issued before any
    // update, so that a thread's rows do not wait on one another
    constexpr int U = 4;
    const spvt::Tables &T = g_spv_tables;
    const long long n = (long long)P.ctrl->n_rows;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; r0 < n; r0 += U * stride) {
        uint32_t mq[U], opq[U], wcq[U], ridq[U];
        #pragma unroll
        for (int q = 0; q < U; q++) {
            const long long row = r0 + q * stride;
            mq[q] = ~0u; opq[q] = 0; wcq[q] = 0; ridq[q] = 0;
            if (row < n) { mq[q] = P.mod[row]; opq[q] = P.op[row]; wcq[q] = P.wc[row]; ridq[q] = P.rid[row]; }
        }
        uint32_t okq[U], boundq[U], slotsq[U], namedq[U];
        long long aoq[U], frq[U];
        #pragma unroll
        for (int q = 0; q < U; q++) {
            okq[q] = 0; boundq[q] = 0; slotsq[q] = 0; namedq[q] = 0; aoq[q] = 0; frq[q] = 0;
            if (mq[q] != ~0u) {
                const DisMod &md = P.dm[mq[q]];
                okq[q] = md.ok; boundq[q] = md.bound; slotsq[q] = md.slots; namedq[q] = md.named;
                aoq[q] = md.arena_off; frq[q] = P.first_row[mq[q]];
            }
        }
        #pragma unroll
        for (int q = 0; q < U; q++) {
            if (!okq[q]) continue;
            const long long row = r0 + q * stride;
            const uint32_t m = mq[q], op = opq[q], wc = wcq[q], bound = boundq[q], slots = slotsq[q];
            const uint32_t local = (uint32_t)(row - frq[q]);
            uint32_t *tab = P.arena + aoq[q];
            if (op == 5 && wc >= 2 && P.inline_names) {
                uint32_t target = __ldg(P.words + P.off[row] + 1);
                if (target < bound) {
                    if (!namedq[q]) P.dm[m].named = 1;
                    atomicOr(&P.dm[m].bloom, 1ull << name_hash(target));
                    atomicMin(&idtab_entry(tab, bound, slots, target, true)[0], local);
                    if (!slots) atomicAnd(&tab[3ull * bound + (target >> 5)], ~(1u << (target & 31)));
                }
            }
            if (op < 256 && (T.ops[op].flags & 4)) {
                uint32_t qq = 1 + ((T.ops[op].flags >> 1) & 1);
                if (qq < wc && ridq[q] < bound) atomicMin(&idtab_entry(tab, bound, slots, ridq[q], true)[2], local);
            }
        }
    }
}

// name length of each id's first OpName: its string's bytes before the first
// NUL, or to the instruction's end
__global__ void k_dis_namelen(DP P)
{
    if (!P.inline_names) return;
    // the op column is scanned eight rows per thread and step (loads issued
    // together); the few OpName rows do the work
    constexpr int U = 8;
    long long n = (long long)P.ctrl->n_rows;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; r0 < n; r0 += U * stride) {
        uint32_t hit = 0;
        #pragma unroll
        for (int q = 0; q < U; q++) {
            const long long row = r0 + q * stride;
            if (row < n && P.op[row] == 5) hit |= 1u << q;
        }
        while (hit) {
            const int q = __ffs(hit) - 1;
            hit &= hit - 1;
            const long long row = r0 + q * stride;
            uint32_t wc = P.wc[row];
            if (wc < 2) continue;
            uint32_t m = P.mod[row];
            const DisMod &md = P.dm[m];
            if (!md.ok) continue;
            const uint32_t *iw = P.words + P.off[row];
            uint32_t target = __ldg(iw + 1);
            if (target >= md.bound) continue;
            uint32_t *e = idtab_entry(P.arena + md.arena_off, md.bound, md.slots, target, false);
            if (!e || e[0] != (uint32_t)(row - P.first_row[m])) continue;
            uint32_t len = 0;
            for (uint32_t i = 2; i < wc; i++) {
                uint32_t v = __ldg(iw + i);
                uint32_t z = (v - 0x01010101u) & ~v & 0x80808080u;
                if (z) { len += (uint32_t)((__ffs(z) - 1) >> 3); break; }
                len += 4;
            }
            e[1] = len;
        }
    }
}

constexpr int NSHAPE = 64;

struct MainSmem {
    char text[TEXT_SMEM + 16];
    int ibase[ITEMS + 2];           // item_base - i0 of modules m0 .. m0 + nm, then of the next module (or
                                    // n_items), clamped to [-1, ITEMS + 1]
    int im[ITEMS];                  // per item: its module, -1 past the end
    uint32_t ilen[ITEMS];           // per item: text bytes
    uint32_t ioff[ITEMS];           // per item: offset in the tile's text
    uint16_t perm[ITEMS];           // items grouped by text shape
    uint16_t rank[ITEMS];           // per item: position within its shape group
    uint32_t irel[ITEMS];           // per item: its words at wst[irel], NOSTAGE when not staged
    uint16_t iop[ITEMS], iwc[ITEMS];// per item: opcode and word count
    uint8_t icls[ITEMS];            // per item: shape class
    uint8_t iok[ITEMS];             // per item: operands parse (else raw words)
    uint8_t ihdr[ITEMS];            // per item: a module's header item
    alignas(16) uint32_t wst[STAGE_WORDS];  // words [wa, wa + STAGE_WORDS) of the batch (wa: wlo aligned down)
    unsigned long long wlo, whi;
    // per CTA, once: the opcode and enumerant names, each opcode's text form
    // for the fast line writer, powers of ten, bit-enum tables
    char names[spvt::NAME_POOL];
    uint2 otx[256];
    uint32_t pow10[10];
    uint8_t bnp[spvt::NUM_BKINDS][16];   // literal parameters of the known bits of a mask's low 4 bits
    uint8_t btl[spvt::NUM_BKINDS][16];   // text bytes of a mask of known bits ("None" for 0)
    uint8_t bknown[spvt::NUM_BKINDS];    // the kind's known bits
    uint32_t cls_n[NSHAPE];
    // the first MCACHE modules of the tile: what formatting reads of them
    struct MC { uint32_t ok, bound, slots, named; unsigned long long bloom; long long arena_off, first; } mc[32];
    uint32_t warp_tot[DNT / 32];
    long long tile;
    unsigned long long base;
    int m0, nm;
    int gave_up;
    unsigned int fnext;             // next chunk of items to format
    unsigned int mnext;             // next chunk of items to measure
};

// ---------------------------------------------------------------------------
// the fast line form: an opcode in the fast operand form (fixed ids and
// literals, then a tail of ids, literals, id pairs or one bit-enum word with
// its literal parameters; no context-dependent literal), its word count
// valid for the form, and no named id among its operands. Its length is
// counted arithmetically and its text written backwards from the line's end,
// digits straight from the values; every other line takes format_row. Both
// give the same bytes (section 3.4.4's text form as format_row defines it).
// ---------------------------------------------------------------------------
constexpr uint32_t NOTFAST = 0xFFFFFFFFu;

// otx[op]: x = name offset | name length << 16 | form << 24 (bit 0 fast text,
// bits 1-3 tail, bit 4 the bit-enum word may be absent); y = id mask | fixed
// words << 16 | result type / id flags (bits 1, 2) << 24 | bit-enum kind << 28
__device__ void init_text_tables(MainSmem &s)
{
    const spvt::Tables &T = g_spv_tables;
    for (int i = threadIdx.x; i < spvt::NAME_POOL; i += blockDim.x) s.names[i] = T.names[i];
    for (int o = threadIdx.x; o < 256; o += blockDim.x) {
        const spvt::OpDesc &d = T.ops[o];
        bool ctx = false;
        for (int q = 0; q < d.nprog; q++) if ((d.prog[q] & 0x7f) == spvt::A_CTX) ctx = true;
        const uint32_t form = ((d.flags & 1) && (d.fast & 1) && !ctx) ? (uint32_t)d.fast : 0u;
        s.otx[o] = make_uint2((uint32_t)d.name_off | ((uint32_t)d.name_len << 16) | (form << 24),
                              (uint32_t)d.id_mask | ((uint32_t)d.nfixed << 16) | ((uint32_t)(d.flags & 6) << 24) |
                                  ((uint32_t)d.bkind << 28));
    }
    if (threadIdx.x < 10) {
        uint32_t v = 1;
        for (uint32_t i = 0; i < threadIdx.x; i++) v *= 10u;
        s.pow10[threadIdx.x] = v;
    }
    if (threadIdx.x < spvt::NUM_BKINDS * 16) {
        const int kind = threadIdx.x >> 4, m = threadIdx.x & 15;
        uint32_t known = 0, np = 0, tl = 0, nb = 0;
        for (int b = 0; b < 32; b++) if (T.benum[kind][b].known) known |= 1u << b;
        for (int b = 0; b < 4; b++)
            if (((m >> b) & 1) && T.benum[kind][b].known) { np += T.benum[kind][b].nparam; tl += T.benum[kind][b].name_len; nb++; }
        s.bnp[kind][m] = (uint8_t)np;
        s.btl[kind][m] = (uint8_t)(m == 0 ? 4 : tl + nb - 1);
        if (m == 0) s.bknown[kind] = (uint8_t)known;
    }
}

// decimal digits of v: t = floor(bits(v) * 1233 / 4096) is the digit count
// or one more than it
__device__ __forceinline__ uint32_t dlen_s(const MainSmem &s, uint32_t v)
{
    const uint32_t u = v | 1u;                         // 0 prints like 1: one digit
    const uint32_t t = ((32u - __clz(u)) * 1233u) >> 12;
    return t + 1u - (u < s.pow10[t] ? 1u : 0u);
}

// an id that prints with its name (inline names on, a name recorded for it)
__device__ __forceinline__ bool named_id(const RowCtx &c, uint32_t id, unsigned long long bloom)
{
    return ((bloom >> name_hash(id)) & 1ull) && c.named && id < c.bound &&
           (c.slots || !((c.tab[3ull * c.bound + (id >> 5)] >> (id & 31)) & 1u));
}

// the line's length in the fast form, or NOTFAST
__device__ uint32_t fast_len(const MainSmem &s, const RowCtx &c, unsigned long long bloom)
{
    const uint2 ot = s.otx[c.op < 256 ? c.op : 0];
    const uint32_t form = ot.x >> 24;
    if (c.op >= 256 || !(form & 1u)) return NOTFAST;
    const uint32_t need = 1u + ((ot.y >> 16) & 0xffu), tail = (form >> 1) & 7u, wc = c.wc;
    bool ok;
    uint32_t mask = 0;
    const uint32_t bk = ot.y >> 28;
    if (tail == 4) {
        if (wc == need) ok = (form & 16u) != 0;
        else if (wc > need) { mask = c.iw[need]; ok = wc == need + 1u + s.bnp[bk][mask & 15u]; }
        else ok = false;
    } else {
        ok = tail == 0 ? wc == need : (wc >= need && (tail != 3 || ((wc - need) & 1u) == 0));
    }
    if (!ok) return NOTFAST;
    const uint32_t idm = ot.y & 0xffffu;
    uint32_t len = ((ot.x >> 16) & 0xffu) + 1u + (((ot.y >> 24) & 4u) ? 2u : 0u);   // name, '\n', " = " past " "
    for (uint32_t i = 1; i < need; i++) {
        const uint32_t v = c.iw[i];
        const uint32_t isid = (idm >> i) & 1u;
        if (isid && named_id(c, v, bloom)) return NOTFAST;
        len += 1u + isid + dlen_s(s, v);
    }
    if (tail == 1 || tail == 3) {
        for (uint32_t i = need; i < wc; i++) {
            const uint32_t v = c.iw[i];
            if (named_id(c, v, bloom)) return NOTFAST;
            len += 2u + dlen_s(s, v);
        }
    } else if (tail == 2) {
        for (uint32_t i = need; i < wc; i++) len += 1u + dlen_s(s, c.iw[i]);
    } else if (tail == 4 && wc > need) {
        len += 1u + ((mask & ~(uint32_t)s.bknown[bk]) ? dlen_s(s, mask) : (uint32_t)s.btl[bk][mask & 15u]);
        for (uint32_t i = need + 1; i < wc; i++) len += 1u + dlen_s(s, c.iw[i]);
    }
    return len;
}

__device__ __forceinline__ uint32_t put_dec_back(uint32_t e, uint32_t v)
{
    do { const uint32_t q = v / 10u; stext()[--e] = (char)('0' + (v - 10u * q)); v = q; } while (v);
    return e;
}
__device__ __forceinline__ uint32_t put_name_back(const MainSmem &s, uint32_t e, uint32_t off, uint32_t len)
{
    for (uint32_t i = len; i > 0; i--) stext()[--e] = s.names[off + i - 1];
    return e;
}

// the line of a fast-form row, written backwards so that it ends at byte end
// of the shared text buffer
__device__ void fast_write(const MainSmem &s, const RowCtx &c, uint32_t end)
{
    const uint2 ot = s.otx[c.op];
    const uint32_t form = ot.x >> 24;
    const uint32_t need = 1u + ((ot.y >> 16) & 0xffu), tail = (form >> 1) & 7u, wc = c.wc;
    const uint32_t idm = ot.y & 0xffffu, fl = (ot.y >> 24) & 6u, bk = ot.y >> 28;
    uint32_t e = end;
    stext()[--e] = '\n';
    if (tail == 1 || tail == 3) {
        for (uint32_t i = wc; i > need; i--) { e = put_dec_back(e, c.iw[i - 1]); stext()[--e] = '%'; stext()[--e] = ' '; }
    } else if (tail == 2) {
        for (uint32_t i = wc; i > need; i--) { e = put_dec_back(e, c.iw[i - 1]); stext()[--e] = ' '; }
    } else if (tail == 4 && wc > need) {
        for (uint32_t i = wc; i > need + 1; i--) { e = put_dec_back(e, c.iw[i - 1]); stext()[--e] = ' '; }
        const uint32_t mask = c.iw[need];
        if (mask == 0) {
            stext()[--e] = 'e'; stext()[--e] = 'n'; stext()[--e] = 'o'; stext()[--e] = 'N';
        } else if (mask & ~(uint32_t)s.bknown[bk]) {
            e = put_dec_back(e, mask);
        } else {
            for (int b = 31 - __clz(mask); b >= 0; b--) {
                if (!((mask >> b) & 1u)) continue;
                const spvt::EnDesc &en = g_spv_tables.benum[bk][b];
                e = put_name_back(s, e, ((uint32_t)en.name_hi << 8) | en.name_lo, en.name_len);
                if (mask & ((1u << b) - 1u)) stext()[--e] = '|';
            }
        }
        stext()[--e] = ' ';
    }
    // fixed words after the result type and id, last first; then the result type
    const uint32_t first = 1u + (fl & 2u ? 1u : 0u) + (fl & 4u ? 1u : 0u);
    for (uint32_t i = need - 1; i >= first; i--) {
        e = put_dec_back(e, c.iw[i]);
        if ((idm >> i) & 1u) stext()[--e] = '%';
        stext()[--e] = ' ';
    }
    if (fl & 2u) { e = put_dec_back(e, c.iw[1]); stext()[--e] = '%'; stext()[--e] = ' '; }
    e = put_name_back(s, e, ot.x & 0xffffu, (ot.x >> 16) & 0xffu);
    if (fl & 4u) {
        stext()[--e] = ' '; stext()[--e] = '='; stext()[--e] = ' ';
        e = put_dec_back(e, c.iw[(fl & 2u) ? 2 : 1]);
        stext()[--e] = '%';
    }
}

__device__ __forceinline__ bool make_ctx(const DP &P, const MainSmem &s, int j, int m, long long row, RowCtx &c,
                                         int walk_ok)
{
    const int mi = m - s.m0;
    if (mi < 32) {                       // the tile's first modules: from shared memory
        const MainSmem::MC &mc = s.mc[mi];
        if (!mc.ok) return false;
        c.bound = mc.bound;
        c.slots = mc.slots;
        c.named = P.inline_names && mc.named;
        c.tab = P.arena + mc.arena_off;
        c.first = mc.first;
    } else {
        const DisMod &md = P.dm[m];
        if (!md.ok) return false;
        c.bound = md.bound;
        c.slots = md.slots;
        c.named = P.inline_names && md.named;
        c.tab = P.arena + md.arena_off;
        c.first = P.first_row[m];
    }
    c.iw = s.irel[j] != NOSTAGE ? s.wst + s.irel[j] : P.words + P.off[row];
    c.wc = s.iwc[j];
    c.op = s.iop[j];
    c.words = P.words;
    c.off = P.off;
    c.opcol = P.op;
    c.inline_names = P.inline_names != 0;
    if (walk_ok >= 0) c.walk_ok = walk_ok != 0;
    else {
        c.walk_ok = true;
        if (c.op < 256 && (g_spv_tables.ops[c.op].flags & 1)) {
            auto word = [&](uint32_t i) -> uint32_t { return c.iw[i]; };
            c.walk_ok = walk_instruction(word, c.wc, g_spv_tables.ops[c.op], 0xffffffffu).ok;
        }
    }
    return true;
}

// Warp 0: tile t's text offset, the sum of all earlier tiles' byte counts
// (decoupled look-back over the published aggregates / inclusive prefixes).
// Publishes tile t's inclusive prefix; a wait that runs out sets the timeout
// flag and leaves s.gave_up set.
__device__ void dis_lookback(const DP &P, MainSmem &s, long long t, uint32_t total, int lane, bool last_tile)
{
    unsigned long long excl = 0;
    if (t > 0) {
        bool gave_up;
        // 128 states a poll: with one tile in flight per SM the nearest
        // inclusive state is often a few hundred tiles back
        excl = warp_lookback_sum<4>(P.tstate, t - 1, F_INC, F_MSK, P.max_spins, lane, gave_up);
        if (gave_up && lane == 0) { atomicExch(&P.ctrl->timeout, 1u); s.gave_up = 1; }
        if (lane == 0 && t != P.stall_tile) st_relaxed(&P.tstate[t], F_INC | (excl + total));
    }
    if (lane == 0) {
        s.base = excl;
        if (last_tile) P.text_off[P.n_mod] = excl + total;
    }
}

// One tile of items: locate, group by text shape (so the lines a warp
// formats share their control flow), measure, scan, publish the tile's byte
// count, format into shared memory, look back for the tile's offset, copy
// out. Formatting before the look-back gives the earlier tiles time to
// publish, so the look-back seldom waits.
__global__ void __launch_bounds__(DNT, SPV_DIS_MIN_BLOCKS) k_dis_main(DP P)
{
    MainSmem &s = *reinterpret_cast<MainSmem *>(smem_raw);
    static_assert(offsetof(MainSmem, text) == 0, "the sinks write at offsets from the start of shared memory");
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n_items = (long long)P.ctrl->n_items;
    const long long ntiles = (n_items + ITEMS - 1) / ITEMS;
    init_text_tables(s);
    // warp 0: take the next tile's ticket; its modules and their first items
    auto setup_tile = [&]() {
            unsigned int ticket = 0;
            if (lane == 0) ticket = atomicAdd(&P.ctrl->next_tile, 1u);
            const long long tt = (long long)__shfl_sync(0xffffffffu, ticket, 0);
            if (lane == 0) {
                s.tile = tt;
                s.fnext = 0;
                s.mnext = 0;
                s.wlo = ~0ull;
                s.whi = 0;
            }
            if (tt < ntiles) {
                const int m0 = P.tile_m0[tt];
                const int nm = (tt + 1 < ntiles ? P.tile_m0[tt + 1] : P.n_mod - 1) - m0 + 1;   // <= ITEMS + 1
                if (lane == 0) { s.m0 = m0; s.nm = nm; }
                const long long i0 = tt * ITEMS;
                for (int j = lane; j <= nm; j += 32) {
                    long long b = j < nm ? P.dm[m0 + j].item_base
                                         : (m0 + nm < P.n_mod ? P.dm[m0 + nm].item_base : n_items);
                    b -= i0;
                    s.ibase[j] = (int)(b < -1 ? -1 : (b > ITEMS + 1 ? ITEMS + 1 : b));
                }
                if (lane < nm) {
                    const DisMod &md = P.dm[m0 + lane];
                    MainSmem::MC &mc = s.mc[lane];
                    mc.ok = md.ok; mc.bound = md.bound; mc.slots = md.slots; mc.named = md.named;
                    mc.bloom = md.bloom; mc.arena_off = md.arena_off; mc.first = P.first_row[m0 + lane];
                }
            }
            };
    bool prefetched = false;          // warp 0 set up the next tile already
    // a ticket is taken when its tile starts: a tile waits only on lower
    // tiles, whose holders are running, so the look-backs always end; a
    // ticket taken a tile ahead would hold back every later tile's look-back
    for (;;) {
        // warp 0: the tile, its modules and their first items (done already
        // when it was set up during the last tile's copy-out)
        if (wid == 0 && !prefetched) setup_tile();
        prefetched = false;
        if (tid < NSHAPE) s.cls_n[tid] = 0;
        // the look-back's timeout flag is cleared here, where every thread has
        // read the last tile's (warp 0 sets up the next tile while the others
        // may still be reading it)
        if (tid == 0) s.gave_up = 0;
        __syncthreads();
        const long long t = s.tile;
        if (t >= ntiles) break;
        const long long i0 = t * ITEMS;
        const int m0 = s.m0, nm = s.nm;

        // 1. locate every item (op, word count and word offset read once,
        //    coalesced: all of a thread's loads are issued before any is
        //    used), count the shape classes, find the tile's word range
        {
            unsigned long long lo_w = ~0ull, hi_w = 0;
            int mq[IPT];
            bool hq[IPT];
            long long rq[IPT];
            #pragma unroll
            for (int q = 0; q < IPT; q++) {
                const int j = tid + q * DNT;
                const long long i = i0 + j;
                int m = -1;
                bool hdr = false;
                if (i < n_items) {
                    int lo = 0, hi = nm;                 // last k with ibase[k] <= j
                    while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (s.ibase[mid] <= j) lo = mid; else hi = mid; }
                    m = m0 + lo;
                    hdr = j == s.ibase[lo];
                }
                mq[q] = m;
                hq[q] = hdr;
                rq[q] = m >= 0 && !hdr ? i - m - 1 : -1;  // module m's rows follow its header item
            }
            uint32_t opq[IPT], wcq[IPT];
            unsigned long long oq[IPT];
            #pragma unroll
            for (int q = 0; q < IPT; q++) {
                opq[q] = 0; wcq[q] = 0; oq[q] = 0;
                if (rq[q] >= 0) { opq[q] = P.op[rq[q]]; wcq[q] = P.wc[rq[q]]; oq[q] = P.off[rq[q]]; }
            }
            #pragma unroll
            for (int q = 0; q < IPT; q++) {
                const int j = tid + q * DNT;
                int cls = 0;
                if (rq[q] >= 0) {
                    lo_w = oq[q] < lo_w ? oq[q] : lo_w;
                    hi_w = oq[q] + wcq[q] > hi_w ? oq[q] + wcq[q] : hi_w;
                    cls = opq[q] < 256 ? g_spv_tables.shape[opq[q]] : 1;
                }
                s.im[j] = mq[q];
                s.ihdr[j] = hq[q];
                s.irel[j] = (uint32_t)oq[q];             // low word offset bits, made relative below
                s.iop[j] = (uint16_t)opq[q];
                s.iwc[j] = (uint16_t)wcq[q];
                s.icls[j] = (uint8_t)cls;
                // rank within the class: one shared atomic per distinct class of the warp
                const unsigned peers = __match_any_sync(0xffffffffu, cls);
                const int leader = __ffs(peers) - 1;
                uint32_t first = 0;
                if (lane == leader) first = atomicAdd(&s.cls_n[cls], (uint32_t)__popc(peers));
                first = __shfl_sync(0xffffffffu, first, leader);
                s.rank[j] = (uint16_t)(first + __popc(peers & ((1u << lane) - 1u)));
            }
            #pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                unsigned long long x = __shfl_xor_sync(0xffffffffu, lo_w, d), y = __shfl_xor_sync(0xffffffffu, hi_w, d);
                lo_w = x < lo_w ? x : lo_w;
                hi_w = y > hi_w ? y : hi_w;
            }
            if (lane == 0 && hi_w) { atomicMin(&s.wlo, lo_w); atomicMax(&s.whi, hi_w); }
        }
        __syncthreads();
        // stage the words [wa, min(whi, wa + STAGE_WORDS)) with asynchronous
        // copies (wa = wlo aligned down to 16 bytes when the words buffer is);
        // an item whose words all lie inside reads them from shared memory. A
        // tile's words span less than 2^32, so the low 32 bits of an offset
        // give its distance from wa.
        {
            const unsigned long long wlo = s.wlo, whi = s.whi;
            const bool al16 = (((uintptr_t)P.words) & 15) == 0;
            const unsigned long long wa = whi ? (al16 ? (wlo & ~3ull) : wlo) : 0;
            const uint32_t wn = whi > wa ? (uint32_t)(whi - wa < STAGE_WORDS ? whi - wa : STAGE_WORDS) : 0u;
            if (al16) {
                for (uint32_t k = 4 * tid; k < wn; k += 4 * DNT)
                    cp_async16(&s.wst[k], P.words + wa + k, wn - k >= 4 ? 16u : 4u * (wn - k));
            } else {
                for (uint32_t k = tid; k < wn; k += DNT) cp_async4(&s.wst[k], P.words + wa + k);
            }
            #pragma unroll
            for (int q = 0; q < IPT; q++) {
                const int j = tid + q * DNT;
                uint32_t rel = s.irel[j] - (uint32_t)wa;
                bool row = s.im[j] >= 0 && !s.ihdr[j];
                s.irel[j] = row && rel + s.iwc[j] <= wn ? rel : NOSTAGE;
            }
            cp_async_wait_all();
        }
        if (wid == 0) {                               // exclusive scan of the class counts
            uint32_t a = s.cls_n[lane], b = s.cls_n[lane + 32];
            uint32_t ia = a, ib = b;
            #pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t x = __shfl_up_sync(0xffffffffu, ia, d), y = __shfl_up_sync(0xffffffffu, ib, d);
                if (lane >= d) { ia += x; ib += y; }
            }
            uint32_t tot_a = __shfl_sync(0xffffffffu, ia, 31);
            s.cls_n[lane] = ia - a;
            s.cls_n[lane + 32] = tot_a + ib - b;
        }
        __syncthreads();
        for (int j = tid; j < ITEMS; j += DNT) s.perm[s.cls_n[s.icls[j]] + s.rank[j]] = (uint16_t)j;
        __syncthreads();

        // 2. measure, in shape order, 32 items at a time from a shared
        //    counter: the few shapes without the fast line form (a module's
        //    preamble) come first, and their long formatting overlaps the
        //    other warps' chunks
        for (;;) {
            unsigned cb = 0;
            if (lane == 0) cb = atomicAdd(&s.mnext, 32u);
            cb = __shfl_sync(0xffffffffu, cb, 0);
            if (cb >= (unsigned)ITEMS) break;
            const int q = (int)cb + lane;
            if (q >= ITEMS) continue;
            int j = s.perm[q];
            int m = s.im[j];
            uint32_t len = 0;
            uint8_t ok = 1;
            if (m >= 0) {
                if (s.ihdr[j]) len = P.dm[m].header_len;
                else {
                    RowCtx c;
                    if (make_ctx(P, s, j, m, i0 + j - m - 1, c, 1)) {
                        const int mi = m - s.m0;
                        const unsigned long long bloom = mi < 32 ? s.mc[mi].bloom : P.dm[m].bloom;
                        const uint32_t fl = fast_len(s, c, bloom);
                        if (fl != NOTFAST) { len = fl; ok = 2; }
                        else {
                            make_ctx(P, s, j, m, i0 + j - m - 1, c, -1);
                            CountSink k; format_row(k, c); len = k.n; ok = c.walk_ok;
                        }
                    }
                }
            }
            s.ilen[j] = len;
            s.iok[j] = ok;
        }
        __syncthreads();
        // 3. scan in item order (IPT consecutive items per thread)
        {
            uint32_t mine = 0;
            #pragma unroll
            for (int q = 0; q < IPT; q++) mine += s.ilen[IPT * tid + q];
            uint32_t incl = mine;
            #pragma unroll
            for (int d = 1; d < 32; d <<= 1) { uint32_t v = __shfl_up_sync(0xffffffffu, incl, d); if (lane >= d) incl += v; }
            if (lane == 31) s.warp_tot[wid] = incl;
            __syncthreads();
            uint32_t wpre = 0;
            #pragma unroll
            for (int w = 0; w < DNT / 32; w++) if (w < wid) wpre += s.warp_tot[w];
            uint32_t ex = wpre + incl - mine;
            #pragma unroll
            for (int q = 0; q < IPT; q++) { s.ioff[IPT * tid + q] = ex; ex += s.ilen[IPT * tid + q]; }
        }
        uint32_t total = 0;
        #pragma unroll
        for (int w = 0; w < DNT / 32; w++) total += s.warp_tot[w];
        // the tile's byte count, published before any wait of this tile
        if (tid == 0 && t != P.stall_tile) st_relaxed(&P.tstate[t], (t == 0 ? F_INC : F_AGG) | total);
        const bool last_tile = i0 + ITEMS >= n_items;
        const bool staged = total <= (uint32_t)TEXT_SMEM;
        auto format_item = [&](auto &k, int j) {
            if (s.ihdr[j]) format_header(k, P.words + P.mod_off[s.im[j]]);
            else { RowCtx c; make_ctx(P, s, j, s.im[j], i0 + j - s.im[j] - 1, c, s.iok[j]); format_row(k, c); }
        };
        if (!staged && wid == 0) dis_lookback(P, s, t, total, lane, last_tile);   // oversized tile: its offset first
        __syncthreads();                              // every item's offset (and an oversized tile's base)
        // 4. format once, in shape order, into shared memory; then the offset
        if (staged) {
            // warp 0 looks back for the tile's offset first, while the other
            // warps format: items go out 32 at a time (in shape order) from a
            // shared counter, and warp 0 joins when its look-back is done
            if (wid == 0) dis_lookback(P, s, t, total, lane, last_tile);
            if (P.text_cap > 0) {
                for (;;) {
                    unsigned cb = 0;
                    if (lane == 0) cb = atomicAdd(&s.fnext, 32u);
                    cb = __shfl_sync(0xffffffffu, cb, 0);
                    if (cb >= (unsigned)ITEMS) break;
                    const int q = (int)cb + lane;
                    if (q >= ITEMS) continue;
                    const int j = s.perm[q];
                    if (s.im[j] < 0 || s.ilen[j] == 0) continue;
                    if (s.iok[j] == 2) {
                        RowCtx c;
                        make_ctx(P, s, j, s.im[j], i0 + j - s.im[j] - 1, c, 1);
                        fast_write(s, c, s.ioff[j] + s.ilen[j]);
                    } else {
                        WriteSink k{s.ioff[j]};
                        format_item(k, j);
                    }
                }
            }
            __syncthreads();
        }
        const unsigned long long base = s.base;
        for (int j = tid; j < ITEMS; j += DNT)
            if (s.im[j] >= 0 && s.ihdr[j]) P.text_off[s.im[j]] = base + s.ioff[j];
        const bool write = !s.gave_up && base + total <= P.text_cap;
        // a tile formatted in one window: warp 0 sets up the next tile while
        // the other warps copy this one out
        if (staged && wid == 0) { setup_tile(); prefetched = true; }
        const int ct = staged ? tid - 32 : tid, cs = staged ? DNT - 32 : DNT;
        // 5. copy out, window by window of TEXT_SMEM bytes: a tile with more
        //    text formats each window in turn (a line crossing a window edge
        //    is formatted once per window it touches, clipped to it)
        if (write && total) {
            const uint32_t nwin = staged ? 1u : (total + TEXT_SMEM - 1) / TEXT_SMEM;
            for (uint32_t r = 0; r < nwin; r++) {
                const uint32_t lo = r * (uint32_t)TEXT_SMEM, hi = total - lo < (uint32_t)TEXT_SMEM ? total : lo + TEXT_SMEM;
                if (!staged) {
                    for (int q = tid; q < ITEMS; q += DNT) {
                        int j = s.perm[q];
                        if (s.im[j] < 0 || s.ilen[j] == 0) continue;
                        const uint32_t a = s.ioff[j], e = a + s.ilen[j];
                        if (e <= lo || a >= hi) continue;
                        if (a >= lo && e <= hi) { WriteSink k{a - lo}; format_item(k, j); }
                        else { ClipSink k{(long long)a - lo, (long long)(hi - lo)}; format_item(k, j); }
                    }
                    __syncthreads();
                }
                // the window's bytes go to [g0, g1): global words (or, with a
                // 16-byte aligned text buffer, 16-byte chunks) wholly inside
                // are stored whole, each word assembled from two aligned
                // shared words (the shift between shared and global alignment
                // is the same for the whole window); the partial ends byte by
                // byte
                const unsigned long long g0 = base + lo, g1 = base + hi;
                const unsigned long long w0 = g0 >> 2, w1 = (g1 + 3) >> 2;
                const uint32_t sh = (uint32_t)(g0 & 3);      // global word w starts at shared byte 4(w - w0) - sh
                const uint32_t *sw = reinterpret_cast<const uint32_t *>(s.text);
                auto gword = [&](uint32_t k) -> uint32_t {   // k = w - w0 (>= 1 when sh != 0)
                    return sh == 0 ? sw[k] : __funnelshift_r(sw[k - 1], sw[k], 8 * (4 - sh));
                };
                if (staged && wid == 0) {
                    // setting up the next tile
                } else if ((((uintptr_t)P.text) & 15) == 0) {
                    const unsigned long long c0 = (g0 + 15) >> 4, c1 = g1 >> 4;   // whole chunks [c0, c1)
                    uint4 *t4 = reinterpret_cast<uint4 *>(P.text);
                    for (unsigned long long c = c0 + ct; c < c1; c += cs) {
                        const uint32_t k = (uint32_t)((c << 2) - w0);
                        t4[c] = make_uint4(gword(k), gword(k + 1), gword(k + 2), gword(k + 3));
                    }
                    const unsigned long long h1 = (c0 << 4) < g1 ? (c0 << 4) : g1;
                    for (unsigned long long g = g0 + ct; g < h1; g += cs) P.text[g] = s.text[g - g0];
                    if (c1 >= c0)
                        for (unsigned long long g = (c1 << 4) + ct; g < g1; g += cs) P.text[g] = s.text[g - g0];
                } else {
                    const bool aligned = (((uintptr_t)P.text) & 3) == 0;
                    uint32_t *tw = reinterpret_cast<uint32_t *>(P.text);
                    for (unsigned long long w = w0 + ct; w < w1; w += cs) {
                        unsigned long long gb = w << 2;
                        if (aligned && gb >= g0 && gb + 4 <= g1) {
                            tw[w] = gword((uint32_t)(w - w0));
                        } else {
                            for (int b = 0; b < 4; b++) {
                                unsigned long long g = gb + b;
                                if (g >= g0 && g < g1) P.text[g] = s.text[g - g0];
                            }
                        }
                    }
                }
                __syncthreads();
            }
        } else {
            __syncthreads();
        }
    }
}

__global__ void k_dis_status(DP P)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < P.n_mod && P.dis_status) P.dis_status[m] = P.ctrl->timeout ? S_TIMEOUT : P.dm[m].status;
}

struct DLayout { size_t ctrl, dm, tstate, tile_m0, arena, total; long long arena_words; };
size_t dal(size_t x) { return (x + 255) & ~size_t(255); }
DLayout dlayout(int n_mod, long long n_words, long long rows_cap, long long arena_words)
{
    DLayout L{};
    L.arena_words = arena_words > 0 ? arena_words : 4 * n_words + 256LL * n_mod + 64;
    size_t o = 0;
    L.ctrl = o; o = dal(o + sizeof(DisCtrl));
    L.dm = o; o = dal(o + sizeof(DisMod) * (size_t)n_mod);
    L.tstate = o; o = dal(o + 8 * (size_t)((rows_cap + n_mod) / ITEMS + 2));
    L.tile_m0 = o; o = dal(o + 4 * (size_t)((rows_cap + n_mod) / ITEMS + 2));
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
    P.first_row = table->mod_first_row; P.cap_rows = table->capacity_rows;
    P.inline_names = opts ? opts->inline_names : 1;
    P.header = opts ? opts->header : 1;
    P.text = text; P.text_cap = text_capacity; P.text_off = text_off; P.dis_status = dis_status;
    P.ctrl = (DisCtrl *)(w + L.ctrl); P.dm = (DisMod *)(w + L.dm);
    P.tstate = (unsigned long long *)(w + L.tstate);
    P.tile_m0 = (int *)(w + L.tile_m0);
    P.arena = (uint32_t *)(w + L.arena); P.arena_words = L.arena_words;
    P.max_spins = opts && opts->max_spins > 0 ? opts->max_spins : 1LL << 20;
    P.stall_tile = opts && opts->test_stall_tile > 0 ? opts->test_stall_tile - 1 : -1;
    // device properties and occupancy, once per device
    static int cached_nsm[64] = {}, cached_per_sm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int nsm = dev < 64 ? cached_nsm[dev] : 0, per_sm = dev < 64 ? cached_per_sm[dev] : 0;
    if (nsm <= 0 || per_sm <= 0) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
        if (cudaFuncSetAttribute(k_dis_main, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MainSmem)) !=
            cudaSuccess)
            return SPV_E_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dis_main, DNT, sizeof(MainSmem)) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        if (dev < 64) { cached_nsm[dev] = nsm; cached_per_sm[dev] = per_sm; }
    }
    int nb = (batch->n_modules + 255) / 256;
    SPV_LAUNCH("k_dis_premod", st, k_dis_premod<<<nsm * 4, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_prescan", st, k_dis_prescan<<<1, 1024, 0, st>>>(P));
    SPV_LAUNCH("k_dis_clear", st, k_dis_clear<<<nsm * 4, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_ids", st, k_dis_ids<<<nsm * 8, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_namelen", st, k_dis_namelen<<<nsm * 8, 256, 0, st>>>(P));
    SPV_LAUNCH("k_dis_main", st, k_dis_main<<<nsm * per_sm, DNT, sizeof(MainSmem), st>>>(P));
    SPV_LAUNCH("k_dis_status", st, k_dis_status<<<nb, 256, 0, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}
