// spv_device.cuh -- device helpers shared by the batch kernels: memory
// ordering primitives, the workspace structures, the header check and the
// operand walk of one instruction (section 3.2.1 operand kinds with their
// '?' / '*' quantifiers; checks of section 3.4.5).
#pragma once
#include <stdint.h>
#include "spv_tables.cuh"

namespace spvd {

constexpr uint32_t MAGIC = 0x07230203u;
constexpr uint32_t DEAD = 0xFFFFFFFFu;     // chain ended (framing error or no chain)
constexpr uint32_t UNRES = 0xFFFFFFFEu;    // tile map cannot tell the exit for this entry
constexpr uint64_t NO_KEY = ~0ull;

// status codes (mirror of spv.h)
enum : uint32_t {
    S_OK = 0, S_BAD_MAGIC = 1, S_BAD_HEADER = 2, S_TRUNCATED = 3, S_ZERO_WORDCOUNT = 4,
    S_UNKNOWN_OPCODE = 5, S_BAD_OPERANDS = 6, S_ID_OUT_OF_BOUND = 7, S_DUP_RESULT_ID = 8,
    S_NO_CAPABILITY = 9, S_NO_MEMORY_MODEL = 10, S_MULTI_MEMORY_MODEL = 11, S_NO_ENTRY_POINT = 12,
    S_NO_FUNCTION = 13, S_MISSING_CAPABILITY = 14, S_TIMEOUT = 15, S_CAPACITY = 16
};

// error keys: (global row << 8) | (rank << 4) | sub; the smallest key is the
// module's first error (lowest row, then lowest rank within the row).
enum : uint32_t { R_UNKNOWN = 0, R_BADOP = 1, R_OOB = 2, R_DUP = 3, R_MISSING = 4, R_FRAME = 5 };
__host__ __device__ inline uint64_t make_key(uint64_t row, uint32_t rank, uint32_t sub)
{
    return (row << 8) | (rank << 4) | sub;
}
__host__ __device__ inline uint32_t key_status(uint64_t key)
{
    switch ((key >> 4) & 15) {
    case R_UNKNOWN: return S_UNKNOWN_OPCODE;
    case R_BADOP: return S_BAD_OPERANDS;
    case R_OOB: return S_ID_OUT_OF_BOUND;
    case R_DUP: return S_DUP_RESULT_ID;
    case R_MISSING: return S_MISSING_CAPABILITY;
    default: return (key & 15) ? S_TRUNCATED : S_ZERO_WORDCOUNT;
    }
}

// module flags
enum : uint32_t { MF_DUP = 1, MF_CAPACITY = 2, MF_TIMEOUT = 4, MF_NOARENA = 8, MF_FIXUP = 16 };

struct Ctrl {                        // one per call, at the start of the workspace
    unsigned int next_tile;          // tile claim counter
    unsigned int timeout;            // any bounded wait gave up
    unsigned long long n_tiles;      // tiles in the batch
    unsigned long long arena_used;   // words of the id-bitmap arena the batch needs
    unsigned long long total_rows;   // rows of the whole batch (written by the last tile)
    unsigned int n_fix;              // modules queued for the exact fixup pass
    unsigned int spec_failed;        // a tile's guessed entry was not its predecessor's exit: redo the call
};

struct ModState {                    // one per module
    uint32_t hdr;                    // header status (S_OK when the header is valid)
    uint32_t bound;
    unsigned long long err_key;      // smallest instruction-level error key
    uint32_t n_cap, n_mm, n_ep, n_fn;
    uint32_t decl_lo, decl_hi;       // capabilities declared by OpCapability (< 64)
    uint32_t req_lo, req_hi;         // capabilities required by some instruction
    uint32_t max_rid;
    uint32_t flags;
    long long arena_off;             // first word of this module's id set, -1 none
    uint32_t id_slots;               // 0: bitmap of ceil(bound / 32) words; else hash set of this many keys
    uint32_t n_ids;                  // result ids inserted into a bitmap id set
    uint32_t n_set;                  // bits set in the bitmap afterwards (fewer than n_ids: a duplicate)
    uint32_t pad2;
};

// ---------------- per-module set of result ids ----------------
// A module whose bound is small against its length (bound <= 32 * (len + 64))
// keeps a bitmap of ceil(bound / 32) words; any other module (a bound far
// above what its words could use) keeps an open-addressing hash set of
// 2 * len + 64 keys (a module of len words defines at most len / 2 ids, so
// the set never fills). Either way a module needs at most 2 * len + 64
// words, whatever its header says.
__host__ __device__ inline bool idset_dense(uint32_t bound, long long len)
{
    return (unsigned long long)bound <= 32ull * (unsigned long long)(len + 64);
}
__host__ __device__ inline unsigned long long idset_words(uint32_t bound, long long len)
{
    return idset_dense(bound, len) ? ((unsigned long long)bound + 31) / 32 : 2ull * (unsigned long long)len + 64;
}
__device__ __forceinline__ uint32_t id_hash(uint32_t id, uint32_t slots) { return (uint32_t)(((unsigned long long)id * 2654435761ull) % slots); }
// insert id (>= 1); returns true if it was already present
__device__ __forceinline__ bool idset_insert(uint32_t *base, uint32_t slots, uint32_t id)
{
    if (!slots) {
        uint32_t bit = 1u << (id & 31);
        return (atomicOr(&base[id >> 5], bit) & bit) != 0;
    }
    uint32_t h = id_hash(id, slots);
    for (;;) {
        uint32_t prev = atomicCAS(&base[h], 0u, id);
        if (prev == 0u) return false;
        if (prev == id) return true;
        h = h + 1 == slots ? 0 : h + 1;
    }
}
__device__ __forceinline__ bool idset_contains(const uint32_t *base, uint32_t slots, uint32_t id)
{
    if (!slots) return (base[id >> 5] >> (id & 31)) & 1u;
    uint32_t h = id_hash(id, slots);
    for (;;) {
        uint32_t k = base[h];
        if (k == id) return true;
        if (k == 0u) return false;
        h = h + 1 == slots ? 0 : h + 1;
    }
}

// ---------------- memory ordering ----------------
// Look-back states carry their whole value in the state word, and the
// entries of a published tile map are each valid on their own (a map entry
// is never 0 once written), so both are written and polled with relaxed
// strong accesses: nothing is read on the strength of another location.
// Acquire loads in a poll loop, and fences on the publishing path, would sit
// on the critical path of every later tile.
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed32(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void spin_pause() { __nanosleep(32); }

// x << n with the shift clamped at 32 (PTX shl): 0 for n >= 32
__device__ __forceinline__ uint32_t shl_clamp(uint32_t x, uint32_t n)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(n));
    return r;
}

// Decoupled look-back by one warp (all 32 lanes) over state[0 .. hi]: a state
// is 0 (not yet published), inclusive (flag `incl`: the sum of every state up
// to and including its own) or an aggregate (any other flag: its own count);
// the count is the state's low 62 bits. Returns the sum of the aggregates
// down to and including the nearest inclusive state (0 for hi < 0). Each poll
// reads U x 32 states, all in flight at once, so a look-back that has to
// reach far behind takes few memory round trips. A poll that finds a state
// not yet published inside the reach is repeated, after a pause that starts
// at 32 ns and doubles up to max_ns; after max_spins polls the warp gives up
// (gave_up set, the sum so far returned).
template <int U, unsigned max_ns = 32>
__device__ __forceinline__ unsigned long long warp_lookback_sum(const unsigned long long *state, long long hi,
                                                                unsigned long long incl, unsigned long long mask,
                                                                long long max_spins, int lane, bool &gave_up)
{
    unsigned long long excl = 0;
    long long spins = 0;
    unsigned ns = 32;
    gave_up = false;
    while (hi >= 0) {
        unsigned long long st[U];
        #pragma unroll
        for (int u = 0; u < U; u++) {
            const long long j = hi - 32 * u - lane;
            st[u] = j >= 0 ? ld_relaxed(&state[j]) : incl;     // before state 0: inclusive 0
        }
        int reach = 32 * U;                                    // distance of the nearest inclusive state
        bool wait = false;
        #pragma unroll
        for (int u = 0; u < U; u++) {
            if (reach < 32 * U || wait) continue;
            const unsigned long long f = st[u] & mask;
            const unsigned im = __ballot_sync(0xffffffffu, f == incl);
            const unsigned nm = __ballot_sync(0xffffffffu, f == 0);
            const int le = im ? __ffs(im) - 1 : 32;
            const unsigned below = le == 32 ? 0xffffffffu : ((1u << le) - 1u);
            if (nm & below) wait = true;
            else if (im) reach = 32 * u + le;
        }
        if (wait) {
            if (++spins > max_spins) { gave_up = true; break; }
            __nanosleep(ns);
            ns = ns < max_ns ? 2 * ns : max_ns;
            continue;
        }
        unsigned long long v = 0;
        #pragma unroll
        for (int u = 0; u < U; u++)
            if (32 * u + lane <= reach) v += st[u] & ~mask;
        #pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        excl += v;
        if (reach < 32 * U) break;
        hi -= 32 * U;
    }
    return excl;
}

// ---------------- header ----------------
// Listing 4 header: magic, version 0x00MMmm00 (major 1, minor <= 6),
// generator, bound, schema 0.
__device__ __forceinline__ uint32_t header_status(const uint32_t *w, long long n)
{
    if (n < 5) return S_TRUNCATED;
    const uint32_t w0 = w[0], v = w[1], w4 = w[4];     // one round trip for the three words
    if (w0 != MAGIC) return S_BAD_MAGIC;
    if ((v & 0xff0000ffu) != 0 || ((v >> 16) & 0xffu) != 1 || ((v >> 8) & 0xffu) > 6) return S_BAD_HEADER;
    if (w4 != 0) return S_BAD_HEADER;
    return S_OK;
}

// ---------------- capability closure ----------------
__device__ __forceinline__ uint64_t cap_closure(uint64_t d)
{
    const spvt::Tables &T = g_spv_tables;
    for (int it = 0; it < 8; it++) {
        uint64_t n = d;
        uint64_t x = d;
        while (x) {
            int b = __ffsll((long long)x) - 1;
            x &= x - 1;
            n |= T.cap_dep[b];
        }
        if (n == d) break;
        d = n;
    }
    return d;
}

// asynchronous global -> shared copies (completed by cp_async_wait_all and
// made visible to the block by the next barrier); the 16-byte form reads
// src_bytes (4..16) and fills the rest of the 16 bytes with zeros
__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---------------- literal strings ----------------
// Words [pos, wc) hold a NUL-terminated string whose last word is zero
// after the NUL. Returns the word count of the string, or 0 when malformed.
template <class WordFn>
__device__ __forceinline__ uint32_t string_words(const WordFn &word, uint32_t pos, uint32_t wc)
{
    for (uint32_t i = pos; i < wc; i++) {
        uint32_t v = word(i);
        uint32_t z = (v - 0x01010101u) & ~v & 0x80808080u;
        if (z) {
            int b = (__ffs(z) - 1) >> 3;          // first zero byte (little-endian order)
            uint32_t rest = b == 3 ? 0u : (v >> (8 * (b + 1)));
            return rest == 0 ? i - pos + 1 : 0;
        }
    }
    return 0;
}

// Result of walking one instruction's operands.
struct Walk {
    bool ok;                 // words match the opcode's operand list exactly
    bool oob;                // some id operand (incl. result type / id) is 0 or >= bound
    uint64_t req;            // capabilities the instruction requires
};

// Walk the operands of an instruction of wc words whose opcode descriptor is
// d. word(i) returns the instruction's word i (1 <= i < wc).
template <class WordFn>
__device__ Walk walk_instruction(const WordFn &word, uint32_t wc, const spvt::OpDesc &d, uint32_t bound)
{
    const spvt::Tables &T = g_spv_tables;
    Walk r{true, false, 0};
    if (d.fast & 1) {
        // only fixed ids / literals and a plain tail: a length check and a
        // range check of the id words (same result as the walk below)
        const uint32_t need = 1u + d.nfixed, tail = (d.fast >> 1) & 7u;
        if (tail == 4) {
            // one bit-enum word: it and the literal parameters of its known
            // bits must fill the instruction exactly
            if (wc == need) r.ok = (d.fast & 16) != 0;
            else if (wc > need) {
                uint32_t x = word(need), np = 0;
                while (x) {
                    int b = __ffs(x) - 1;
                    x &= x - 1;
                    const spvt::EnDesc &e = T.benum[d.bkind][b];
                    if (e.known) np += e.nparam;
                }
                r.ok = wc == need + 1u + np;
            } else r.ok = false;
        } else {
            r.ok = tail == 0 ? wc == need : (wc >= need && (tail != 3 || ((wc - need) & 1u) == 0));
        }
        if (r.ok) {
            uint32_t mask = d.id_mask;
            while (mask) {
                int i = __ffs(mask) - 1;
                mask &= mask - 1;
                uint32_t v = word((uint32_t)i);
                if (v == 0 || v >= bound) r.oob = true;
            }
            if (tail == 1 || tail == 3)
                for (uint32_t i = need; i < wc; i++) { uint32_t v = word(i); if (v == 0 || v >= bound) r.oob = true; }
        }
        if (d.cap >= 0) r.req |= 1ull << d.cap;
        return r;
    }
    uint32_t pos = 1;
#define SPV_ID_AT(p) do { uint32_t _v = word(p); if (_v == 0 || _v >= bound) r.oob = true; } while (0)
    if (d.flags & 2) { if (pos >= wc) { r.ok = false; return r; } SPV_ID_AT(pos); pos++; }
    if (d.flags & 4) { if (pos >= wc) { r.ok = false; return r; } SPV_ID_AT(pos); pos++; }
    for (int k = 0; k < d.nprog && r.ok; k++) {
        uint8_t c = d.prog[k];
        bool opt = (c & spvt::A_OPT) != 0;
        c &= 0x7f;
        if (c == spvt::A_IDS) { for (; pos < wc; pos++) SPV_ID_AT(pos); continue; }
        if (c == spvt::A_LITS) { pos = wc; continue; }
        if (c == spvt::A_IDPAIRS) {
            if ((wc - pos) & 1) { r.ok = false; break; }
            for (; pos < wc; pos++) SPV_ID_AT(pos);
            continue;
        }
        if (pos >= wc) { if (opt) continue; r.ok = false; break; }
        if (c == spvt::A_ID) { SPV_ID_AT(pos); pos++; }
        else if (c == spvt::A_LIT) { pos++; }
        else if (c == spvt::A_STR) {
            uint32_t n = string_words(word, pos, wc);
            if (!n) { r.ok = false; break; }
            pos += n;
        } else if (c == spvt::A_CTX) { pos = wc; }
        else if (c >= spvt::A_ENUM && c < spvt::A_ENUM + spvt::NUM_VKINDS) {
            int kind = c - spvt::A_ENUM;
            uint32_t v = word(pos++);
            // the enumerant's parameter codes, packed in one register
            uint32_t packed = 0;
            int np = 0;
            if (v < 64 && T.venum[kind][v].known) {
                const spvt::EnDesc &e = T.venum[kind][v];
                if (e.cap >= 0) r.req |= 1ull << e.cap;
                np = e.nparam;
                packed = (uint32_t)e.param[0] | ((uint32_t)e.param[1] << 8) | ((uint32_t)e.param[2] << 16);
            } else if (T.vunknown[kind]) {
                packed = T.vunknown[kind]; np = 1;
            }
            for (int q = 0; q < np && r.ok; q++) {
                uint8_t pc = (uint8_t)(packed >> (8 * q));
                if (pc == spvt::A_LITS) { pos = wc; continue; }
                if (pos >= wc) { r.ok = false; break; }
                if (pc == spvt::A_ID) { SPV_ID_AT(pos); pos++; }
                else if (pc == spvt::A_LIT) { pos++; }
                else if (pc == spvt::A_STR) {
                    uint32_t n = string_words(word, pos, wc);
                    if (!n) { r.ok = false; break; }
                    pos += n;
                } else {                    // a nested value enum without parameters
                    int k2 = pc - spvt::A_ENUM;
                    uint32_t v2 = word(pos++);
                    if (v2 < 64 && T.venum[k2][v2].known && T.venum[k2][v2].cap >= 0)
                        r.req |= 1ull << T.venum[k2][v2].cap;
                }
            }
        } else {                            // bit enum
            int kind = c - spvt::A_BITS;
            uint32_t v = word(pos++);
            uint32_t x = v;
            while (x && r.ok) {
                int b = __ffs(x) - 1;
                x &= x - 1;
                const spvt::EnDesc &e = T.benum[kind][b];
                if (!e.known) continue;
                for (int q = 0; q < e.nparam; q++) {
                    if (pos >= wc) { r.ok = false; break; }
                    pos++;                  // bit-enum parameters are literals
                }
            }
        }
    }
#undef SPV_ID_AT
    if (r.ok && pos != wc) r.ok = false;
    if (d.cap >= 0) r.req |= 1ull << d.cap;
    return r;
}

// Width rules of OpTypeInt / OpTypeFloat (8/16/64-bit integers, 16/64-bit floats).
template <class WordFn>
__device__ __forceinline__ uint64_t width_caps(const WordFn &word, uint32_t op, uint32_t wc)
{
    if (wc < 3) return 0;
    uint32_t w = word(2);
    if (op == 21) return w == 8 ? (1ull << 39) : w == 16 ? (1ull << 22) : w == 64 ? (1ull << 11) : 0;
    if (op == 22) return w == 16 ? (1ull << 9) : w == 64 ? (1ull << 10) : 0;
    return 0;
}

}  // namespace spvd
