// spv_asm.cu -- batched assembler (section 3.4.4, Dis/Assembler): the text
// form that the disassembler prints, read back into words, for every module
// of a batch at once. The text form is the one include/spv.h documents for
// spv_assemble_batch.
//
// The paper's assembler keeps a hash table from id names to SPIRVId objects.
// Here each module gets a device hash table that every line naming an id
// fills concurrently; the names are then numbered in order of first
// appearance by a scan over their occurrences.
//
// Steps, all on the caller's stream with no host synchronisation:
//   1. lines: a bitmap of module starts, then per 8 KB tile of text the line
//      starts (after a '\n', or at a module start), counted, scanned and
//      written; each module's first line by binary search, each line's
//      module.
//   2. measure: one thread per line parses it: word count, named-id
//      occurrences, the largest explicit id, header comment lines, type
//      declarations, and the first bad line of each module.
//   3. named ids: every occurrence goes into its module's hash table (the
//      first position of each name by atomicMin); a scan over occurrences in
//      text order ranks the first ones; a name's id is the module's largest
//      explicit id + 1 + its rank.
//   4. types: the first OpTypeInt / OpTypeFloat of each id, into a
//      per-module hash table; an OpConstant value of one token takes its
//      width from it.
//   5. a scan of the word counts places every line; a module's words start
//      with its five header words; every line is parsed once more and
//      writes its words.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spv.h"
#include "spv_prof.h"
#include "spv_scan.cuh"
#include "spv_tables.cuh"

namespace {

// ---------------------------------------------------------------------------
// name -> opcode / enumerant hash tables, built at compile time from the
// opcode and enumerant tables (open addressing, linear probing)
// ---------------------------------------------------------------------------
constexpr uint32_t FNV0 = 2166136261u, FNVP = 16777619u;
constexpr int OPH = 1024, ENH = 1024;
struct AsmNames {
    uint16_t op[OPH];        // opcode + 1, 0 empty
    uint16_t en[ENH];        // (kind << 8 | index) + 1; value kinds 0.., bit kinds 16..
    int max_len;             // longest name
};
constexpr uint32_t en_seed(int kind) { return FNV0 ^ ((uint32_t)(kind + 1) * 0x9E3779B1u); }

constexpr void put_en(AsmNames &a, const spvt::Tables &t, int kind, int idx, const spvt::EnDesc &e)
{
    const int off = (e.name_hi << 8) | e.name_lo;
    uint32_t h = en_seed(kind);
    for (int k = 0; k < e.name_len; k++) h = (h ^ (uint8_t)t.names[off + k]) * FNVP;
    uint32_t s = h & (ENH - 1);
    while (a.en[s]) s = (s + 1) & (ENH - 1);
    a.en[s] = (uint16_t)(((kind << 8) | idx) + 1);
    if (e.name_len > a.max_len) a.max_len = e.name_len;
}

constexpr AsmNames build_asm_names(const spvt::Tables &t)
{
    AsmNames a{};
    for (int o = 0; o < 256; o++) {
        const spvt::OpDesc &d = t.ops[o];
        if (!(d.flags & 1)) continue;
        uint32_t h = FNV0;
        for (int k = 0; k < d.name_len; k++) h = (h ^ (uint8_t)t.names[d.name_off + k]) * FNVP;
        uint32_t s = h & (OPH - 1);
        while (a.op[s]) s = (s + 1) & (OPH - 1);
        a.op[s] = (uint16_t)(o + 1);
        if (d.name_len > a.max_len) a.max_len = d.name_len;
    }
    for (int k = 0; k < spvt::NUM_VKINDS; k++)
        for (int v = 0; v < 64; v++)
            if (t.venum[k][v].known) put_en(a, t, k, v, t.venum[k][v]);
    for (int k = 0; k < spvt::NUM_BKINDS; k++)
        for (int b = 0; b < 32; b++)
            if (t.benum[k][b].known) put_en(a, t, 16 + k, b, t.benum[k][b]);
    return a;
}

static __device__ const AsmNames g_asm_names = build_asm_names(SPV_TABLES_HOST);

__device__ __constant__ double c_p10[23] = {1e0,  1e1,  1e2,  1e3,  1e4,  1e5,  1e6,  1e7,  1e8,  1e9,  1e10, 1e11,
                                            1e12, 1e13, 1e14, 1e15, 1e16, 1e17, 1e18, 1e19, 1e20, 1e21, 1e22};

__device__ __forceinline__ bool same_bytes(const uint8_t *a, const char *b, uint32_t n)
{
    for (uint32_t k = 0; k < n; k++)
        if (a[k] != (uint8_t)b[k]) return false;
    return true;
}

__device__ int find_op(const uint8_t *s, uint32_t n)
{
    if (n == 0 || n > (uint32_t)g_asm_names.max_len) return -1;
    uint32_t h = FNV0;
    for (uint32_t k = 0; k < n; k++) h = (h ^ s[k]) * FNVP;
    for (uint32_t i = h & (OPH - 1), p = 0; p < OPH; p++, i = (i + 1) & (OPH - 1)) {
        const uint32_t e = g_asm_names.op[i];
        if (!e) return -1;
        const spvt::OpDesc &d = g_spv_tables.ops[e - 1];
        if (d.name_len == n && same_bytes(s, g_spv_tables.names + d.name_off, n)) return (int)(e - 1);
    }
    return -1;
}

// kind: value kind k, or 16 + bit kind k; returns the value (value kinds) or
// the bit index (bit kinds), -1 when the name is not one of the kind's
__device__ int find_en(int kind, const uint8_t *s, uint32_t n)
{
    if (n == 0 || n > (uint32_t)g_asm_names.max_len) return -1;
    uint32_t h = en_seed(kind);
    for (uint32_t k = 0; k < n; k++) h = (h ^ s[k]) * FNVP;
    for (uint32_t i = h & (ENH - 1), p = 0; p < ENH; p++, i = (i + 1) & (ENH - 1)) {
        const uint32_t e = g_asm_names.en[i];
        if (!e) return -1;
        const int kk = (int)((e - 1) >> 8), idx = (int)((e - 1) & 255);
        if (kk != kind) continue;
        const spvt::EnDesc &d = kind < 16 ? g_spv_tables.venum[kind][idx] : g_spv_tables.benum[kind - 16][idx];
        if (d.name_len == n && same_bytes(s, g_spv_tables.names + ((d.name_hi << 8) | d.name_lo), n)) return idx;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// literals
// ---------------------------------------------------------------------------
__device__ __forceinline__ int hexv(uint32_t c)
{
    if (c - '0' < 10u) return (int)(c - '0');
    if (c - 'a' < 6u) return (int)(c - 'a' + 10);
    if (c - 'A' < 6u) return (int)(c - 'A' + 10);
    return -1;
}
__device__ __forceinline__ bool isdig(uint32_t c) { return c - '0' < 10u; }

// decimal digits only, at least one, value <= max
__device__ bool dec_u64(const uint8_t *s, uint32_t n, uint64_t max, uint64_t &v)
{
    if (n == 0) return false;
    uint64_t a = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint32_t d = (uint32_t)s[i] - '0';
        if (d > 9u) return false;
        if (a > (max - d) / 10) return false;
        a = a * 10 + d;
    }
    v = a;
    return true;
}

__device__ bool raw_word(const uint8_t *s, uint32_t n, uint32_t &v)
{
    if (n != 10 || s[0] != '0' || s[1] != 'x') return false;
    uint32_t a = 0;
    for (int k = 2; k < 10; k++) {
        const int h = hexv(s[k]);
        if (h < 0) return false;
        a = (a << 4) | (uint32_t)h;
    }
    v = a;
    return true;
}

// 0 explicit (id set), 1 named, -1 not an id
__device__ int classify_id(const uint8_t *s, uint32_t n, uint32_t &id)
{
    if (n < 2 || s[0] != '%') return -1;
    uint32_t j = n;
    while (j > 1 && isdig(s[j - 1])) j--;
    if (j == n || (j != 1 && s[j - 1] != '_')) return 1;
    uint64_t v;
    if (!dec_u64(s + j, n - j, 0xffffffffull, v)) return -1;
    id = (uint32_t)v;
    return 0;
}

// Round m * 2^E (+ a nonzero amount below m's last bit when sticky) to a
// binary format with P significand bits and exponents [EMIN, EMAX], to
// nearest even; returns the bits without the sign.
template <int P, int EMIN, int EMAX>
__device__ uint64_t round_bin(uint64_t m, long long E, bool sticky)
{
    if (m == 0) return 0;
    const int lz = __clzll((long long)m);
    m <<= lz;
    E -= lz;
    long long ue = 63 + E;                       // exponent of the leading bit
    if (ue > EMAX) return (uint64_t)(EMAX - EMIN + 2) << (P - 1);   // infinity
    long long sh = 64 - P + (ue < EMIN ? EMIN - ue : 0);
    if (sh >= 65) return 0;
    uint64_t keep, rem, half;
    if (sh == 64) { keep = 0; rem = m; half = 1ull << 63; }
    else { keep = m >> sh; rem = m & ((1ull << sh) - 1); half = 1ull << (sh - 1); }
    if (rem > half || (rem == half && (sticky || (keep & 1)))) keep++;
    if (ue < EMIN) return keep;                  // subnormal (or, rounded up, the smallest normal)
    if (keep >> P) { keep >>= 1; ue++; }
    if (ue > EMAX) return (uint64_t)(EMAX - EMIN + 2) << (P - 1);
    return ((uint64_t)(ue - EMIN + 1) << (P - 1)) | (keep & ((1ull << (P - 1)) - 1));
}
__device__ __forceinline__ uint64_t round_double(uint64_t m, long long E, bool sticky)
{
    return round_bin<53, -1022, 1023>(m, E, sticky);
}

// the double (bits) rounded to float, to nearest even
__device__ uint32_t double_to_float_bits(uint64_t d)
{
    const uint32_t sign = (uint32_t)(d >> 32) & 0x80000000u;
    const uint32_t be = (uint32_t)(d >> 52) & 0x7ff;
    const uint64_t frac = d & ((1ull << 52) - 1);
    if (be == 0x7ff) return sign | (frac ? 0x7fc00000u : 0x7f800000u);
    if (be == 0 && frac == 0) return sign;
    const uint64_t m = be ? (frac | (1ull << 52)) : frac;
    const long long E = (be ? (long long)be : 1) - 1075;
    return sign | (uint32_t)round_bin<24, -126, 127>(m, E, false);
}

// ---- little bignums, base 2^32, little-endian: the exact decimal path ----
constexpr int BN = 124;
struct Big { uint32_t w[BN]; int n; };

__device__ void big_mul_add(Big &a, uint32_t mul, uint32_t add)
{
    uint64_t c = add;
    for (int i = 0; i < a.n; i++) {
        const uint64_t t = (uint64_t)a.w[i] * mul + c;
        a.w[i] = (uint32_t)t;
        c = t >> 32;
    }
    if (c && a.n < BN) a.w[a.n++] = (uint32_t)c;
}
__device__ int big_bits(const Big &a)
{
    int n = a.n;
    while (n > 0 && a.w[n - 1] == 0) n--;
    return n ? 32 * (n - 1) + (32 - __clz((int)a.w[n - 1])) : 0;
}
__device__ void big_shl(Big &a, int s)
{
    const int ws = s >> 5, bs = s & 31;
    int n = a.n + ws + 1;
    if (n > BN) n = BN;
    for (int i = n - 1; i >= 0; i--) {
        const int j = i - ws;
        uint32_t v = 0;
        if (j >= 0 && j < a.n) v = a.w[j] << bs;
        if (bs && j - 1 >= 0 && j - 1 < a.n) v |= a.w[j - 1] >> (32 - bs);
        a.w[i] = v;
    }
    a.n = n;
}
__device__ void big_shr1(Big &a)
{
    for (int i = 0; i < a.n; i++) a.w[i] = (a.w[i] >> 1) | (i + 1 < a.n ? a.w[i + 1] << 31 : 0u);
}
__device__ int big_cmp(const Big &a, const Big &b)
{
    const int n = a.n > b.n ? a.n : b.n;
    for (int i = n - 1; i >= 0; i--) {
        const uint32_t x = i < a.n ? a.w[i] : 0u, y = i < b.n ? b.w[i] : 0u;
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}
__device__ void big_sub(Big &a, const Big &b)   // a -= b, a >= b
{
    long long br = 0;
    for (int i = 0; i < a.n; i++) {
        long long t = (long long)a.w[i] - (i < b.n ? (long long)b.w[i] : 0) - br;
        br = t < 0;
        a.w[i] = (uint32_t)(t + (br << 32));
    }
}
__device__ bool big_zero(const Big &a)
{
    for (int i = 0; i < a.n; i++)
        if (a.w[i]) return false;
    return true;
}
__device__ void big_pow10(Big &a, int k)
{
    a.n = 1; a.w[0] = 1;
    for (; k >= 9; k -= 9) big_mul_add(a, 1000000000u, 0);
    uint32_t p = 1;
    for (; k > 0; k--) p *= 10;
    big_mul_add(a, p, 0);
}

constexpr int DEC_KEEP = 780;      // significant digits kept; the rest decide only a sticky digit

// The exact value of a decimal literal's digits [m0, m1) (one '.' allowed)
// times 10^ex, rounded to double (no sign). The 780 leading significant
// digits decide the result together with whether any later digit is nonzero
// (a double's halfway points have at most 767 significant digits).
__device__ __noinline__ uint64_t dec_value(const uint8_t *s, uint32_t m0, uint32_t m1, long long ex)
{
    // pass 1: count significant digits, digits after the point, sticky
    long long frac_digits = 0, nd = 0, dropped = 0;
    bool after = false, started = false, sticky = false;
    for (uint32_t k = m0; k < m1; k++) {
        const uint32_t c = s[k];
        if (c == '.') { after = true; continue; }
        if (after) frac_digits++;
        if (!started && c == '0') continue;
        started = true;
        if (nd < DEC_KEEP) nd++;
        else { dropped++; sticky |= c != '0'; }
    }
    if (nd == 0) return 0;
    // value = D * 10^q (+ a sticky digit), D the nd kept digits
    long long q = ex - frac_digits + dropped;
    if (nd + q >= 310) return 0x7ff0000000000000ull;
    if (nd + q <= -324) return 0;
    Big D;
    D.n = 1; D.w[0] = 0;
    {
        uint32_t chunk = 0, cm = 1;
        long long taken = 0;
        started = false;
        for (uint32_t k = m0; k < m1 && taken < nd; k++) {
            const uint32_t c = s[k];
            if (c == '.') continue;
            if (!started && c == '0') continue;
            started = true;
            chunk = chunk * 10 + (c - '0');
            cm *= 10;
            taken++;
            if (cm == 1000000000u) { big_mul_add(D, cm, chunk); chunk = 0; cm = 1; }
        }
        if (cm > 1) big_mul_add(D, cm, chunk);
        if (sticky) { big_mul_add(D, 10, 1); q--; }
    }
    // fast path: D below 2^53 and a power of ten that is exact in double
    if (D.n <= 2 && q >= -22 && q <= 22) {
        const uint64_t d = (uint64_t)D.w[0] | (D.n > 1 ? (uint64_t)D.w[1] << 32 : 0ull);
        if (d < (1ull << 53)) {
            const double r = q >= 0 ? (double)d * c_p10[q] : (double)d / c_p10[-q];
            return (uint64_t)__double_as_longlong(r);
        }
    }
    if (q >= 0) {
        for (long long k = q; k >= 9; k -= 9) big_mul_add(D, 1000000000u, 0);
        uint32_t p = 1;
        for (long long k = q % 9; k > 0; k--) p *= 10;
        big_mul_add(D, p, 0);
        const int bl = big_bits(D);
        uint64_t m = 0;
        bool st = false;
        for (int b = bl - 1, k = 0; b >= 0; b--, k++) {
            const uint32_t bit = (D.w[b >> 5] >> (b & 31)) & 1u;
            if (k < 64) m = (m << 1) | bit;
            else st |= bit != 0;
        }
        const long long E = bl > 64 ? bl - 64 : 0;
        return round_double(m, E, st);
    }
    // q < 0: Q = floor(D * 2^s / 10^-q), with 63 or 64 significant bits
    Big V;
    big_pow10(V, (int)-q);
    const int s_sh = 63 + big_bits(V) - big_bits(D);
    if (s_sh >= 0) big_shl(D, s_sh);
    else big_shl(V, -s_sh);
    big_shl(V, 63);
    uint64_t Q = 0;
    for (int b = 63; b >= 0; b--) {
        if (big_cmp(D, V) >= 0) { big_sub(D, V); Q |= 1ull << b; }
        big_shr1(V);
    }
    return round_double(Q, -(long long)s_sh, !big_zero(D));
}

// hexadecimal digits [m0, m1) (one '.' allowed) times 2^ex, rounded to
// double (no sign)
__device__ uint64_t hex_value(const uint8_t *s, uint32_t m0, uint32_t m1, long long ex)
{
    uint64_t m = 0;
    long long e2 = 0;
    bool sticky = false, after = false;
    for (uint32_t k = m0; k < m1; k++) {
        const uint32_t c = s[k];
        if (c == '.') { after = true; continue; }
        const uint32_t d = (uint32_t)hexv(c);
        if ((m >> 60) == 0) {
            m = (m << 4) | d;
            if (after) e2 -= 4;
        } else {
            sticky |= d != 0;
            if (!after) e2 += 4;
        }
    }
    return round_double(m, e2 + ex, sticky);
}

// A float literal (the whole token):
//   [+-]? ( inf | nan | 0[xX] H* [. H*] [[pP] [+-]? D+] | D* [. D*] [[eE] [+-]? D+] )
// with at least one mantissa digit. Returns false if the token is not one;
// with VALUE, *bits is the double.
template <bool VALUE>
__device__ bool float_literal(const uint8_t *s, uint32_t n, uint64_t *bits)
{
    uint32_t i = 0;
    uint64_t sign = 0;
    if (i < n && (s[i] == '+' || s[i] == '-')) { sign = s[i] == '-' ? 1ull << 63 : 0; i++; }
    if (n - i == 3) {
        if (s[i] == 'i' && s[i + 1] == 'n' && s[i + 2] == 'f') {
            if (VALUE) *bits = sign | 0x7ff0000000000000ull;
            return true;
        }
        if (s[i] == 'n' && s[i + 1] == 'a' && s[i + 2] == 'n') {
            if (VALUE) *bits = sign | 0x7ff8000000000000ull;
            return true;
        }
    }
    const bool hex = n - i >= 2 && s[i] == '0' && (s[i + 1] == 'x' || s[i + 1] == 'X');
    if (hex) i += 2;
    const uint32_t m0 = i;
    uint32_t ndig = 0;
    bool dot = false;
    while (i < n) {
        const uint32_t c = s[i];
        if (c == '.' && !dot) { dot = true; i++; continue; }
        if (hex ? hexv(c) >= 0 : isdig(c)) { ndig++; i++; continue; }
        break;
    }
    if (!ndig) return false;
    const uint32_t m1 = i;
    long long ex = 0;
    if (i < n && (hex ? (s[i] == 'p' || s[i] == 'P') : (s[i] == 'e' || s[i] == 'E'))) {
        i++;
        bool neg = false;
        if (i < n && (s[i] == '+' || s[i] == '-')) { neg = s[i] == '-'; i++; }
        const uint32_t e0 = i;
        while (i < n && isdig(s[i])) {
            if (ex < (1ll << 40)) ex = ex * 10 + (s[i] - '0');
            i++;
        }
        if (i == e0) return false;
        if (neg) ex = -ex;
    }
    if (i != n) return false;
    if (VALUE) *bits = sign | (hex ? hex_value(s, m0, m1, ex) : dec_value(s, m0, m1, ex));
    return true;
}

// ---------------------------------------------------------------------------
// workspace records
// ---------------------------------------------------------------------------
struct AsmCtrl {
    long long need_lines, need_occ;         // what the last call needed (spv_asm_required); first
    long long t0, t1, base_al;              // text range [t0, t1); 16-byte aligned tile base (may be < 0)
    long long n_tiles;
    long long n_lines;                      // all line starts (may exceed the line capacity)
    long long ls_limit;                     // start of the first line not stored (t1 if all are)
    long long n_occ;                        // named-id occurrences (may exceed the capacity)
    long long arena_used;
    long long n_mod;
    long long n_special;                    // lines the passes after the measuring one revisit
    unsigned int bad_offsets;
    unsigned int pad;
};

enum : uint32_t { MF_FIT_LINES = 1, MF_FIT_OCC = 2, MF_FIT_ARENA = 4 };
struct AsmMod {
    unsigned long long hdr[4];      // (line + 1) << 32 | value of the last valid header line; 0 none
    unsigned long long err;         // line << 8 | code of the first bad line; ~0 none
    long long first_line, end_line; // lines [first_line, end_line)
    unsigned int max_explicit;
    unsigned int n_types;           // type declaration lines
    unsigned int flags;             // MF_*
    unsigned int pad;
    long long occ0, occ1;           // named occurrences [occ0, occ1)
    long long names_at, names_cap;  // name hash table: names_cap slots of 2 words at arena[names_at]
    long long types_at, types_cap;  // type hash table: types_cap slots of 2 words
    unsigned long long distinct;    // distinct names
};

// line flags; LF_SLOT: the line's final words (at most SLOT_WORDS) are in its slot
enum : uint8_t { LF_TYPEDECL = 1, LF_CONST1 = 2, LF_W64 = 4, LF_SLOT = 8 };
constexpr int SLOT_WORDS = 8;

struct AsmP {
    const uint8_t *text;
    const uint64_t *text_off;
    int n_mod;
    unsigned long long text_bytes;
    AsmCtrl *ctrl;
    AsmMod *mod;
    uint32_t *bitmap;
    long long bitmap_words;
    long long tile_cap;
    uint32_t *tile_cnt;
    unsigned long long *tile_off;
    long long line_cap;
    unsigned long long *ls;
    int32_t *lmod;
    uint32_t *lw, *lnm;
    uint8_t *lfl;
    uint32_t *lslot;                // SLOT_WORDS words per line
    unsigned long long *special;    // lines with named ids, one-token constants, type declarations or unrecorded words
    unsigned long long *lwo, *occ_off;
    long long occ_cap;
    unsigned long long *occ_slot, *occ_pos;
    uint32_t *occ_first;
    unsigned long long *occ_rank;
    unsigned long long *arena;
    long long arena_cap;
    unsigned long long *msize, *moff;
    // outputs
    uint32_t *words;
    long long words_cap;
    int64_t *word_off;
    uint32_t *status;
    int64_t *err_line;
};

constexpr int LT_THREADS = 256, LT_BYTES = 32, LT_TILE = LT_THREADS * LT_BYTES;   // 8 KB tiles

// ---------------------------------------------------------------------------
// setup and line split
// ---------------------------------------------------------------------------
// after k_asm_mod_init (which flags decreasing offsets)
__global__ void k_asm_setup(AsmP P)
{
    AsmCtrl *c = P.ctrl;
    const unsigned long long a = P.text_off[0], b = P.text_off[P.n_mod];
    unsigned int bad = c->bad_offsets | (b > P.text_bytes || a > b || b >= (1ull << 40));
    const long long t0 = bad ? 0 : (long long)a, t1 = bad ? 0 : (long long)b;
    c->t0 = t0; c->t1 = t1;
    const long long mis = (long long)(((uintptr_t)P.text + (uintptr_t)t0) & 15u);
    c->base_al = t0 - mis;
    c->n_tiles = t1 > t0 ? (t1 - c->base_al + LT_TILE - 1) / LT_TILE : 0;
    if (c->n_tiles > P.tile_cap) { c->n_tiles = 0; bad = 1; }
    c->n_lines = 0;
    c->ls_limit = t1;
    c->n_occ = 0;
    c->arena_used = 0;
    c->n_mod = P.n_mod;
    c->bad_offsets = bad;
}

// per module: clear the record, check the offsets
__global__ void k_asm_mod_init(AsmP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        AsmMod &M = P.mod[m];
        for (int k = 0; k < 4; k++) M.hdr[k] = 0;
        M.err = ~0ull;
        M.first_line = M.end_line = 0;
        M.max_explicit = 0; M.n_types = 0; M.flags = 0;
        M.occ0 = M.occ1 = 0;
        M.names_at = M.names_cap = M.types_at = M.types_cap = 0;
        M.distinct = 0;
        if (P.text_off[m] > P.text_off[m + 1]) atomicOr(&P.ctrl->bad_offsets, 1u);
    }
}

__global__ void k_asm_mark(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        const long long a = (long long)P.text_off[m], b = (long long)P.text_off[m + 1];
        if (a < b && a > c.t0) {
            const long long r = a - c.base_al;
            atomicOr(&P.bitmap[r >> 5], 1u << (r & 31));
        }
    }
}

// bit j: text position c0 + j starts a line
__device__ uint32_t line_start_mask(const AsmP &P, const AsmCtrl &c, long long c0)
{
    if (c0 + LT_BYTES <= c.t0 || c0 >= c.t1) return 0;
    uint32_t nl = 0;        // bit j: byte c0 + j is '\n'
    if (c0 >= c.t0 && c0 + LT_BYTES <= c.t1) {
        const uint4 *p = reinterpret_cast<const uint4 *>(P.text + c0);
        const uint4 a = p[0], b = p[1];
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        #pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t e = __vcmpeq4(w[k], 0x0a0a0a0au) & 0x01010101u;
            nl |= ((e | (e >> 7) | (e >> 14) | (e >> 21)) & 15u) << (4 * k);
        }
    } else {
        for (int j = 0; j < LT_BYTES; j++) {
            const long long q = c0 + j;
            if (q >= c.t0 && q < c.t1 && P.text[q] == '\n') nl |= 1u << j;
        }
    }
    const uint32_t prev_nl = (c0 > c.t0 && c0 - 1 < c.t1 && P.text[c0 - 1] == '\n') ? 1u : 0u;
    uint32_t s = (nl << 1) | prev_nl | P.bitmap[(c0 - c.base_al) >> 5];
    if (c0 <= c.t0 && c.t0 < c0 + LT_BYTES) s |= 1u << (c.t0 - c0);
    // only positions in [t0, t1)
    uint32_t valid = ~0u;
    if (c0 < c.t0) valid &= ~0u << (c.t0 - c0);
    if (c0 + LT_BYTES > c.t1) valid &= (1u << (c.t1 - c0)) - 1u;
    return s & valid;
}

template <int PASS>
__global__ void __launch_bounds__(LT_THREADS) k_asm_lines(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    const long long nt = c.n_tiles;
    for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
        const long long c0 = c.base_al + t * LT_TILE + (long long)threadIdx.x * LT_BYTES;
        uint32_t mask = line_start_mask(P, c, c0);
        unsigned long long total;
        const unsigned long long pre = block_exscan(__popc(mask), &total);
        if (PASS == 0) {
            if (threadIdx.x == 0) P.tile_cnt[t] = (uint32_t)total;
        } else {
            unsigned long long idx = P.tile_off[t] + pre;
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                if ((long long)idx < P.line_cap) P.ls[idx] = (unsigned long long)(c0 + j);
                else if ((long long)idx == P.line_cap) P.ctrl->ls_limit = c0 + j;
                idx++;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// module line ranges
// ---------------------------------------------------------------------------
__device__ long long lower_bound_ls(const unsigned long long *ls, long long n, unsigned long long q)
{
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (ls[mid] < q) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// one warp per module: line range, fit, and each line's module
__global__ void k_asm_modlines(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    const long long stored = c.n_lines < P.line_cap ? c.n_lines : P.line_cap;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < P.n_mod; m += warps) {
        AsmMod &M = P.mod[m];
        const unsigned long long a = P.text_off[m], b = P.text_off[m + 1];
        const bool fits = !c.bad_offsets && (long long)b <= c.ls_limit;
        long long f = 0, e = 0;
        if (!c.bad_offsets && a < b) {          // the stored lines of every module get their module
            f = lower_bound_ls(P.ls, stored, a);
            e = lower_bound_ls(P.ls, stored, b);
        }
        if (lane == 0) {
            M.first_line = f;
            M.end_line = e;
            M.flags = fits ? MF_FIT_LINES : 0u;
        }
        for (long long l = f + lane; l < e; l += 32) P.lmod[l] = m;
    }
}

// ---------------------------------------------------------------------------
// the line walker
// ---------------------------------------------------------------------------
enum { M_MEASURE = 0, M_NAMES = 1, M_TYPES = 2, M_CONST = 3, M_EMIT = 4 };
enum : uint32_t { E_SYNTAX = SPV_ASM_SYNTAX };

struct Tok { uint32_t b, n; bool open; };

__device__ __forceinline__ bool next_tok(const uint8_t *s, uint32_t n, uint32_t &i, Tok &t)
{
    while (i < n && s[i] == ' ') i++;
    if (i >= n) return false;
    const uint32_t b = i;
    bool open = false;
    if (s[i] == '"') {
        i++;
        while (i < n && s[i] != '"') i += s[i] == '\\' ? 2u : 1u;
        if (i >= n) { open = true; i = n; }
        else i++;
    } else {
        while (i < n && s[i] != ' ') i++;
    }
    t.b = b; t.n = i - b; t.open = open;
    return true;
}
__device__ __forceinline__ bool more_toks(const uint8_t *s, uint32_t n, uint32_t i)
{
    while (i < n && s[i] == ' ') i++;
    return i < n;
}

// name hash of a named id token (24 bits kept in the slot key)
__device__ __forceinline__ uint32_t tok_hash(const uint8_t *s, uint32_t n)
{
    uint32_t h = FNV0;
    for (uint32_t k = 0; k < n; k++) h = (h ^ s[k]) * FNVP;
    return h;
}

struct Walk {
    // line
    const uint8_t *s;
    uint32_t n;
    unsigned long long pos;         // text position of s[0]
    // module and tables
    AsmMod *M;
    const uint8_t *text, *mod_end;  // the text; one past the module's last byte
    unsigned long long *arena, *occ_slot, *occ_pos;
    long long rel;                  // line number in the module, from 0
    // cursor and results
    uint32_t i;
    uint32_t words;
    uint32_t named;                 // named-id tokens so far on this line
    uint32_t max_explicit;
    uint32_t first_lit;             // value of the first literal operand
    bool have_lit;
    uint8_t flags;                  // LF_*
    bool w64;                       // the constant's type is 64 bits wide (CONST, EMIT)
    // occurrences of this line start here (NAMES, TYPES, CONST, EMIT)
    unsigned long long occ;
    // output (EMIT); the line's slot (MEASURE, CONST)
    uint32_t *out;
    long long out_at, out_cap;
    uint32_t *slot;
};

template <int MODE>
__device__ __forceinline__ void put(Walk &w, uint32_t v)
{
    if (MODE == M_EMIT) {
        const long long at = w.out_at + w.words;
        if (at < w.out_cap) w.out[at] = v;
    }
    if (MODE == M_MEASURE || MODE == M_CONST) {
        if (w.words < SLOT_WORDS) w.slot[w.words] = v;
    }
    w.words++;
}

// insert a named id token into the module's hash table; returns the slot
__device__ unsigned long long name_insert(Walk &w, const uint8_t *t, uint32_t n, unsigned long long tpos)
{
    unsigned long long *tab = w.arena + w.M->names_at;
    const unsigned long long cap = (unsigned long long)w.M->names_cap;
    const uint32_t h = tok_hash(t, n);
    const unsigned long long key = ((unsigned long long)(h >> 8) << 40) | (tpos + 1);
    unsigned long long i = h % cap;
    for (unsigned long long probes = 0; probes < cap; probes++, i = i + 1 == cap ? 0 : i + 1) {
        unsigned long long k = tab[2 * i];
        if (k == 0) {
            k = atomicCAS(&tab[2 * i], 0ull, key);
            if (k == 0) { atomicMin(&tab[2 * i + 1], tpos); return i; }
        }
        if ((k >> 40) != (key >> 40)) continue;
        // same hash bits: compare the bytes with the token at the slot's position
        const uint8_t *o = w.text + ((k & ((1ull << 40) - 1)) - 1);
        bool same = true;
        for (uint32_t j = 0; j < n && same; j++) same = o + j < w.mod_end && o[j] == t[j];
        if (same && o + n < w.mod_end && o[n] != ' ' && o[n] != '\n') same = false;
        if (same) { atomicMin(&tab[2 * i + 1], tpos); return i; }
    }
    return ~0ull;       // cannot happen: the table has more slots than occurrences
}

// resolve an id token; false if it is not one
template <int MODE>
__device__ bool take_id(Walk &w, const Tok &t, uint32_t &id)
{
    const uint8_t *s = w.s + t.b;
    const int c = classify_id(s, t.n, id);
    if (c < 0) return false;
    if (c == 0) {
        if (MODE == M_MEASURE && id > w.max_explicit) w.max_explicit = id;
        return true;
    }
    const unsigned long long k = w.occ + w.named++;
    if (MODE == M_MEASURE) { id = 0; return true; }
    if (MODE == M_NAMES) {
        const unsigned long long slot = name_insert(w, s, t.n, w.pos + t.b);
        if (slot == ~0ull) {            // a full table (cannot happen: it has more slots than occurrences)
            atomicMin(&w.M->err, ((unsigned long long)w.rel << 8) | E_SYNTAX);
            return false;
        }
        w.occ_slot[k] = (unsigned long long)w.M->names_at + 2 * slot;
        w.occ_pos[k] = w.pos + t.b;
        id = 0;
        return true;
    }
    id = (uint32_t)w.arena[w.occ_slot[k]];            // the fresh id (written over the key by the ranking)
    return true;
}

__device__ bool type_w64(const Walk &w, uint32_t id)
{
    const AsmMod &M = *w.M;
    if (M.types_cap == 0) return false;
    const unsigned long long *tab = w.arena + M.types_at;
    const unsigned long long cap = (unsigned long long)M.types_cap;
    unsigned long long i = (id * 2654435761u) % cap;
    for (unsigned long long probes = 0; probes < cap; probes++, i = i + 1 == cap ? 0 : i + 1) {
        const unsigned long long k = tab[2 * i];
        if (k == 0) return false;
        if (k == (unsigned long long)id + 1) return tab[2 * i + 1] & 1ull;
    }
    return false;
}

__device__ void type_insert(const Walk &w, uint32_t id, bool is_float, bool w64, long long line)
{
    unsigned long long *tab = w.arena + w.M->types_at;
    const unsigned long long cap = (unsigned long long)w.M->types_cap;
    const unsigned long long val = ((unsigned long long)line << 2) | (is_float ? 2ull : 0ull) | (w64 ? 1ull : 0ull);
    unsigned long long i = (id * 2654435761u) % cap;
    for (unsigned long long probes = 0; probes < cap; probes++, i = i + 1 == cap ? 0 : i + 1) {
        unsigned long long k = tab[2 * i];
        if (k == 0) k = atomicCAS(&tab[2 * i], 0ull, (unsigned long long)id + 1);
        if (k == 0 || k == (unsigned long long)id + 1) { atomicMin(&tab[2 * i + 1], val); return; }
    }
}

// a string token: bytes, NUL, zero padding
template <int MODE>
__device__ bool take_string(Walk &w, const Tok &t)
{
    if (t.n < 2 || w.s[t.b] != '"' || t.open) return false;
    const uint8_t *b = w.s + t.b + 1;
    const uint32_t n = t.n - 2;
    uint32_t i = 0, acc = 0, k = 0;
    while (i < n) {
        uint32_t ch = b[i];
        if (ch == '\\') {
            int h1, h2;
            if (i + 3 < n && b[i + 1] == 'x' && (h1 = hexv(b[i + 2])) >= 0 && (h2 = hexv(b[i + 3])) >= 0) {
                ch = (uint32_t)(h1 * 16 + h2);
                i += 4;
            } else {
                if (i + 1 >= n) return false;
                ch = b[i + 1];
                i += 2;
            }
        } else {
            i++;
        }
        if (MODE == M_EMIT || MODE == M_MEASURE || MODE == M_CONST) acc |= ch << (8 * k);
        if (++k == 4) { put<MODE>(w, acc); acc = 0; k = 0; }
    }
    put<MODE>(w, acc);
    return true;
}

template <int MODE>
__device__ bool take_lit(Walk &w, const Tok &t)
{
    uint64_t v;
    if (!dec_u64(w.s + t.b, t.n, 0xffffffffull, v)) return false;
    if (!w.have_lit) { w.have_lit = true; w.first_lit = (uint32_t)v; }
    put<MODE>(w, (uint32_t)v);
    return true;
}

// OpConstant's value (context-dependent literal)
template <int MODE>
__device__ bool take_ctx(Walk &w, const Tok &t)
{
    if (more_toks(w.s, w.n, w.i)) {         // two or more tokens: one word each
        Tok u = t;
        do {
            if (!take_lit<MODE>(w, u)) return false;
        } while (next_tok(w.s, w.n, w.i, u));
        return true;
    }
    const uint8_t *s = w.s + t.b;
    uint64_t v;
    if (dec_u64(s, t.n, ~0ull, v)) {
        if (MODE == M_MEASURE) { w.flags |= LF_CONST1; put<MODE>(w, 0); return true; }
        put<MODE>(w, (uint32_t)v);
        if (w.w64 || (v >> 32)) put<MODE>(w, (uint32_t)(v >> 32));
        return true;
    }
    if (MODE != M_EMIT && MODE != M_CONST) {
        if (!float_literal<false>(s, t.n, nullptr)) return false;
        if (MODE == M_MEASURE) w.flags |= LF_CONST1;
        put<MODE>(w, 0);
        return true;
    }
    uint64_t bits;
    if (!float_literal<true>(s, t.n, &bits)) return false;
    if (w.w64) { put<MODE>(w, (uint32_t)bits); put<MODE>(w, (uint32_t)(bits >> 32)); }
    else put<MODE>(w, double_to_float_bits(bits));
    return true;
}

template <int MODE, int DEPTH>
__device__ bool take_operand(Walk &w, uint8_t code);

// a value-enum (kind < 16) or bit-enum (16 + kind) operand and its parameters
template <int MODE, int DEPTH>
__device__ bool take_enum(Walk &w, int kind, const Tok &t)
{
    const uint8_t *s = w.s + t.b;
    uint64_t v64;
    uint32_t v = 0;
    if (dec_u64(s, t.n, 0xffffffffull, v64)) {
        v = (uint32_t)v64;
    } else if (kind < 16) {
        const int e = find_en(kind, s, t.n);
        if (e < 0) return false;
        v = (uint32_t)e;
    } else if (t.n == 4 && s[0] == 'N' && s[1] == 'o' && s[2] == 'n' && s[3] == 'e') {
        v = 0;
    } else {
        uint32_t a = 0, b = 0;
        for (;;) {
            while (b < t.n && s[b] != '|') b++;
            const int e = find_en(kind, s + a, b - a);
            if (e < 0) return false;
            v |= 1u << e;
            if (b == t.n) break;
            a = ++b;
        }
    }
    put<MODE>(w, v);
    if constexpr (DEPTH >= 2) {
        return true;                        // parameters of parameters are never enums with parameters
    } else {
    if (kind < 16) {
        const spvt::EnDesc *d = v < 64 && g_spv_tables.venum[kind][v].known ? &g_spv_tables.venum[kind][v] : nullptr;
        if (d) {
            for (int k = 0; k < d->nparam; k++)
                if (!take_operand<MODE, DEPTH + 1>(w, d->param[k])) return false;
        } else if (g_spv_tables.vunknown[kind] != spvt::A_END) {
            if (!take_operand<MODE, DEPTH + 1>(w, g_spv_tables.vunknown[kind])) return false;
        }
        return true;
    }
    for (int bit = 0; bit < 32; bit++) {
        if (!((v >> bit) & 1u)) continue;
        const spvt::EnDesc &d = g_spv_tables.benum[kind - 16][bit];
        if (!d.known) continue;
        for (int k = 0; k < d.nparam; k++)
            if (!take_operand<MODE, DEPTH + 1>(w, d.param[k])) return false;
    }
    return true;
    }
}

template <int MODE, int DEPTH>
__device__ bool take_operand(Walk &w, uint8_t code)
{
    const bool opt = code & spvt::A_OPT;
    const uint8_t c = code & (uint8_t)~spvt::A_OPT;
    Tok t;
    if (c == spvt::A_IDS || c == spvt::A_IDPAIRS) {
        uint32_t id;
        while (next_tok(w.s, w.n, w.i, t)) {
            if (!take_id<MODE>(w, t, id)) return false;
            put<MODE>(w, id);
        }
        return true;
    }
    if (c == spvt::A_LITS) {
        while (next_tok(w.s, w.n, w.i, t))
            if (!take_lit<MODE>(w, t)) return false;
        return true;
    }
    if (!next_tok(w.s, w.n, w.i, t)) return opt;
    switch (c) {
    case spvt::A_ID: {
        uint32_t id;
        if (!take_id<MODE>(w, t, id)) return false;
        put<MODE>(w, id);
        return true;
    }
    case spvt::A_LIT: return take_lit<MODE>(w, t);
    case spvt::A_STR: return take_string<MODE>(w, t);
    case spvt::A_CTX: return take_ctx<MODE>(w, t);
    default:
        if (c >= spvt::A_BITS) return take_enum<MODE, DEPTH>(w, 16 + (c - spvt::A_BITS), t);
        if (c >= spvt::A_ENUM) return take_enum<MODE, DEPTH>(w, c - spvt::A_ENUM, t);
        return false;
    }
}

// The start of an instruction line: the first token, whether it is a
// "%r =" result id, the opcode-name token and its opcode (-1 if no name of
// the table). False if the line has no token.
struct Prefix { Tok t0, nm; int op; bool has_rid; };
__device__ bool line_prefix(const uint8_t *s, uint32_t n, Prefix &p)
{
    uint32_t i = 0;
    if (!next_tok(s, n, i, p.t0)) return false;
    p.has_rid = false;
    uint32_t k = i;
    Tok t1;
    if (s[p.t0.b] == '%' && next_tok(s, n, k, t1) && t1.n == 1 && s[t1.b] == '=' && more_toks(s, n, k)) {
        p.has_rid = true;
        next_tok(s, n, k, p.nm);
    } else {
        p.nm = p.t0;
    }
    p.op = find_op(s + p.nm.b, p.nm.n);
    return true;
}
// packed in 64 bits for lines whose prefix positions are below 2048
__device__ __forceinline__ unsigned long long pack_prefix(const Prefix &p, bool ok)
{
    if (!ok) return 1ull << 10;                        // no token
    if ((p.t0.b | p.t0.n | p.nm.b | p.nm.n) >= 2048u) return 0;   // not packed
    return (unsigned long long)(p.op + 1) | ((unsigned long long)p.has_rid << 9) | (3ull << 10) |
           ((unsigned long long)p.t0.b << 12) | ((unsigned long long)p.t0.n << 23) |
           ((unsigned long long)p.nm.b << 34) | ((unsigned long long)p.nm.n << 45);
}
__device__ __forceinline__ void unpack_prefix(unsigned long long v, Prefix &p)
{
    p.op = (int)(v & 511) - 1;
    p.has_rid = (v >> 9) & 1;
    p.t0.b = (uint32_t)(v >> 12) & 2047; p.t0.n = (uint32_t)(v >> 23) & 2047; p.t0.open = false;
    p.nm.b = (uint32_t)(v >> 34) & 2047; p.nm.n = (uint32_t)(v >> 45) & 2047; p.nm.open = false;
}

// Walk one instruction line. Returns 0 or E_SYNTAX. In EMIT, words_total is
// the line's word count (known from the scan). pre: the line's prefix when
// already known.
template <int MODE>
__device__ uint32_t walk_line(Walk &w, long long line, uint32_t words_total, const Prefix *pre = nullptr)
{
    const uint8_t *s = w.s;
    const uint32_t n = w.n;
    w.i = 0; w.words = 0; w.named = 0; w.flags = 0; w.have_lit = false; w.first_lit = 0;
    Prefix px;
    if (pre) px = *pre;
    else if (!line_prefix(s, n, px)) return E_SYNTAX;
    const Tok t0 = px.t0, nm = px.nm;
    const bool has_rid = px.has_rid;
    const int op = px.op;
    uint32_t i = nm.b + nm.n;
    uint32_t opn;
    if (op >= 0) {
        opn = (uint32_t)op;
    } else {
        uint64_t v;
        if (nm.n < 3 || s[nm.b] != 'O' || s[nm.b + 1] != 'p' || !dec_u64(s + nm.b + 2, nm.n - 2, 0xffff, v))
            return E_SYNTAX;
        opn = (uint32_t)v;
    }
    put<MODE>(w, MODE == M_EMIT ? (words_total << 16) | opn : 0u);
    Tok f;
    uint32_t v;
    {
        uint32_t k = i;
        const bool hasf = next_tok(s, n, k, f);
        if (op < 0 || (hasf && raw_word(s + f.b, f.n, v))) {
            if (has_rid) return E_SYNTAX;
            while (next_tok(s, n, i, f)) {
                if (!raw_word(s + f.b, f.n, v)) return E_SYNTAX;
                put<MODE>(w, v);
            }
            if (w.words > 65535) return E_SYNTAX;
            if (MODE == M_MEASURE || MODE == M_CONST) w.slot[0] = (w.words << 16) | opn;
            return 0;
        }
    }
    const spvt::OpDesc &d = g_spv_tables.ops[op];
    w.i = i;
    uint32_t rid = 0, rtype = 0;
    if (has_rid && !take_id<MODE>(w, t0, rid)) return E_SYNTAX;
    if (d.flags & 2) {
        if (!next_tok(s, n, w.i, f) || !take_id<MODE>(w, f, rtype)) return E_SYNTAX;
        put<MODE>(w, rtype);
        if (MODE == M_CONST) w.w64 = type_w64(w, rtype);
    }
    if (d.flags & 4) {
        if (!has_rid) return E_SYNTAX;
        put<MODE>(w, rid);
    } else if (has_rid) {
        return E_SYNTAX;
    }
    for (int k = 0; k < d.nprog; k++)
        if (!take_operand<MODE, 0>(w, d.prog[k])) return E_SYNTAX;
    if (more_toks(s, n, w.i)) return E_SYNTAX;
    if (w.words > 65535) return E_SYNTAX;
    if ((opn == 21 || opn == 22) && w.have_lit) {
        if (MODE == M_MEASURE) w.flags |= LF_TYPEDECL;
        if (MODE == M_TYPES) type_insert(w, rid, opn == 22, w.first_lit == 64, line);
    }
    if (MODE == M_MEASURE || MODE == M_CONST) w.slot[0] = (w.words << 16) | opn;
    return 0;
}

// ---------------------------------------------------------------------------
// header comment lines
// ---------------------------------------------------------------------------
__device__ bool scan_num(const uint8_t *s, uint32_t n, uint32_t &i, int base, uint64_t max, uint64_t &v)
{
    const uint32_t b = i;
    uint64_t a = 0;
    while (i < n) {
        const int d = hexv(s[i]);
        if (d < 0 || d >= base) break;
        a = a * (uint64_t)base + (uint64_t)d;
        if (a > max) return false;
        i++;
    }
    if (i == b) return false;
    v = a;
    return true;
}
__device__ bool prefix(const uint8_t *s, uint32_t n, const char *p, uint32_t &i)
{
    uint32_t k = 0;
    while (p[k]) {
        if (k >= n || s[k] != (uint8_t)p[k]) return false;
        k++;
    }
    i = k;
    return true;
}
// field 0..3 (version, generator, bound, schema) and value, or -1
__device__ int header_line(const uint8_t *s, uint32_t n, uint32_t &value)
{
    uint32_t i;
    uint64_t a, c;
    if (prefix(s, n, "; Version: ", i)) {
        if (scan_num(s, n, i, 10, 255, a) && i < n && s[i] == '.') {
            i++;
            if (scan_num(s, n, i, 10, 255, c) && i == n) { value = (uint32_t)((a << 16) | (c << 8)); return 0; }
        }
        return -1;
    }
    if (prefix(s, n, "; Generator: 0x", i)) {
        if (scan_num(s, n, i, 16, 0xffffffffull, a) && i == n) { value = (uint32_t)a; return 1; }
        return -1;
    }
    if (prefix(s, n, "; Bound: ", i)) {
        if (scan_num(s, n, i, 10, 0xffffffffull, a) && i == n) { value = (uint32_t)a; return 2; }
        return -1;
    }
    if (prefix(s, n, "; Schema: ", i)) {
        if (scan_num(s, n, i, 10, 0xffffffffull, a) && i == n) { value = (uint32_t)a; return 3; }
        return -1;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// per-line passes
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool module_ready(const AsmMod &M, uint32_t need)
{
    return (M.flags & need) == need && M.err == ~0ull;
}

// One line in one mode. sline: the line's bytes staged in shared memory,
// or null to read them from the text.
template <int MODE>
__device__ __forceinline__ void parse_line(const AsmP &P, long long l, const uint8_t *sline)
{
    if (MODE == M_NAMES && P.lnm[l] == 0) return;
    if (MODE == M_TYPES && !(P.lfl[l] & LF_TYPEDECL)) return;
    if (MODE == M_CONST && !(P.lfl[l] & LF_CONST1)) return;
    if (MODE == M_EMIT && ((P.lfl[l] & LF_SLOT) || P.lw[l] == 0)) return;   // k_asm_copy writes slot lines
    if (MODE == M_MEASURE) { P.lw[l] = 0; P.lnm[l] = 0; P.lfl[l] = 0; }
    const int m = P.lmod[l];
    AsmMod &M = P.mod[m];
    if (MODE == M_MEASURE) {
        if (!(M.flags & MF_FIT_LINES)) return;
    } else {
        if (!module_ready(M, MF_FIT_LINES | MF_FIT_OCC | MF_FIT_ARENA)) return;
    }
    const unsigned long long q = P.ls[l];
    const unsigned long long mend = P.text_off[m + 1];
    unsigned long long e = l + 1 < M.end_line ? P.ls[l + 1] - 1 : mend;
    if (l + 1 >= M.end_line && e > q && P.text[e - 1] == '\n') e--;
    const long long rel = l - M.first_line;
    if (e == q) return;
    if (e - q >= (1ull << 31)) {
        if (MODE == M_MEASURE) atomicMin(&M.err, ((unsigned long long)rel << 8) | E_SYNTAX);
        return;
    }
    Walk w;
    w.s = sline ? sline : P.text + q; w.n = (uint32_t)(e - q); w.pos = q;
    w.M = &M; w.text = P.text; w.mod_end = P.text + mend; w.rel = rel;
    w.arena = P.arena; w.occ_slot = P.occ_slot; w.occ_pos = P.occ_pos;
    w.max_explicit = 0; w.w64 = false; w.occ = 0; w.out = nullptr; w.out_at = 0; w.out_cap = 0;
    w.slot = P.lslot + (size_t)SLOT_WORDS * l;
    if (w.s[0] == ';') {
        if (MODE == M_MEASURE) {
            uint32_t value;
            const int f = header_line(w.s, w.n, value);
            if (f >= 0) atomicMax(&M.hdr[f], ((unsigned long long)(rel + 1) << 32) | value);
        }
        return;
    }
    if (MODE != M_MEASURE) w.occ = P.occ_off[l];
    if (MODE == M_EMIT) {
        w.w64 = (P.lfl[l] & LF_W64) != 0;
        w.out = P.words; w.out_cap = P.words_cap;
        w.out_at = (long long)P.lwo[l] + (long long)P.moff[m];
    }
    const uint32_t st = walk_line<MODE>(w, rel, MODE == M_EMIT ? P.lw[l] : 0u);
    if (MODE == M_MEASURE) {
        if (st) {
            atomicMin(&M.err, ((unsigned long long)rel << 8) | st);
            return;
        }
        uint8_t fl = w.flags;
        if (w.words <= SLOT_WORDS && w.named == 0 && !(fl & LF_CONST1)) fl |= LF_SLOT;
        P.lw[l] = w.words;
        P.lnm[l] = w.named;
        P.lfl[l] = fl;
        if (w.max_explicit > 0) atomicMax(&M.max_explicit, w.max_explicit);
        if (w.flags & LF_TYPEDECL) atomicAdd(&M.n_types, 1u);
    } else if (MODE == M_CONST) {
        P.lw[l] = w.words;
        uint8_t fl = P.lfl[l];
        if (w.w64) fl |= LF_W64;
        if (w.words <= SLOT_WORDS) fl |= LF_SLOT;
        P.lfl[l] = fl;
    }
}

// the words the measuring (or constant) pass recorded in each line's slot
__global__ void __launch_bounds__(256) k_asm_copy(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    const long long nl = c.n_lines < P.line_cap ? c.n_lines : P.line_cap;
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < nl;
         l += (long long)gridDim.x * blockDim.x) {
        if (!(P.lfl[l] & LF_SLOT)) continue;
        const int m = P.lmod[l];
        if (P.status[m] != SPV_ASM_OK) continue;
        const long long at = (long long)P.lwo[l] + (long long)P.moff[m];
        const uint32_t n = P.lw[l];
        const uint4 *sl = reinterpret_cast<const uint4 *>(P.lslot + (size_t)SLOT_WORDS * l);
        const uint4 x = sl[0], y = n > 4 ? sl[1] : make_uint4(0, 0, 0, 0);
        const uint32_t v[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
        #pragma unroll
        for (uint32_t k = 0; k < 8; k++)
            if (k < n && at + k < P.words_cap) P.words[at + k] = v[k];
    }
}

// the passes after the measuring one: the lines of the special list
template <int MODE>
__global__ void __launch_bounds__(256) k_asm_parse(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    if (MODE == M_NAMES && c.n_occ == 0) return;
    const long long n = c.n_special < P.line_cap ? c.n_special : P.line_cap;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        parse_line<MODE>(P, (long long)P.special[k], nullptr);
}

// The measuring pass by tiles of MT_LINES consecutive lines: the tile's text
// is staged in shared memory; each line's prefix (result id, opcode name) is
// read once, and the lines are sorted by the text shape of their opcode, so
// that a warp takes lines that walk the same code; each line's words are
// recorded in shared memory and written to its slot as whole 32-byte
// sectors.
constexpr int MT_THREADS = 256, MT_LINES = 1024, MT_TEXT = 44 * 1024, MT_KEYS = 256;
struct MTSmem {
    alignas(16) uint8_t text[MT_TEXT];
    alignas(16) uint32_t slot[MT_THREADS][SLOT_WORDS];
    unsigned long long pre[MT_LINES];    // packed prefix (0: not packed); then the packed outputs
    int32_t mod[MT_LINES];               // the line's module; -1: its module does not fit, or an empty line
    uint32_t qoff[MT_LINES];             // line start - the tile's first line start
    uint16_t perm[MT_LINES];
    uint16_t len[MT_LINES];              // line length; 0xffff: longer
    uint8_t key[MT_LINES];
    uint32_t hist[MT_KEYS];
};

// returns the line's packed outputs: words | named << 20 | flags << 40; the
// largest explicit id goes to max_explicit
// (the line's module fits the line capacity and the line is not empty)
__device__ __forceinline__ unsigned long long measure_line(const AsmP &P, long long l, int m, unsigned long long q,
                                                           const uint8_t *s, uint32_t n, const Prefix *pre,
                                                           uint32_t *sslot, uint32_t &max_explicit)
{
    AsmMod &M = P.mod[m];
    uint32_t lw = 0, lnm = 0;
    uint8_t fl = 0;
    max_explicit = 0;
    {
        if (s[0] == ';') {
            uint32_t value;
            const int f = header_line(s, n, value);
            if (f >= 0) atomicMax(&M.hdr[f], ((unsigned long long)(l - M.first_line + 1) << 32) | value);
        } else {
            Walk w;
            w.s = s; w.n = n; w.pos = q;
            w.M = &M; w.text = P.text; w.mod_end = nullptr; w.rel = 0;
            w.arena = P.arena; w.occ_slot = P.occ_slot; w.occ_pos = P.occ_pos;
            w.max_explicit = 0; w.w64 = false; w.occ = 0; w.out = nullptr; w.out_at = 0; w.out_cap = 0;
            w.slot = sslot;
            const uint32_t st = walk_line<M_MEASURE>(w, 0, 0u, pre);
            if (st) {
                atomicMin(&M.err, ((unsigned long long)(l - M.first_line) << 8) | st);
            } else {
                fl = w.flags;
                lw = w.words;
                lnm = w.named;
                if (w.words <= SLOT_WORDS && w.named == 0 && !(fl & LF_CONST1)) {
                    fl |= LF_SLOT;
                    uint4 *g = reinterpret_cast<uint4 *>(P.lslot + (size_t)SLOT_WORDS * l);
                    const uint4 *a = reinterpret_cast<const uint4 *>(sslot);
                    g[0] = a[0];
                    g[1] = a[1];
                }
                max_explicit = w.max_explicit;
                if (w.flags & LF_TYPEDECL) atomicAdd(&M.n_types, 1u);
            }
        }
    }
    return (unsigned long long)lw | ((unsigned long long)lnm << 20) | ((unsigned long long)fl << 40);
}


// one 16-byte asynchronous copy from global to shared memory (both
// addresses 16-byte aligned), completed by cp.async.wait_all
__device__ __forceinline__ void stage16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__global__ void __launch_bounds__(MT_THREADS, 3) k_asm_measure(AsmP P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MTSmem &S = *reinterpret_cast<MTSmem *>(smem_raw);
    const AsmCtrl &c = *P.ctrl;
    if (c.bad_offsets) return;
    const long long nl = c.n_lines < P.line_cap ? c.n_lines : P.line_cap;
    const long long ntiles = (nl + MT_LINES - 1) / MT_LINES;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long l0 = t * MT_LINES;
        const int nt = (int)(nl - l0 < MT_LINES ? nl - l0 : MT_LINES);
        const long long a = (long long)P.ls[l0];
        const long long e = l0 + nt < nl ? (long long)P.ls[l0 + nt] : c.t1;
        const long long a_al = a - (long long)(((uintptr_t)P.text + (uintptr_t)a) & 15u);
        const long long se = e < a_al + MT_TEXT ? e : a_al + MT_TEXT;     // bytes [a, se) staged
        for (long long k = threadIdx.x; a_al + 16 * k < se; k += MT_THREADS) {
            const long long g = a_al + 16 * k;
            if (g >= a && g + 16 <= se) {
                stage16(S.text + 16 * k, P.text + g);      // one round trip for the whole tile
            } else {
                for (int j = 0; j < 16; j++) {
                    const long long q = g + j;
                    if (q >= a && q < se) S.text[16 * k + j] = P.text[q];
                }
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        for (int i = threadIdx.x; i < MT_KEYS; i += MT_THREADS) S.hist[i] = 0;
        __syncthreads();
        // each line's length (up to the next line start, less its '\n'),
        // prefix and key: 0 comments and empty lines, 1 unknown names, else
        // the opcode's shape
        for (int i = threadIdx.x; i < nt; i += MT_THREADS) {
            const long long q = (long long)P.ls[l0 + i];
            long long qe = i + 1 < nt ? (long long)P.ls[l0 + i + 1] : e;
            if (qe > q && (qe <= se ? S.text[qe - 1 - a_al] : P.text[qe - 1]) == '\n') qe--;
            const long long n = qe - q;
            const int m = P.lmod[l0 + i];
            const bool live = n > 0 && (P.mod[m].flags & MF_FIT_LINES);
            uint32_t key = 0;
            unsigned long long pk = 0;
            if (!live) {
            } else if (qe <= se && S.text[q - a_al] != ';') {
                Prefix px;
                const bool ok = line_prefix(S.text + (q - a_al), (uint32_t)n, px);
                pk = pack_prefix(px, ok);
                key = !ok || px.op < 0 ? 1u : g_spv_tables.shape[px.op];
            } else if (qe > se) {
                key = 1;
            }
            S.len[i] = (uint16_t)(n < 0xffff ? n : 0xffff);
            S.pre[i] = pk;
            S.mod[i] = live ? m : -1;
            S.qoff[i] = q - a < 0xffffffffll ? (uint32_t)(q - a) : 0xffffffffu;   // else read again
            S.key[i] = (uint8_t)key;
            atomicAdd(&S.hist[key], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {                      // exclusive scan of the histogram, one warp
            const int lane = threadIdx.x;
            uint32_t v[MT_KEYS / 32], sum = 0;
            #pragma unroll
            for (int k = 0; k < MT_KEYS / 32; k++) { v[k] = S.hist[lane * (MT_KEYS / 32) + k]; sum += v[k]; }
            uint32_t x = sum;
            #pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += y;
            }
            uint32_t pre = x - sum;
            #pragma unroll
            for (int k = 0; k < MT_KEYS / 32; k++) { S.hist[lane * (MT_KEYS / 32) + k] = pre; pre += v[k]; }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += MT_THREADS) S.perm[atomicAdd(&S.hist[S.key[i]], 1u)] = (uint16_t)i;
        __syncthreads();
        for (int j = threadIdx.x; j < nt; j += MT_THREADS) {
            const int i = S.perm[j];
            const long long l = l0 + i;
            const int m = S.mod[i];
            if (m < 0) {                                  // empty, or its module does not fit
                S.pre[i] = 0;
                continue;
            }
            const long long q = S.qoff[i] != 0xffffffffu ? a + S.qoff[i] : (long long)P.ls[l];
            long long n = S.len[i];
            if (n == 0xffff) {
                long long qe = i + 1 < nt ? (long long)P.ls[l + 1] : e;
                if (qe > q && P.text[qe - 1] == '\n') qe--;
                n = qe - q;
            }
            uint32_t mx = 0;
            unsigned long long out = 0;
            if (n >= (1ll << 31)) {
                AsmMod &M = P.mod[m];
                if (M.flags & MF_FIT_LINES) atomicMin(&M.err, ((unsigned long long)(l - M.first_line) << 8) | E_SYNTAX);
            } else {
                const bool staged = q + n <= se;
                const unsigned long long pk = S.pre[i];
                Prefix px;
                const Prefix *pre = nullptr;
                if (staged && (pk >> 11) & 1) { unpack_prefix(pk, px); pre = &px; }
                out = measure_line(P, l, m, (unsigned long long)q, staged ? S.text + (q - a_al) : P.text + q,
                                   (uint32_t)n, pre, S.slot[threadIdx.x], mx);
            }
            S.pre[i] = out;
            if (mx) atomicMax(&P.mod[m].max_explicit, mx);
            // lines that a later pass revisits, appended (one atomic per warp)
            const uint32_t ofl = (uint32_t)(out >> 40), olw = (uint32_t)(out & 0xfffff);
            const bool sp = (ofl & (LF_CONST1 | LF_TYPEDECL)) || ((out >> 20) & 0xfffff) || (olw && !(ofl & LF_SLOT));
            const unsigned act = __activemask();
            const unsigned b = __ballot_sync(act, sp);
            if (b) {
                const int lane = threadIdx.x & 31, leader = __ffs(b) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(reinterpret_cast<unsigned long long *>(&P.ctrl->n_special),
                                                     (unsigned long long)__popc(b));
                base = __shfl_sync(act, base, leader);
                if (sp) {
                    const unsigned long long at = base + __popc(b & ((1u << lane) - 1));
                    if ((long long)at < P.line_cap) P.special[at] = (unsigned long long)l;
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += MT_THREADS) {       // the outputs, coalesced
            const unsigned long long o = S.pre[i];
            P.lw[l0 + i] = (uint32_t)(o & 0xfffff);
            P.lnm[l0 + i] = (uint32_t)((o >> 20) & 0xfffff);
            P.lfl[l0 + i] = (uint8_t)(o >> 40);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// named ids and per-module tables
// ---------------------------------------------------------------------------
// occurrence ranges and hash-table sizes
__global__ void k_asm_modsize(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        AsmMod &M = P.mod[m];
        unsigned long long need = 0;
        if ((M.flags & MF_FIT_LINES) && !c.bad_offsets) {
            M.occ0 = (long long)P.occ_off[M.first_line];
            M.occ1 = (long long)P.occ_off[M.end_line];
            if (M.occ1 <= P.occ_cap) M.flags |= MF_FIT_OCC;
            const long long occ = M.occ1 - M.occ0;
            M.names_cap = occ ? occ + occ / 2 + 1 : 0;
            M.types_cap = M.n_types ? 2 * (long long)M.n_types + 1 : 0;
            if ((M.flags & MF_FIT_OCC) && M.err == ~0ull) need = 2ull * (M.names_cap + M.types_cap);
        }
        P.msize[m] = need;
    }
}

__global__ void k_asm_modplace(AsmP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        AsmMod &M = P.mod[m];
        const long long at = (long long)P.moff[m];
        M.names_at = at;
        M.types_at = at + 2 * M.names_cap;
        if (P.msize[m] && at + (long long)P.msize[m] <= P.arena_cap) M.flags |= MF_FIT_ARENA;
        else if (!P.msize[m]) M.flags |= MF_FIT_ARENA;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long used = (long long)P.moff[P.n_mod];
        P.ctrl->arena_used = used < P.arena_cap ? used : P.arena_cap;
        P.ctrl->need_lines = P.ctrl->n_lines;
    }
}

__global__ void k_asm_clear_arena(AsmP P)
{
    const long long n = 0 + P.ctrl->arena_used;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        P.arena[i] = (i & 1) ? ~0ull : 0ull;      // slot pairs: key 0 (empty), value ~0 (for atomicMin)
}

// first occurrence of its name?
__global__ void k_asm_first(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    const long long n = c.n_occ < P.occ_cap ? c.n_occ : P.occ_cap;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long slot = P.occ_slot[k];      // ~0: a module that was not walked
        P.occ_first[k] = slot != ~0ull && P.arena[slot + 1] == P.occ_pos[k] ? 1u : 0u;
    }
}

__global__ void k_asm_clear_occ(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    const long long n = c.n_occ < P.occ_cap ? c.n_occ : P.occ_cap;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        P.occ_slot[k] = ~0ull;
}

// the first occurrence of each name writes its fresh id over the slot key
__global__ void k_asm_rank(AsmP P)
{
    for (int m = blockIdx.x; m < P.n_mod; m += gridDim.x) {
        AsmMod &M = P.mod[m];
        if (!module_ready(M, MF_FIT_LINES | MF_FIT_OCC | MF_FIT_ARENA) || M.occ1 == M.occ0) continue;
        const unsigned long long r0 = P.occ_rank[M.occ0];
        const unsigned long long base = (unsigned long long)M.max_explicit + 1;
        for (long long k = M.occ0 + threadIdx.x; k < M.occ1; k += blockDim.x) {
            if (!P.occ_first[k]) continue;
            const unsigned long long fresh = base + (P.occ_rank[k] - r0);
            if (fresh > 0xffffffffull) {
                // the line of this occurrence
                const unsigned long long pos = P.occ_pos[k];
                const long long l = lower_bound_ls(P.ls + M.first_line, M.end_line - M.first_line, pos + 1) - 1;
                atomicMin(&M.err, ((unsigned long long)l << 8) | E_SYNTAX);
            }
            P.arena[P.occ_slot[k]] = fresh;
        }
        if (threadIdx.x == 0) M.distinct = P.occ_rank[M.occ1] - r0;
    }
}

// ---------------------------------------------------------------------------
// module results
// ---------------------------------------------------------------------------
__global__ void k_asm_modfinal(AsmP P)
{
    const AsmCtrl &c = *P.ctrl;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        AsmMod &M = P.mod[m];
        uint32_t st = SPV_ASM_OK;
        long long line = -1;
        unsigned long long nw = 0;
        if (c.bad_offsets) st = SPV_ASM_BAD_OFFSETS;
        else if (!(M.flags & MF_FIT_LINES)) st = SPV_ASM_CAPACITY;
        else if (M.err != ~0ull) { st = (uint32_t)(M.err & 255u); line = (long long)(M.err >> 8) + 1; }
        else if ((M.flags & (MF_FIT_OCC | MF_FIT_ARENA)) != (MF_FIT_OCC | MF_FIT_ARENA)) st = SPV_ASM_CAPACITY;
        else nw = 5 + (P.lwo[M.end_line] - P.lwo[M.first_line]);
        P.status[m] = st;
        if (P.err_line) P.err_line[m] = line;
        P.msize[m] = nw;
    }
}

// header words; moff[m] becomes the offset from a line's word position in
// the line scan to its place in words[]
__global__ void k_asm_head(AsmP P)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.n_mod; m += gridDim.x * blockDim.x) {
        if (P.status[m] != SPV_ASM_OK) continue;
        const AsmMod &M = P.mod[m];
        const long long at = P.word_off[m];
        P.moff[m] = (unsigned long long)(at + 5 - (long long)P.lwo[M.first_line]);
        uint32_t h[5];
        h[0] = 0x07230203u;
        h[1] = M.hdr[0] ? (uint32_t)M.hdr[0] : 0x00010200u;
        h[2] = M.hdr[1] ? (uint32_t)M.hdr[1] : 0u;
        h[3] = M.hdr[2] ? (uint32_t)M.hdr[2] : (uint32_t)((unsigned long long)M.max_explicit + M.distinct + 1);
        h[4] = M.hdr[3] ? (uint32_t)M.hdr[3] : 0u;
        for (int k = 0; k < 5; k++)
            if (at + k < P.words_cap) P.words[at + k] = h[k];
    }
}

__global__ void k_asm_need(AsmP P)
{
    AsmCtrl *c = P.ctrl;
    c->need_lines = c->n_lines;
    c->need_occ = c->n_occ;
}

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct ALayout {
    size_t ctrl, mod, bitmap, tile_cnt, tile_off, ls, lmod, lw, lnm, lfl, lslot, special, lwo, occ_off, occ_slot, occ_pos, occ_first,
        occ_rank, arena, msize, moff, sums, total;
    long long line_cap, occ_cap, arena_cap, tile_cap, bitmap_words, sums_cap;
};

ALayout alayout(int32_t n_mod, uint64_t text_bytes, int64_t line_cap, int64_t name_cap)
{
    ALayout L{};
    L.line_cap = line_cap > 0 ? line_cap : (long long)(text_bytes / 16) + n_mod + 64;
    L.occ_cap = name_cap > 0 ? name_cap : (long long)(text_bytes / 32) + 64;
    L.arena_cap = 3 * L.occ_cap + (long long)(text_bytes / 64) + 4ll * n_mod + 64;
    L.tile_cap = (long long)((text_bytes + 16) / LT_TILE) + 2;
    L.bitmap_words = (long long)((text_bytes + 16) / 32) + 2;
    long long mx = L.line_cap + 1;
    if (L.occ_cap + 1 > mx) mx = L.occ_cap + 1;
    if (L.tile_cap + 1 > mx) mx = L.tile_cap + 1;
    if (n_mod + 1 > mx) mx = n_mod + 1;
    L.sums_cap = mx / SC_TILE + 2;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    L.ctrl = take(sizeof(AsmCtrl));
    L.mod = take(sizeof(AsmMod) * (size_t)(n_mod > 0 ? n_mod : 1));
    L.bitmap = take(4 * (size_t)L.bitmap_words);
    L.tile_cnt = take(4 * (size_t)L.tile_cap);
    L.tile_off = take(8 * (size_t)(L.tile_cap + 1));
    L.ls = take(8 * (size_t)L.line_cap);
    L.lmod = take(4 * (size_t)L.line_cap);
    L.lw = take(4 * (size_t)L.line_cap);
    L.lnm = take(4 * (size_t)L.line_cap);
    L.lfl = take((size_t)L.line_cap);
    L.lslot = take(4 * (size_t)SLOT_WORDS * (size_t)L.line_cap);
    L.special = take(8 * (size_t)L.line_cap);
    L.lwo = take(8 * (size_t)(L.line_cap + 1));
    L.occ_off = take(8 * (size_t)(L.line_cap + 1));
    L.occ_slot = take(8 * (size_t)L.occ_cap);
    L.occ_pos = take(8 * (size_t)L.occ_cap);
    L.occ_first = take(4 * (size_t)L.occ_cap);
    L.occ_rank = take(8 * (size_t)(L.occ_cap + 1));
    L.arena = take(8 * (size_t)L.arena_cap);
    L.msize = take(8 * (size_t)(n_mod + 1));
    L.moff = take(8 * (size_t)(n_mod + 1));
    L.sums = take(8 * (size_t)(L.sums_cap + 1));
    L.total = o;
    return L;
}

}  // namespace

extern "C" size_t spv_asm_workspace_bytes(int32_t n_modules, uint64_t text_bytes, int64_t line_capacity,
                                          int64_t name_capacity)
{
    if (n_modules < 0 || line_capacity < 0 || name_capacity < 0) return 0;
    return alayout(n_modules, text_bytes, line_capacity, name_capacity).total;
}

extern "C" int spv_assemble_batch(const char *text, uint64_t text_bytes, const uint64_t *text_off, int32_t n_modules,
                                  uint32_t *words, int64_t words_capacity, int64_t *word_off, uint32_t *asm_status,
                                  int64_t *asm_err_line, void *workspace, size_t workspace_bytes,
                                  int64_t line_capacity, int64_t name_capacity, spv_stream_t stream)
{
    if (n_modules < 0 || !text_off || !word_off || (n_modules && !asm_status) || line_capacity < 0 ||
        name_capacity < 0 || words_capacity < 0 || (words_capacity && !words) || (text_bytes && !text))
        return SPV_E_ARG;
    const ALayout L = alayout(n_modules, text_bytes, line_capacity, name_capacity);
    if (!workspace || workspace_bytes < L.total) return SPV_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)workspace;
    if (n_modules == 0) {
        if (cudaMemsetAsync(word_off, 0, 8, st) != cudaSuccess) return SPV_E_CUDA;
        return cudaMemsetAsync(w + L.ctrl, 0, sizeof(AsmCtrl), st) == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
    }
    AsmP P{};
    P.text = (const uint8_t *)text; P.text_off = text_off; P.n_mod = n_modules; P.text_bytes = text_bytes;
    P.ctrl = (AsmCtrl *)(w + L.ctrl);
    P.mod = (AsmMod *)(w + L.mod);
    P.bitmap = (uint32_t *)(w + L.bitmap); P.bitmap_words = L.bitmap_words;
    P.tile_cap = L.tile_cap;
    P.tile_cnt = (uint32_t *)(w + L.tile_cnt); P.tile_off = (unsigned long long *)(w + L.tile_off);
    P.line_cap = L.line_cap;
    P.ls = (unsigned long long *)(w + L.ls); P.lmod = (int32_t *)(w + L.lmod);
    P.lw = (uint32_t *)(w + L.lw); P.lnm = (uint32_t *)(w + L.lnm); P.lfl = (uint8_t *)(w + L.lfl);
    P.lslot = (uint32_t *)(w + L.lslot);
    P.special = (unsigned long long *)(w + L.special);
    P.lwo = (unsigned long long *)(w + L.lwo); P.occ_off = (unsigned long long *)(w + L.occ_off);
    P.occ_cap = L.occ_cap;
    P.occ_slot = (unsigned long long *)(w + L.occ_slot); P.occ_pos = (unsigned long long *)(w + L.occ_pos);
    P.occ_first = (uint32_t *)(w + L.occ_first); P.occ_rank = (unsigned long long *)(w + L.occ_rank);
    P.arena = (unsigned long long *)(w + L.arena); P.arena_cap = L.arena_cap;
    P.msize = (unsigned long long *)(w + L.msize); P.moff = (unsigned long long *)(w + L.moff);
    P.words = words; P.words_cap = words_capacity; P.word_off = word_off;
    P.status = asm_status; P.err_line = asm_err_line;
    unsigned long long *sums = (unsigned long long *)(w + L.sums);
    AsmCtrl *c = P.ctrl;
    const long long n_mod_ll = n_modules;
    const long long *n_mod_dev = &c->n_mod;

    const int gm = grid_for(n_modules, 256);
    const long long line_work = L.line_cap;
    if (cudaMemsetAsync(c, 0, sizeof(AsmCtrl), st) != cudaSuccess) return SPV_E_CUDA;
    if (cudaMemsetAsync(P.bitmap, 0, 4 * (size_t)L.bitmap_words, st) != cudaSuccess) return SPV_E_CUDA;
    SPV_LAUNCH("k_asm_mod_init", st, k_asm_mod_init<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_setup", st, k_asm_setup<<<1, 1, 0, st>>>(P));
    SPV_LAUNCH("k_asm_mark", st, k_asm_mark<<<gm, 256, 0, st>>>(P));
    const int gt = grid_for(L.tile_cap * LT_THREADS, LT_THREADS);
    SPV_LAUNCH("k_asm_lines", st, k_asm_lines<0><<<gt, LT_THREADS, 0, st>>>(P));
    scan(P.tile_cnt, &c->n_tiles, L.tile_cap, sums, P.tile_off, &c->n_lines, st);
    SPV_LAUNCH("k_asm_lines", st, k_asm_lines<1><<<gt, LT_THREADS, 0, st>>>(P));
    SPV_LAUNCH("k_asm_modlines", st, k_asm_modlines<<<grid_for(32ll * n_modules, 256), 256, 0, st>>>(P));
    const int gl = grid_for(line_work, 256);
    {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_asm_measure, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MTSmem));
            attr = true;
        }
        const int gmt = grid_for((L.line_cap + MT_LINES - 1) / MT_LINES * MT_THREADS, MT_THREADS);
        SPV_LAUNCH("k_asm_measure", st, k_asm_measure<<<gmt, MT_THREADS, sizeof(MTSmem), st>>>(P));
    }
    // named-id occurrences per line, then per module
    const long long *lines_dev = &c->n_lines;
    scan(P.lnm, lines_dev, L.line_cap, sums, P.occ_off, &c->n_occ, st);
    SPV_LAUNCH("k_asm_modsize", st, k_asm_modsize<<<gm, 256, 0, st>>>(P));
    scan(P.msize, n_mod_dev, n_mod_ll, sums, P.moff, nullptr, st);
    SPV_LAUNCH("k_asm_modplace", st, k_asm_modplace<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_clear_arena", st, k_asm_clear_arena<<<grid_for(L.arena_cap, 256), 256, 0, st>>>(P));
    const int go = grid_for(L.occ_cap, 256);
    SPV_LAUNCH("k_asm_clear_occ", st, k_asm_clear_occ<<<go, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_names", st, k_asm_parse<M_NAMES><<<gl, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_first", st, k_asm_first<<<go, 256, 0, st>>>(P));
    scan(P.occ_first, &c->n_occ, L.occ_cap, sums, P.occ_rank, nullptr, st);
    SPV_LAUNCH("k_asm_rank", st, k_asm_rank<<<grid_for(256ll * n_modules, 256), 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_types", st, k_asm_parse<M_TYPES><<<gl, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_const", st, k_asm_parse<M_CONST><<<gl, 256, 0, st>>>(P));
    scan(P.lw, lines_dev, L.line_cap, sums, P.lwo, nullptr, st);
    SPV_LAUNCH("k_asm_modfinal", st, k_asm_modfinal<<<gm, 256, 0, st>>>(P));
    scan(P.msize, n_mod_dev, n_mod_ll, sums, (unsigned long long *)word_off, nullptr, st);
    SPV_LAUNCH("k_asm_head", st, k_asm_head<<<gm, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_copy", st, k_asm_copy<<<gl, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_emit", st, k_asm_parse<M_EMIT><<<gl, 256, 0, st>>>(P));
    SPV_LAUNCH("k_asm_need", st, k_asm_need<<<1, 1, 0, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}

extern "C" int spv_asm_required(const void *workspace, int64_t *lines, int64_t *names)
{
    if (!workspace) return SPV_E_ARG;
    AsmCtrl c;
    if (cudaMemcpy(&c, workspace, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return SPV_E_CUDA;
    if (lines) *lines = c.need_lines;
    if (names) *names = c.need_occ;
    return SPV_SUCCESS;
}
