// spv_batch.cu -- batched decode / validate / encode of SPIR-V modules.
//
// One persistent launch processes every module of a batch, split into tiles
// of T words laid on 16-byte boundaries (a module owns at least one). Each
// CTA claims tiles in order from an atomic counter and, per tile:
//   1. stages the tile (+ a halo) into shared memory with 16-byte copies;
//   2. finds instruction starts. Starts form a chain p -> p + wc(p) from
//      word 5 of the module (section 3.4.6: instructions are word-counted
//      32-bit word sequences). Every word whose opcode and word count could
//      start an instruction is a guessed start; the guess is the chain when
//      each guessed start but one is the successor of exactly one other and
//      exactly one leaves the tile. A module's first tile drops false guesses
//      (literals that read as instructions) round by round from its known
//      entry; a later tile takes its first guessed start as its entry,
//      publishes its exit and row count at once and checks the entry against
//      its predecessor's exit at the end (a wrong guess redoes the batch
//      without guesses). A tile whose guess is not a chain takes the exact
//      path: per-segment exits, warp maps, the tile map, and its entry from a
//      decoupled look-back over the predecessors' exits and maps. Waits are
//      bounded (max_spins) and end in SPV_TIMEOUT, never a hang;
//   3. re-encodes the staged words (fused path) and validates the rows
//      (section 3.4.5 rules; ids below the bound and each result id set once,
//      section 3.4.2) into per-tile aggregates, in chunks of 32 rows;
//   4. gets the tile's global first row from a second decoupled look-back
//      (sum of predecessors' counts) and writes one structure-of-arrays row
//      per instruction.
// A prepass reads headers and lays out tiles and id bitmaps; a finalize pass
// turns per-module aggregates into status codes; an exact fixup pass runs
// only for modules with a duplicate result id or a missing capability.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <vector>
#include <algorithm>
#include <mutex>

#include "../../include/spv.h"
#include "spv_device.cuh"
#include "spv_prof.h"

using namespace spvd;

namespace {

constexpr int HALO = 64;          // words staged past the tile end
static_assert(HALO >= 3, "a start's result type and id are read from the staged words");
constexpr int NCAND = 32;         // candidate entries in a tile map
constexpr uint16_t NONE16 = 0xFFFF;
constexpr unsigned long long F_MAP = 1ull << 62, F_EXIT = 2ull << 62, F_MASK = 3ull << 62;
// a tile whose guessed starts form a chain publishes, beside its map, the
// state F_FMAP: bits 0-31 mark the candidate entries that leave the tile at
// the guessed chain's exit, bits 32-49 hold that exit (tile-local), so a
// later tile entering at a marked candidate needs no map entry
constexpr unsigned long long F_FMAP = 3ull << 62;


// What a tile of k_tile needs to know about itself, one 32-byte load.
struct TileRec {
    long long base;          // the module's first word
    uint32_t m, k;           // module, tile index within the module
    uint32_t len_rel;        // the module's end, counted from the tile's first staged word (0: a module too large)
    uint32_t hdr;            // the module's header status
    uint32_t ph;             // words from the 16-byte boundary below the module's first word to that word
    uint32_t pad;
};

struct Params {
    const uint32_t *words;
    const int64_t *mod_off;
    int32_t n_modules;
    // table
    uint16_t *op; uint16_t *wc; uint64_t *off; uint32_t *rtype; uint32_t *rid; uint32_t *mod;
    int64_t *first_row; uint32_t *n_instr; int64_t cap_rows;
    uint32_t *status; int64_t *err_row;
    uint32_t *out;                 // encode target or null
    int validate, recompute_bound;
    // workspace
    Ctrl *ctrl; int64_t *tile_off; TileRec *tile_rec; unsigned long long *tstate; uint32_t *tmap;
    unsigned long long *cstate; ModState *ms; uint32_t *arena; int64_t arena_words; uint32_t *fixlist;
    int64_t *abase;                // [n_modules + 1] prefix of the id-set words each module asks for
    long long max_spins;
    long long stall_tile;          // test hook: this tile never publishes its look-back states (-1: none)
    long long stall_map_tile;      // test hook: this tile publishes its MAP state but never its map entries,
                                   // exit or row count (-1: none)
    int persistent;
    int table_mode;                // validating a caller's table: never write its columns
    int tile_words;                // words per tile of k_tile
    int out_vec;                   // out and words share their 16-byte phase: 16-byte stores
    int spec;                      // tiles may take their first guessed start as their entry
    int rerun;                     // the redo pass: every kernel returns unless a guess failed
};

// a kernel of the redo pass has nothing to do unless the first pass's entry
// guesses failed somewhere
__device__ __forceinline__ bool skip_pass(const Params &P) { return P.rerun && !P.ctrl->spec_failed; }

// words from the 16-byte boundary below word o of the batch to that word
__host__ __device__ inline uint32_t word_phase(const uint32_t *words, long long o)
{
    return (uint32_t)((((unsigned long long)(uintptr_t)words) >> 2) + (unsigned long long)o) & 3u;
}

// ---------------------------------------------------------------------------
// prepass, in two kernels: per module (many CTAs) the header status, bound,
// tile count and id-set words; then one CTA scans the counts into the tile
// and id-set layout
// ---------------------------------------------------------------------------
__global__ void k_prepass_mod(Params P, int tile_words)
{
    if (skip_pass(P)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long mm = blockIdx.x * (long long)blockDim.x + threadIdx.x; mm < P.n_modules; mm += stride) {
        const int m = (int)mm;
        unsigned long long nt = 0, nb = 0;
        uint32_t hdr = S_OK, bound = 0, flags = 0;
        long long o = P.mod_off[m], len = P.mod_off[m + 1] - o;
        if (len < 0 || len > 0x7fffffffLL) { hdr = S_CAPACITY; flags = MF_CAPACITY; len = 0; }
        else hdr = header_status(P.words + o, len);
        if (len >= 4) bound = P.words[o + 3];
        // tiles start on 16-byte boundaries: the first one also holds the
        // ph words below the module's first word
        const uint32_t ph = word_phase(P.words, o);
        nt = len > 0 ? ((unsigned long long)len + ph + (unsigned)tile_words - 1) >> (31 - __clz(tile_words)) : 1;  // tile_words: a power of two
        if (hdr == S_OK && P.validate) nb = idset_words(bound, len);
        P.tile_off[m] = (int64_t)nt;              // counts; k_prepass_scan makes them offsets
        P.abase[m] = (int64_t)nb;
        ModState st;
        st.hdr = hdr; st.bound = bound; st.err_key = NO_KEY;
        st.n_cap = st.n_mm = st.n_ep = st.n_fn = 0;
        st.decl_lo = st.decl_hi = st.req_lo = st.req_hi = 0;
        st.max_rid = 0;
        st.arena_off = -1;
        st.id_slots = 0; st.n_ids = 0; st.n_set = 0; st.pad2 = 0;
        if (hdr == S_OK && P.validate && !idset_dense(bound, len)) st.id_slots = (uint32_t)nb;
        st.flags = flags;
        P.ms[m] = st;
    }
}

__global__ void __launch_bounds__(1024) k_prepass_scan(Params P)
{
    if (skip_pass(P)) return;
    __shared__ unsigned long long s_tiles[32], s_arena[32];
    __shared__ unsigned long long s_base_tiles, s_base_arena;
    int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) { s_base_tiles = 0; s_base_arena = 0; }
    __syncthreads();
    for (int base = 0; base < P.n_modules; base += 1024) {
        int m = base + tid;
        unsigned long long nt = 0, nb = 0;
        if (m < P.n_modules) { nt = (unsigned long long)P.tile_off[m]; nb = (unsigned long long)P.abase[m]; }
        // block exclusive scan of (nt, nb)
        unsigned long long it = nt, ib = nb;
        for (int d = 1; d < 32; d <<= 1) {
            unsigned long long a = __shfl_up_sync(0xffffffffu, it, d), b = __shfl_up_sync(0xffffffffu, ib, d);
            if (lane >= d) { it += a; ib += b; }
        }
        if (lane == 31) { s_tiles[wid] = it; s_arena[wid] = ib; }
        __syncthreads();
        if (wid == 0) {
            unsigned long long a = s_tiles[lane], b = s_arena[lane];
            for (int d = 1; d < 32; d <<= 1) {
                unsigned long long x = __shfl_up_sync(0xffffffffu, a, d), y = __shfl_up_sync(0xffffffffu, b, d);
                if (lane >= d) { a += x; b += y; }
            }
            s_tiles[lane] = a; s_arena[lane] = b;
        }
        __syncthreads();
        unsigned long long wt = wid ? s_tiles[wid - 1] : 0, wb = wid ? s_arena[wid - 1] : 0;
        unsigned long long et = s_base_tiles + wt + it - nt, eb = s_base_arena + wb + ib - nb;
        if (m < P.n_modules) {
            P.tile_off[m] = (int64_t)et;
            P.abase[m] = (int64_t)eb;
            if (P.validate && P.ms[m].hdr == S_OK) {
                if ((long long)(eb + nb) <= P.arena_words) P.ms[m].arena_off = (long long)eb;
                else P.ms[m].flags |= MF_NOARENA | MF_CAPACITY;
            }
        }
        __syncthreads();
        if (tid == 1023) { s_base_tiles = et + nt; s_base_arena = eb + nb; }
        __syncthreads();
    }
    if (tid == 0) {
        P.tile_off[P.n_modules] = (int64_t)s_base_tiles;
        P.abase[P.n_modules] = (int64_t)s_base_arena;
        P.ctrl->n_tiles = s_base_tiles;
        P.ctrl->arena_used = s_base_arena < (unsigned long long)P.arena_words ? s_base_arena
                                                                              : (unsigned long long)P.arena_words;
        P.ctrl->next_tile = 0;
        P.ctrl->timeout = 0;
        P.ctrl->total_rows = 0;
        P.ctrl->n_fix = 0;
        if (!P.rerun) P.ctrl->spec_failed = 0;
    }
}

// per tile: its record (owning module and where it starts), cleared
// look-back states and map entries (0: not written); clears the id arena
__global__ void k_tile_setup(Params P)
{
    if (skip_pass(P)) return;
    unsigned long long nt = P.ctrl->n_tiles;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < (long long)nt; g += stride) {
        int lo = 0, hi = P.n_modules;              // last m with tile_off[m] <= g
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (P.tile_off[mid] <= g) lo = mid; else hi = mid;
        }
        TileRec r{};
        r.m = (uint32_t)lo;
        r.k = (uint32_t)(g - P.tile_off[lo]);
        r.base = P.mod_off[lo];
        r.hdr = P.ms[lo].hdr;
        r.ph = word_phase(P.words, r.base);
        long long lr = (P.mod_off[lo + 1] - r.base) + r.ph - (long long)r.k * P.tile_words;
        if (r.hdr == S_CAPACITY) lr = 0;
        r.len_rel = (uint32_t)(lr < 0 ? 0 : lr);
        P.tile_rec[g] = r;
        P.tstate[g] = 0;
        P.cstate[g] = 0;
        uint4 *mp = reinterpret_cast<uint4 *>(P.tmap + g * NCAND);
        #pragma unroll
        for (int i = 0; i < NCAND / 4; i++) mp[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (P.validate) {
        unsigned long long aw = P.ctrl->arena_used;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)aw; i += stride)
            P.arena[i] = 0;
    }
}

// ---------------------------------------------------------------------------
// the fused tile kernel
//
// Tiles sit on 16-byte boundaries of the word buffer: when a module's first
// word lies ph words past such a boundary, its tile k covers the module
// positions [k*T - ph, (k+1)*T - ph). Every tile, and every thread's
// segment of L words, is then staged and read with 16-byte copies. Inside a
// tile positions are tile-local (0 .. T-1); published exits and map entries
// are module positions.
//
// Instruction starts (section 3.4.6: an instruction's first word holds its
// word count) form the chain p -> p + wc(p). The kernel first guesses the
// tile's starts word by word: a word is a candidate start when its opcode is
// in the table and its word count fits that opcode's operand list. The
// guess is kept only if it is itself a chain: every candidate's successor
// is the next candidate, except one whose successor leaves the tile (counts
// of successor marks against candidates, over the whole tile). A chain that
// holds the tile's true entry gives every start from that entry on. Any
// other case (a framing error, an unknown opcode, a wrong operand count, or
// a word that merely looks like a start and breaks the chain) takes the
// exact path: per-segment exits by a backward pass, warp maps, and walks.
// ---------------------------------------------------------------------------
template <int L> __device__ __forceinline__ int pw(int i) { return i + 4 * (i / L); }   // staged word index
template <int L> __device__ __forceinline__ uint32_t pwu(uint32_t i) { return i + 4u * (i / L); }
template <int L> __device__ __forceinline__ int pe(int i) { return i + i / L; }         // exit-array index

// What validating one row needs of its opcode, in two words.
//   x: the word positions that hold ids when the row has 32 words (the fixed
//      ids, then every position of an id tail); a row of wc words takes the
//      low wc bits
//   y: bits 0-4 need (1 + fixed operand words); bits 5-10 r: the words past
//      them, d = wc - need, are valid for d < r (1: none, 32: any tail, 0:
//      only a bit-enum word with its parameters); bit 11 d must be even (id
//      pairs); bit 12 the tail is one bit-enum word (d = 1 + its parameters
//      is valid); bits 13-14 its bit-enum kind; bit 15 the fast form applies
//      (known, fixed ids / literals and a plain tail, not counted by
//      validation); bit 16 known; bit 17 has a result id; bit 18 has a
//      result type (the result id is word 2, else word 1); bits 24-31 the
//      required capability (int8, -1 none)
__host__ __device__ inline uint2 vdesc(const spvt::OpDesc &d)
{
    if (!(d.flags & 1)) return make_uint2(0u, 0u);
    uint32_t x = 0, y = (1u << 16) | ((uint32_t)(uint8_t)d.cap << 24);
    if (d.flags & 4) y |= 1u << 17;
    if (d.flags & 2) y |= 1u << 18;
    if ((d.fast & 1) && !(d.flags & 8)) {
        const uint32_t need = 1u + d.nfixed, tail = (d.fast >> 1) & 7u;
        x = d.id_mask;
        if (tail == 1 || tail == 3) x |= 0xffffffffu << need;
        const uint32_t r = tail == 0 ? 1u : tail == 4 ? ((d.fast & 16) ? 1u : 0u) : 32u;
        y |= need | (r << 5) | (tail == 3 ? 1u << 11 : 0u) | (tail == 4 ? 1u << 12 : 0u) |
             ((uint32_t)(d.bkind & 3) << 13) | (1u << 15);
    }
    return make_uint2(x, y);
}

template <int NT, int L>
struct TileSmem {
    static constexpr int T = NT * L;
    static constexpr int NW = NT / 32;
    static constexpr int TH = T + HALO;                 // staged words: the tile and its halo
    static constexpr int WPAD = TH + 4 * (TH / L);      // 4 spare words per segment: conflict-free 16-byte reads
    static constexpr int NE = T + T / L + 1;
    uint4 w4[WPAD / 4];
    uint16_t E[NE];                 // exact path: exit past each position's segment (relative); then the start list
    uint32_t fwc[257];              // per opcode: word counts a start may have, as min | (max - min + 1) << 16
    uint2 vd[257];                  // per opcode: what validating a row needs (vdesc)
    uint8_t bnp[4][16];             // per bit-enum kind and mask: literal parameters of its known bits
    uint32_t far[T / 32];           // successor marks two or more segments ahead
    uint32_t sl_hi[NW];             // each warp's last segment's marks for the next warp's first segment
    uint16_t X[NT];                 // guessed starts per segment
    uint16_t seg_entry[NT];
    uint32_t wmap[NW][32];          // per warp: exit for its 32 candidate entries
    uint32_t warp_entry[NW];
    uint32_t warp_tot[NW];
    // tile scalars
    long long tile;
    long long mod_base;
    int m;
    uint32_t k, end_s, tile_n, hdr, ph;
    uint32_t entry, exitp, exitX, cnt1, cnt2, xfirst;
    int need_exact;
    int count_pub;                  // the row count is published already
    unsigned long long row_base;
    int timeout;
    // aggregates flushed once per tile
    unsigned long long err_key;
    uint32_t n_cap, n_mm, n_ep, n_fn, decl_lo, decl_hi, req_lo, req_hi, max_rid, flags, n_ids;
    unsigned int vnext;                             // next row chunk to validate
};

// The full operand walk of row r starting at tile position p: forms with
// strings, value enums and their parameters; rows that validation counts or
// measures (capabilities, memory model, entry points, functions, integer and
// float widths); rows longer than 32 words. Returns the row's required
// capabilities and whether it inserted a result id into a bitmap. (Inlined:
// an out-of-line call measured slower, with more instruction-fetch stalls.)
struct SlowOut { uint32_t lo, hi, ins; };
template <int NT, int L>
__device__ __forceinline__ SlowOut slow_row(TileSmem<NT, L> &s, const uint32_t *src, uint32_t p, unsigned r,
                                         uint32_t bound, uint32_t *arena, long long arena_off, uint32_t id_slots)
{
    constexpr int TH = TileSmem<NT, L>::TH;
    const uint32_t *ws = reinterpret_cast<const uint32_t *>(s.w4);
    SlowOut o{0u, 0u, 0u};
    const uint32_t w0 = ws[pwu<L>(p)];
    const uint32_t op = w0 & 0xffffu, wc = w0 >> 16;
    const spvt::OpDesc &d = g_spv_tables.ops[op];          // a known opcode (< 256)
    auto iw = [&](uint32_t q) -> uint32_t {
        const uint32_t a = p + q;
        return a < (uint32_t)TH ? ws[pwu<L>(a)] : __ldg(src + a);
    };
    uint32_t ri = 0;
    if (d.flags & 4) {
        const uint32_t q = (d.flags & 2) ? 2u : 1u;
        if (q < wc) ri = iw(q);
    }
    if (d.flags & 8) {            // the few opcodes validation counts or measures
        if (op == 17) {
            atomicAdd(&s.n_cap, 1u);
            if (wc >= 2) { const uint32_t c = iw(1); if (c < 32) atomicOr(&s.decl_lo, 1u << c); else if (c < 64) atomicOr(&s.decl_hi, 1u << (c - 32)); }
        }
        else if (op == 14) atomicAdd(&s.n_mm, 1u);
        else if (op == 15) atomicAdd(&s.n_ep, 1u);
        else if (op == 54) atomicAdd(&s.n_fn, 1u);
    }
    const Walk wk = walk_instruction(iw, wc, d, bound);
    if (!wk.ok) atomicMin(&s.err_key, make_key(r, R_BADOP, 0));
    else if (wk.oob) atomicMin(&s.err_key, make_key(r, R_OOB, 0));
    else {
        if ((d.flags & 4) && arena_off >= 0) {
            if (id_slots == 0) {
                atomicOr(&arena[arena_off + (ri >> 5)], 1u << (ri & 31));
                o.ins = 1;
            } else if (idset_insert(arena + arena_off, id_slots, ri)) {
                atomicOr(&s.flags, MF_DUP);
            }
        }
        uint64_t req = wk.req;
        if (d.flags & 8) req |= width_caps(iw, op, wc);
        o.lo = (uint32_t)req;
        o.hi = (uint32_t)(req >> 32);
    }
    return o;
}

template <int NT, int L>
__global__ void __launch_bounds__(NT, 1536 / NT) k_tile(Params P)
{
    using S = TileSmem<NT, L>;
    constexpr int T = S::T;
    constexpr int NW = S::NW;
    constexpr int TH = S::TH;
    constexpr int WSPAN = 32 * L;                  // words per warp segment
    constexpr uint32_t SEGM = (1u << L) - 1u;
    constexpr uint32_t FULL = 0xffffffffu;
    static_assert(L == 8 || L == 16, "segments of 8 or 16 words");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &s = *reinterpret_cast<S *>(smem_raw);
    uint32_t *ws = reinterpret_cast<uint32_t *>(s.w4);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int lo = tid * L;
    const spvt::Tables &TB = g_spv_tables;
    if (skip_pass(P)) return;

    // per-opcode tables, once per CTA
    for (int o = tid; o < 257; o += NT) {
        uint32_t f = 0u;                           // no word count fits
        if (o < 256) {
            const spvt::OpDesc &d = TB.ops[o];
            if (d.flags & 1) {
                uint32_t mn, mx = 0xffffu;
                if (d.fast & 1) {
                    const uint32_t need = 1u + d.nfixed, tail = (d.fast >> 1) & 7u;
                    mn = need;
                    if (tail == 0) mx = need;
                    else if (tail == 4 && !(d.fast & 16)) mn = need + 1;
                } else {
                    mn = 1u + ((d.flags >> 1) & 1u) + ((d.flags >> 2) & 1u);
                }
                f = mn | ((mx - mn + 1u) << 16);
            }
            s.vd[o] = vdesc(d);
        } else {
            s.vd[o] = make_uint2(0u, 0u);          // opcodes past the table: unknown
        }
        s.fwc[o] = f;
    }
    // a bit-enum word's parameters: its known bits all lie below bit 4
    static_assert(spvt::NUM_BKINDS == 4, "bit-enum kinds");
    for (int i = tid; i < 64; i += NT) {
        const int kind = i >> 4, x = i & 15;
        uint32_t np = 0;
        for (int b = 0; b < 32; b++) {
            const spvt::EnDesc &e = TB.benum[kind][b];
            if (e.known && b < 4 && ((x >> b) & 1)) np += e.nparam;
        }
        s.bnp[kind][x] = (uint8_t)np;
    }

    // a ticket is taken only when its tile starts: tiles wait on their
    // predecessors' published states, and a ticket held while its CTA works
    // on another tile would stall every later tile of the module
    const long long n_tiles = (long long)P.ctrl->n_tiles;
    for (;;) {
        if (tid == 0) {
            const long long g0 = (long long)atomicAdd(&P.ctrl->next_tile, 1u);
            s.tile = g0;
            if (g0 < n_tiles) {
                const TileRec r = P.tile_rec[g0];
                s.m = (int)r.m; s.k = r.k; s.mod_base = r.base; s.hdr = r.hdr; s.ph = r.ph;
                s.end_s = r.len_rel;
                s.tile_n = r.len_rel < (uint32_t)T ? r.len_rel : (uint32_t)T;
                s.timeout = 0;
                s.err_key = NO_KEY;
                s.n_cap = s.n_mm = s.n_ep = s.n_fn = 0;
                s.decl_lo = s.decl_hi = s.req_lo = s.req_hi = 0;
                s.max_rid = 0; s.flags = 0; s.n_ids = 0; s.vnext = 0;
                s.cnt1 = 0; s.cnt2 = 0; s.exitX = DEAD; s.need_exact = 0; s.count_pub = 0; s.xfirst = DEAD;
            }
        }
        for (int i = tid; i < T / 32; i += NT) s.far[i] = 0u;
        __syncthreads();
        const long long g = s.tile;
        if (g >= n_tiles) break;
        const uint32_t end_s = s.end_s, tile_n = s.tile_n, k = s.k, ph = s.ph;
        const int m = s.m;
        const bool live = (s.hdr == S_OK);
        const long long tbase = s.mod_base - (long long)ph + (long long)k * T;   // word index of tile-local 0
        const uint32_t tb_rel = k * (uint32_t)T - ph;                         // its module position (k > 0)
        const uint32_t *src = P.words + tbase;
        const int lo_ok = k == 0 ? (int)ph : 0;                               // first module word of the tile

        // 1. stage the tile and its halo with 16-byte asynchronous copies (one
        //    round trip); the ragged ends of the module by smaller copies,
        //    words outside the module as zeros
        {
            const int e = (int)(end_s < (uint32_t)TH ? end_s : (uint32_t)TH);
            for (int c = tid; c < TH / 4; c += NT) {
                const int s0 = 4 * c;
                uint32_t *dst = ws + pw<L>(s0);
                if (s0 >= e) {
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
                } else if (s0 >= lo_ok) {
                    cp_async16(dst, src + s0, (uint32_t)((e - s0 < 4 ? e - s0 : 4) * 4));
                } else {
                    #pragma unroll
                    for (int q = 0; q < 4; q++) {
                        if (s0 + q >= lo_ok && s0 + q < e) cp_async4(dst + q, src + s0 + q);
                        else dst[q] = 0u;
                    }
                }
            }
            cp_async_wait_all();
        }
        __syncthreads();

        // 2. guessed starts of my segment, and where each one's successor lies;
        //    my segment's words also go straight to the encoded output
        uint32_t X = 0, sl = 0, ne = 0;
        const int n_copy = (int)(end_s < (uint32_t)T ? end_s : (uint32_t)T);   // tile-local end of the module's words
        if (P.out && P.out_vec) {
            // 5. encode: in the fused path every field an instruction writes back
            // (first word from wc/op, result type, result id) is decoded from the
            // staged words themselves, so the re-encoded tile is the staged tile;
            // the header bound is patched by the finalize pass
            uint32_t *dst = P.out + tbase;
            #pragma unroll
            for (int c = 0; c < L / 4; c++) {
                const int s0 = lo + 4 * c;
                const uint4 v = *reinterpret_cast<const uint4 *>(ws + pw<L>(s0));
                if (s0 >= lo_ok && s0 + 4 <= n_copy) {
                    *reinterpret_cast<uint4 *>(dst + s0) = v;
                } else if (s0 < n_copy && s0 + 4 > lo_ok) {
                    const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
                    #pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (s0 + q >= lo_ok && s0 + q < n_copy) dst[s0 + q] = vv[q];
                }
            }
        }
        {
            if (live) {
                if (k == 0 && tid == 0) {
                    // the module header is never a start: its staged words are
                    // cleared while this thread guesses (only it reads them here)
                    // and put back afterwards
                    #pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (j < (int)ph + 5) ws[pw<L>(j)] = 0u;
                }
                const int lim = (int)tile_n - lo;      // a successor at or past lim leaves the tile
                // a word w is a candidate when, with its opcode's entry f = min |
                // (max - min + 1) << 16, w - (min << 16) < (max - min + 1) << 16: the
                // word count lies in [min, max] (the opcode bits stay below bit 16,
                // and a count below min wraps to a value no smaller than the
                // bound). Successors in this or the next segment are marked
                // here; farther ones (long instructions, or leaving the tile) are
                // listed in `big` and settled after the loop.
                constexpr uint32_t SLM = 2 * L >= 32 ? FULL : (1u << (2 * L)) - 1u;
                uint32_t ex = 0, big = 0;
                #pragma unroll
                for (int c = 0; c < L / 4; c++) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(ws + pw<L>(lo + 4 * c));
                    const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
                    #pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int j = 4 * c + q;
                        const uint32_t w = vv[q], op = w & 0xffffu;
                        const uint32_t f = s.fwc[op < 256u ? op : 256u];
                        const uint32_t nx = (uint32_t)j + (w >> 16);
                        if (w - (f << 16) < (f & 0xffff0000u)) {
                            X |= 1u << j;
                            sl |= shl_clamp(1u, nx) & SLM;
                            if (nx >= 2u * L) big |= 1u << j;
                        }
                    }
                }
                if (lim < 2 * L) {
                    // the tile ends inside this segment or the next: successors
                    // at or past lim leave the tile instead of being marked
                    sl = 0; big = 0;
                    for (uint32_t x = X; x; x &= x - 1) {
                        const int j = __ffs(x) - 1;
                        const int nx = j + (int)(ws[pw<L>(lo + j)] >> 16);
                        if (nx >= lim) { ne++; ex = (uint32_t)(lo + nx); }
                        else if (nx < 2 * L) sl |= 1u << nx;
                        else big |= 1u << j;
                    }
                }
                while (big) {                          // successors two or more segments ahead
                    const int j = __ffs(big) - 1;
                    big &= big - 1;
                    const int nx = j + (int)(ws[pw<L>(lo + j)] >> 16);
                    if (nx >= lim) { ne++; ex = (uint32_t)(lo + nx); continue; }
                    const int at = lo + nx;
                    atomicOr(&s.far[at >> 5], 1u << (at & 31));
                }
                if (k == 0 && tid == 0) {
                    #pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (j >= (int)ph && j < (int)ph + 5) ws[pw<L>(j)] = __ldg(src + j);
                }
                s.X[tid] = (uint16_t)X;
                if (lane == 31) s.sl_hi[wid] = sl;
                if (ne) s.exitX = ex;                  // one writer when the guess is a chain
            }
        }
        __syncthreads();
        // the guess is a chain when the successor marks are exactly the
        // candidates but one (the first), each mark made once, and exactly
        // one candidate leaves the tile
        uint32_t succ = 0;
        auto chain_test = [&]() {
            if (live) {
                uint32_t prev = __shfl_up_sync(FULL, sl, 1);
                if (lane == 0) prev = wid ? s.sl_hi[wid - 1] : 0u;
                succ = (sl & SEGM) | (prev >> L) | ((s.far[lo >> 5] >> (lo & 31)) & SEGM);
                uint32_t r1 = (uint32_t)__popc(X & ~succ) | ((uint32_t)__popc(succ & ~X) << 16);
                uint32_t r2 = ne | ((uint32_t)__popc(X) << 16);
                r1 = __reduce_add_sync(FULL, r1);
                r2 = __reduce_add_sync(FULL, r2);
                // the first guessed start: a minimum per warp, then one shared atomic per warp
                const uint32_t xf = __reduce_min_sync(FULL, X ? (uint32_t)(lo + __ffs(X) - 1) : DEAD);
                if (lane == 0) { atomicAdd(&s.cnt1, r1); atomicAdd(&s.cnt2, r2); if (xf != DEAD) atomicMin(&s.xfirst, xf); }
            }
            __syncthreads();
        };
        auto is_chain = [&]() {
            const uint32_t c1 = s.cnt1, c2 = s.cnt2;
            const uint32_t nA = c1 & 0xffffu, nB = c1 >> 16, nE = c2 & 0xffffu, nX = c2 >> 16;
            return live && (nX == 0 || (nA == 1 && nB == 0 && nE == 1 && s.exitX <= end_s));
        };
        chain_test();
        // A module's first tile whose guess is not a chain. Its first start
        // (word 5) is known, so no other candidate without a predecessor
        // starts an instruction, and neither does a candidate that only such
        // candidates lead to: a false candidate is a literal or string word
        // that reads as an instruction, and the few words it leads to soon
        // fall on a non-candidate, join the chain or leave the tile. They are
        // dropped round by round, each round marking successors afresh from
        // the remaining candidates and testing again; a tile still not a
        // chain after the last round takes the exact path.
        if (live && k == 0 && !is_chain()) {
            const uint32_t e0 = ph + 5;
            const bool e0_cand = e0 < tile_n && ((s.X[e0 / L] >> (e0 % L)) & 1u);
            const uint32_t keep = e0 >= (uint32_t)lo && e0 < (uint32_t)(lo + L) ? 1u << (e0 - (uint32_t)lo) : 0u;
            const int lim = (int)tile_n - lo;
            #pragma unroll 1
            for (int round = 0; round < 4 && e0_cand && !is_chain(); round++) {
                __syncthreads();                       // every thread has read the counts
                X &= succ | keep;
                if (tid == 0) { s.cnt1 = 0; s.cnt2 = 0; s.exitX = DEAD; s.xfirst = DEAD; }
                for (int i = tid; i < T / 32; i += NT) s.far[i] = 0u;
                __syncthreads();
                uint32_t ex = 0, farm = 0;
                sl = 0; ne = 0;
                for (uint32_t x = X; x; x &= x - 1) {
                    const int j = __ffs(x) - 1;
                    const int nx = j + (int)(ws[pw<L>(lo + j)] >> 16);
                    const bool leaves = nx >= lim;
                    ne += leaves ? 1u : 0u;
                    ex = leaves ? (uint32_t)(lo + nx) : ex;
                    sl |= (!leaves && nx < 2 * L) ? (1u << (nx & 31)) : 0u;
                    farm |= (!leaves && nx >= 2 * L) ? (1u << j) : 0u;
                }
                while (farm) {
                    const int j = __ffs(farm) - 1;
                    farm &= farm - 1;
                    const int at = lo + j + (int)(ws[pw<L>(lo + j)] >> 16);
                    atomicOr(&s.far[at >> 5], 1u << (at & 31));
                }
                s.X[tid] = (uint16_t)X;
                if (lane == 31) s.sl_hi[wid] = sl;
                if (ne) s.exitX = ex;
                __syncthreads();
                chain_test();
            }
        }
        const uint32_t exitX = s.exitX;
        bool fast = false, spec_tile = false;
        {
            const uint32_t c2 = s.cnt2;
            const uint32_t nX = c2 >> 16;
            fast = is_chain();
            // a later tile of its module whose guessed starts form a chain takes
            // the chain's first start as its entry: its exit and row count are
            // known now; the guess is checked against the predecessor's exit at
            // the end of the tile
            spec_tile = P.spec && fast && k > 0 && nX > 0;
            // a guessed chain that holds the tile's entry (its first start when
            // guessing, word 5 of a module's first tile) gives the tile's exit
            // and row count at once: published here, before anything else of
            // the tile, since every later tile waits on the count
            if (tid == 0 && fast && nX > 0 && g != P.stall_tile && g != P.stall_map_tile) {
                const uint32_t e0 = ph + 5;
                const bool first_on_chain = k == 0 && e0 < tile_n && ((s.X[e0 / L] >> (e0 % L)) & 1u);
                if (spec_tile || first_on_chain) {
                    st_relaxed(&P.tstate[g], F_EXIT | (unsigned long long)(exitX + tb_rel));
                    st_relaxed(&P.cstate[g], (g == 0 ? F_EXIT : F_MAP) | (unsigned long long)nX);
                    s.count_pub = 2;          // exit and count published
                }
            }
        }

        // exact path: per-position exits of each segment (backward pass),
        // then per warp the exits of its 32 candidate entries
        auto Eabs = [&](uint32_t x) -> uint32_t {   // x < tile_n
            const uint32_t e = s.E[pe<L>((int)x)];
            if (e == 0xffffu) return DEAD;
            const uint32_t seg_hi = (x / L + 1) * L;
            return (seg_hi < tile_n ? seg_hi : tile_n) + e;
        };
        auto exact_maps = [&]() {
            {
                const int hi = lo + L < (int)tile_n ? lo + L : (int)tile_n;
                for (int q = hi - 1; q >= lo; q--) {
                    const uint32_t wc = ws[pw<L>(q)] >> 16;
                    uint32_t e;
                    if (wc == 0 || (uint32_t)q + wc > end_s) e = 0xffffu;
                    else if (q + (int)wc >= hi) e = (uint32_t)(q + (int)wc - hi);
                    else e = s.E[pe<L>(q + (int)wc)];
                    s.E[pe<L>(q)] = (uint16_t)e;
                }
            }
            __syncthreads();
            {
                const uint32_t wb = (uint32_t)wid * WSPAN;
                const uint32_t we = wb + WSPAN < tile_n ? wb + WSPAN : tile_n;
                uint32_t x = wb + lane;
                while (x < we) { x = Eabs(x); if (x == DEAD) break; }
                s.wmap[wid][lane] = x;
            }
            __syncthreads();
        };
        // exact path: from the tile entry e through the warp maps; the warps'
        // entries and the tile's exit (lane 0 of warp 0)
        auto exact_compose = [&](uint32_t x0) {
            uint32_t xw = x0;
            for (int w2 = 0; w2 < NW; w2++) {
                const uint32_t wb = (uint32_t)w2 * WSPAN;
                const uint32_t we = wb + WSPAN < tile_n ? wb + WSPAN : tile_n;
                if (xw == DEAD || xw >= tile_n || xw >= we) { s.warp_entry[w2] = DEAD; continue; }
                s.warp_entry[w2] = xw;
                if (xw - wb < 32) xw = s.wmap[w2][xw - wb];
                else { while (xw < we) { xw = Eabs(xw); if (xw == DEAD) break; } }
            }
            return xw;
        };
        if (live && !fast) exact_maps();

        // A tile whose entry every thread knows (its first guessed start, or
        // word 5 of a module's first tile on the guessed chain) has published
        // its exit and row count above: it skips warp 0's section and the
        // barrier after it.
        bool quick = false;
        {
            const uint32_t e0 = ph + 5;
            const bool first_on_chain = k == 0 && e0 < tile_n && ((s.X[e0 / L] >> (e0 % L)) & 1u);
            const uint32_t nX = s.cnt2 >> 16;
            quick = live && fast && nX > 0 && g != P.stall_tile && g != P.stall_map_tile && (spec_tile || first_on_chain);
        }
        const uint32_t qentry = quick ? (spec_tile ? s.xfirst : ph + 5) : DEAD;
        if (quick) {
            if (P.out && !P.out_vec) {
                // encode word by word when the output buffer's 16-byte phase is not the words'
                uint32_t *dst = P.out + tbase;
                for (int i = tid + lo_ok; i < n_copy; i += NT) dst[i] = ws[pw<L>(i)];
            }
        } else {
        // 3. warp 0: the tile map for entries 0..31, published; the look-back
        //    for the tile's entry; the tile's exit, published. Meanwhile the
        //    other warps encode.
        if (wid == 0) {
            uint32_t x = UNRES;
            if (spec_tile) {
                // no map: later tiles read this tile's exit
            } else if (fast) {
                // a candidate entry on the guessed chain leaves with it; any
                // other is followed a few steps until it joins the chain,
                // dies or leaves the tile (else the map cannot tell)
                uint32_t pos = (uint32_t)lane;
                x = UNRES;
                #pragma unroll 1
                for (int st = 0; st < 4; st++) {
                    if (pos >= tile_n) { x = pos; break; }
                    if ((s.X[pos / L] >> (pos % L)) & 1u) { x = exitX; break; }
                    const uint32_t wc = ws[pw<L>((int)pos)] >> 16;
                    if (wc == 0 || pos + wc > end_s) { x = DEAD; break; }
                    pos += wc;
                }
            } else {
                x = s.wmap[0][lane];
                for (int w2 = 1; w2 < NW; w2++) {
                    if (x == DEAD || x >= tile_n) break;
                    const uint32_t wb = (uint32_t)w2 * WSPAN;
                    if (x - wb < 32) x = s.wmap[w2][x - wb];
                    else if (x < wb + WSPAN) { x = UNRES; break; }
                }
            }
            const uint32_t mv = (x == DEAD || x == UNRES) ? x : x + tb_rel;
            const long long first = g - (long long)k;
            const bool stalled = (g == P.stall_tile);
            const bool map_only = (g == P.stall_map_tile);
            const bool need_lookback = live && k > 0 && !spec_tile;
            if (need_lookback && !stalled) {
                // a map entry of a tile after a module's first is never 0 (an
                // exit lies past the tile's start, DEAD and UNRES are not 0),
                // so an entry read as 0 is not written yet: the entries need no
                // ordering against the MAP state, which only tells the
                // look-back that the map is on its way
                if (!map_only) st_relaxed32(&P.tmap[g * NCAND + lane], mv);
                const bool inline_map = fast && !map_only && exitX != DEAD;
                const uint32_t cm = __ballot_sync(FULL, inline_map && x == exitX);
                __syncwarp();
                if (lane == 0)
                    st_relaxed(&P.tstate[g], inline_map ? (F_FMAP | ((unsigned long long)exitX << 32) | cm) : F_MAP);
            }
            // entry of this tile (tile-local)
            uint32_t entry;
            if (!live) entry = DEAD;
            else if (k == 0) entry = ph + 5;
            else if (spec_tile) entry = s.xfirst;
            else {
                // find the nearest predecessor with a published exit
                long long hi_j = g - 1;
                long long spins = 0;
                long long anchor = -1;
                uint32_t ax = DEAD;
                bool gave_up = false;
                unsigned long long st_last = 0;
                for (;;) {
                    long long j = hi_j - lane;
                    unsigned long long st = j >= first ? ld_relaxed(&P.tstate[j]) : F_EXIT;
                    st_last = st;
                    unsigned long long f = st & F_MASK;
                    unsigned exitm = __ballot_sync(FULL, j < first || f == F_EXIT);
                    unsigned nonem = __ballot_sync(FULL, j >= first && f == 0);
                    if (exitm) {
                        int le = __ffs(exitm) - 1;
                        if (nonem & ((1u << le) - 1u)) {
                            if (++spins > P.max_spins) { gave_up = true; break; }
                            spin_pause();
                            continue;
                        }
                        unsigned long long sv = __shfl_sync(FULL, st, le);
                        anchor = hi_j - le;
                        ax = anchor < first ? 5u : (uint32_t)(sv & 0xffffffffu);
                        break;
                    }
                    if (nonem) {
                        if (++spins > P.max_spins) { gave_up = true; break; }
                        spin_pause();
                        continue;
                    }
                    hi_j -= 32;
                }
                // apply predecessors' maps from the anchor forward, 32 tiles'
                // states per read (the last poll's when it holds them all): a
                // published exit is taken as it is, an inline map settles a
                // marked entry, anything else reads the map entry (one read as
                // 0 is not visible yet and is read again)
                uint32_t xx = ax;
                for (long long t0 = anchor + 1; t0 < g && !gave_up; t0 += 32) {
                  const bool in_regs = (hi_j == g - 1);
                  const long long tl = t0 + lane;
                  const unsigned long long stb = in_regs ? 0ull : (tl < g ? ld_relaxed(&P.tstate[tl]) : 0ull);
                  for (long long tt = t0; tt < g && tt < t0 + 32 && !gave_up; tt++) {
                    {
                        uint32_t kt = (uint32_t)(tt - first);
                        uint32_t tb = kt * (uint32_t)T - ph;
                        if (xx == DEAD || xx >= tb + (uint32_t)T) continue;
                        const unsigned long long stt = in_regs ? __shfl_sync(FULL, st_last, (int)(hi_j - tt))
                                                               : __shfl_sync(FULL, stb, (int)(tt - t0));
                        if ((stt & F_MASK) == F_EXIT) { xx = (uint32_t)(stt & 0xffffffffu); continue; }
                        if ((stt & F_MASK) == F_FMAP && xx - tb < 32 && ((stt >> (xx - tb)) & 1ull)) {
                            xx = tb + (uint32_t)((stt >> 32) & 0x3ffffu);
                            continue;
                        }
                        uint32_t val = xx - tb < 32 ? __shfl_sync(FULL, ld_relaxed32(&P.tmap[tt * NCAND + lane]), (int)((xx - tb) & 31u)) : 0u;
                        while (xx - tb < 32 && val == 0u) {
                            if (++spins > P.max_spins) { gave_up = true; break; }
                            spin_pause();
                            val = __shfl_sync(FULL, ld_relaxed32(&P.tmap[tt * NCAND + lane]), (int)((xx - tb) & 31u));
                        }
                        if (gave_up) break;
                        if (xx - tb < 32 && val != UNRES) { xx = val; continue; }
                        // the map cannot tell: wait for this tile's own exit
                        unsigned long long st;
                        for (;;) {
                            st = 0;
                            if (lane == 0) st = ld_relaxed(&P.tstate[tt]);
                            st = __shfl_sync(FULL, st, 0);
                            if ((st & F_MASK) == F_EXIT) break;
                            if (++spins > P.max_spins) { gave_up = true; break; }
                            spin_pause();
                        }
                        if (gave_up) break;
                        xx = (uint32_t)(st & 0xffffffffu);
                    }
                  }
                }
                entry = gave_up ? DEAD : (xx == DEAD ? DEAD : xx - tb_rel);
                if (gave_up && lane == 0) s.timeout = 1;
            }
            if (lane == 0) {
                uint32_t xw = DEAD;
                bool known_exit = true;
                if (!live || entry == DEAD) xw = DEAD;
                else if (fast) {
                    if (entry >= tile_n) xw = entry;
                    else if ((s.X[entry / L] >> (entry % L)) & 1u) xw = exitX;
                    else { known_exit = false; s.need_exact = 1; }     // the entry is not on the guessed chain
                } else {
                    xw = exact_compose(entry);
                }
                s.entry = entry;
                s.exitp = xw;
                if (known_exit && live && g != P.stall_tile && g != P.stall_map_tile && s.count_pub != 2) {
                    const uint32_t mx = xw == DEAD ? DEAD : xw + tb_rel;
                    st_relaxed(&P.tstate[g], F_EXIT | (unsigned long long)mx);
                }
            }
            __syncwarp();
            // the tile's row count, published as soon as its entry is known: the
            // guessed chain's starts from the entry on (none without a live
            // entry). Every later tile's first row waits on this count.
            if (s.count_pub == 0 && (!live || entry == DEAD || (fast && s.need_exact == 0))) {
                uint32_t c = 0;
                if (live && entry != DEAD && entry < tile_n) {
                    for (int t = lane; t < NT; t += 32) {
                        const uint32_t lo_t = (uint32_t)t * L;
                        uint32_t x = s.X[t];
                        if (lo_t + L <= entry) x = 0;
                        else if (lo_t < entry) x &= ~((1u << (entry - lo_t)) - 1u);
                        c += (uint32_t)__popc(x);
                    }
                }
                c = __reduce_add_sync(FULL, c);
                if (lane == 0) {
                    s.count_pub = 1;
                    if (g != P.stall_tile && g != P.stall_map_tile)
                        st_relaxed(&P.cstate[g], (g == 0 ? F_EXIT : F_MAP) | c);
                }
            }
        } else if (P.out && !P.out_vec) {
            // encode word by word when the output buffer's 16-byte phase is not
            // the words' (the other warps, while warp 0 looks back)
            uint32_t *dst = P.out + tbase;
            for (int i = tid - 32 + lo_ok; i < n_copy; i += NT - 32) dst[i] = ws[pw<L>(i)];
        }
        __syncthreads();
        }
        // the entry missed the guessed chain: the exact path for this tile's starts
        const bool need_exact = !quick && s.need_exact != 0;
        if (need_exact) {
            exact_maps();
            if (tid == 0) {
                const uint32_t xw = exact_compose(s.entry);
                s.exitp = xw;
                if (g != P.stall_tile && g != P.stall_map_tile) {
                    const uint32_t mx = xw == DEAD ? DEAD : xw + tb_rel;
                    st_relaxed(&P.tstate[g], F_EXIT | (unsigned long long)mx);
                }
            }
            __syncthreads();
        }
        // 4. my segment's starts; the framing error if the chain dies here
        uint32_t mask = 0;
        int ferr = -1;          // 0 zero word count, 1 truncated
        if (fast && !need_exact) {
            const uint32_t e = quick ? qentry : s.entry;
            if (e != DEAD && e < tile_n) {
                if (e <= (uint32_t)lo) mask = X;
                else if (e < (uint32_t)(lo + L)) mask = X & ~((1u << (e - (uint32_t)lo)) - 1u);
            }
        } else if (live) {
            // per warp: entry of each segment (serial walk by lane 0), then the
            // starts of my segment
            s.seg_entry[tid] = NONE16;
            __syncwarp();
            if (lane == 0) {
                uint32_t x = s.warp_entry[wid];
                uint32_t wb = (uint32_t)wid * WSPAN;
                uint32_t we = wb + WSPAN < tile_n ? wb + WSPAN : tile_n;
                while (x != DEAD && x < we) {
                    s.seg_entry[x / L] = (uint16_t)x;
                    x = Eabs(x);
                }
            }
            __syncwarp();
            const int hi = lo + L < (int)tile_n ? lo + L : (int)tile_n;
            uint32_t p = s.seg_entry[tid];
            if (p != NONE16) {
                while ((int)p < hi) {
                    uint32_t wc = ws[pw<L>((int)p)] >> 16;
                    if (wc == 0) { ferr = 0; break; }
                    if (p + wc > end_s) { ferr = 1; break; }
                    mask |= 1u << (p - lo);
                    p += wc;
                }
            }
        }
        const unsigned cnt = __popc(mask);
        unsigned incl = cnt;
        #pragma unroll
        for (int d = 1; d < 32; d <<= 1) { unsigned v = __shfl_up_sync(FULL, incl, d); if (lane >= d) incl += v; }
        if (lane == 31) s.warp_tot[wid] = incl;
        __syncthreads();
        // every warp scans the warp counts itself (no barrier after a scan by
        // one warp); warp 0 publishes the tile's count
        const bool stalled = (g == P.stall_tile || g == P.stall_map_tile);
        unsigned wv = lane < NW ? s.warp_tot[lane] : 0;
        #pragma unroll
        for (int d = 1; d < NW; d <<= 1) { unsigned u = __shfl_up_sync(FULL, wv, d); if (lane >= d) wv += u; }
        const unsigned tile_count = __shfl_sync(FULL, wv, NW - 1);
        const unsigned wpre = __shfl_sync(FULL, wv, wid > 0 ? wid - 1 : 0);
        if (wid == 0 && lane == 0 && !stalled && !s.count_pub)
            st_relaxed(&P.cstate[g], (g == 0 ? F_EXIT : F_MAP) | tile_count);
        const unsigned my_off = (wid ? wpre : 0u) + incl - cnt;
        // error keys hold tile-local rows until the flush adds the tile's first row
        if (ferr >= 0 && live) atomicMin(&s.err_key, make_key(my_off + cnt, R_FRAME, (uint32_t)ferr));
        // start list (reuses E)
        uint16_t *S16 = s.E;
        {
            uint32_t x = mask;
            unsigned o = my_off;
            while (x) { int b = __ffs(x) - 1; x &= x - 1; S16[o++] = (uint16_t)(lo + b); }
        }
        __syncthreads();
        const uint32_t bound = P.ms[m].bound;
        const long long arena_off = P.ms[m].arena_off;
        const uint32_t id_slots = P.ms[m].id_slots;
        uint32_t acc_lo = 0, acc_hi = 0, acc_ins = 0;  // this lane's requirements and insertions
        if (P.validate) {
            // rows in chunks of 32 from a shared counter. A row in the fast
            // operand form (fixed ids and literals, then a plain tail or one
            // bit-enum word; at most 32 words, all staged: p < T and the halo
            // holds 64 more) is checked here, in the order of section 3.4.5's
            // checks: known opcode, its word count against the form, every id
            // operand in [1, bound); then its result id goes into the module's
            // id set and the opcode's capability into the tile's requirements.
            // Any other row takes the full operand walk (slow_row).
            static_assert(HALO >= 32, "fast rows read up to 32 staged words");
            for (;;) {
                unsigned rb = 0;
                if (lane == 0) rb = atomicAdd(&s.vnext, 32u);
                rb = __shfl_sync(FULL, rb, 0);
                if (rb >= tile_count) break;
                const unsigned r = rb + (unsigned)lane;
                const bool have = r < tile_count;
                const uint32_t p = have ? (uint32_t)S16[r] : 0u;
                const uint32_t a0 = pwu<L>(p);
                // words 1..8 of the row lie at a0 + i, or 4 further once past
                // the segment's end (position `cross`): one boundary at most
                const uint32_t cross = (uint32_t)L - p % (uint32_t)L;
                const uint32_t w0 = ws[a0];
                const uint32_t op = w0 & 0xffffu, wc = w0 >> 16;
                const uint2 vd = s.vd[op < 256u ? op : 256u];
                const bool known = have && ((vd.y >> 16) & 1u);
                const bool fastrow = have && ((vd.y >> 15) & 1u) && wc <= 32u;
                const uint32_t need = vd.y & 31u;
                const uint32_t dw = wc - need;                    // words past the fixed operands
                const uint32_t np = s.bnp[(vd.y >> 13) & 3u][ws[pwu<L>(p + need)] & 15u];
                bool ok = (dw < ((vd.y >> 5) & 63u) && !(dw & (vd.y >> 11) & 1u)) ||
                          (((vd.y >> 12) & 1u) && dw == 1u + np);
                ok = ok && fastrow;
                const uint32_t idm = ok ? vd.x & (shl_clamp(2u, wc - 1u) - 1u) : 0u;
                uint32_t mx = 0, ri = 0;                          // largest id - 1; the result id
                const uint32_t qi = 1u + ((vd.y >> 18) & 1u);     // the result id's word
                #pragma unroll
                for (int i = 1; i <= 8; i++) {
                    const uint32_t v = ws[a0 + (uint32_t)i + ((uint32_t)i >= cross ? 4u : 0u)];
                    if ((idm >> i) & 1u) mx = max(mx, v - 1u);
                    if (i <= 2 && (uint32_t)i == qi) ri = v;
                }
                if (idm >> 9) {                                   // ids past word 8 (long id tails)
                    for (uint32_t x = idm >> 9 << 9; x; x &= x - 1)
                        mx = max(mx, ws[pwu<L>(p + (uint32_t)(__ffs(x) - 1))] - 1u);
                }
                const bool oob = idm != 0 && mx >= bound - 1u;
                if (have && (!known || (fastrow && !ok) || oob))
                    atomicMin(&s.err_key, make_key(r, !known ? R_UNKNOWN : (!ok ? R_BADOP : R_OOB), 0));
                const bool good = ok && !oob;
                const uint32_t cap = vd.y >> 24;                  // 0xff: none
                if (good && cap < 64u) { if (cap & 32u) acc_hi |= 1u << (cap & 31u); else acc_lo |= 1u << cap; }
                if (good && ((vd.y >> 17) & 1u) && arena_off >= 0) {
                    if (id_slots == 0) {
                        // no wait on the old value: duplicates show up later as
                        // fewer bits set than ids inserted
                        atomicOr(&P.arena[arena_off + (ri >> 5)], 1u << (ri & 31));
                        acc_ins++;
                    } else if (idset_insert(P.arena + arena_off, id_slots, ri)) {
                        atomicOr(&s.flags, MF_DUP);
                    }
                }
                const bool slow = known && !fastrow;
                if (__any_sync(FULL, slow) && slow) {
                    const SlowOut so = slow_row<NT, L>(s, src, p, r, bound, P.arena, arena_off, id_slots);
                    acc_lo |= so.lo; acc_hi |= so.hi; acc_ins += so.ins;
                }
            }
            // this warp's requirements and insertions, once for all its chunks
            const uint32_t rlo = __reduce_or_sync(FULL, acc_lo);
            const uint32_t rhi = __reduce_or_sync(FULL, acc_hi);
            const uint32_t nins = __reduce_add_sync(FULL, acc_ins);
            if (lane == 0) {
                if (rlo) atomicOr(&s.req_lo, rlo);
                if (rhi) atomicOr(&s.req_hi, rhi);
                if (nins) atomicAdd(&s.n_ids, nins);
            }
        }
        // warp 0: the tile's first row (decoupled look-back over all tiles'
        // counts), after its share of the validation (which needs no global
        // row index): by then the predecessors' counts are mostly published,
        // and a warp that waits sleeps longer between polls
        if (wid == 0) {
            unsigned long long excl = 0;
            if (g > 0) {
                bool gave_up;
                // 32 states a poll: the nearest inclusive state is seldom far back
                excl = warp_lookback_sum<1, 512>(P.cstate, g - 1, F_EXIT, F_MASK, P.max_spins, lane, gave_up);
                if (gave_up) { excl = 0; if (lane == 0) s.timeout = 1; }
                if (lane == 0 && !stalled) st_relaxed(&P.cstate[g], F_EXIT | (excl + tile_count));
            }
            if (lane == 0) {
                s.row_base = excl;
                if (k == 0) P.first_row[m] = (int64_t)excl;
                if (g == n_tiles - 1) P.ctrl->total_rows = excl + tile_count;
            }
        }
        __syncthreads();
        // the table rows, at the tile's first row (each warp its chunks of 32
        // rows); the largest result id
        const unsigned long long row_base = s.row_base;
        {
            uint32_t rmax = 0;
            for (unsigned rb = 32u * (unsigned)wid; rb < tile_count; rb += NT) {
                const unsigned r = rb + (unsigned)lane;
                if (r < tile_count) {
                    // a start lies in the tile and the result type and id within two
                    // words of it, inside the 64-word halo: staged, read directly
                    const uint32_t p = S16[r];
                    const uint32_t w0 = ws[pwu<L>(p)];
                    const uint32_t op = w0 & 0xffffu, wc = w0 >> 16;
                    const uint32_t vy = s.vd[op < 256u ? op : 256u].y;
                    const uint32_t flags = ((vy >> 17) & 1u ? 4u : 0u) | ((vy >> 18) & 1u ? 2u : 0u);
                    const uint32_t w1 = ws[pwu<L>(p + 1)], w2 = ws[pwu<L>(p + 2)];
                    uint32_t rt = 0, ri = 0;
                    if (flags & 2u) { if (wc > 1) rt = w1; if ((flags & 4u) && wc > 2) ri = w2; }
                    else if ((flags & 4u) && wc > 1) ri = w1;
                    rmax = ri > rmax ? ri : rmax;
                    const unsigned long long row = row_base + r;
                    if ((long long)row < P.cap_rows) {
                        P.op[row] = (uint16_t)op; P.wc[row] = (uint16_t)wc;
                        P.off[row] = (uint64_t)(tbase + p);
                        P.rtype[row] = rt; P.rid[row] = ri; P.mod[row] = (uint32_t)m;
                    } else {
                        atomicOr(&s.flags, MF_CAPACITY);
                    }
                }
            }
            rmax = __reduce_max_sync(FULL, rmax);
            if (lane == 0 && rmax) atomicMax(&s.max_rid, rmax);
        }

        __syncthreads();
        // the entry guess of a speculating tile against its predecessor's exit
        if (spec_tile && tid == 0) {
            unsigned long long st = 0;
            long long spins = 0;
            for (;;) {
                st = ld_relaxed(&P.tstate[g - 1]);
                if ((st & F_MASK) == F_EXIT) break;
                if (++spins > P.max_spins) { s.timeout = 1; break; }
                spin_pause();
            }
            if ((st & F_MASK) == F_EXIT) {
                const uint32_t xp = (uint32_t)(st & 0xffffffffu);
                if (xp == DEAD || xp - tb_rel != s.xfirst) atomicExch(&P.ctrl->spec_failed, 1u);
            }
        }
        // 6. flush the tile's aggregates to the module
        if (tid == 0) {
            ModState *ms = &P.ms[m];
            if (s.err_key != NO_KEY) atomicMin(&ms->err_key, s.err_key + (s.row_base << 8));
            if (s.n_cap) atomicAdd(&ms->n_cap, s.n_cap);
            if (s.n_mm) atomicAdd(&ms->n_mm, s.n_mm);
            if (s.n_ep) atomicAdd(&ms->n_ep, s.n_ep);
            if (s.n_fn) atomicAdd(&ms->n_fn, s.n_fn);
            if (s.decl_lo) atomicOr(&ms->decl_lo, s.decl_lo);
            if (s.decl_hi) atomicOr(&ms->decl_hi, s.decl_hi);
            if (s.req_lo) atomicOr(&ms->req_lo, s.req_lo);
            if (s.req_hi) atomicOr(&ms->req_hi, s.req_hi);
            if (s.max_rid) atomicMax(&ms->max_rid, s.max_rid);
            if (s.n_ids) atomicAdd(&ms->n_ids, s.n_ids);
            uint32_t fl = s.flags | (s.timeout ? MF_TIMEOUT : 0u);
            if (fl) atomicOr(&ms->flags, fl);
            if (s.timeout) atomicExch(&P.ctrl->timeout, 1u);
        }
        if (!P.persistent) break;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// bits set in each module's bitmap id set (chunks of the arena in parallel;
// abase is the prefix of the words each module asked for)
// ---------------------------------------------------------------------------
__global__ void k_id_popcount(Params P)
{
    if (skip_pass(P)) return;
    const long long aw = (long long)P.ctrl->arena_used;
    const int CH = 64;
    const long long nch = (aw + CH - 1) / CH;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nch; c += stride) {
        long long w = c * CH, w1 = w + CH < aw ? w + CH : aw;
        int lo = 0, hi = P.n_modules;          // last m with abase[m] <= w
        while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (P.abase[mid] <= w) lo = mid; else hi = mid; }
        int m = lo;
        while (w < w1 && m < P.n_modules) {
            long long mend = P.abase[m + 1];
            long long e = mend < w1 ? mend : w1;
            const ModState &ms = P.ms[m];
            if (e > w && ms.arena_off >= 0 && ms.id_slots == 0) {
                uint32_t cnt = 0;
                for (long long k = w; k < e; k++) cnt += __popc(P.arena[k]);
                if (cnt) atomicAdd(&P.ms[m].n_set, cnt);
            }
            if (e > w) w = e;
            m++;
        }
    }
}

// ---------------------------------------------------------------------------
// finalize: per module status, row counts, bound of the encoded header
// ---------------------------------------------------------------------------
__device__ void module_status(const Params &P, int m, unsigned long long key, uint32_t *st, int64_t *er)
{
    const ModState &s = P.ms[m];
    int64_t first = P.first_row[m];
    if (P.ctrl->timeout || (s.flags & MF_TIMEOUT)) { *st = S_TIMEOUT; *er = -1; return; }
    if (s.hdr != S_OK) { *st = s.hdr; *er = -1; return; }
    if (s.flags & MF_CAPACITY) { *st = S_CAPACITY; *er = -1; return; }
    if (key != NO_KEY) {
        uint32_t code = key_status(key);
        *st = code;
        *er = (int64_t)(key >> 8) - first;
        return;
    }
    *er = -1;
    if (!P.validate) { *st = S_OK; return; }
    if (s.n_cap == 0) *st = S_NO_CAPABILITY;
    else if (s.n_mm == 0) *st = S_NO_MEMORY_MODEL;
    else if (s.n_mm > 1) *st = S_MULTI_MEMORY_MODEL;
    else if (s.n_ep == 0) *st = S_NO_ENTRY_POINT;
    else if (s.n_fn == 0) *st = S_NO_FUNCTION;
    else *st = S_OK;
}

__global__ void k_finalize(Params P)
{
    if (skip_pass(P)) return;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= P.n_modules) return;
    if (!P.table_mode) {
        unsigned long long total = P.ctrl->total_rows;
        int64_t first = P.first_row[m];
        int64_t next = m + 1 < P.n_modules ? P.first_row[m + 1] : (int64_t)total;
        P.n_instr[m] = (uint32_t)(next - first);
        if (m == P.n_modules - 1) P.first_row[P.n_modules] = (int64_t)total;
    }
    ModState &s = P.ms[m];
    if (P.out && P.recompute_bound && s.hdr == S_OK) P.out[P.mod_off[m] + 3] = s.max_rid + 1;
    if (P.validate && s.arena_off >= 0 && s.id_slots == 0 && s.n_set < s.n_ids) s.flags |= MF_DUP;
    if (P.validate && s.hdr == S_OK && !(s.flags & (MF_CAPACITY | MF_TIMEOUT)) && !P.ctrl->timeout) {
        uint64_t decl = ((uint64_t)s.decl_hi << 32) | s.decl_lo;
        uint64_t req = ((uint64_t)s.req_hi << 32) | s.req_lo;
        uint64_t missing = req & ~cap_closure(decl);
        if (missing || (s.flags & MF_DUP)) {
            s.flags |= MF_FIXUP;
            unsigned slot = atomicAdd(&P.ctrl->n_fix, 1u);
            P.fixlist[slot] = (uint32_t)m;
            return;
        }
    }
    uint32_t st; int64_t er;
    module_status(P, m, s.err_key, &st, &er);
    P.status[m] = st;
    P.err_row[m] = er;
}

// ---------------------------------------------------------------------------
// exact fixup for the few modules with a missing capability or a duplicate
// result id: one CTA per module, over its table rows.
//   missing capability: min row (passing the earlier checks) requiring a
//     capability outside the closure of the declared ones;
//   duplicate: min row r whose result id some row < r already defines --
//     rows are taken in order, chunk by chunk: a row is a duplicate if the
//     id bitmap (rows of earlier chunks) has its id, or a lower row of the
//     same chunk has it (shared-memory hash of the chunk's ids).
// ---------------------------------------------------------------------------
constexpr int FIX_NT = 512;
constexpr int FIX_CHUNK = 2048;
constexpr int FIX_HASH = 4096;

__global__ void __launch_bounds__(FIX_NT) k_fixup(Params P)
{
    if (skip_pass(P)) return;
    __shared__ unsigned long long s_best;
    __shared__ uint32_t h_key[FIX_HASH];
    __shared__ uint32_t h_min[FIX_HASH];
    __shared__ int s_stop;
    const spvt::Tables &TB = g_spv_tables;
    unsigned n_fix = P.ctrl->n_fix;
    for (unsigned f = blockIdx.x; f < n_fix; f += gridDim.x) {
        int m = (int)P.fixlist[f];
        ModState &ms = P.ms[m];
        int64_t first = P.first_row[m];
        int64_t n = P.n_instr[m];
        uint32_t bound = ms.bound;
        uint64_t decl = ((uint64_t)ms.decl_hi << 32) | ms.decl_lo;
        uint64_t req = ((uint64_t)ms.req_hi << 32) | ms.req_lo;
        uint64_t missing = req & ~cap_closure(decl);
        if (threadIdx.x == 0) { s_best = ms.err_key; s_stop = 0; }
        __syncthreads();
        if (missing) {
            for (int64_t r = threadIdx.x; r < n; r += FIX_NT) {
                int64_t row = first + r;
                uint32_t op = P.op[row], wc = P.wc[row];
                if (op >= 256 || !(TB.ops[op].flags & 1)) continue;
                const uint32_t *iwp = P.words + P.off[row];
                auto iw = [&](uint32_t i) -> uint32_t { return __ldg(iwp + i); };
                Walk wk = walk_instruction(iw, wc, TB.ops[op], bound);
                if (!wk.ok) continue;
                uint64_t rq = wk.req | width_caps(iw, op, wc);
                if (rq & missing) atomicMin(&s_best, make_key((unsigned long long)row, R_MISSING, 0));
            }
        }
        if ((ms.flags & MF_DUP) && ms.arena_off >= 0) {
            uint32_t *bm = P.arena + ms.arena_off;
            const uint32_t slots = ms.id_slots;
            long long len_m = P.mod_off[m + 1] - P.mod_off[m];
            unsigned long long nbw = idset_words(bound, len_m);
            for (unsigned long long i = threadIdx.x; i < nbw; i += FIX_NT) bm[i] = 0;
            __syncthreads();
            for (int64_t c0 = 0; c0 < n; c0 += FIX_CHUNK) {
                for (int i = threadIdx.x; i < FIX_HASH; i += FIX_NT) { h_key[i] = 0; h_min[i] = 0xffffffffu; }
                __syncthreads();
                // ids of this chunk's defining rows: first occurrence in the chunk
                for (int i = threadIdx.x; i < FIX_CHUNK; i += FIX_NT) {
                    int64_t r = c0 + i;
                    if (r >= n) break;
                    int64_t row = first + r;
                    uint32_t op = P.op[row];
                    if (op >= 256 || !(TB.ops[op].flags & 4)) continue;
                    uint32_t id = P.rid[row];
                    if (id == 0 || id >= bound) continue;
                    uint32_t h = (id * 2654435761u) & (FIX_HASH - 1);
                    for (;;) {
                        uint32_t prev = atomicCAS(&h_key[h], 0u, id);
                        if (prev == 0 || prev == id) { atomicMin(&h_min[h], (uint32_t)i); break; }
                        h = (h + 1) & (FIX_HASH - 1);
                    }
                }
                __syncthreads();
                for (int i = threadIdx.x; i < FIX_CHUNK; i += FIX_NT) {
                    int64_t r = c0 + i;
                    if (r >= n) break;
                    int64_t row = first + r;
                    uint32_t op = P.op[row];
                    if (op >= 256 || !(TB.ops[op].flags & 4)) continue;
                    uint32_t id = P.rid[row];
                    if (id == 0 || id >= bound) continue;
                    bool dup = idset_contains(bm, slots, id);
                    if (!dup) {
                        uint32_t h = (id * 2654435761u) & (FIX_HASH - 1);
                        while (h_key[h] != id) h = (h + 1) & (FIX_HASH - 1);
                        dup = h_min[h] < (uint32_t)i;
                    }
                    if (dup) { atomicMin(&s_best, make_key((unsigned long long)row, R_DUP, 0)); s_stop = 1; }
                }
                __syncthreads();
                for (int i = threadIdx.x; i < FIX_CHUNK; i += FIX_NT) {
                    int64_t r = c0 + i;
                    if (r >= n) break;
                    int64_t row = first + r;
                    uint32_t op = P.op[row];
                    if (op >= 256 || !(TB.ops[op].flags & 4)) continue;
                    uint32_t id = P.rid[row];
                    if (id == 0 || id >= bound) continue;
                    idset_insert(bm, slots, id);
                }
                __syncthreads();
                if (s_stop) break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t st; int64_t er;
            module_status(P, m, s_best, &st, &er);
            P.status[m] = st;
            P.err_row[m] = er;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// validate from an existing table
// ---------------------------------------------------------------------------
__global__ void k_validate_rows(Params P)
{
    const spvt::Tables &TB = g_spv_tables;
    long long n_rows = P.first_row[P.n_modules];
    if (n_rows > P.cap_rows) n_rows = P.cap_rows;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < n_rows; row += stride) {
        uint32_t m = P.mod[row];
        ModState *ms = &P.ms[m];
        if (ms->hdr != S_OK) continue;
        uint32_t op = P.op[row], wc = P.wc[row];
        const uint32_t *iwp = P.words + P.off[row];
        auto iw = [&](uint32_t i) -> uint32_t { return __ldg(iwp + i); };
        uint32_t ri = P.rid[row];
        if (ri) atomicMax(&ms->max_rid, ri);
        if (op == 17) { atomicAdd(&ms->n_cap, 1u); if (wc >= 2) { uint32_t c = iw(1); if (c < 32) atomicOr(&ms->decl_lo, 1u << c); else if (c < 64) atomicOr(&ms->decl_hi, 1u << (c - 32)); } }
        else if (op == 14) atomicAdd(&ms->n_mm, 1u);
        else if (op == 15) atomicAdd(&ms->n_ep, 1u);
        else if (op == 54) atomicAdd(&ms->n_fn, 1u);
        if (op >= 256 || !(TB.ops[op].flags & 1)) { atomicMin(&ms->err_key, make_key((unsigned long long)row, R_UNKNOWN, 0)); continue; }
        const spvt::OpDesc &d = TB.ops[op];
        Walk wk = walk_instruction(iw, wc, d, ms->bound);
        if (!wk.ok) { atomicMin(&ms->err_key, make_key((unsigned long long)row, R_BADOP, 0)); continue; }
        if (wk.oob) { atomicMin(&ms->err_key, make_key((unsigned long long)row, R_OOB, 0)); continue; }
        if ((d.flags & 4) && ms->arena_off >= 0) {
            if (ms->id_slots == 0) {
                atomicOr(&P.arena[ms->arena_off + (ri >> 5)], 1u << (ri & 31));
                atomicAdd(&ms->n_ids, 1u);
            } else if (idset_insert(P.arena + ms->arena_off, ms->id_slots, ri)) {
                atomicOr(&ms->flags, MF_DUP);
            }
        }
        uint64_t req = wk.req | width_caps(iw, op, wc);
        if ((uint32_t)req) atomicOr(&ms->req_lo, (uint32_t)req);
        if ((uint32_t)(req >> 32)) atomicOr(&ms->req_hi, (uint32_t)(req >> 32));
    }
}

// framing errors of a decoded table: the rows of module m end before the
// module's last word exactly when decode stopped at a framing error
__global__ void k_table_framing(Params P)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= P.n_modules) return;
    ModState &s = P.ms[m];
    if (s.hdr != S_OK) return;
    int64_t first = P.first_row[m];
    uint32_t n = P.n_instr[m];
    long long base = P.mod_off[m], len = P.mod_off[m + 1] - base;
    long long endp = n ? (long long)(P.off[first + n - 1] - base) + P.wc[first + n - 1] : 5;
    if (endp < len) {
        uint32_t wc = P.words[base + endp] >> 16;
        atomicMin(&s.err_key, make_key((unsigned long long)(first + n), R_FRAME, wc == 0 ? 0u : 1u));
    }
}

// ---------------------------------------------------------------------------
// encode from a table
// ---------------------------------------------------------------------------
__global__ void k_encode_bound_init(const uint32_t *words, const int64_t *mod_off, int n_mod, uint32_t *out)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_mod) return;
    long long o = mod_off[m], n = mod_off[m + 1] - o;
    if (n >= 0 && n <= 0x7fffffffLL && header_status(words + o, n) == S_OK) out[o + 3] = 1;
}

__global__ void k_encode_rows(const uint32_t *words, const int64_t *mod_off, const uint16_t *op,
                              const uint16_t *wc, const uint64_t *off, const uint32_t *rtype,
                              const uint32_t *rid, const uint32_t *mod, const int64_t *first_row,
                              int n_mod, long long cap_rows, uint32_t *out, int recompute)
{
    const spvt::Tables &TB = g_spv_tables;
    long long n_rows = first_row[n_mod];
    if (n_rows > cap_rows) n_rows = cap_rows;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rows; r += stride) {
        uint32_t m = mod[r];
        long long o = mod_off[m], n = mod_off[m + 1] - o;
        if (n > 0x7fffffffLL || header_status(words + o, n) != S_OK) continue;
        uint64_t p = off[r];
        uint32_t c = wc[r], opc = op[r];
        out[p] = (c << 16) | opc;
        if (opc < 256 && (TB.ops[opc].flags & 1)) {
            uint32_t q = 1;
            if (TB.ops[opc].flags & 2) { if (q < c) out[p + q] = rtype[r]; q++; }
            if (TB.ops[opc].flags & 4) { if (q < c) out[p + q] = rid[r]; }
        }
        if (recompute) atomicMax(&out[o + 3], rid[r] + 1);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Layout {
    size_t ctrl, tile_off, tile_rec, tstate, tmap, cstate, ms, fixlist, abase, arena, total;
    long long max_tiles, arena_words;
};

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int n_mod, long long n_words, long long arena_words, int tile_words)
{
    Layout L{};
    // a module of len words (first word ph < 4 past a 16-byte boundary) has
    // ceil((len + ph) / T) tiles, at least one: at most (len + T + 2) / T
    L.max_tiles = (n_words + 2LL * n_mod) / tile_words + n_mod + 1;
    L.arena_words = arena_words > 0 ? arena_words : 2 * n_words + 64LL * n_mod + 64;
    size_t o = 0;
    L.ctrl = o; o = al(o + sizeof(Ctrl));
    L.tile_off = o; o = al(o + 8 * (size_t)(n_mod + 1));
    L.tile_rec = o; o = al(o + sizeof(TileRec) * (size_t)L.max_tiles);
    L.tstate = o; o = al(o + 8 * (size_t)L.max_tiles);
    L.tmap = o; o = al(o + 4 * (size_t)NCAND * L.max_tiles);
    L.cstate = o; o = al(o + 8 * (size_t)L.max_tiles);
    L.ms = o; o = al(o + sizeof(ModState) * (size_t)n_mod);
    L.fixlist = o; o = al(o + 4 * (size_t)n_mod);
    L.abase = o; o = al(o + 8 * (size_t)(n_mod + 1));
    L.arena = o; o = al(o + 4 * (size_t)L.arena_words);
    L.total = o;
    return L;
}

struct Cfg { int T, NT, L, ctas_per_sm, per_module; long long max_spins, stall_tile, stall_map_tile; int spec; };

// A tile shape left unset (tile_words and threads both 0) follows the batch:
// batches of small modules (mean under 4,096 words) take 2,048-word tiles
// of 128 threads, others 4,096-word tiles of 256 threads (measured on
// 1,000-module bins of 200 to 50,000 instructions).
int resolve_cfg(const spv_config *c, Cfg *out, int n_modules, long long n_words)
{
    Cfg r{4096, 256, 16, 0, 0, 1LL << 20, -1, -1, 1};
    const bool auto_shape = !c || (!c->tile_words && !c->threads);
    if (auto_shape && n_modules > 0 && n_words / n_modules < 4096) { r.T = 2048; r.NT = 128; }
    if (c) {
        if (c->tile_words) r.T = c->tile_words;
        if (c->threads) r.NT = c->threads;
        if (c->ctas_per_sm < 0 || c->max_spins < 0) return SPV_E_ARG;
        r.ctas_per_sm = c->ctas_per_sm;
        r.per_module = c->per_module;
        if (c->max_spins) r.max_spins = c->max_spins;
        if (c->test_stall_tile > 0) r.stall_tile = c->test_stall_tile - 1;
        if (c->test_stall_tile < 0) r.stall_map_tile = -c->test_stall_tile - 1;
        if (c->no_speculation || c->test_stall_tile) r.spec = 0;
    }
    if (r.NT != 64 && r.NT != 128 && r.NT != 256 && r.NT != 512) return SPV_E_ARG;
    if (r.T % r.NT) return SPV_E_ARG;
    r.L = r.T / r.NT;
    if (r.L != 8 && r.L != 16) return SPV_E_ARG;
    if ((r.NT == 512 && r.L != 16) || (r.NT == 64 && r.L != 8)) return SPV_E_ARG;
    *out = r;
    return 0;
}

template <int NT, int L>
int launch_tile_kernel(const Params &P, int grid, cudaStream_t st)
{
    size_t sm = sizeof(TileSmem<NT, L>);
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev]) {
        if (cudaFuncSetAttribute(k_tile<NT, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return SPV_E_CUDA;
        configured[dev] = true;
    }
    SPV_LAUNCH("k_tile", st, k_tile<NT, L><<<grid, NT, sm, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? 0 : SPV_E_CUDA;
}

template <int NT, int L>
int occupancy(int *per_sm)
{
    // computed once per device
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && cached[dev] > 0) { *per_sm = cached[dev]; return 0; }
    size_t sm = sizeof(TileSmem<NT, L>);
    cudaFuncSetAttribute(k_tile<NT, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_tile<NT, L>, NT, sm) != cudaSuccess) return SPV_E_CUDA;
    if (dev < 64) cached[dev] = *per_sm;
    return 0;
}

int dispatch_tile(const Params &P, const Cfg &c, int grid, cudaStream_t st)
{
    if (c.NT == 512 && c.L == 16) return launch_tile_kernel<512, 16>(P, grid, st);
    if (c.NT == 256 && c.L == 16) return launch_tile_kernel<256, 16>(P, grid, st);
    if (c.NT == 256 && c.L == 8) return launch_tile_kernel<256, 8>(P, grid, st);
    if (c.NT == 128 && c.L == 16) return launch_tile_kernel<128, 16>(P, grid, st);
    if (c.NT == 128 && c.L == 8) return launch_tile_kernel<128, 8>(P, grid, st);
    if (c.NT == 64 && c.L == 8) return launch_tile_kernel<64, 8>(P, grid, st);
    return SPV_E_ARG;
}

int dispatch_occupancy(const Cfg &c, int *per_sm)
{
    if (c.NT == 512 && c.L == 16) return occupancy<512, 16>(per_sm);
    if (c.NT == 256 && c.L == 16) return occupancy<256, 16>(per_sm);
    if (c.NT == 256 && c.L == 8) return occupancy<256, 8>(per_sm);
    if (c.NT == 128 && c.L == 16) return occupancy<128, 16>(per_sm);
    if (c.NT == 128 && c.L == 8) return occupancy<128, 8>(per_sm);
    if (c.NT == 64 && c.L == 8) return occupancy<64, 8>(per_sm);
    return SPV_E_ARG;
}

bool check_batch(const spv_batch *b)
{
    return b && b->n_modules >= 0 && b->n_words >= 0 && (b->n_words == 0 || b->words) && b->mod_off;
}

Params base_params(const spv_batch *b, void *ws, const Layout &L, int tile_words)
{
    Params P{};
    P.tile_words = tile_words;
    P.stall_tile = -1;                 // test hooks off unless a call sets them
    P.stall_map_tile = -1;
    char *w = (char *)ws;
    P.words = b->words; P.mod_off = b->mod_off; P.n_modules = b->n_modules;
    P.ctrl = (Ctrl *)(w + L.ctrl);
    P.tile_off = (int64_t *)(w + L.tile_off);
    P.tile_rec = (TileRec *)(w + L.tile_rec);
    P.tstate = (unsigned long long *)(w + L.tstate);
    P.tmap = (uint32_t *)(w + L.tmap);
    P.cstate = (unsigned long long *)(w + L.cstate);
    P.ms = (ModState *)(w + L.ms);
    P.fixlist = (uint32_t *)(w + L.fixlist);
    P.abase = (int64_t *)(w + L.abase);
    P.arena = (uint32_t *)(w + L.arena);
    P.arena_words = L.arena_words;
    return P;
}

int sm_count()
{
    static int cached[64] = {};
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    if (dev < 64) cached[dev] = n;
    return n;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" size_t spv_workspace_bytes(int32_t n_modules, int64_t n_words, int64_t arena_words, const spv_config *cfg)
{
    Cfg c;
    if (n_modules < 0 || n_words < 0 || resolve_cfg(cfg, &c, n_modules, n_words)) return 0;
    return make_layout(n_modules, n_words, arena_words, c.T).total;
}

extern "C" int spv_process_batch(const spv_batch *batch, spv_table *table, uint32_t *status, int64_t *err_row,
                                 int validate, uint32_t *out_words, int recompute_bound, void *workspace,
                                 size_t workspace_bytes, int64_t arena_words, const spv_config *cfg,
                                 spv_stream_t stream)
{
    Cfg c;
    if (!check_batch(batch) || !table || !status || !err_row || resolve_cfg(cfg, &c, batch->n_modules, batch->n_words))
        return SPV_E_ARG;
    if (!table->op || !table->wc || !table->off || !table->rtype || !table->rid || !table->mod ||
        !table->mod_first_row || !table->mod_n_instr || table->capacity_rows < 0)
        return SPV_E_ARG;
    Layout L = make_layout(batch->n_modules, batch->n_words, arena_words, c.T);
    if (!workspace || workspace_bytes < L.total) return SPV_E_WORKSPACE;
    if (batch->n_modules == 0) return SPV_SUCCESS;
    cudaStream_t st = (cudaStream_t)stream;
    Params P = base_params(batch, workspace, L, c.T);
    P.op = table->op; P.wc = table->wc; P.off = table->off; P.rtype = table->rtype; P.rid = table->rid;
    P.mod = table->mod; P.first_row = table->mod_first_row; P.n_instr = table->mod_n_instr;
    P.cap_rows = table->capacity_rows;
    P.status = status; P.err_row = err_row;
    P.out = out_words; P.validate = validate ? 1 : 0; P.recompute_bound = recompute_bound ? 1 : 0;
    P.out_vec = out_words && ((((uintptr_t)out_words) - ((uintptr_t)batch->words)) & 15) == 0;
    P.max_spins = c.max_spins;
    P.stall_tile = c.stall_tile;
    P.stall_map_tile = c.stall_map_tile;
    int nsm = sm_count();
    std::vector<int64_t> off;
    if (c.per_module) {
        // comparison path: one launch per module, each CTA one tile
        off.resize(batch->n_modules + 1);
        if (cudaMemcpyAsync(off.data(), batch->mod_off, 8 * off.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SPV_E_CUDA;
    }
    // one pass of the kernels; with speculation a redo pass follows whose
    // kernels return at once unless a tile's entry guess failed, and
    // otherwise redo the batch without guesses
    auto pass = [&](int rerun) -> int {
        P.rerun = rerun;
        P.spec = (!rerun && !c.per_module) ? c.spec : 0;
        SPV_LAUNCH("k_prepass_mod", st, k_prepass_mod<<<nsm * 4, 256, 0, st>>>(P, c.T));
        SPV_LAUNCH("k_prepass_scan", st, k_prepass_scan<<<1, 1024, 0, st>>>(P));
        SPV_LAUNCH("k_tile_setup", st, k_tile_setup<<<nsm * 4, 256, 0, st>>>(P));
        if (cudaPeekAtLastError() != cudaSuccess) return SPV_E_CUDA;
        int rc;
        if (!c.per_module) {
            int per_sm = c.ctas_per_sm;
            if (per_sm <= 0) { if (dispatch_occupancy(c, &per_sm)) return SPV_E_CUDA; if (per_sm < 1) per_sm = 1; }
            P.persistent = 1;
            rc = dispatch_tile(P, c, nsm * per_sm, st);
        } else {
            P.persistent = 0;
            rc = 0;
            for (int m = 0; m < batch->n_modules && !rc; m++) {
                long long len = off[m + 1] - off[m];
                long long ph = word_phase(batch->words, off[m]);
                long long nt = len > 0 ? (len + ph + c.T - 1) / c.T : 1;
                rc = dispatch_tile(P, c, (int)nt, st);
            }
        }
        if (rc) return rc;
        int nb = (batch->n_modules + 255) / 256;
        if (validate) SPV_LAUNCH("k_id_popcount", st, k_id_popcount<<<nsm * 4, 256, 0, st>>>(P));
        SPV_LAUNCH("k_finalize", st, k_finalize<<<nb, 256, 0, st>>>(P));
        if (validate) SPV_LAUNCH("k_fixup", st, k_fixup<<<64, FIX_NT, 0, st>>>(P));
        return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
    };
    int rc = pass(0);
    if (rc == SPV_SUCCESS && P.spec) rc = pass(1);
    return rc;
}

// The tile shapes k_tile is built for, tried by the autotuner.
static const int kTileShapes[][2] = {{4096, 256}, {8192, 512}, {2048, 256}, {2048, 128}, {1024, 128}, {512, 64}};

extern "C" int spv_autotune_batch(const spv_batch *batch, spv_table *table, uint32_t *status, int64_t *err_row,
                                  int validate, uint32_t *out_words, void *workspace, size_t workspace_bytes,
                                  int reps, spv_config *best, float *best_ms, spv_stream_t stream)
{
    if (!best || !check_batch(batch)) return SPV_E_ARG;
    if (reps <= 0) reps = 3;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SPV_E_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SPV_E_CUDA; }
    int rc = SPV_SUCCESS, found = 0;
    float bms = 0.f;
    spv_config b{};
    for (const auto &shape : kTileShapes) {
        spv_config c{};
        c.tile_words = shape[0];
        c.threads = shape[1];
        if (spv_workspace_bytes(batch->n_modules, batch->n_words, 0, &c) > workspace_bytes) continue;
        rc = spv_process_batch(batch, table, status, err_row, validate, out_words, 1, workspace, workspace_bytes, 0,
                               &c, stream);                       // warm-up
        if (rc != SPV_SUCCESS) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = SPV_E_CUDA; break; }
        for (int r = 0; r < reps && rc == SPV_SUCCESS; r++)
            rc = spv_process_batch(batch, table, status, err_row, validate, out_words, 1, workspace,
                                   workspace_bytes, 0, &c, stream);
        if (rc != SPV_SUCCESS) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = SPV_E_CUDA; break; }
        ms /= (float)reps;
        if (!found || ms < bms) { found = 1; bms = ms; b = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPV_SUCCESS) return rc;
    if (!found) return SPV_E_WORKSPACE;
    // leave the outputs of the chosen shape behind
    rc = spv_process_batch(batch, table, status, err_row, validate, out_words, 1, workspace, workspace_bytes, 0, &b,
                           stream);
    if (rc != SPV_SUCCESS) return rc;
    *best = b;
    if (best_ms) *best_ms = bms;
    return cudaStreamSynchronize(st) == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}

extern "C" int spv_decode_batch(const spv_batch *batch, spv_table *table, uint32_t *status, int64_t *err_row,
                                void *workspace, size_t workspace_bytes, const spv_config *cfg, spv_stream_t stream)
{
    return spv_process_batch(batch, table, status, err_row, 0, nullptr, 0, workspace, workspace_bytes, 0, cfg,
                             stream);
}

extern "C" int spv_validate_batch(const spv_batch *batch, const spv_table *table, uint32_t *status,
                                  int64_t *err_row, void *workspace, size_t workspace_bytes, int64_t arena_words,
                                  spv_stream_t stream)
{
    Cfg c;
    if (!check_batch(batch) || !table || !status || !err_row ||
        resolve_cfg(nullptr, &c, batch->n_modules, batch->n_words))
        return SPV_E_ARG;
    if (!table->op || !table->wc || !table->off || !table->rid || !table->mod || !table->mod_first_row ||
        !table->mod_n_instr)
        return SPV_E_ARG;
    Layout L = make_layout(batch->n_modules, batch->n_words, arena_words, c.T);
    if (!workspace || workspace_bytes < L.total) return SPV_E_WORKSPACE;
    if (batch->n_modules == 0) return SPV_SUCCESS;
    cudaStream_t st = (cudaStream_t)stream;
    Params P = base_params(batch, workspace, L, c.T);
    P.op = table->op; P.wc = table->wc; P.off = table->off; P.rtype = table->rtype; P.rid = table->rid;
    P.mod = table->mod; P.first_row = table->mod_first_row; P.n_instr = table->mod_n_instr;
    P.cap_rows = table->capacity_rows;
    P.status = status; P.err_row = err_row;
    P.validate = 1;
    P.table_mode = 1;
    P.max_spins = c.max_spins;
    P.stall_tile = -1;
    P.stall_map_tile = -1;
    int nsm = sm_count();
    int nb = (batch->n_modules + 255) / 256;
    SPV_LAUNCH("k_prepass_mod", st, k_prepass_mod<<<sm_count() * 4, 256, 0, st>>>(P, c.T));
    SPV_LAUNCH("k_prepass_scan", st, k_prepass_scan<<<1, 1024, 0, st>>>(P));
    SPV_LAUNCH("k_tile_setup", st, k_tile_setup<<<nsm * 4, 256, 0, st>>>(P));
    SPV_LAUNCH("k_table_framing", st, k_table_framing<<<nb, 256, 0, st>>>(P));
    SPV_LAUNCH("k_validate_rows", st, k_validate_rows<<<nsm * 8, 256, 0, st>>>(P));
    SPV_LAUNCH("k_id_popcount", st, k_id_popcount<<<nsm * 4, 256, 0, st>>>(P));
    SPV_LAUNCH("k_finalize", st, k_finalize<<<nb, 256, 0, st>>>(P));
    SPV_LAUNCH("k_fixup", st, k_fixup<<<64, FIX_NT, 0, st>>>(P));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}

extern "C" int spv_encode_batch(const spv_batch *src, const spv_table *table, uint32_t *out_words,
                                int recompute_bound, spv_stream_t stream)
{
    if (!check_batch(src) || !table || !out_words || !table->mod_first_row || !table->op || !table->wc ||
        !table->off || !table->rtype || !table->rid || !table->mod)
        return SPV_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (src->n_words &&
        cudaMemcpyAsync(out_words, src->words, 4 * (size_t)src->n_words, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SPV_E_CUDA;
    if (src->n_modules == 0) return SPV_SUCCESS;
    if (recompute_bound)
        SPV_LAUNCH("k_encode_bound_init", st, k_encode_bound_init<<<(src->n_modules + 255) / 256, 256, 0, st>>>(src->words, src->mod_off, src->n_modules,
                                                                          out_words));
    int nsm = sm_count();
    SPV_LAUNCH("k_encode_rows", st, k_encode_rows<<<nsm * 8, 256, 0, st>>>(src->words, src->mod_off, table->op, table->wc, table->off,
                                           table->rtype, table->rid, table->mod, table->mod_first_row,
                                           src->n_modules, table->capacity_rows, out_words, recompute_bound));
    return cudaPeekAtLastError() == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
}

// ---------------------------------------------------------------------------
// spv_process_batch_noalloc: the fused decode / validate / encode without any
// allocation by the caller or the library. Some callers cannot allocate
// device memory: a host runtime that reserves all of a GPU's memory in its
// own pool up front and forbids other allocations, or a latency-bound
// serving loop where cudaMalloc could stall the device or fail under memory
// pressure. They still own inputs and outputs; the scratch the kernels need
// (tile look-back states, per-module aggregates, the result-id sets) lives
// in the fixed array below instead of a caller-provided workspace.
// ---------------------------------------------------------------------------
namespace {
// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SPV_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
// Per device: the array's device address (host code cannot use its name) and
// the context it was looked up in. A context torn down and made again (for
// example after cudaDeviceReset) loads the module again, and the array may
// then sit elsewhere, so the address is looked up again whenever the current
// context differs from the cached one.
struct NoallocSlot { void *addr; void *ctx; };
NoallocSlot g_noalloc_slot[1024];
typedef int (*CtxGetCurrentFn)(void **);
CtxGetCurrentFn g_ctx_get_current;     // the driver's cuCtxGetCurrent, found once
bool g_ctx_lookup_done;

void *current_context()
{
    if (!g_ctx_lookup_done) {
        g_ctx_lookup_done = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = (CtxGetCurrentFn)fn;
    }
    void *ctx = nullptr;
    if (!g_ctx_get_current || g_ctx_get_current(&ctx) != 0) return nullptr;
    return ctx;
}
}  // namespace

extern "C" int spv_process_batch_noalloc(const spv_batch *batch, spv_table *table, uint32_t *status,
                                         int64_t *err_row, int validate, uint32_t *out_words,
                                         int recompute_bound, const spv_config *cfg, spv_stream_t stream)
{
    // the argument checks of spv_process_batch come first, so a bad argument
    // is SPV_E_ARG whatever the batch's size
    Cfg c;
    if (!check_batch(batch) || !table || !status || !err_row || resolve_cfg(cfg, &c, batch->n_modules, batch->n_words))
        return SPV_E_ARG;
    if (!table->op || !table->wc || !table->off || !table->rtype || !table->rid || !table->mod ||
        !table->mod_first_row || !table->mod_n_instr || table->capacity_rows < 0)
        return SPV_E_ARG;
    if (c.per_module) return SPV_E_UNSUPPORTED;
    if (make_layout(batch->n_modules, batch->n_words, 0, c.T).total > (size_t)SPV_NOALLOC_SCRATCH_BYTES)
        return SPV_E_WORKSPACE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 1024) return SPV_E_CUDA;
    void *scratch = nullptr;
    {
        // set-up, once per device (and again after its context is made anew),
        // with that device current
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        void *ctx = current_context();          // null before the runtime has made one current
        NoallocSlot &sl = g_noalloc_slot[dev];
        if (!sl.addr || !ctx || ctx != sl.ctx) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPV_E_CUDA;
            sl.addr = p;
            sl.ctx = current_context();         // the context the lookup ran in
        }
        scratch = sl.addr;
    }
    // the kernels initialise every part of the scratch they read (look-back
    // states, counters, module states and id sets are cleared on the device
    // at the start of each call), so the previous call's contents never leak
    return spv_process_batch(batch, table, status, err_row, validate, out_words, recompute_bound, scratch,
                             (size_t)SPV_NOALLOC_SCRATCH_BYTES, 0, cfg, stream);
}
