/*
 * spv_synth.c -- seeded generator of synthetic SPIR-V compute modules.
 *
 * Input generation only: it writes modules and records where it put each
 * instruction, nothing more. It neither decodes, validates nor prints
 * modules, and it shares no code with the CUDA library or the CPU oracle,
 * both of which consume its output.
 *
 * Shape: what a JIT backend emits for OpenCL-style compute kernels (the
 * paper's use case, section 4): capabilities Addresses / Kernel / Int64, the
 * OpenCL.std extended set, Physical64 OpenCL memory model, one entry point
 * per kernel with a LocalSize execution mode, decorations, a block of types
 * and constants, a GlobalInvocationId input variable, then functions made of
 * basic blocks of integer / float arithmetic, pointer access chains, loads,
 * stores, conversions, comparisons, phis and structured branches. Optional
 * OpString / OpName instructions carry random printable ASCII strings.
 * Operand ids are drawn uniformly from already-defined ids of the right kind,
 * so every module is valid; the header bound is the largest id plus one.
 *
 * Random numbers: xoshiro256** seeded through splitmix64 (Blackman & Vigna,
 * "Scrambled linear pseudorandom number generators", 2021).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- random numbers ---------------- */
typedef struct { uint64_t s[4]; } Rng;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static void rng_seed(Rng *r, uint64_t seed)
{
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
static uint64_t rng_next(Rng *r)
{
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return result;
}
static uint32_t rng_below(Rng *r, uint32_t n) { return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)n) >> 32); }
static double rng_unit(Rng *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static double rng_normal(Rng *r)
{
    double u1 = rng_unit(r), u2 = rng_unit(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ---------------- growable word sections ---------------- */
typedef struct { uint32_t *w; int64_t n, cap; int64_t *st; int64_t ns, scap; int64_t cur; } Sec;

static void sec_word(Sec *s, uint32_t v)
{
    if (s->n == s->cap) { s->cap = s->cap ? s->cap * 2 : 1024; s->w = (uint32_t *)realloc(s->w, (size_t)s->cap * 4); }
    s->w[s->n++] = v;
}
static void sec_begin(Sec *s, uint32_t opcode)
{
    if (s->ns == s->scap) { s->scap = s->scap ? s->scap * 2 : 256; s->st = (int64_t *)realloc(s->st, (size_t)s->scap * 8); }
    s->st[s->ns++] = s->n;
    s->cur = s->n;
    sec_word(s, opcode);
}
static void sec_end(Sec *s) { s->w[s->cur] |= (uint32_t)(s->n - s->cur) << 16; }
static void sec_str(Sec *s, const char *str, int len)
{
    int nw = len / 4 + 1;
    for (int i = 0; i < nw; i++) {
        uint32_t v = 0;
        for (int b = 0; b < 4; b++) {
            int k = 4 * i + b;
            if (k < len) v |= (uint32_t)(uint8_t)str[k] << (8 * b);
        }
        sec_word(s, v);
    }
}
static void sec_free(Sec *s) { free(s->w); free(s->st); memset(s, 0, sizeof *s); }

/* ---------------- id pools ---------------- */
typedef struct { uint32_t *v; int n, cap; } Pool;
static void pool_add(Pool *p, uint32_t id)
{
    if (p->n == p->cap) { p->cap = p->cap ? p->cap * 2 : 64; p->v = (uint32_t *)realloc(p->v, (size_t)p->cap * 4); }
    p->v[p->n++] = id;
}
static uint32_t pool_pick(Rng *r, const Pool *p) { return p->v[rng_below(r, (uint32_t)p->n)]; }
static void pool_free(Pool *p) { free(p->v); memset(p, 0, sizeof *p); }

/* opcodes and enumerants written by the generator (SPIR-V 1.2 numbering) */
enum {
    O_Source = 3, O_Name = 5, O_String = 7, O_ExtInstImport = 11, O_ExtInst = 12, O_MemoryModel = 14,
    O_EntryPoint = 15, O_ExecutionMode = 16, O_Capability = 17, O_TypeVoid = 19, O_TypeBool = 20,
    O_TypeInt = 21, O_TypeFloat = 22, O_TypeVector = 23, O_TypePointer = 32, O_TypeFunction = 33,
    O_ConstantTrue = 41, O_ConstantFalse = 42, O_Constant = 43, O_ConstantNull = 46, O_Function = 54,
    O_FunctionParameter = 55, O_FunctionEnd = 56, O_FunctionCall = 57, O_Variable = 59, O_Load = 61,
    O_Store = 62, O_PtrAccessChain = 67, O_InBoundsPtrAccessChain = 70, O_Decorate = 71,
    O_CompositeExtract = 81, O_ConvertFToU = 109, O_ConvertUToF = 112, O_UConvert = 113,
    O_Bitcast = 124, O_SNegate = 126, O_FNegate = 127, O_IAdd = 128, O_FAdd = 129, O_ISub = 130,
    O_FSub = 131, O_IMul = 132, O_FMul = 133, O_UDiv = 134, O_FDiv = 136, O_UMod = 137,
    O_Select = 169, O_IEqual = 170, O_UGreaterThan = 172, O_ULessThan = 176, O_FOrdEqual = 180,
    O_FOrdLessThan = 184, O_FOrdGreaterThan = 186, O_ShiftRightLogical = 194, O_ShiftLeftLogical = 196,
    O_BitwiseOr = 197, O_BitwiseXor = 198, O_BitwiseAnd = 199, O_Not = 200, O_ControlBarrier = 224,
    O_AtomicIAdd = 234, O_Phi = 245, O_LoopMerge = 246, O_SelectionMerge = 247, O_Label = 248,
    O_Branch = 249, O_BranchConditional = 250, O_Return = 253
};

typedef struct {
    Rng rng;
    uint32_t next_id;
    Sec caps, head, entries, modes, debug, annot, types, funcs;
    /* types */
    uint32_t t_void, t_bool, t_uint, t_ulong, t_float, t_v3ulong, t_ptr_in_v3, t_ptr_uint, t_ptr_float, t_fn;
    uint32_t ext, v_gid;
    Pool c_uint, c_float, c_ulong, c_bool;    /* global constants */
    Pool all_ids, funcs_ids, params;
} Gen;

static uint32_t new_id(Gen *g) { uint32_t id = g->next_id++; pool_add(&g->all_ids, id); return id; }

/* first id handed out (1 normally); synth_oplist_batch generates each module
 * a second time from a high base to tell id words from literal words */
static uint32_t s_id_base = 1;

static void random_ascii(Rng *r, char *buf, int len)
{
    for (int i = 0; i < len; i++) buf[i] = (char)(0x20 + rng_below(r, 0x7f - 0x20));
}

/* one basic block body step; appends instructions, returns how many */
static int body_step(Gen *g, Sec *s, Pool *vu, Pool *vf, Pool *vb, Pool *vl, const uint32_t *prm)
{
    Rng *r = &g->rng;
    uint32_t k = rng_below(r, 100);
    if (k < 25) {
        static const uint32_t ops[] = {O_IAdd, O_ISub, O_IMul, O_UDiv, O_UMod, O_ShiftLeftLogical,
                                       O_ShiftRightLogical, O_BitwiseAnd, O_BitwiseOr, O_BitwiseXor};
        uint32_t id = new_id(g);
        sec_begin(s, ops[rng_below(r, 10)]); sec_word(s, g->t_uint); sec_word(s, id);
        sec_word(s, pool_pick(r, vu)); sec_word(s, pool_pick(r, vu)); sec_end(s);
        pool_add(vu, id); return 1;
    }
    if (k < 45) {
        static const uint32_t ops[] = {O_FAdd, O_FSub, O_FMul, O_FDiv};
        uint32_t id = new_id(g);
        sec_begin(s, ops[rng_below(r, 4)]); sec_word(s, g->t_float); sec_word(s, id);
        sec_word(s, pool_pick(r, vf)); sec_word(s, pool_pick(r, vf)); sec_end(s);
        pool_add(vf, id); return 1;
    }
    if (k < 55) {   /* load through an access chain */
        int is_f = rng_below(r, 2);
        uint32_t ptr = new_id(g), val = new_id(g);
        sec_begin(s, rng_below(r, 4) ? O_InBoundsPtrAccessChain : O_PtrAccessChain);
        sec_word(s, is_f ? g->t_ptr_float : g->t_ptr_uint); sec_word(s, ptr);
        sec_word(s, is_f ? prm[1] : prm[0]); sec_word(s, pool_pick(r, vl)); sec_end(s);
        sec_begin(s, O_Load); sec_word(s, is_f ? g->t_float : g->t_uint); sec_word(s, val); sec_word(s, ptr);
        sec_word(s, 0x2); sec_word(s, 4); sec_end(s);
        pool_add(is_f ? vf : vu, val); return 2;
    }
    if (k < 63) {   /* store through an access chain */
        int is_f = rng_below(r, 2);
        uint32_t ptr = new_id(g);
        sec_begin(s, O_InBoundsPtrAccessChain);
        sec_word(s, is_f ? g->t_ptr_float : g->t_ptr_uint); sec_word(s, ptr);
        sec_word(s, is_f ? prm[1] : prm[0]); sec_word(s, pool_pick(r, vl)); sec_end(s);
        sec_begin(s, O_Store); sec_word(s, ptr); sec_word(s, pool_pick(r, is_f ? vf : vu));
        if (rng_below(r, 2)) { sec_word(s, 0x2); sec_word(s, 4); }
        sec_end(s);
        return 2;
    }
    if (k < 70) {   /* conversions */
        uint32_t c = rng_below(r, 3), id = new_id(g);
        if (c == 0) { sec_begin(s, O_ConvertUToF); sec_word(s, g->t_float); sec_word(s, id); sec_word(s, pool_pick(r, vu)); pool_add(vf, id); }
        else if (c == 1) { sec_begin(s, O_ConvertFToU); sec_word(s, g->t_uint); sec_word(s, id); sec_word(s, pool_pick(r, vf)); pool_add(vu, id); }
        else { sec_begin(s, O_UConvert); sec_word(s, g->t_ulong); sec_word(s, id); sec_word(s, pool_pick(r, vu)); pool_add(vl, id); }
        sec_end(s); return 1;
    }
    if (k < 75) {   /* comparisons */
        uint32_t id = new_id(g);
        if (rng_below(r, 2)) {
            static const uint32_t ops[] = {O_IEqual, O_ULessThan, O_UGreaterThan};
            sec_begin(s, ops[rng_below(r, 3)]); sec_word(s, g->t_bool); sec_word(s, id);
            sec_word(s, pool_pick(r, vu)); sec_word(s, pool_pick(r, vu));
        } else {
            static const uint32_t ops[] = {O_FOrdEqual, O_FOrdLessThan, O_FOrdGreaterThan};
            sec_begin(s, ops[rng_below(r, 3)]); sec_word(s, g->t_bool); sec_word(s, id);
            sec_word(s, pool_pick(r, vf)); sec_word(s, pool_pick(r, vf));
        }
        sec_end(s); pool_add(vb, id); return 1;
    }
    if (k < 79) {
        uint32_t id = new_id(g);
        sec_begin(s, O_Select); sec_word(s, g->t_uint); sec_word(s, id); sec_word(s, pool_pick(r, vb));
        sec_word(s, pool_pick(r, vu)); sec_word(s, pool_pick(r, vu)); sec_end(s);
        pool_add(vu, id); return 1;
    }
    if (k < 83) {   /* OpenCL.std call: fabs 23, sqrt 61, exp 19, fmax 27 */
        static const uint32_t ext_ops[] = {23, 61, 19, 27};
        uint32_t e = rng_below(r, 4), id = new_id(g);
        sec_begin(s, O_ExtInst); sec_word(s, g->t_float); sec_word(s, id); sec_word(s, g->ext);
        sec_word(s, ext_ops[e]); sec_word(s, pool_pick(r, vf));
        if (e == 3) sec_word(s, pool_pick(r, vf));
        sec_end(s); pool_add(vf, id); return 1;
    }
    if (k < 88) {   /* unary */
        uint32_t c = rng_below(r, 4), id = new_id(g);
        if (c == 0) { sec_begin(s, O_SNegate); sec_word(s, g->t_uint); sec_word(s, id); sec_word(s, pool_pick(r, vu)); pool_add(vu, id); }
        else if (c == 1) { sec_begin(s, O_FNegate); sec_word(s, g->t_float); sec_word(s, id); sec_word(s, pool_pick(r, vf)); pool_add(vf, id); }
        else if (c == 2) { sec_begin(s, O_Not); sec_word(s, g->t_uint); sec_word(s, id); sec_word(s, pool_pick(r, vu)); pool_add(vu, id); }
        else { sec_begin(s, O_Bitcast); sec_word(s, g->t_float); sec_word(s, id); sec_word(s, pool_pick(r, vu)); pool_add(vf, id); }
        sec_end(s); return 1;
    }
    if (k < 91 && g->funcs_ids.n > 0) {
        uint32_t id = new_id(g);
        sec_begin(s, O_FunctionCall); sec_word(s, g->t_void); sec_word(s, id); sec_word(s, pool_pick(r, &g->funcs_ids));
        sec_word(s, prm[0]); sec_word(s, prm[1]); sec_word(s, pool_pick(r, vu)); sec_end(s);
        return 1;
    }
    if (k < 95) {
        uint32_t ptr = new_id(g), id = new_id(g);
        sec_begin(s, O_InBoundsPtrAccessChain); sec_word(s, g->t_ptr_uint); sec_word(s, ptr);
        sec_word(s, prm[0]); sec_word(s, pool_pick(r, vl)); sec_end(s);
        sec_begin(s, O_AtomicIAdd); sec_word(s, g->t_uint); sec_word(s, id); sec_word(s, ptr);
        sec_word(s, pool_pick(r, &g->c_uint)); sec_word(s, pool_pick(r, &g->c_uint)); sec_word(s, pool_pick(r, vu));
        sec_end(s); pool_add(vu, id); return 2;
    }
    if (k < 97) {
        sec_begin(s, O_ControlBarrier); sec_word(s, pool_pick(r, &g->c_uint)); sec_word(s, pool_pick(r, &g->c_uint));
        sec_word(s, pool_pick(r, &g->c_uint)); sec_end(s);
        return 1;
    }
    {
        uint32_t id = new_id(g);
        sec_begin(s, O_IAdd); sec_word(s, g->t_ulong); sec_word(s, id);
        sec_word(s, pool_pick(r, vl)); sec_word(s, pool_pick(r, vl)); sec_end(s);
        pool_add(vl, id); return 1;
    }
}

/* one function of about budget instructions in blocks of about block_len */
static void gen_function(Gen *g, uint32_t fid, int64_t budget, int block_len)
{
    Rng *r = &g->rng;
    Sec *s = &g->funcs;
    if (budget < 12) budget = 12;
    int64_t nblocks = budget / (block_len > 4 ? block_len : 4);
    if (nblocks < 1) nblocks = 1;
    uint32_t *labels = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nblocks);
    for (int64_t b = 0; b < nblocks; b++) labels[b] = new_id(g);
    Pool vu = {0}, vf = {0}, vb = {0}, vl = {0};
    for (int i = 0; i < g->c_uint.n; i++) pool_add(&vu, g->c_uint.v[i]);
    for (int i = 0; i < g->c_float.n; i++) pool_add(&vf, g->c_float.v[i]);
    for (int i = 0; i < g->c_bool.n; i++) pool_add(&vb, g->c_bool.v[i]);
    for (int i = 0; i < g->c_ulong.n; i++) pool_add(&vl, g->c_ulong.v[i]);
    int64_t used = 0;
    uint32_t prm[3];
    sec_begin(s, O_Function); sec_word(s, g->t_void); sec_word(s, fid); sec_word(s, 0); sec_word(s, g->t_fn); sec_end(s);
    uint32_t ptys[3] = {g->t_ptr_uint, g->t_ptr_float, g->t_uint};
    for (int i = 0; i < 3; i++) {
        prm[i] = new_id(g);
        sec_begin(s, O_FunctionParameter); sec_word(s, ptys[i]); sec_word(s, prm[i]); sec_end(s);
        pool_add(&g->params, prm[i]);
    }
    pool_add(&vu, prm[2]);
    used += 5;   /* OpFunction, 3 parameters, OpFunctionEnd */
    for (int64_t b = 0; b < nblocks; b++) {
        sec_begin(s, O_Label); sec_word(s, labels[b]); sec_end(s); used++;
        if (b == 0) {
            uint32_t g3 = new_id(g), gx = new_id(g);
            sec_begin(s, O_Load); sec_word(s, g->t_v3ulong); sec_word(s, g3); sec_word(s, g->v_gid);
            sec_word(s, 0x2); sec_word(s, 32); sec_end(s);
            sec_begin(s, O_CompositeExtract); sec_word(s, g->t_ulong); sec_word(s, gx); sec_word(s, g3);
            sec_word(s, 0); sec_end(s);
            pool_add(&vl, gx); used += 2;
        } else {
            int nphi = (int)rng_below(r, 3);
            for (int k = 0; k < nphi; k++) {
                uint32_t id = new_id(g);
                int pairs = 1 + (int)rng_below(r, 3);
                sec_begin(s, O_Phi); sec_word(s, g->t_uint); sec_word(s, id);
                for (int q = 0; q < pairs; q++) { sec_word(s, pool_pick(r, &vu)); sec_word(s, labels[rng_below(r, (uint32_t)b)]); }
                sec_end(s); pool_add(&vu, id); used++;
            }
        }
        int64_t remaining_blocks = nblocks - b;
        int64_t target = (budget - used) / remaining_blocks - 3;
        if (target < 0) target = 0;
        for (int64_t k = 0; k < target;) { int n = body_step(g, s, &vu, &vf, &vb, &vl, prm); k += n; used += n; }
        if (b == nblocks - 1) { sec_begin(s, O_Return); sec_end(s); used++; }
        else {
            uint32_t choice = rng_below(r, 3);
            uint32_t tgt = labels[b + 1];
            uint32_t other = labels[b + 1 + rng_below(r, (uint32_t)(nblocks - b - 1))];
            if (choice == 0) { sec_begin(s, O_Branch); sec_word(s, tgt); sec_end(s); used++; }
            else {
                if (choice == 1) { sec_begin(s, O_SelectionMerge); sec_word(s, other); sec_word(s, 0); sec_end(s); }
                else { sec_begin(s, O_LoopMerge); sec_word(s, other); sec_word(s, tgt); sec_word(s, rng_below(r, 2)); sec_end(s); }
                sec_begin(s, O_BranchConditional); sec_word(s, pool_pick(r, &vb)); sec_word(s, tgt); sec_word(s, other);
                sec_end(s); used += 2;
            }
        }
    }
    sec_begin(s, O_FunctionEnd); sec_end(s);
    free(labels);
    pool_free(&vu); pool_free(&vf); pool_free(&vb); pool_free(&vl);
}

static void sec_cat(Sec *dst, const Sec *src)
{
    for (int64_t i = 0; i < src->ns; i++) {
        if (dst->ns == dst->scap) { dst->scap = dst->scap ? dst->scap * 2 : 256; dst->st = (int64_t *)realloc(dst->st, (size_t)dst->scap * 8); }
        dst->st[dst->ns++] = dst->n + src->st[i];
    }
    for (int64_t i = 0; i < src->n; i++) sec_word(dst, src->w[i]);
}

/* Generate one module.
 *   func_instr       instructions across all function bodies
 *   n_kernels        entry points (>= 1); n_funcs >= n_kernels functions
 *   block_len        mean instructions per basic block
 *   n_decorations    OpDecorate instructions
 *   n_consts         constants besides the type block
 *   string_permille  OpString / OpName instructions per 1000 of the total
 * Writes at most cap words to out (out may be NULL to size), the module's
 * instruction start offsets to starts (up to starts_cap; may be NULL), the
 * instruction count to *n_instr and the header bound to *bound.
 * Returns the module's length in words. */
int64_t synth_module(uint64_t seed, int64_t func_instr, int32_t n_kernels, int32_t n_funcs,
                     int32_t block_len, int32_t n_decorations, int32_t n_consts, int32_t string_permille,
                     uint32_t *out, int64_t cap, int64_t *starts, int64_t starts_cap,
                     int64_t *n_instr, uint32_t *bound)
{
    Gen *g = (Gen *)calloc(1, sizeof(Gen));
    rng_seed(&g->rng, seed);
    Rng *r = &g->rng;
    g->next_id = s_id_base;
    if (n_kernels < 1) n_kernels = 1;
    if (n_funcs < n_kernels) n_funcs = n_kernels;

    /* capabilities, import, memory model */
    static const uint32_t caps[] = {4, 6, 11};   /* Addresses, Kernel, Int64 */
    for (int i = 0; i < 3; i++) { sec_begin(&g->caps, O_Capability); sec_word(&g->caps, caps[i]); sec_end(&g->caps); }
    g->ext = new_id(g);
    sec_begin(&g->head, O_ExtInstImport); sec_word(&g->head, g->ext); sec_str(&g->head, "OpenCL.std", 10); sec_end(&g->head);
    sec_begin(&g->head, O_MemoryModel); sec_word(&g->head, 2); sec_word(&g->head, 2); sec_end(&g->head);

    /* types */
    Sec *t = &g->types;
    g->t_void = new_id(g); sec_begin(t, O_TypeVoid); sec_word(t, g->t_void); sec_end(t);
    g->t_bool = new_id(g); sec_begin(t, O_TypeBool); sec_word(t, g->t_bool); sec_end(t);
    g->t_uint = new_id(g); sec_begin(t, O_TypeInt); sec_word(t, g->t_uint); sec_word(t, 32); sec_word(t, 0); sec_end(t);
    g->t_ulong = new_id(g); sec_begin(t, O_TypeInt); sec_word(t, g->t_ulong); sec_word(t, 64); sec_word(t, 0); sec_end(t);
    g->t_float = new_id(g); sec_begin(t, O_TypeFloat); sec_word(t, g->t_float); sec_word(t, 32); sec_end(t);
    g->t_v3ulong = new_id(g); sec_begin(t, O_TypeVector); sec_word(t, g->t_v3ulong); sec_word(t, g->t_ulong); sec_word(t, 3); sec_end(t);
    g->t_ptr_in_v3 = new_id(g); sec_begin(t, O_TypePointer); sec_word(t, g->t_ptr_in_v3); sec_word(t, 1); sec_word(t, g->t_v3ulong); sec_end(t);
    g->t_ptr_uint = new_id(g); sec_begin(t, O_TypePointer); sec_word(t, g->t_ptr_uint); sec_word(t, 5); sec_word(t, g->t_uint); sec_end(t);
    g->t_ptr_float = new_id(g); sec_begin(t, O_TypePointer); sec_word(t, g->t_ptr_float); sec_word(t, 5); sec_word(t, g->t_float); sec_end(t);
    g->t_fn = new_id(g); sec_begin(t, O_TypeFunction); sec_word(t, g->t_fn); sec_word(t, g->t_void);
    sec_word(t, g->t_ptr_uint); sec_word(t, g->t_ptr_float); sec_word(t, g->t_uint); sec_end(t);
    /* constants: a few of each kind always exist so every pool is non-empty */
    for (int i = 0; i < 4 + n_consts; i++) {
        uint32_t kind = i < 4 ? (uint32_t)i : rng_below(r, 6);
        uint32_t id = new_id(g);
        if (kind == 0 || kind == 4) {
            sec_begin(t, O_Constant); sec_word(t, g->t_uint); sec_word(t, id); sec_word(t, rng_below(r, 1u << 20)); sec_end(t);
            pool_add(&g->c_uint, id);
        } else if (kind == 1 || kind == 5) {
            float f = (float)((rng_unit(r) - 0.5) * 256.0);
            if (rng_below(r, 4) == 0) f = (float)(int)f;
            uint32_t bits; memcpy(&bits, &f, 4);
            sec_begin(t, O_Constant); sec_word(t, g->t_float); sec_word(t, id); sec_word(t, bits); sec_end(t);
            pool_add(&g->c_float, id);
        } else if (kind == 2) {
            uint64_t v = rng_next(r) >> rng_below(r, 64);
            sec_begin(t, O_Constant); sec_word(t, g->t_ulong); sec_word(t, id); sec_word(t, (uint32_t)v); sec_word(t, (uint32_t)(v >> 32)); sec_end(t);
            pool_add(&g->c_ulong, id);
        } else {
            uint32_t which = rng_below(r, 3);
            sec_begin(t, which == 0 ? O_ConstantTrue : which == 1 ? O_ConstantFalse : O_ConstantNull);
            sec_word(t, g->t_bool); sec_word(t, id); sec_end(t);
            pool_add(&g->c_bool, id);
        }
    }
    g->v_gid = new_id(g);
    sec_begin(t, O_Variable); sec_word(t, g->t_ptr_in_v3); sec_word(t, g->v_gid); sec_word(t, 1); sec_end(t);

    /* module-level instruction count so far and string budget */
    int64_t fixed = 3 + 2 + 2 * (int64_t)n_kernels + 1 + n_decorations + g->types.ns + n_kernels;
    int64_t total_target = fixed + func_instr;
    int64_t n_strings = (int64_t)((double)total_target * string_permille / (1000.0 - string_permille));

    /* functions: kernels first; helpers are callable from later functions */
    uint32_t *fids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_funcs);
    for (int f = 0; f < n_funcs; f++) fids[f] = new_id(g);
    int64_t per = func_instr / n_funcs;
    for (int f = n_funcs - 1; f >= 0; f--) {
        int64_t b = (f == 0) ? func_instr - per * (n_funcs - 1) : per;
        gen_function(g, fids[f], b, block_len);
        if (f >= n_kernels) pool_add(&g->funcs_ids, fids[f]);
    }

    /* entry points, execution modes, kernel names */
    for (int k = 0; k < n_kernels; k++) {
        char nm[32]; int len = 0;
        { const char *pfx = "kernel_"; while (pfx[len]) { nm[len] = pfx[len]; len++; } }
        { char d[12]; int nd = 0; int v = k; do { d[nd++] = (char)('0' + v % 10); v /= 10; } while (v); while (nd) nm[len++] = d[--nd]; }
        sec_begin(&g->entries, O_EntryPoint); sec_word(&g->entries, 6); sec_word(&g->entries, fids[k]);
        sec_str(&g->entries, nm, len); sec_word(&g->entries, g->v_gid); sec_end(&g->entries);
        sec_begin(&g->modes, O_ExecutionMode); sec_word(&g->modes, fids[k]); sec_word(&g->modes, 17);
        sec_word(&g->modes, 1u << (5 + rng_below(r, 4))); sec_word(&g->modes, 1); sec_word(&g->modes, 1); sec_end(&g->modes);
        sec_begin(&g->debug, O_Name); sec_word(&g->debug, fids[k]); sec_str(&g->debug, nm, len); sec_end(&g->debug);
    }
    sec_begin(&g->debug, O_Source); sec_word(&g->debug, 3); sec_word(&g->debug, 200000); sec_end(&g->debug);
    for (int64_t i = 0; i < n_strings; i++) {
        char buf[64];
        int len = 1 + (int)rng_below(r, 64);
        random_ascii(r, buf, len);
        if (i % 2 == 0) {
            uint32_t id = new_id(g);
            sec_begin(&g->debug, O_String); sec_word(&g->debug, id); sec_str(&g->debug, buf, len); sec_end(&g->debug);
        } else {
            uint32_t target = g->all_ids.v[rng_below(r, (uint32_t)g->all_ids.n)];
            sec_begin(&g->debug, O_Name); sec_word(&g->debug, target); sec_str(&g->debug, buf, len); sec_end(&g->debug);
        }
    }

    /* decorations */
    sec_begin(&g->annot, O_Decorate); sec_word(&g->annot, g->v_gid); sec_word(&g->annot, 11); sec_word(&g->annot, 28); sec_end(&g->annot);
    for (int i = 1; i < n_decorations; i++) {
        uint32_t target = g->params.n ? pool_pick(r, &g->params) : g->v_gid;
        uint32_t kind = rng_below(r, 6);
        sec_begin(&g->annot, O_Decorate); sec_word(&g->annot, target);
        if (kind == 0) { sec_word(&g->annot, 38); sec_word(&g->annot, 5); }          /* FuncParamAttr NoCapture */
        else if (kind == 1) { sec_word(&g->annot, 44); sec_word(&g->annot, 4); }     /* Alignment 4 */
        else if (kind == 2) { sec_word(&g->annot, 19); }                            /* Restrict */
        else if (kind == 3) { sec_word(&g->annot, 24); }                            /* NonWritable */
        else if (kind == 4) { sec_word(&g->annot, 21); }                            /* Volatile */
        else { sec_word(&g->annot, 38); sec_word(&g->annot, 4); }                   /* FuncParamAttr NoAlias */
        sec_end(&g->annot);
    }

    /* assemble in logical-layout order behind the 5-word header */
    Sec all = {0};
    for (int i = 0; i < 5; i++) sec_word(&all, 0);
    sec_cat(&all, &g->caps); sec_cat(&all, &g->head); sec_cat(&all, &g->entries); sec_cat(&all, &g->modes);
    sec_cat(&all, &g->debug); sec_cat(&all, &g->annot); sec_cat(&all, &g->types); sec_cat(&all, &g->funcs);
    all.w[0] = 0x07230203u; all.w[1] = 0x00010200u; all.w[2] = 32; all.w[3] = g->next_id; all.w[4] = 0;

    int64_t n = all.n;
    if (out) memcpy(out, all.w, (size_t)(n < cap ? n : cap) * 4);
    if (starts) memcpy(starts, all.st, (size_t)(all.ns < starts_cap ? all.ns : starts_cap) * 8);
    if (n_instr) *n_instr = all.ns;
    if (bound) *bound = g->next_id;

    sec_free(&all); sec_free(&g->caps); sec_free(&g->head); sec_free(&g->entries); sec_free(&g->modes);
    sec_free(&g->debug); sec_free(&g->annot); sec_free(&g->types); sec_free(&g->funcs);
    pool_free(&g->c_uint); pool_free(&g->c_float); pool_free(&g->c_ulong); pool_free(&g->c_bool);
    pool_free(&g->all_ids); pool_free(&g->funcs_ids); pool_free(&g->params);
    free(fids); free(g);
    return n;
}

/* Per-module shape of a batch: module m draws, from seed seed0 + m, an
 * instruction count exp(ln(median) + sigma * N(0,1)) clipped to [lo, hi] and
 * a kernel count uniform in [1, max_kernels]. */
void synth_batch_shape(int32_t n_mod, uint64_t seed0, double median, double sigma, int64_t lo, int64_t hi,
                       int32_t max_kernels, int64_t *n_instr, int32_t *n_kernels)
{
    for (int32_t m = 0; m < n_mod; m++) {
        Rng r; rng_seed(&r, (seed0 + (uint64_t)m) ^ 0x5bd1e995ull);
        double x = exp(log(median) + sigma * rng_normal(&r));
        int64_t n = (int64_t)(x + 0.5);
        if (n < lo) n = lo;
        if (n > hi) n = hi;
        n_instr[m] = n;
        n_kernels[m] = 1 + (int32_t)rng_below(&r, (uint32_t)max_kernels);
    }
}

/* Generate a batch: module m uses seed seed0 + m, n_instr[m] instructions in
 * total (about 100 of them module-level) and n_kernels[m] kernels. mod_off
 * receives M+1 offsets; out may be NULL to size. Returns the total words. */
int64_t synth_batch(int32_t n_mod, uint64_t seed0, const int64_t *n_instr, const int32_t *n_kernels,
                    int32_t string_permille, uint32_t *out, int64_t cap, int64_t *mod_off)
{
    int64_t total = 0;
    for (int32_t m = 0; m < n_mod; m++) {
        int32_t nk = n_kernels[m];
        int64_t module_level = 3 + 2 + 3 * nk + 1 + 20 + 24;
        int64_t fi = n_instr[m] - module_level;
        if (fi < 12 * nk) fi = 12 * nk;
        mod_off[m] = total;
        int64_t ni; uint32_t b;
        int64_t n = synth_module(seed0 + (uint64_t)m, fi, nk, nk, 40, 20, 10, string_permille,
                                 out ? out + total : NULL, out ? cap - total : 0, NULL, 0, &ni, &b);
        total += n;
    }
    mod_off[n_mod] = total;
    return total;
}

/* ---------------- op lists: the same modules as a JIT backend's rows ----------------
 * Each instruction of a batch becomes one row: its opcode and its operands,
 * the result id left out; an operand that is an id becomes a reference to
 * the row (within the module) whose result it is. The generator knows which
 * words are ids by generating every module twice, with ids from 1 and from
 * 2^30: exactly the id words differ. The result id's place is word 2 for the
 * opcodes below that have a result type, word 1 for the others with a result
 * id (the generator's own opcodes only). */
static int res_pos(uint32_t op)
{
    switch (op) {
    case O_String: case O_ExtInstImport: case O_TypeVoid: case O_TypeBool: case O_TypeInt: case O_TypeFloat:
    case O_TypeVector: case O_TypePointer: case O_TypeFunction: case O_Label:
        return 1;
    case O_Source: case O_Name: case O_MemoryModel: case O_EntryPoint: case O_ExecutionMode: case O_Capability:
    case O_FunctionEnd: case O_Store: case O_Decorate: case O_ControlBarrier: case O_LoopMerge:
    case O_SelectionMerge: case O_Branch: case O_BranchConditional: case O_Return:
        return 0;
    default:
        return 2;
    }
}

/* Generates the batch of synth_batch (same arguments, same words and
 * mod_off) and its op list: op[r], opd_off[r..r+1) into opd / opd_ref,
 * row_off[m..m+1] the rows of module m, is_id[w] = 1 for id words (header
 * words excluded). Outputs may be NULL to size: *n_rows and *n_opd are set
 * either way. Returns the total words. */
int64_t synth_oplist_batch(int32_t n_mod, uint64_t seed0, const int64_t *n_instr, const int32_t *n_kernels,
                           int32_t string_permille, uint32_t *out, int64_t *mod_off, uint8_t *is_id,
                           uint16_t *op, int64_t *opd_off, uint32_t *opd, uint8_t *opd_ref, int64_t *row_off,
                           int64_t *n_rows, int64_t *n_opd)
{
    int64_t total = 0, rows = 0, nopd = 0;
    for (int32_t m = 0; m < n_mod; m++) {
        int32_t nk = n_kernels[m];
        int64_t module_level = 3 + 2 + 3 * nk + 1 + 20 + 24;
        int64_t fi = n_instr[m] - module_level;
        if (fi < 12 * nk) fi = 12 * nk;
        int64_t ni; uint32_t b;
        s_id_base = 1;
        int64_t n = synth_module(seed0 + (uint64_t)m, fi, nk, nk, 40, 20, 10, string_permille, NULL, 0, NULL, 0, &ni, &b);
        uint32_t *w1 = (uint32_t *)malloc((size_t)n * 4), *w2 = (uint32_t *)malloc((size_t)n * 4);
        int64_t *st = (int64_t *)malloc((size_t)ni * 8);
        synth_module(seed0 + (uint64_t)m, fi, nk, nk, 40, 20, 10, string_permille, w1, n, st, ni, &ni, &b);
        s_id_base = 1u << 30;
        int64_t ni2; uint32_t b2;
        synth_module(seed0 + (uint64_t)m, fi, nk, nk, 40, 20, 10, string_permille, w2, n, NULL, 0, &ni2, &b2);
        s_id_base = 1;
        /* the row that defines each id */
        int64_t *def = (int64_t *)malloc((size_t)b * 8);
        for (uint32_t k = 0; k < b; k++) def[k] = -1;
        for (int64_t i = 0; i < ni; i++) {
            int p = res_pos(w1[st[i]] & 0xffffu);
            if (p) def[w1[st[i] + p]] = i;
        }
        if (mod_off) mod_off[m] = total;
        if (row_off) row_off[m] = rows;
        for (int64_t k = 0; k < n; k++) {
            if (out) out[total + k] = w1[k];
            if (is_id) is_id[total + k] = (uint8_t)(k >= 5 && w1[k] != w2[k]);
        }
        for (int64_t i = 0; i < ni; i++) {
            int64_t a = st[i], e = i + 1 < ni ? st[i + 1] : n;
            int p = res_pos(w1[a] & 0xffffu);
            if (op) op[rows] = (uint16_t)(w1[a] & 0xffffu);
            if (opd_off) opd_off[rows] = nopd;
            for (int64_t k = a + 1; k < e; k++) {
                if (p && k == a + p) continue;
                int ref = w1[k] != w2[k];
                if (opd) opd[nopd] = ref ? (uint32_t)def[w1[k]] : w1[k];
                if (opd_ref) opd_ref[nopd] = (uint8_t)ref;
                nopd++;
            }
            rows++;
        }
        total += n;
        free(w1); free(w2); free(st); free(def);
    }
    if (mod_off) mod_off[n_mod] = total;
    if (row_off) row_off[n_mod] = rows;
    if (opd_off) opd_off[rows] = nopd;
    *n_rows = rows;
    *n_opd = nopd;
    return total;
}
