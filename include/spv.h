/*
 * spv.h -- C ABI of the batched SPIR-V library for NVIDIA B300 (sm_103a).
 *
 * The library decodes, validates, re-encodes and disassembles many SPIR-V
 * binary modules at once on one GPU. It implements the data-parallel core of
 * the toolkit described in arXiv 2305.09493 ("Experiences in Building a
 * Composable and Functional API for Runtime SPIR-V Code Generation"):
 *   decode       the binary layout of section 3.4.6 ("Compliance": modules are
 *                32-bit words holding opcodes and operands) and Listing 4
 *                (header: version, generator, bound, schema);
 *   validate     the rules of section 3.4.5 plus the SSA rule of section 3.4.2;
 *   encode       section 3.2.1 (instructions write themselves as words) with
 *                the write-time bound recomputation of section 3.4.1;
 *   disassemble  section 3.4.4 with the "inline names" and "header" options
 *                of Listing 10, one line per instruction as in Listing 8.
 *
 * Conventions for every call below.
 *   - All array arguments are DEVICE pointers unless marked "host". They are
 *     owned by the caller; the library never frees or keeps them.
 *   - Calls are asynchronous on the given CUDA stream and never synchronise
 *     unless stated. A call returns a negative SPV_E_* code when an argument
 *     is invalid or a CUDA call fails (nothing is launched in the first case);
 *     per-module results go to status[] and never make a call fail.
 *   - "workspace" is caller-owned device scratch of at least the size the
 *     matching *_workspace_bytes function returns. It is fully rewritten by
 *     each call; two calls that overlap on the GPU must not share one.
 *   - Module m is words[mod_off[m] .. mod_off[m+1]) (little-endian 32-bit
 *     words, never byte-swapped); mod_off is non-decreasing, mod_off[0] = 0,
 *     mod_off[n_modules] = n_words, every module is shorter than 2^31 words.
 */
#ifndef SPV_H
#define SPV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *spv_stream_t;   /* a cudaStream_t; NULL = legacy default stream */

/* Per-module status codes (status[m]). When several errors apply the one at
 * the lowest instruction index wins; within one instruction the order is
 * UNKNOWN_OPCODE, BAD_OPERANDS, ID_OUT_OF_BOUND, DUP_RESULT_ID,
 * MISSING_CAPABILITY; a framing error (TRUNCATED, ZERO_WORDCOUNT) counts as
 * the instruction after the last decoded one; module-level rules
 * (NO_CAPABILITY .. NO_FUNCTION) apply only when no instruction-level error
 * exists. */
enum spv_status {
    SPV_OK = 0,
    SPV_BAD_MAGIC = 1,          /* word 0 is not 0x07230203 */
    SPV_BAD_HEADER = 2,         /* version word not 0x00MMmm00 with major 1, minor <= 6; or schema != 0 */
    SPV_TRUNCATED = 3,          /* fewer than 5 words, or an instruction runs past the module's end */
    SPV_ZERO_WORDCOUNT = 4,     /* an instruction's word count is 0 */
    SPV_UNKNOWN_OPCODE = 5,     /* opcode outside the library's compute-subset table */
    SPV_BAD_OPERANDS = 6,       /* operand words do not match the opcode's operand list */
    SPV_ID_OUT_OF_BOUND = 7,    /* an id operand, result type or result id is 0 or >= bound */
    SPV_DUP_RESULT_ID = 8,      /* a result id defined by an earlier instruction */
    SPV_NO_CAPABILITY = 9,      /* no OpCapability (section 3.4.5) */
    SPV_NO_MEMORY_MODEL = 10,   /* no OpMemoryModel (section 3.4.5) */
    SPV_MULTI_MEMORY_MODEL = 11,/* more than one OpMemoryModel */
    SPV_NO_ENTRY_POINT = 12,    /* no OpEntryPoint (section 3.4.5) */
    SPV_NO_FUNCTION = 13,       /* no OpFunction (section 3.4.5) */
    SPV_MISSING_CAPABILITY = 14,/* an instruction needs a capability the module does not declare */
    SPV_TIMEOUT = 15,           /* a bounded wait inside a kernel gave up; results of the module are void */
    SPV_CAPACITY = 16           /* output rows or workspace arena too small for this module */
};

/* Call-level return codes. */
#define SPV_SUCCESS 0
#define SPV_E_ARG (-1)          /* invalid argument; nothing was launched */
#define SPV_E_WORKSPACE (-2)    /* workspace smaller than required; nothing was launched */
#define SPV_E_CUDA (-3)         /* a CUDA launch or runtime call failed */
#define SPV_E_UNSUPPORTED (-4)  /* requested configuration not available */

/* A batch of modules (device pointers). */
typedef struct spv_batch {
    const uint32_t *words;      /* [n_words] */
    const int64_t *mod_off;     /* [n_modules + 1] */
    int32_t n_modules;
    int64_t n_words;
} spv_batch;

/* The structure-of-arrays instruction table (one row per decoded
 * instruction, rows of module m contiguous and in module order). All columns
 * are device arrays of capacity_rows entries written by decode; the per-module
 * arrays have n_modules (+1) entries. A decode call writes mod_first_row[m]
 * (first row of module m) for every m and mod_first_row[n_modules] = total
 * rows; rows beyond capacity_rows are not written and their modules get
 * SPV_CAPACITY. capacity_rows >= n_words always suffices. */
typedef struct spv_table {
    uint16_t *op;               /* opcode */
    uint16_t *wc;               /* word count */
    uint64_t *off;              /* absolute word index of the instruction in batch.words */
    uint32_t *rtype;            /* result type id, 0 if the opcode has none */
    uint32_t *rid;              /* result id, 0 if the opcode has none */
    uint32_t *mod;              /* module index */
    int64_t *mod_first_row;     /* [n_modules + 1] */
    uint32_t *mod_n_instr;      /* [n_modules] */
    int64_t capacity_rows;
} spv_table;

/* Tuning of the batched kernels; zero fields take defaults. */
typedef struct spv_config {
    int32_t tile_words;         /* words per tile: 512, 1024, 2048, 4096 or 8192 */
    int32_t threads;            /* threads per CTA: 64, 128, 256 or 512; tile_words/threads must be 8 or 16,
                                   512 threads only with 16 and 64 only with 8. Tiles start on 16-byte
                                   boundaries of the word buffer. Both 0 (default): 2048 x 128 for batches whose
                                   mean module is under 4,096 words, else 4096 x 256; one of them 0: that one
                                   takes its default (4096 words, 256 threads) */
    int32_t ctas_per_sm;        /* resident CTAs per SM for the persistent grid (default: occupancy maximum) */
    int32_t per_module;         /* 1: one launch sequence per module instead of one persistent launch
                                   (comparison path; copies mod_off to the host and synchronises) */
    int64_t max_spins;          /* bound on every wait inside a kernel (0: default 1 << 20 polls); a
                                   wait that runs out ends with SPV_TIMEOUT for every module of the call */
    int64_t test_stall_tile;    /* test hook, 0 = off: with n > 0, tile n-1 never publishes its look-back
                                   states, so the waits of the tiles after it run out; with n < 0, tile
                                   -n-1 announces its tile map but never writes the map's entries, its
                                   exit or its row count, so a later tile of its module waits on a map
                                   entry that nothing writes (either hook turns speculation off) */
    int32_t no_speculation;     /* 1: every tile after a module's first finds its entry by the look-back
                                   over its predecessors. 0 (default): a tile whose guessed instruction
                                   starts form a chain takes its first guessed start as its entry and
                                   publishes its exit and row count at once, checking the guess against
                                   its predecessor's exit at the end; if any check fails the call redoes
                                   the batch without speculation (on the same stream, same outputs) */
    int32_t reserved;           /* 0 */
} spv_config;

/* Workspace bytes needed by spv_process_batch / spv_decode_batch /
 * spv_validate_batch for a batch of this shape. arena_words is the capacity,
 * in 32-bit words, of the arena holding each module's set of result ids: a
 * bitmap of ceil(bound / 32) words when bound <= 32 * (len + 64), else a
 * hash set of 2 * len + 64 words (len = the module's words). 0 selects the
 * default 2 * n_words + 64 * n_modules + 64, which always fits every module;
 * with a smaller arena the modules that do not fit get SPV_CAPACITY. */
size_t spv_workspace_bytes(int32_t n_modules, int64_t n_words, int64_t arena_words, const spv_config *cfg);

/*
 * spv_process_batch -- decode (+ validate) (+ encode) in one persistent launch.
 *
 * Decode (Listing 4 header; section 3.4.6 word layout): per module check the
 * header, then walk instructions from word 5 by the word count in the high
 * half of each instruction's first word, stopping at the first word count of
 * 0 or at an instruction running past the module's end; fill the table.
 * validate != 0 adds the rules of section 3.4.5 and the id rules of section
 * 3.4.2 (status codes above). out_words != NULL re-encodes every module into
 * out_words[n_words] (same offsets): each instruction's first word, result
 * type and result id are written from the decoded columns, every other word
 * is copied, and with recompute_bound the header bound becomes 1 + the
 * largest result id (section 3.4.1; 1 if none).
 *
 * status[n_modules]: the module's status; err_row[n_modules]: the
 * module-local index of the instruction the status refers to, -1 for header
 * and module-level errors and for SPV_OK. With validate == 0 only header and
 * framing errors are reported.
 */
int spv_process_batch(const spv_batch *batch, spv_table *table, uint32_t *status, int64_t *err_row,
                      int validate, uint32_t *out_words, int recompute_bound,
                      void *workspace, size_t workspace_bytes, int64_t arena_words,
                      const spv_config *cfg, spv_stream_t stream);

/* Size of the fixed device scratch used by spv_process_batch_noalloc. */
#define SPV_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * spv_process_batch_noalloc -- spv_process_batch for callers that cannot
 * allocate device memory (the paper has no counterpart; this is a library
 * service). A host runtime that keeps all of a GPU's memory in its own pool,
 * or a latency-bound serving loop where cudaMalloc could stall the device or
 * fail under memory pressure, still passes its inputs and outputs but no
 * workspace: the kernels' scratch is a fixed 32 MiB device array inside the
 * library (SPV_NOALLOC_SCRATCH_BYTES), which every GPU that loads the
 * library holds until the process exits. Nothing is allocated by the call.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture. The address is kept per device together
 *     with the context it was found in, and looked up again when a call runs
 *     in another context (after cudaDeviceReset, say).
 *   - Arguments are checked first, as by spv_process_batch (SPV_E_ARG), then
 *     the scratch size.
 *   - A batch whose workspace (spv_workspace_bytes with the default arena)
 *     exceeds SPV_NOALLOC_SCRATCH_BYTES is rejected with SPV_E_WORKSPACE and
 *     nothing is launched; cfg->per_module is rejected with
 *     SPV_E_UNSUPPORTED.
 *   - Every call on a device shares the array and leaves its contents behind;
 *     each call clears on the device what it needs cleared. Two calls that
 *     overlap on the GPU (different streams, no ordering) race on the array.
 * Arguments and results are those of spv_process_batch.
 */
int spv_process_batch_noalloc(const spv_batch *batch, spv_table *table, uint32_t *status, int64_t *err_row,
                              int validate, uint32_t *out_words, int recompute_bound,
                              const spv_config *cfg, spv_stream_t stream);

/*
 * spv_autotune_batch -- pick the fastest tile shape (tile_words x threads)
 * of spv_process_batch for a batch (a library service; the paper has no
 * counterpart). Runs the batch once to warm up and reps times (0: 3) timed
 * with CUDA events on the stream for every built shape whose workspace fits
 * in workspace_bytes, then once more with the fastest, so the outputs are
 * that shape's; arguments as spv_process_batch (recompute_bound = 1).
 * Writes *best (tile_words, threads; other fields 0) and *best_ms (mean
 * time of one call). Synchronises the stream; not for use under stream
 * capture. SPV_E_WORKSPACE when no shape fits.
 */
int spv_autotune_batch(const spv_batch *batch, spv_table *table, uint32_t *status, int64_t *err_row, int validate,
                       uint32_t *out_words, void *workspace, size_t workspace_bytes, int reps, spv_config *best,
                       float *best_ms, spv_stream_t stream);

/*
 * spv_layout_batch -- logical layout and scopes of every module's decoded
 * rows (section 3.4.1: module, function and block scopes; the checks follow
 * the SPIR-V logical layout the paper builds on). Module-scope rows must
 * come in section order: capabilities (1), extensions (2), extended-
 * instruction imports (3), memory model (4), entry points (5), execution
 * modes (6), debug instructions (7), decorations (8), types, constants and
 * global variables (9), functions (10). OpFunction opens a function at
 * module scope; its parameters follow; then OpFunctionEnd (a declaration)
 * or blocks, each opened by OpLabel and closed by a terminator (OpBranch,
 * OpBranchConditional, OpReturn, OpReturnValue, OpUnreachable), the last
 * followed by OpFunctionEnd. OpVariable and OpUndef are global declarations
 * at module scope and body instructions in a block; OpNop and opcodes
 * outside the table are allowed anywhere. Reads table->op and
 * table->mod_first_row of a decode (rows of module m: mod_first_row[m] ..
 * mod_first_row[m + 1] - 1, capped at capacity_rows). Writes
 * layout_status[n_modules] (spv_layout_status) and layout_err_row: the
 * module-local row of the first error in row order (the row count for
 * SPV_LAYOUT_UNCLOSED), -1 when OK. Asynchronous on stream. workspace:
 * device scratch of at least spv_layout_workspace_bytes(n_modules,
 * table->capacity_rows) bytes (modules of more than 16,384 rows are split
 * into segments whose summaries it holds).
 */
enum spv_layout_status {
    SPV_LAYOUT_OK = 0,
    SPV_LAYOUT_SECTION_ORDER = 1,      /* a module-scope row of a lower section after one of a higher section */
    SPV_LAYOUT_OUTSIDE_FUNCTION = 2,   /* a parameter, label, body instruction, terminator or OpFunctionEnd at module scope */
    SPV_LAYOUT_IN_FUNCTION = 3,        /* a module-scope instruction, or a second OpFunction, inside a function */
    SPV_LAYOUT_BLOCK = 4,              /* body or terminator before the first label or after a terminator; a label in an
                                          open block; a parameter after a label; OpFunctionEnd in an open block */
    SPV_LAYOUT_UNCLOSED = 5            /* the rows end inside a function */
};
size_t spv_layout_workspace_bytes(int32_t n_modules, int64_t capacity_rows);
int spv_layout_batch(const spv_table *table, int32_t n_modules, uint32_t *layout_status, int64_t *layout_err_row,
                     void *workspace, size_t workspace_bytes, spv_stream_t stream);
/* Layout class of an opcode in the library's table (host query):
 * 0 neutral, 1 module section, 2 OpUndef / OpVariable (section 9 at module
 * scope, body in a block), 3 OpFunction (section 10), 4 OpFunctionParameter,
 * 5 OpFunctionEnd, 6 OpLabel, 7 terminator, 8 body; *section is the module
 * section (0 when none). Returns 0. */
int spv_op_layout(uint32_t opcode, int *layout_class, int *section);

/* spv_decode_batch -- spv_process_batch with validate = 0 and no encode. */
int spv_decode_batch(const spv_batch *batch, spv_table *table, uint32_t *status, int64_t *err_row,
                     void *workspace, size_t workspace_bytes, const spv_config *cfg, spv_stream_t stream);

/* spv_validate_batch -- validate modules from an already decoded table
 * (section 3.4.5 rules and section 3.4.2 id rules over the table's rows; the
 * operand words are read from batch.words at each row's offset). The table
 * must come from a decode of the same batch; its rows may have been edited
 * as long as every row still lies inside its module. Writes status/err_row
 * as spv_process_batch with validate = 1 (framing errors come from the
 * table: a module whose rows end before its last word is reported as the
 * decode reported it). */
int spv_validate_batch(const spv_batch *batch, const spv_table *table, uint32_t *status, int64_t *err_row,
                       void *workspace, size_t workspace_bytes, int64_t arena_words, spv_stream_t stream);

/* spv_encode_batch -- write out_words[n_words] from a table over the source
 * words (section 3.2.1 "write"; bound per section 3.4.1). out_words starts as
 * a copy of the source; for every module with a valid header and every row
 * of it, the row's first word becomes (wc << 16) | op and, when the opcode
 * has them, its result type / result id words take the row's rtype / rid;
 * with recompute_bound the header bound becomes 1 + the largest rid of the
 * module's rows (1 if none). The table may be edited between decode and
 * encode; rows must stay inside their module. No workspace. */
int spv_encode_batch(const spv_batch *src, const spv_table *table, uint32_t *out_words,
                     int recompute_bound, spv_stream_t stream);

/* Disassembly options (Listing 10): inline_names prints ids as
 * %<name>_<id> using each id's first OpName; header prints the five header
 * fields as comment lines first. max_spins bounds every wait of the text
 * offset look-back (0: 1 << 20 polls); a wait that runs out ends the call
 * with SPV_TIMEOUT in dis_status for every module (the text is then not
 * complete). test_stall_tile is a test hook, 0 = off: with n > 0, text tile
 * n-1 never publishes its byte count, so the waits of the tiles after it run
 * out. Zero-initialised fields take the defaults. */
typedef struct spv_dis_opts {
    int32_t inline_names;
    int32_t header;
    int64_t max_spins;
    int64_t test_stall_tile;
} spv_dis_opts;

/* Workspace bytes for spv_disassemble_batch. arena_words is the capacity,
 * in 32-bit words, of the per-module id tables (first OpName and first
 * definition of each id): 3 * bound words plus a bitmap of ceil(bound / 32)
 * words when bound <= len + 64 (len = the module's words), else a hash map of
 * 4 * (len + 64) words. 0 selects the default 4 * n_words + 256 * n_modules
 * + 64, which always fits every module. */
size_t spv_dis_workspace_bytes(int32_t n_modules, int64_t n_words, int64_t n_rows_capacity, int64_t arena_words);

/*
 * spv_disassemble_batch -- text of every module (section 3.4.4): every
 * line is measured, the lengths are scanned into 64-bit offsets, and every
 * line is written once. Module m's text is text[text_off[m] .. text_off[m+1]);
 * text_off has n_modules + 1 entries (device). No byte at or past
 * text_capacity is ever written; when text_off[n_modules] exceeds the
 * capacity the text is incomplete and the caller calls again with a buffer of
 * text_off[n_modules] bytes (text_off is always filled). A module with a
 * header error has no text; a
 * module whose id tables do not fit the arena gets status SPV_CAPACITY in
 * dis_status (device, n_modules entries, may be NULL) and no text.
 * The text form: optional "; SPIR-V", "; Version: M.m",
 * "; Generator: 0x%08x", "; Bound: B", "; Schema: S" lines; then one line
 * per row: "[%R = ]OpName[ operands]" with the result type first; ids %<id>
 * or %<name>_<id> (name bytes outside [A-Za-z0-9_] become '_'); literals in
 * unsigned decimal; strings quoted with \" \\ \xhh escapes; enumerants by
 * name (bit enums A|B, 0 as None, unknown values in decimal); float
 * constants as C99 "%a" hexadecimal floating point; rows with an unknown
 * opcode as Op<decimal> and rows whose operands do not parse as the opcode
 * name, followed by the remaining words as 0x%08x.
 */
int spv_disassemble_batch(const spv_batch *batch, const spv_table *table, const spv_dis_opts *opts,
                          char *text, uint64_t text_capacity, uint64_t *text_off, uint32_t *dis_status,
                          void *workspace, size_t workspace_bytes, int64_t arena_words, spv_stream_t stream);

/*
 * Assembler: text back to words (section 3.4.4, Dis/Assembler), for every
 * module of a batch at once; the inverse of spv_disassemble_batch, with the
 * paper's hash table from id names to ids.
 *
 * The text form, per module (lines end at '\n'; a final '\n' does not start
 * another line; lines are numbered from 1 in each module):
 *   - an empty line is skipped;
 *   - a line starting with ';' is a comment; exactly "; Version: A.B"
 *     (A, B <= 255), "; Generator: 0xH", "; Bound: N" and "; Schema: N"
 *     (values < 2^32, nothing after them) set header words, the last such
 *     line of each field winning;
 *   - any other line is one instruction: tokens split by spaces, a token that
 *     starts with '"' running to the next '"' not escaped by '\' (an unclosed
 *     one is an error): "[%r =] OpName operands" in the operand order of the
 *     opcode table (result type first), or "Op<decimal> 0xHHHHHHHH ..." (raw
 *     words; also after a known name when its first operand token is one).
 * Ids: "%<digits>" and "%<name>_<digits>" are the id <digits> (< 2^32); any
 * other "%<name>" is a named id: a module's distinct names get the ids M+1,
 * M+2, ... in order of first appearance in its text, M its largest explicit
 * id (0 if none). Literals are decimal, < 2^32. Strings: "\xHH" is the byte
 * HH, '\' before any other byte is that byte. Enumerants: the name or a
 * decimal number; bit enums also "None" and "A|B". An OpConstant value of two
 * or more tokens is one word per token; of one token it is a decimal integer
 * (< 2^64) or a float literal ([+-] then inf, nan, C99 hexadecimal or
 * decimal), as wide as the result type: the first OpTypeInt / OpTypeFloat of
 * the module defining that id, else 32-bit. Float literals round exactly to
 * double, to nearest even; a 32-bit constant is that double rounded again to
 * float. An instruction has at most 65535 words.
 * Each module's words: magic, version (default 1.2), generator (0), bound
 * (the Bound line, else the largest id + 1), schema (0), then one
 * instruction per instruction line.
 *
 * text: device, text_bytes bytes; module m is text[text_off[m] ..
 * text_off[m+1]) (text_off: device, n_modules + 1 entries, non-decreasing,
 * text_off[n_modules] <= text_bytes; otherwise every module gets
 * SPV_ASM_BAD_OFFSETS). Module m's words go to words[word_off[m] ..
 * word_off[m+1]) (word_off: device, n_modules + 1 entries, always filled); a
 * module that is not SPV_ASM_OK has no words. No word at or past
 * words_capacity is written: when word_off[n_modules] exceeds it, call again
 * with a larger buffer. asm_status (device, n_modules) gets spv_asm_status
 * codes; asm_err_line (device, may be NULL) the first bad line of a
 * SPV_ASM_SYNTAX module, else -1.
 * line_capacity / name_capacity bound the lines and the named-id occurrences
 * the workspace holds (0: text_bytes / 16 + n_modules + 64 lines and
 * text_bytes / 32 + 64 occurrences); modules past them get SPV_ASM_CAPACITY
 * and spv_asm_required then tells what the call needed.
 */
typedef enum spv_asm_status {
    SPV_ASM_OK = 0,
    SPV_ASM_SYNTAX = 1,         /* a line that does not parse (asm_err_line) */
    SPV_ASM_CAPACITY = 2,       /* the workspace's line or name capacity is too small */
    SPV_ASM_BAD_OFFSETS = 3     /* text_off decreasing or past text_bytes */
} spv_asm_status;

size_t spv_asm_workspace_bytes(int32_t n_modules, uint64_t text_bytes, int64_t line_capacity, int64_t name_capacity);

int spv_assemble_batch(const char *text, uint64_t text_bytes, const uint64_t *text_off, int32_t n_modules,
                       uint32_t *words, int64_t words_capacity, int64_t *word_off, uint32_t *asm_status,
                       int64_t *asm_err_line, void *workspace, size_t workspace_bytes, int64_t line_capacity,
                       int64_t name_capacity, spv_stream_t stream);

/* Lines and named-id occurrences the last spv_assemble_batch on this
 * workspace needed (synchronous: waits for that call). */
int spv_asm_required(const void *workspace, int64_t *lines, int64_t *names);

/*
 * Builder: modules from op lists (section 3.4.2, "Enabling Function
 * Composition"), for a whole batch at once. In the paper each instruction
 * is added to its scope in order and each one with a result first asks the
 * module for the next id (getNextId). Here a module is a list of rows: row r
 * is an opcode op[r] and its operands opd[opd_off[r] .. opd_off[r+1]), the
 * result id left out; operand k is a literal word (opd_ref[k] = 0) or a
 * reference to row opd[k] of the same module, counted from the module's
 * first row (opd_ref[k] = 1), which stands for that row's result id. The
 * rows whose opcode has a result id (by the opcode table) get the ids 1, 2,
 * ... of their module in row order; the result id is written after the
 * result type (the first operand) when the opcode has one, else first.
 * Opcodes outside the table have no result id; their operands are copied.
 * Checks, the first bad row of a module winning (in a row: the first two
 * before the references, in operand order): an opcode with a result type
 * and no operand, or an instruction over 65535 words, is SPV_BUILD_BAD_ROW;
 * a reference outside the module or to a row without a result id is
 * SPV_BUILD_BAD_REF. A module that is not SPV_BUILD_OK has no words.
 * Module m's words: magic, version, generator, bound (its ids + 1), schema
 * 0, then its rows' instructions; they go to words[word_off[m] ..
 * word_off[m+1]) (word_off: device, n_modules + 1 entries, always filled);
 * no word at or past words_capacity is written. ids (device, n_rows, may be
 * NULL) gets each row's id, 0 for rows without one. status (device,
 * n_modules) gets spv_build_status codes, err_row (device, may be NULL) the
 * module-relative first bad row, else -1. All arrays are device memory.
 * row_off and opd_off must not decrease, row_off[n_modules] <= n_rows;
 * otherwise every module is SPV_BUILD_BAD_OFFSETS.
 */
typedef struct spv_oplist {
    const uint16_t *op;         /* [n_rows] */
    const int64_t *opd_off;     /* [n_rows + 1] */
    const uint32_t *opd;        /* [opd_off[n_rows]] operand values */
    const uint8_t *opd_ref;     /* [opd_off[n_rows]] 1: opd is a row index within the module */
    const int64_t *row_off;     /* [n_modules + 1] module m is rows row_off[m] .. row_off[m+1] */
    int32_t n_modules;
    int64_t n_rows;
} spv_oplist;

typedef enum spv_build_status {
    SPV_BUILD_OK = 0,
    SPV_BUILD_BAD_REF = 1,
    SPV_BUILD_BAD_ROW = 2,
    SPV_BUILD_BAD_OFFSETS = 3
} spv_build_status;

size_t spv_build_workspace_bytes(int32_t n_modules, int64_t n_rows);

int spv_build_batch(const spv_oplist *ol, uint32_t version, uint32_t generator, uint32_t *words,
                    int64_t words_capacity, int64_t *word_off, uint32_t *ids, uint32_t *status, int64_t *err_row,
                    void *workspace, size_t workspace_bytes, spv_stream_t stream);

/*
 * Serving: continuous batching of modules that arrive one by one, as a JIT
 * backend produces them (the paper's use case, section 4). A server owns a
 * device pool and a pinned host pool. Submitted modules wait in a queue; a
 * scheduler thread takes every waiting module (up to max_batch_modules /
 * max_batch_words) as soon as a batch slot is free and runs decode +
 * validate + disassembly on it as one batch (spv_process_batch and
 * spv_disassemble_batch), on two streams so that the copies of one batch
 * overlap the kernels of the next. Requests that arrive while a batch is on
 * the GPU go into the next one. Admission is by footprint: a module of n
 * words holds 28 * n + 64 bytes of the device pool (its words and decoded
 * table) from submit until release; a submit that would exceed
 * hbm_cap_bytes returns SPV_E_BUSY and changes nothing. Results (status,
 * error row, text on the host, and the decoded rows still on the device)
 * are owned by the server until spv_serve_release.
 */
#define SPV_E_BUSY (-5)         /* serving: admission cap or staging space exhausted; retry later */

typedef struct spv_serve_cfg {
    uint64_t hbm_cap_bytes;     /* admission cap on device-resident bytes (0: 8 GiB) */
    int64_t max_batch_words;    /* largest batch (0: 32M words) */
    int32_t max_batch_modules;  /* most modules per batch (0: 4096; 1: one module per launch sequence) */
    int32_t inline_names;       /* disassembly options (Listing 10) */
    int32_t header;
    int32_t device;             /* CUDA device ordinal */
} spv_serve_cfg;

typedef struct spv_result {
    int32_t error;              /* SPV_SUCCESS, or the SPV_E_* code of a failed batch */
    uint32_t status;            /* module status (enum spv_status) */
    int64_t err_row;
    uint32_t n_instr;
    const char *text;           /* host, text_len bytes, valid until release */
    uint64_t text_len;
    const uint16_t *op;         /* device: this module's rows of the decoded table */
    const uint16_t *wc;
    const uint32_t *rtype;
    const uint32_t *rid;
    const uint64_t *off;        /* word offsets into words_base */
    const uint32_t *words_base; /* device: the batch's word buffer holding this module */
    uint64_t submit_ns;         /* CLOCK_MONOTONIC times of submit and completion */
    uint64_t done_ns;
    uint32_t batch_modules;     /* size of the batch the module ran in */
} spv_result;

typedef struct spv_server spv_server;

/* Create a server (allocates its pools; returns NULL on failure). */
spv_server *spv_serve_create(const spv_serve_cfg *cfg);
/* Copy a module (host words) into the server; *ticket identifies it.
 * SPV_E_BUSY when admitting it would exceed the cap. */
int spv_serve_submit(spv_server *s, const uint32_t *host_words, int64_t n_words, uint64_t *ticket);
/* 1 and *out filled when the module is done, 0 while it is pending, SPV_E_ARG for an unknown ticket. */
int spv_serve_poll(spv_server *s, uint64_t ticket, spv_result *out);
/* Like poll, but waits up to timeout_us microseconds. */
int spv_serve_wait(spv_server *s, uint64_t ticket, spv_result *out, int64_t timeout_us);
/* Release a done module's results and its share of the device pool. */
int spv_serve_release(spv_server *s, uint64_t ticket);
/* Stop the scheduler, wait for in-flight batches, free everything (modules still queued are dropped). */
void spv_serve_destroy(spv_server *s);
/*
 * Load replay, for measuring the server under an arrival process: module i
 * (mods[i], n_words[i] words in host memory) is submitted arrive_ns[i]
 * nanoseconds (non-decreasing) after the start, from a native thread,
 * retrying while admission says SPV_E_BUSY; the calling thread waits for the
 * modules in order and releases them. Per module (host arrays of n):
 * latency_ns from its scheduled arrival to its completion, and optionally
 * server_ns from submission to completion and batch_modules; busy_retries
 * (optional) counts the refused submissions. Returns SPV_SUCCESS, SPV_E_ARG,
 * or the first failing call's code.
 */
int spv_serve_replay(spv_server *s, int32_t n, const uint32_t *const *mods, const int64_t *n_words,
                     const int64_t *arrive_ns, int64_t *latency_ns, int64_t *server_ns, uint32_t *batch_modules,
                     int64_t *busy_retries);

/*
 * Host-resident batches, transfers overlapped with the kernels (a library
 * service; the paper has no counterpart). A batch that starts and ends in
 * host memory is bound by the PCIe copies: its words go up once and its text,
 * several times larger, comes back. spv_pipe_run splits the batch into
 * chunks of whole modules (about chunk_words words each; a larger module is
 * a chunk of its own) that rotate over `depth` slots, each with its own
 * stream and device buffers, so one chunk's text copy-back overlaps the next
 * chunk's kernels and the upload of the one after.
 */
typedef struct spv_pipe spv_pipe;
typedef struct spv_pipe_cfg {
    int64_t chunk_words;        /* target words per chunk (0: 8M words) */
    int32_t depth;              /* slots in flight, 2..8 (0: 3) */
    int32_t validate;           /* nonzero: validate (else decode-only statuses) */
    int32_t encode;             /* nonzero: re-encode on the device (copied back when h_out_words != NULL) */
    int32_t inline_names;       /* disassembly options as in spv_dis_opts */
    int32_t header;
} spv_pipe_cfg;
/* A handle on the current device, holding its slots' streams; device and
 * pinned buffers are allocated by the first run and grown when a later batch
 * needs more. NULL on failure. */
spv_pipe *spv_pipe_create(const spv_pipe_cfg *cfg);
/*
 * Process a batch in host memory: h_words[n_words], h_mod_off[n_modules + 1]
 * (non-decreasing, h_mod_off[n_modules] <= n_words). Outputs, all host
 * memory: h_status / h_err_row [n_modules] as spv_process_batch;
 * h_text_off[n_modules + 1] and h_text[text_capacity] as
 * spv_disassemble_batch over the whole batch (h_text_off[n_modules] is the
 * total size; no byte at or past text_capacity is written); optional
 * h_out_words[n_words] (encoded words, needs cfg.encode) and
 * h_dis_status[n_modules]. Page-locked host buffers let the copies overlap;
 * pageable ones work but serialise. Returns when every output is in place:
 * SPV_SUCCESS, SPV_E_ARG (nothing done), SPV_E_CUDA. With n_modules == 0
 * only h_text_off[0] = 0 is written (the other outputs may be NULL).
 */
int spv_pipe_run(spv_pipe *p, const uint32_t *h_words, int64_t n_words, const int64_t *h_mod_off, int32_t n_modules,
                 uint32_t *h_status, int64_t *h_err_row, uint64_t *h_text_off, char *h_text, uint64_t text_capacity,
                 uint32_t *h_out_words, uint32_t *h_dis_status);
/* Wait for the handle's streams, free its buffers and streams. */
void spv_pipe_destroy(spv_pipe *p);

/* Sizes of a batch's outputs (a convenience for sizing buffers):
 * *rows_upper (may be NULL) = n_words - 5 * n_modules, at least 0, an upper
 * bound of the decoded rows from the batch's shape alone (an instruction
 * holds at least one word, a header five). *text_bytes (may be NULL) = the
 * exact size of spv_disassemble_batch's text with these options, found by
 * decoding and measuring the batch on the stream.
 * EXCEPTION to the conventions of every other call in this header: when
 * text_bytes is given, this call ALLOCATES its own device scratch
 * (cudaMallocAsync on the stream, freed with cudaFreeAsync before it
 * returns) and is SYNCHRONOUS (it waits for the stream to read the size
 * back). It is a sizing helper for setting up buffers, not a hot-path call:
 * do not use it inside a stream capture or where allocation is forbidden;
 * there, size the text buffer from spv_disassemble_batch itself (its
 * text_off[n_modules] is the needed size even when it exceeds
 * text_capacity, and a call with text_capacity 0 writes no text). With
 * text_bytes NULL the call only
 * computes rows_upper on the host and touches no device state.
 * Returns SPV_SUCCESS or an SPV_E_* code. */
int spv_query_sizes(const spv_batch *batch, const spv_dis_opts *opts, int64_t *rows_upper, uint64_t *text_bytes,
                    spv_stream_t stream);

/* Host-side queries of the library's own opcode / enumerant tables (no GPU
 * needed). spv_op_info returns 0 and fills the outputs for a known opcode,
 * -1 otherwise; cap is the capability the opcode requires or -1. */
int spv_op_info(uint32_t opcode, int *has_rtype, int *has_rid, int *cap, const char **name);
/* kind is one of the enumeration names used by the operand lists
 * ("Capability", "Decoration", ...). Returns 0 for a known enumerant. */
int spv_enum_info(const char *kind, uint32_t value, const char **name, int *cap);
/* Library version string. */
const char *spv_version(void);

/* Per-kernel timing of the library's own launches, for benchmarks and
 * profiling (no counterpart in the paper). With profiling on, every launch
 * made by the calls above is bracketed by two CUDA events recorded on the
 * launching stream; do not enable it while a stream is being captured.
 * spv_profile_enable(1) clears the record and starts recording,
 * spv_profile_enable(0) stops. spv_profile_read waits for the recorded
 * events, then fills up to max entries (host arrays) with each kernel's name
 * (static strings), launch count and total milliseconds, and returns the
 * number of kernels (or a negative SPV_E_* code). */
int spv_profile_enable(int on);
int spv_profile_read(int max, const char **names, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* SPV_H */
