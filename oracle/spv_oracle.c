/*
 * spv_oracle.c -- the plain, sequential CPU definition of the batched SPIR-V
 * hot path: decode, validate, encode, disassemble, the logical-layout check,
 * and assemble (text back to words).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference arm may load or call this library. The CUDA
 * library shares no code, header, table or helper with it; both tables were
 * typed separately from the public SPIR-V specification and a test compares
 * them entry by entry.
 *
 * Where each step comes from (arXiv 2305.09493):
 *   header      Listing 4 and the text around it (section 3.4.1): version
 *               major/minor, generator, bound (recomputed when the module is
 *               written), schema, in the specification's order.  The magic
 *               number and the word layout are those of the SPIR-V spec the
 *               paper builds on.
 *   words       section 3.4.6 "Compliance": a module is a stream of 32-bit
 *               words holding opcodes and operands; word 0 of an instruction
 *               is (word count << 16) | opcode.
 *   operands    section 3.2.1 "Parsing Operand Kinds" / "Parsing
 *               Instructions": ids, value and bit enums, literals,
 *               composites; quantifiers '?' (optional) and '*' (variadic).
 *   validate    section 3.4.5: at least one function, one capability, a
 *               memory model and one entry point; instruction capability
 *               requirements and capability dependencies; plus the SSA rule
 *               of section 3.4.2 (each result id defined once, ids below the
 *               bound).
 *   encode      section 3.2.1 (an instruction writes itself as words) and the
 *               bound recomputation of section 3.4.1.
 *   disassemble section 3.4.4 and Listing 10 (options "inline names" and
 *               "header"); one line per instruction as in Listing 8.
 *   assemble    section 3.4.4 "Dis/Assembler": the inverse of the text form,
 *               with a hash table from id names to ids.
 *
 * Every decision the paper leaves open is listed, with its reading, in the
 * repository's design notes; the short form is repeated at each function.
 * Parity unpinned: the exact spelling of float constants (we print C99 "%a"
 * as glibc does, and pin only a few values) and the escape form of strings
 * have no external reference; they are fixed by our own definition.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <ctype.h>

/* ------------------------------------------------------------------ */
/* Status codes (per module).                                         */
/* ------------------------------------------------------------------ */
enum {
    ST_OK = 0, ST_BAD_MAGIC = 1, ST_BAD_HEADER = 2, ST_TRUNCATED = 3,
    ST_ZERO_WORDCOUNT = 4, ST_UNKNOWN_OPCODE = 5, ST_BAD_OPERANDS = 6,
    ST_ID_OUT_OF_BOUND = 7, ST_DUP_RESULT_ID = 8, ST_NO_CAPABILITY = 9,
    ST_NO_MEMORY_MODEL = 10, ST_MULTI_MEMORY_MODEL = 11,
    ST_NO_ENTRY_POINT = 12, ST_NO_FUNCTION = 13, ST_MISSING_CAPABILITY = 14
};

#define ORC_MAGIC 0x07230203u

/* ------------------------------------------------------------------ */
/* Enumerations used by the compute subset (SPIR-V 1.2 numbering).    */
/* Each entry: value, name, capability it requires (-1: none) and the */
/* operands that follow it ("" none, NULL -> kind default).            */
/* ------------------------------------------------------------------ */
typedef struct { uint32_t value; const char *name; int cap; const char *params; } Enumerant;
typedef struct { const char *kind; int is_bits; const Enumerant *e; int n; const char *unknown_params; } EnumKind;

static const Enumerant E_SourceLanguage[] = {
    {0,"Unknown",-1,""},{1,"ESSL",-1,""},{2,"GLSL",-1,""},{3,"OpenCL_C",-1,""},
    {4,"OpenCL_CPP",-1,""},{5,"HLSL",-1,""}};
static const Enumerant E_AddressingModel[] = {
    {0,"Logical",-1,""},{1,"Physical32",4,""},{2,"Physical64",4,""}};
static const Enumerant E_MemoryModel[] = {
    {0,"Simple",1,""},{1,"GLSL450",1,""},{2,"OpenCL",6,""}};
static const Enumerant E_ExecutionModel[] = {
    {0,"Vertex",1,""},{1,"TessellationControl",3,""},{2,"TessellationEvaluation",3,""},
    {3,"Geometry",2,""},{4,"Fragment",1,""},{5,"GLCompute",1,""},{6,"Kernel",6,""}};
static const Enumerant E_ExecutionMode[] = {
    {17,"LocalSize",-1,"L L L"},{18,"LocalSizeHint",6,"L L L"},
    {30,"VecTypeHint",6,"L"},{31,"ContractionOff",6,""}};
static const Enumerant E_Capability[] = {
    {0,"Matrix",-1,""},{1,"Shader",-1,""},{2,"Geometry",-1,""},{3,"Tessellation",-1,""},
    {4,"Addresses",-1,""},{5,"Linkage",-1,""},{6,"Kernel",-1,""},{7,"Vector16",-1,""},
    {8,"Float16Buffer",-1,""},{9,"Float16",-1,""},{10,"Float64",-1,""},{11,"Int64",-1,""},
    {12,"Int64Atomics",-1,""},{13,"ImageBasic",-1,""},{14,"ImageReadWrite",-1,""},
    {15,"ImageMipmap",-1,""},{17,"Pipes",-1,""},{18,"Groups",-1,""},
    {19,"DeviceEnqueue",-1,""},{20,"LiteralSampler",-1,""},{21,"AtomicStorage",-1,""},
    {22,"Int16",-1,""},{23,"TessellationPointSize",-1,""},{24,"GeometryPointSize",-1,""},
    {25,"ImageGatherExtended",-1,""},{27,"StorageImageMultisample",-1,""},
    {28,"UniformBufferArrayDynamicIndexing",-1,""},{29,"SampledImageArrayDynamicIndexing",-1,""},
    {30,"StorageBufferArrayDynamicIndexing",-1,""},{31,"StorageImageArrayDynamicIndexing",-1,""},
    {32,"ClipDistance",-1,""},{33,"CullDistance",-1,""},{34,"ImageCubeArray",-1,""},
    {35,"SampleRateShading",-1,""},{36,"ImageRect",-1,""},{37,"SampledRect",-1,""},
    {38,"GenericPointer",-1,""},{39,"Int8",-1,""},{40,"InputAttachment",-1,""},
    {41,"SparseResidency",-1,""},{42,"MinLod",-1,""},{43,"Sampled1D",-1,""},
    {44,"Image1D",-1,""},{45,"SampledCubeArray",-1,""},{46,"SampledBuffer",-1,""},
    {47,"ImageBuffer",-1,""},{48,"ImageMSArray",-1,""},{49,"StorageImageExtendedFormats",-1,""},
    {50,"ImageQuery",-1,""},{51,"DerivativeControl",-1,""},{52,"InterpolationFunction",-1,""},
    {53,"TransformFeedback",-1,""},{54,"GeometryStreams",-1,""},
    {55,"StorageImageReadWithoutFormat",-1,""},{56,"StorageImageWriteWithoutFormat",-1,""},
    {57,"MultiViewport",-1,""},{58,"SubgroupDispatch",-1,""},{59,"NamedBarrier",-1,""},
    {60,"PipeStorage",-1,""}};
static const Enumerant E_StorageClass[] = {
    {0,"UniformConstant",-1,""},{1,"Input",-1,""},{2,"Uniform",1,""},{3,"Output",1,""},
    {4,"Workgroup",-1,""},{5,"CrossWorkgroup",-1,""},{6,"Private",1,""},{7,"Function",-1,""},
    {8,"Generic",38,""},{9,"PushConstant",1,""},{10,"AtomicCounter",21,""},{11,"Image",-1,""}};
static const Enumerant E_Decoration[] = {
    {0,"RelaxedPrecision",1,NULL},{1,"SpecId",1,NULL},{2,"Block",1,NULL},{3,"BufferBlock",1,NULL},
    {4,"RowMajor",0,NULL},{5,"ColMajor",0,NULL},{6,"ArrayStride",1,NULL},{7,"MatrixStride",0,NULL},
    {8,"GLSLShared",1,NULL},{9,"GLSLPacked",1,NULL},{10,"CPacked",6,NULL},
    {11,"BuiltIn",-1,"E:BuiltIn"},{13,"NoPerspective",1,NULL},{14,"Flat",1,NULL},
    {15,"Patch",3,NULL},{16,"Centroid",1,NULL},{17,"Sample",35,NULL},{18,"Invariant",1,NULL},
    {19,"Restrict",-1,NULL},{20,"Aliased",-1,NULL},{21,"Volatile",-1,NULL},{22,"Constant",6,NULL},
    {23,"Coherent",-1,NULL},{24,"NonWritable",-1,NULL},{25,"NonReadable",-1,NULL},
    {26,"Uniform",1,NULL},{28,"SaturatedConversion",6,NULL},{29,"Stream",54,NULL},
    {30,"Location",1,NULL},{31,"Component",1,NULL},{32,"Index",1,NULL},{33,"Binding",1,NULL},
    {34,"DescriptorSet",1,NULL},{35,"Offset",1,NULL},{36,"XfbBuffer",53,NULL},
    {37,"XfbStride",53,NULL},{38,"FuncParamAttr",6,"E:FuncParamAttr"},
    {39,"FPRoundingMode",6,NULL},{40,"FPFastMathMode",6,NULL},
    {41,"LinkageAttributes",5,"S E:LinkageType"},{42,"NoContraction",1,NULL},
    {43,"InputAttachmentIndex",40,NULL},{44,"Alignment",6,"L"},{45,"MaxByteOffset",4,NULL},
    {46,"AlignmentId",6,"I"},{47,"MaxByteOffsetId",4,"I"}};
static const Enumerant E_BuiltIn[] = {
    {24,"NumWorkgroups",-1,""},{25,"WorkgroupSize",-1,""},{26,"WorkgroupId",-1,""},
    {27,"LocalInvocationId",-1,""},{28,"GlobalInvocationId",-1,""},
    {29,"LocalInvocationIndex",-1,""},{30,"WorkDim",6,""},{31,"GlobalSize",6,""},
    {32,"EnqueuedWorkgroupSize",6,""},{33,"GlobalOffset",6,""},{34,"GlobalLinearId",6,""},
    {36,"SubgroupSize",6,""},{37,"SubgroupMaxSize",6,""},{38,"NumSubgroups",6,""},
    {39,"NumEnqueuedSubgroups",6,""},{40,"SubgroupId",6,""},
    {41,"SubgroupLocalInvocationId",6,""}};
static const Enumerant E_FuncParamAttr[] = {
    {0,"Zext",-1,""},{1,"Sext",-1,""},{2,"ByVal",-1,""},{3,"Sret",-1,""},{4,"NoAlias",-1,""},
    {5,"NoCapture",-1,""},{6,"NoWrite",-1,""},{7,"NoReadWrite",-1,""}};
static const Enumerant E_LinkageType[] = {{0,"Export",-1,""},{1,"Import",-1,""}};
static const Enumerant E_FunctionControl[] = {
    {0x1,"Inline",-1,""},{0x2,"DontInline",-1,""},{0x4,"Pure",-1,""},{0x8,"Const",-1,""}};
static const Enumerant E_MemoryAccess[] = {
    {0x1,"Volatile",-1,""},{0x2,"Aligned",-1,"L"},{0x4,"Nontemporal",-1,""}};
static const Enumerant E_SelectionControl[] = {{0x1,"Flatten",-1,""},{0x2,"DontFlatten",-1,""}};
static const Enumerant E_LoopControl[] = {
    {0x1,"Unroll",-1,""},{0x2,"DontUnroll",-1,""},{0x4,"DependencyInfinite",-1,""},
    {0x8,"DependencyLength",-1,"L"}};

#define NE(a) ((int)(sizeof(a) / sizeof((a)[0])))
static const EnumKind ENUM_KINDS[] = {
    {"SourceLanguage", 0, E_SourceLanguage, NE(E_SourceLanguage), ""},
    {"AddressingModel", 0, E_AddressingModel, NE(E_AddressingModel), ""},
    {"MemoryModel", 0, E_MemoryModel, NE(E_MemoryModel), ""},
    {"ExecutionModel", 0, E_ExecutionModel, NE(E_ExecutionModel), ""},
    {"ExecutionMode", 0, E_ExecutionMode, NE(E_ExecutionMode), "L*"},
    {"Capability", 0, E_Capability, NE(E_Capability), ""},
    {"StorageClass", 0, E_StorageClass, NE(E_StorageClass), ""},
    {"Decoration", 0, E_Decoration, NE(E_Decoration), "L*"},
    {"BuiltIn", 0, E_BuiltIn, NE(E_BuiltIn), ""},
    {"FuncParamAttr", 0, E_FuncParamAttr, NE(E_FuncParamAttr), ""},
    {"LinkageType", 0, E_LinkageType, NE(E_LinkageType), ""},
    {"FunctionControl", 1, E_FunctionControl, NE(E_FunctionControl), ""},
    {"MemoryAccess", 1, E_MemoryAccess, NE(E_MemoryAccess), ""},
    {"SelectionControl", 1, E_SelectionControl, NE(E_SelectionControl), ""},
    {"LoopControl", 1, E_LoopControl, NE(E_LoopControl), ""},
};

static const EnumKind *find_kind(const char *name, size_t len)
{
    for (int i = 0; i < NE(ENUM_KINDS); i++)
        if (strlen(ENUM_KINDS[i].kind) == len && strncmp(ENUM_KINDS[i].kind, name, len) == 0)
            return &ENUM_KINDS[i];
    return NULL;
}

static const Enumerant *find_enumerant(const EnumKind *k, uint32_t v)
{
    for (int i = 0; i < k->n; i++)
        if (k->e[i].value == v) return &k->e[i];
    return NULL;
}

/* Capability dependencies: declaring the left capability implicitly declares
 * the right one (section 3.4.5, "capabilities and dependencies"). */
static const int CAP_DEPENDS[][2] = {
    {1,0},{2,1},{3,1},{7,6},{8,6},{12,11},{13,6},{14,13},{15,13},{17,6},{19,6},{20,6},
    {21,1},{23,3},{24,2},{25,1},{27,1},{28,1},{29,1},{30,1},{31,1},{32,1},{33,1},
    {34,45},{35,1},{36,37},{37,1},{38,4},{40,1},{41,1},{42,1},{44,43},{45,1},{47,46},
    {48,1},{49,1},{50,1},{51,1},{52,1},{53,1},{54,2},{55,1},{56,1},{57,2},{58,19},
    {59,6},{60,17}};

/* ------------------------------------------------------------------ */
/* Instructions of the compute subset.                                */
/* operands: space separated; I id, L literal word, S literal string,  */
/* C context-dependent literal (all remaining words, at least one),    */
/* E:<kind> value enum, B:<kind> bit enum; prefix ? optional; suffix * */
/* repeat to the end of the instruction; "I2*" repeats id pairs.       */
/* ------------------------------------------------------------------ */
typedef struct { uint16_t op; const char *name; uint8_t rtype, rid; const char *operands; int cap; } OpInfo;

#define BIN "I I"
static const OpInfo OPS[] = {
    {0, "OpNop", 0, 0, "", -1},
    {1, "OpUndef", 1, 1, "", -1},
    {3, "OpSource", 0, 0, "E:SourceLanguage L ?I ?S", -1},
    {5, "OpName", 0, 0, "I S", -1},
    {6, "OpMemberName", 0, 0, "I L S", -1},
    {7, "OpString", 0, 1, "S", -1},
    {10, "OpExtension", 0, 0, "S", -1},
    {11, "OpExtInstImport", 0, 1, "S", -1},
    {12, "OpExtInst", 1, 1, "I L I*", -1},
    {14, "OpMemoryModel", 0, 0, "E:AddressingModel E:MemoryModel", -1},
    {15, "OpEntryPoint", 0, 0, "E:ExecutionModel I S I*", -1},
    {16, "OpExecutionMode", 0, 0, "I E:ExecutionMode", -1},
    {17, "OpCapability", 0, 0, "E:Capability", -1},
    {19, "OpTypeVoid", 0, 1, "", -1},
    {20, "OpTypeBool", 0, 1, "", -1},
    {21, "OpTypeInt", 0, 1, "L L", -1},
    {22, "OpTypeFloat", 0, 1, "L", -1},
    {23, "OpTypeVector", 0, 1, "I L", -1},
    {28, "OpTypeArray", 0, 1, "I I", -1},
    {30, "OpTypeStruct", 0, 1, "I*", -1},
    {32, "OpTypePointer", 0, 1, "E:StorageClass I", -1},
    {33, "OpTypeFunction", 0, 1, "I I*", -1},
    {41, "OpConstantTrue", 1, 1, "", -1},
    {42, "OpConstantFalse", 1, 1, "", -1},
    {43, "OpConstant", 1, 1, "C", -1},
    {44, "OpConstantComposite", 1, 1, "I*", -1},
    {46, "OpConstantNull", 1, 1, "", -1},
    {54, "OpFunction", 1, 1, "B:FunctionControl I", -1},
    {55, "OpFunctionParameter", 1, 1, "", -1},
    {56, "OpFunctionEnd", 0, 0, "", -1},
    {57, "OpFunctionCall", 1, 1, "I I*", -1},
    {59, "OpVariable", 1, 1, "E:StorageClass ?I", -1},
    {61, "OpLoad", 1, 1, "I ?B:MemoryAccess", -1},
    {62, "OpStore", 0, 0, "I I ?B:MemoryAccess", -1},
    {65, "OpAccessChain", 1, 1, "I I*", -1},
    {66, "OpInBoundsAccessChain", 1, 1, "I I*", -1},
    {67, "OpPtrAccessChain", 1, 1, "I I I*", 4},
    {70, "OpInBoundsPtrAccessChain", 1, 1, "I I I*", 4},
    {71, "OpDecorate", 0, 0, "I E:Decoration", -1},
    {80, "OpCompositeConstruct", 1, 1, "I*", -1},
    {81, "OpCompositeExtract", 1, 1, "I L*", -1},
    {83, "OpCopyObject", 1, 1, "I", -1},
    {109, "OpConvertFToU", 1, 1, "I", -1},
    {110, "OpConvertFToS", 1, 1, "I", -1},
    {111, "OpConvertSToF", 1, 1, "I", -1},
    {112, "OpConvertUToF", 1, 1, "I", -1},
    {113, "OpUConvert", 1, 1, "I", -1},
    {114, "OpSConvert", 1, 1, "I", -1},
    {115, "OpFConvert", 1, 1, "I", -1},
    {117, "OpConvertPtrToU", 1, 1, "I", 4},
    {120, "OpConvertUToPtr", 1, 1, "I", 4},
    {121, "OpPtrCastToGeneric", 1, 1, "I", 6},
    {122, "OpGenericCastToPtr", 1, 1, "I", 6},
    {124, "OpBitcast", 1, 1, "I", -1},
    {126, "OpSNegate", 1, 1, "I", -1},
    {127, "OpFNegate", 1, 1, "I", -1},
    {128, "OpIAdd", 1, 1, BIN, -1},
    {129, "OpFAdd", 1, 1, BIN, -1},
    {130, "OpISub", 1, 1, BIN, -1},
    {131, "OpFSub", 1, 1, BIN, -1},
    {132, "OpIMul", 1, 1, BIN, -1},
    {133, "OpFMul", 1, 1, BIN, -1},
    {134, "OpUDiv", 1, 1, BIN, -1},
    {135, "OpSDiv", 1, 1, BIN, -1},
    {136, "OpFDiv", 1, 1, BIN, -1},
    {137, "OpUMod", 1, 1, BIN, -1},
    {138, "OpSRem", 1, 1, BIN, -1},
    {139, "OpSMod", 1, 1, BIN, -1},
    {140, "OpFRem", 1, 1, BIN, -1},
    {141, "OpFMod", 1, 1, BIN, -1},
    {164, "OpLogicalEqual", 1, 1, BIN, -1},
    {165, "OpLogicalNotEqual", 1, 1, BIN, -1},
    {166, "OpLogicalOr", 1, 1, BIN, -1},
    {167, "OpLogicalAnd", 1, 1, BIN, -1},
    {168, "OpLogicalNot", 1, 1, "I", -1},
    {169, "OpSelect", 1, 1, "I I I", -1},
    {170, "OpIEqual", 1, 1, BIN, -1},
    {171, "OpINotEqual", 1, 1, BIN, -1},
    {172, "OpUGreaterThan", 1, 1, BIN, -1},
    {173, "OpSGreaterThan", 1, 1, BIN, -1},
    {174, "OpUGreaterThanEqual", 1, 1, BIN, -1},
    {175, "OpSGreaterThanEqual", 1, 1, BIN, -1},
    {176, "OpULessThan", 1, 1, BIN, -1},
    {177, "OpSLessThan", 1, 1, BIN, -1},
    {178, "OpULessThanEqual", 1, 1, BIN, -1},
    {179, "OpSLessThanEqual", 1, 1, BIN, -1},
    {180, "OpFOrdEqual", 1, 1, BIN, -1},
    {181, "OpFUnordEqual", 1, 1, BIN, -1},
    {182, "OpFOrdNotEqual", 1, 1, BIN, -1},
    {183, "OpFUnordNotEqual", 1, 1, BIN, -1},
    {184, "OpFOrdLessThan", 1, 1, BIN, -1},
    {185, "OpFUnordLessThan", 1, 1, BIN, -1},
    {186, "OpFOrdGreaterThan", 1, 1, BIN, -1},
    {187, "OpFUnordGreaterThan", 1, 1, BIN, -1},
    {188, "OpFOrdLessThanEqual", 1, 1, BIN, -1},
    {189, "OpFUnordLessThanEqual", 1, 1, BIN, -1},
    {190, "OpFOrdGreaterThanEqual", 1, 1, BIN, -1},
    {191, "OpFUnordGreaterThanEqual", 1, 1, BIN, -1},
    {194, "OpShiftRightLogical", 1, 1, BIN, -1},
    {195, "OpShiftRightArithmetic", 1, 1, BIN, -1},
    {196, "OpShiftLeftLogical", 1, 1, BIN, -1},
    {197, "OpBitwiseOr", 1, 1, BIN, -1},
    {198, "OpBitwiseXor", 1, 1, BIN, -1},
    {199, "OpBitwiseAnd", 1, 1, BIN, -1},
    {200, "OpNot", 1, 1, "I", -1},
    {224, "OpControlBarrier", 0, 0, "I I I", -1},
    {225, "OpMemoryBarrier", 0, 0, "I I", -1},
    {227, "OpAtomicLoad", 1, 1, "I I I", -1},
    {228, "OpAtomicStore", 0, 0, "I I I I", -1},
    {229, "OpAtomicExchange", 1, 1, "I I I I", -1},
    {234, "OpAtomicIAdd", 1, 1, "I I I I", -1},
    {235, "OpAtomicISub", 1, 1, "I I I I", -1},
    {245, "OpPhi", 1, 1, "I2*", -1},
    {246, "OpLoopMerge", 0, 0, "I I B:LoopControl", -1},
    {247, "OpSelectionMerge", 0, 0, "I B:SelectionControl", -1},
    {248, "OpLabel", 0, 1, "", -1},
    {249, "OpBranch", 0, 0, "I", -1},
    {250, "OpBranchConditional", 0, 0, "I I I L*", -1},
    {253, "OpReturn", 0, 0, "", -1},
    {254, "OpReturnValue", 0, 0, "I", -1},
    {255, "OpUnreachable", 0, 0, "", -1},
};

static const OpInfo *find_op(uint32_t op)
{
    for (int i = 0; i < NE(OPS); i++)
        if (OPS[i].op == op) return &OPS[i];
    return NULL;
}

static const OpInfo *find_op_name(const char *name, size_t len)
{
    for (int i = 0; i < NE(OPS); i++)
        if (strlen(OPS[i].name) == len && strncmp(OPS[i].name, name, len) == 0) return &OPS[i];
    return NULL;
}

/* ------------------------------------------------------------------ */
/* Operand walk: turns one instruction into a list of typed tokens.   */
/* ------------------------------------------------------------------ */
enum { TK_ID, TK_LIT, TK_STR, TK_CLIT, TK_ENUM, TK_BITS };
typedef struct { int type; uint32_t pos, n; const EnumKind *kind; } Tok;
#define MAX_TOKS 70000
typedef struct { Tok t[MAX_TOKS]; int n; } TokList;

static void push_tok(TokList *L, int type, uint32_t pos, uint32_t n, const EnumKind *k)
{
    if (L->n < MAX_TOKS) { L->t[L->n].type = type; L->t[L->n].pos = pos; L->t[L->n].n = n; L->t[L->n].kind = k; L->n++; }
}

/* A literal string starts at word pos: UTF-8 bytes, little-endian within each
 * word, NUL-terminated, the rest of the last word zero. Returns the number of
 * words, or 0 if there is no NUL before word end or the padding is not zero. */
static uint32_t string_words(const uint32_t *w, uint32_t pos, uint32_t end)
{
    for (uint32_t i = pos; i < end; i++) {
        uint32_t x = w[i];
        for (int b = 0; b < 4; b++) {
            if (((x >> (8 * b)) & 0xffu) == 0) {
                for (int c = b + 1; c < 4; c++)
                    if (((x >> (8 * c)) & 0xffu) != 0) return 0;
                return i - pos + 1;
            }
        }
    }
    return 0;
}

static int walk_spec(const uint32_t *w, uint32_t wc, uint32_t *pos, const char *spec, TokList *L);

static int walk_one(const uint32_t *w, uint32_t wc, uint32_t *pos, const char *tok, size_t len, TokList *L)
{
    /* tok has no '?' and no '*' */
    if (len == 1 && tok[0] == 'I') { push_tok(L, TK_ID, *pos, 1, NULL); (*pos)++; return 0; }
    if (len == 1 && tok[0] == 'L') { push_tok(L, TK_LIT, *pos, 1, NULL); (*pos)++; return 0; }
    if (len == 1 && tok[0] == 'S') {
        uint32_t n = string_words(w, *pos, wc);
        if (n == 0) return -1;
        push_tok(L, TK_STR, *pos, n, NULL); *pos += n; return 0;
    }
    if (len == 1 && tok[0] == 'C') {
        if (*pos >= wc) return -1;
        push_tok(L, TK_CLIT, *pos, wc - *pos, NULL); *pos = wc; return 0;
    }
    if (len > 2 && (tok[0] == 'E' || tok[0] == 'B') && tok[1] == ':') {
        const EnumKind *k = find_kind(tok + 2, len - 2);
        uint32_t v = w[*pos];
        push_tok(L, k->is_bits ? TK_BITS : TK_ENUM, *pos, 1, k);
        (*pos)++;
        if (!k->is_bits) {
            const Enumerant *e = find_enumerant(k, v);
            const char *params = (e && e->params) ? e->params : k->unknown_params;
            return walk_spec(w, wc, pos, params, L);
        }
        for (int bit = 0; bit < 32; bit++) {
            if (!(v & (1u << bit))) continue;
            const Enumerant *e = find_enumerant(k, 1u << bit);
            if (e && e->params && e->params[0])
                if (walk_spec(w, wc, pos, e->params, L)) return -1;
        }
        return 0;
    }
    fprintf(stderr, "oracle: bad operand spec token\n");
    abort();
}

/* Walk a spec string from *pos. Required operands must be present; an
 * optional one is taken when words remain; a '*' operand takes every
 * remaining word. Returns 0, or -1 if the words do not fit the spec. */
static int walk_spec(const uint32_t *w, uint32_t wc, uint32_t *pos, const char *spec, TokList *L)
{
    const char *s = spec;
    while (*s) {
        while (*s == ' ') s++;
        if (!*s) break;
        const char *b = s;
        while (*s && *s != ' ') s++;
        size_t len = (size_t)(s - b);
        int optional = 0, star = 0;
        if (b[0] == '?') { optional = 1; b++; len--; }
        if (len >= 1 && b[len - 1] == '*') { star = 1; len--; }
        if (star) {
            if (len == 2 && b[0] == 'I' && b[1] == '2') {
                if ((wc - *pos) % 2 != 0) return -1;
                while (*pos < wc) { push_tok(L, TK_ID, *pos, 1, NULL); (*pos)++; }
            } else if (len == 1 && (b[0] == 'I' || b[0] == 'L')) {
                while (*pos < wc) { push_tok(L, b[0] == 'I' ? TK_ID : TK_LIT, *pos, 1, NULL); (*pos)++; }
            } else {
                fprintf(stderr, "oracle: bad star spec\n"); abort();
            }
            continue;
        }
        if (*pos >= wc) {
            if (optional) continue;
            return -1;
        }
        if (walk_one(w, wc, pos, b, len, L)) return -1;
    }
    return 0;
}

/* Full operand walk of the instruction at w[0 .. wc). Returns 0 if the words
 * match the opcode's operand list exactly, -1 otherwise (BAD_OPERANDS). */
static int walk_instruction(const uint32_t *w, uint32_t wc, const OpInfo *oi, TokList *L)
{
    L->n = 0;
    uint32_t pos = 1;
    if (oi->rtype) { if (pos >= wc) return -1; push_tok(L, TK_ID, pos, 1, NULL); pos++; }
    if (oi->rid) { if (pos >= wc) return -1; push_tok(L, TK_ID, pos, 1, NULL); pos++; }
    if (walk_spec(w, wc, &pos, oi->operands, L)) return -1;
    return pos == wc ? 0 : -1;
}

/* ------------------------------------------------------------------ */
/* Decode (framing).                                                   */
/* ------------------------------------------------------------------ */

/* Header check of one module of n words. Returns a status code. */
static uint32_t header_status(const uint32_t *w, int64_t n)
{
    if (n < 5) return ST_TRUNCATED;
    if (w[0] != ORC_MAGIC) return ST_BAD_MAGIC;
    uint32_t ver = w[1];
    uint32_t major = (ver >> 16) & 0xffu, minor = (ver >> 8) & 0xffu;
    if ((ver & 0xff0000ffu) != 0 || major != 1 || minor > 6) return ST_BAD_HEADER;
    if (w[4] != 0) return ST_BAD_HEADER;
    return ST_OK;
}

/* Decode a whole batch. Module m is words[mod_off[m] .. mod_off[m+1]).
 * Per module: check the header; then from word 5, read word count and opcode
 * from each instruction's first word, stopping at the first word count of 0
 * (ZERO_WORDCOUNT) or at an instruction that runs past the module's end
 * (TRUNCATED). Rows before the error are kept. Row columns are global across
 * the batch; off[] is the absolute word index into words[]. rtype/rid are
 * taken from the opcode's descriptor when the opcode is known and the words
 * exist, else 0. err_row[m] is the module-local row index of a framing error
 * (= n_instr[m]) or -1.
 * Returns the number of rows, or -1 if cap_rows is too small. */
int64_t orc_decode(const uint32_t *words, const int64_t *mod_off, int32_t n_mod,
                   uint16_t *op, uint16_t *wc, uint64_t *off, uint32_t *rtype, uint32_t *rid,
                   uint32_t *mod, int64_t *first_row, uint32_t *n_instr, uint32_t *status,
                   int64_t *err_row, int64_t cap_rows)
{
    int64_t row = 0;
    for (int32_t m = 0; m < n_mod; m++) {
        const uint32_t *w = words + mod_off[m];
        int64_t n = mod_off[m + 1] - mod_off[m];
        first_row[m] = row;
        n_instr[m] = 0;
        err_row[m] = -1;
        status[m] = header_status(w, n);
        if (status[m] != ST_OK) continue;
        int64_t p = 5;
        uint32_t cnt = 0;
        while (p < n) {
            uint32_t c = w[p] >> 16;
            if (c == 0) { status[m] = ST_ZERO_WORDCOUNT; err_row[m] = cnt; break; }
            if (p + c > n) { status[m] = ST_TRUNCATED; err_row[m] = cnt; break; }
            if (row >= cap_rows) return -1;
            uint32_t o = w[p] & 0xffffu;
            const OpInfo *oi = find_op(o);
            op[row] = (uint16_t)o;
            wc[row] = (uint16_t)c;
            off[row] = (uint64_t)(mod_off[m] + p);
            rtype[row] = 0; rid[row] = 0;
            if (oi) {
                uint32_t q = 1;
                if (oi->rtype) { if (q < c) rtype[row] = w[p + q]; q++; }
                if (oi->rid) { if (q < c) rid[row] = w[p + q]; }
            }
            mod[row] = (uint32_t)m;
            row++; cnt++;
            p += c;
        }
        n_instr[m] = cnt;
    }
    return row;
}


/* ------------------------------------------------------------------ */
/* A small open-addressing map from id to a value, sized by the module */
/* (a module of n words names at most n distinct ids), so that a huge  */
/* bound in a header costs nothing.                                    */
/* ------------------------------------------------------------------ */
typedef struct { uint32_t *key; int64_t *val; uint8_t *used; size_t mask; } IdMap;

static void idmap_init(IdMap *m, int64_t n)
{
    size_t cap = 16;
    while (cap < (size_t)(2 * n + 16)) cap <<= 1;
    m->key = (uint32_t *)malloc(cap * sizeof(uint32_t));
    m->val = (int64_t *)malloc(cap * sizeof(int64_t));
    m->used = (uint8_t *)calloc(cap, 1);
    m->mask = cap - 1;
}
static void idmap_free(IdMap *m) { free(m->key); free(m->val); free(m->used); }
/* Returns the value slot for key, or NULL if absent and create is 0. */
static int64_t *idmap_get(IdMap *m, uint32_t key, int create)
{
    size_t h = (size_t)(key * 2654435761u) & m->mask;
    while (m->used[h]) {
        if (m->key[h] == key) return &m->val[h];
        h = (h + 1) & m->mask;
    }
    if (!create) return NULL;
    m->used[h] = 1; m->key[h] = key; m->val[h] = -1;
    return &m->val[h];
}

/* ------------------------------------------------------------------ */
/* Validate.                                                           */
/* ------------------------------------------------------------------ */
typedef struct { int n; int cap[8]; } Needs;

static void need(Needs *nd, int cap) { if (cap >= 0 && nd->n < 8) nd->cap[nd->n++] = cap; }

/* Capabilities an instruction requires (each one alone must be declared):
 * the opcode's own requirement, those of every enumerant operand, and the
 * integer/float width rules of OpTypeInt / OpTypeFloat. */
static void instruction_needs(const uint32_t *w, const OpInfo *oi, const TokList *L, Needs *nd)
{
    nd->n = 0;
    need(nd, oi->cap);
    for (int i = 0; i < L->n; i++) {
        if (L->t[i].type != TK_ENUM) continue;
        const Enumerant *e = find_enumerant(L->t[i].kind, w[L->t[i].pos]);
        if (e) need(nd, e->cap);
    }
    if (oi->op == 21) {            /* OpTypeInt width */
        uint32_t width = w[2];
        if (width == 8) need(nd, 39);
        if (width == 16) need(nd, 22);
        if (width == 64) need(nd, 11);
    }
    if (oi->op == 22) {            /* OpTypeFloat width */
        uint32_t width = w[2];
        if (width == 16) need(nd, 9);
        if (width == 64) need(nd, 10);
    }
}

static uint64_t cap_closure(uint64_t declared)
{
    uint64_t prev;
    do {
        prev = declared;
        for (int i = 0; i < NE(CAP_DEPENDS); i++)
            if (declared & (1ull << CAP_DEPENDS[i][0])) declared |= 1ull << CAP_DEPENDS[i][1];
    } while (declared != prev);
    return declared;
}

/* Validate every module. status[m] is the module's first error and
 * err_row[m] the module-local row it occurred at (-1 for header and
 * module-level errors and for valid modules).
 *
 * Instruction-level errors, checked per row in this order (the first failing
 * check is the row's error): UNKNOWN_OPCODE, BAD_OPERANDS, ID_OUT_OF_BOUND
 * (result type, result id and every id operand must lie in [1, bound)),
 * DUP_RESULT_ID (an earlier row defines the same result id),
 * MISSING_CAPABILITY (a capability the row requires is not in the closure of
 * the module's declared capabilities). The module's error is the one at the
 * lowest row; a framing error counts as a row after the last decoded row.
 * Without such an error the module-level rules follow, in order: no
 * OpCapability, no OpMemoryModel, more than one OpMemoryModel, no
 * OpEntryPoint, no OpFunction. */
void orc_validate(const uint32_t *words, const int64_t *mod_off, int32_t n_mod,
                  uint32_t *status, int64_t *err_row)
{
    TokList *L = (TokList *)malloc(sizeof(TokList));
    for (int32_t m = 0; m < n_mod; m++) {
        const uint32_t *w = words + mod_off[m];
        int64_t n = mod_off[m + 1] - mod_off[m];
        status[m] = header_status(w, n);
        err_row[m] = -1;
        if (status[m] != ST_OK) continue;
        uint32_t bound = w[3];
        /* pass 1: framing, declared capabilities, module counters */
        int64_t p = 5, rows = 0;
        uint32_t framing = ST_OK;
        uint64_t declared = 0;
        int64_t n_cap = 0, n_mm = 0, n_ep = 0, n_fn = 0;
        while (p < n) {
            uint32_t c = w[p] >> 16;
            if (c == 0) { framing = ST_ZERO_WORDCOUNT; break; }
            if (p + c > n) { framing = ST_TRUNCATED; break; }
            uint32_t o = w[p] & 0xffffu;
            if (o == 17) { n_cap++; if (c >= 2 && w[p + 1] < 64) declared |= 1ull << w[p + 1]; }
            if (o == 14) n_mm++;
            if (o == 15) n_ep++;
            if (o == 54) n_fn++;
            rows++;
            p += c;
        }
        uint64_t have = cap_closure(declared);
        /* pass 2: per-row checks in row order */
        IdMap defined;
        idmap_init(&defined, n);
        p = 5;
        int64_t r = 0;
        uint32_t found = ST_OK;
        for (; r < rows; r++) {
            uint32_t c = w[p] >> 16, o = w[p] & 0xffffu;
            const uint32_t *iw = w + p;
            p += c;
            const OpInfo *oi = find_op(o);
            if (!oi) { found = ST_UNKNOWN_OPCODE; break; }
            if (walk_instruction(iw, c, oi, L)) { found = ST_BAD_OPERANDS; break; }
            int oob = 0;
            for (int i = 0; i < L->n; i++)
                if (L->t[i].type == TK_ID) {
                    uint32_t id = iw[L->t[i].pos];
                    if (id == 0 || id >= bound) oob = 1;
                }
            if (oob) { found = ST_ID_OUT_OF_BOUND; break; }
            if (oi->rid) {
                uint32_t id = iw[1 + oi->rtype];
                if (idmap_get(&defined, id, 0)) { found = ST_DUP_RESULT_ID; break; }
                *idmap_get(&defined, id, 1) = r;
            }
            Needs nd;
            instruction_needs(iw, oi, L, &nd);
            int missing = 0;
            for (int i = 0; i < nd.n; i++)
                if (!(have & (1ull << nd.cap[i]))) missing = 1;
            if (missing) { found = ST_MISSING_CAPABILITY; break; }
        }
        idmap_free(&defined);
        if (found != ST_OK) { status[m] = found; err_row[m] = r; continue; }
        if (framing != ST_OK) { status[m] = framing; err_row[m] = rows; continue; }
        if (n_cap == 0) status[m] = ST_NO_CAPABILITY;
        else if (n_mm == 0) status[m] = ST_NO_MEMORY_MODEL;
        else if (n_mm > 1) status[m] = ST_MULTI_MEMORY_MODEL;
        else if (n_ep == 0) status[m] = ST_NO_ENTRY_POINT;
        else if (n_fn == 0) status[m] = ST_NO_FUNCTION;
    }
    free(L);
}

/* ------------------------------------------------------------------ */
/* logical layout and scopes                                            */
/* ------------------------------------------------------------------ */
/*
 * Section 3.4.1, "Handling Different Scopes within a SPIR-V Module": the
 * module scope holds the global declarations (capabilities, memory model,
 * entry points, debug names, decorations, types, constants, global
 * variables) and the functions; a function holds its parameters and its
 * body; a body is a sequence of basic blocks, each opened by a label.  The
 * paper gives the scopes, not the checks; the reading used here:
 *   - module-scope instructions come in the SPIR-V specification's section
 *     order: capabilities (1), extensions (2), extended-instruction imports
 *     (3), memory model (4), entry points (5), execution modes (6), debug
 *     instructions (7), decorations (8), types / constants / global
 *     variables (9), functions (10); a row of a lower section after one of a
 *     higher section is SECTION_ORDER;
 *   - OpFunction opens a function (only at module scope), its parameters
 *     follow directly, then either OpFunctionEnd (a declaration) or blocks;
 *     a block opens with OpLabel and closes with a terminator (OpBranch,
 *     OpBranchConditional, OpReturn, OpReturnValue, OpUnreachable); after a
 *     terminator comes OpLabel or OpFunctionEnd;
 *   - OpVariable and OpUndef are global declarations at module scope and
 *     body instructions inside a function; OpNop and opcodes outside the
 *     table are allowed anywhere;
 *   - errors: OUTSIDE_FUNCTION (a function-scope instruction at module
 *     scope), IN_FUNCTION (a module-scope instruction, or a second
 *     OpFunction, inside a function), BLOCK (a body instruction or
 *     terminator before the first label or after a terminator, a label in
 *     an open block, a parameter after a label, OpFunctionEnd in an open
 *     block), UNCLOSED (the rows end inside a function; its row is the
 *     module's row count).  The first error in row order is the module's.
 */
enum { LC_ANY, LC_SEC, LC_MIXED, LC_FUNCTION, LC_PARAM, LC_FUNCEND, LC_LABEL, LC_TERM, LC_BODY };
enum { LS_OK, LS_SECTION_ORDER, LS_OUTSIDE_FUNCTION, LS_IN_FUNCTION, LS_BLOCK, LS_UNCLOSED };

int orc_layout_class(uint32_t op, int *section)
{
    *section = 0;
    switch (op) {
    case 0: return LC_ANY;                                     /* OpNop */
    case 17: *section = 1; return LC_SEC;                      /* OpCapability */
    case 10: *section = 2; return LC_SEC;                      /* OpExtension */
    case 11: *section = 3; return LC_SEC;                      /* OpExtInstImport */
    case 14: *section = 4; return LC_SEC;                      /* OpMemoryModel */
    case 15: *section = 5; return LC_SEC;                      /* OpEntryPoint */
    case 16: *section = 6; return LC_SEC;                      /* OpExecutionMode */
    case 3: case 5: case 6: case 7: *section = 7; return LC_SEC;  /* OpSource OpName OpMemberName OpString */
    case 71: *section = 8; return LC_SEC;                      /* OpDecorate */
    case 1: case 59: *section = 9; return LC_MIXED;            /* OpUndef, OpVariable */
    case 54: *section = 10; return LC_FUNCTION;                /* OpFunction */
    case 55: return LC_PARAM;                                  /* OpFunctionParameter */
    case 56: return LC_FUNCEND;                                /* OpFunctionEnd */
    case 248: return LC_LABEL;                                 /* OpLabel */
    case 249: case 250: case 253: case 254: case 255: return LC_TERM;
    default: break;
    }
    if (!find_op(op)) return LC_ANY;
    if (op >= 19 && op <= 46) { *section = 9; return LC_SEC; }   /* OpType* and OpConstant* */
    return LC_BODY;
}

/* Per module (rows first_row[m] .. first_row[m] + n_instr[m] - 1 of a decode):
 * layout status and the module-local row it refers to (-1 when LS_OK). */
void orc_layout(const uint16_t *op, const int64_t *first_row, const uint32_t *n_instr, int32_t n_mod,
                uint32_t *status, int64_t *err_row)
{
    enum { MODULE, HEAD, BLOCK, AFTER };
    for (int32_t m = 0; m < n_mod; m++) {
        int st = MODULE, maxsec = 0;
        uint32_t e = LS_OK;
        int64_t row = -1;
        for (uint32_t i = 0; i < n_instr[m] && e == LS_OK; i++) {
            int sec;
            int c = orc_layout_class(op[first_row[m] + i], &sec);
            switch (c) {
            case LC_ANY:
                break;
            case LC_SEC:
            case LC_MIXED:
            case LC_FUNCTION:
                if (st == MODULE) {
                    if (sec < maxsec) e = LS_SECTION_ORDER;
                    else maxsec = sec;
                    if (c == LC_FUNCTION && e == LS_OK) st = HEAD;
                } else if (c == LC_MIXED && st == BLOCK) {
                    /* a variable or undef inside a block */
                } else if (c == LC_MIXED) {
                    e = LS_BLOCK;
                } else {
                    e = LS_IN_FUNCTION;
                }
                break;
            case LC_PARAM:
                if (st != HEAD) e = st == MODULE ? LS_OUTSIDE_FUNCTION : LS_BLOCK;
                break;
            case LC_LABEL:
                if (st == HEAD || st == AFTER) st = BLOCK;
                else e = st == MODULE ? LS_OUTSIDE_FUNCTION : LS_BLOCK;
                break;
            case LC_BODY:
                if (st != BLOCK) e = st == MODULE ? LS_OUTSIDE_FUNCTION : LS_BLOCK;
                break;
            case LC_TERM:
                if (st == BLOCK) st = AFTER;
                else e = st == MODULE ? LS_OUTSIDE_FUNCTION : LS_BLOCK;
                break;
            case LC_FUNCEND:
                if (st == HEAD || st == AFTER) st = MODULE;
                else e = st == MODULE ? LS_OUTSIDE_FUNCTION : LS_BLOCK;
                break;
            }
            if (e != LS_OK) row = i;
        }
        if (e == LS_OK && st != MODULE) { e = LS_UNCLOSED; row = n_instr[m]; }
        status[m] = e;
        err_row[m] = row;
    }
}

/* ------------------------------------------------------------------ */
/* Encode.                                                             */
/* ------------------------------------------------------------------ */

/* Re-encode a decoded table into out[] (same size and module offsets as the
 * source words). out starts as a copy of src; for each module with a valid
 * header, word 3 (bound) becomes 1 + the largest result id of its rows when
 * recompute_bound is set (1 when it has none); each row then writes its first
 * word from (wc, op) and, when its opcode is known, its result type and
 * result id from the table's columns at their operand positions. */
void orc_encode(const uint32_t *src, const int64_t *mod_off, int32_t n_mod, int64_t n_words,
                const uint16_t *op, const uint16_t *wc, const uint64_t *off, const uint32_t *rtype,
                const uint32_t *rid, const int64_t *first_row, const uint32_t *n_instr,
                uint32_t *out, int recompute_bound)
{
    memcpy(out, src, (size_t)n_words * 4);
    for (int32_t m = 0; m < n_mod; m++) {
        int64_t n = mod_off[m + 1] - mod_off[m];
        if (header_status(src + mod_off[m], n) != ST_OK) continue;
        if (recompute_bound) {
            uint32_t mx = 0;
            for (int64_t r = first_row[m]; r < first_row[m] + n_instr[m]; r++)
                if (rid[r] > mx) mx = rid[r];
            out[mod_off[m] + 3] = mx + 1;
        }
        for (int64_t r = first_row[m]; r < first_row[m] + n_instr[m]; r++) {
            uint64_t p = off[r];
            out[p] = ((uint32_t)wc[r] << 16) | op[r];
            const OpInfo *oi = find_op(op[r]);
            if (!oi) continue;
            uint32_t q = 1;
            if (oi->rtype) { if (q < wc[r]) out[p + q] = rtype[r]; q++; }
            if (oi->rid) { if (q < wc[r]) out[p + q] = rid[r]; }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Disassemble.                                                        */
/* ------------------------------------------------------------------ */
typedef struct { char *buf; int64_t len, cap; } Out;

static void out_bytes(Out *o, const char *s, size_t n)
{
    for (size_t i = 0; i < n; i++) {
        if (o->buf && o->len < o->cap) o->buf[o->len] = s[i];
        o->len++;
    }
}
static void out_str(Out *o, const char *s) { out_bytes(o, s, strlen(s)); }
static void out_fmt_u64(Out *o, uint64_t v) { char t[32]; snprintf(t, sizeof t, "%llu", (unsigned long long)v); out_str(o, t); }

/* Per-module lookups the text needs: the first OpName naming each id and the
 * opcode of the first row defining each id. */
typedef struct {
    uint32_t bound;
    IdMap name_at;        /* id -> word index (module-relative) of the first OpName row naming it */
    IdMap def_op;         /* id -> opcode of the first row whose result id it is */
} Ctx;

static int64_t ctx_name_at(const Ctx *cx, uint32_t id)
{
    int64_t *v = idmap_get((IdMap *)&cx->name_at, id, 0);
    return v ? *v : -1;
}
static int64_t ctx_def_op(const Ctx *cx, uint32_t id)
{
    int64_t *v = idmap_get((IdMap *)&cx->def_op, id, 0);
    return v ? *v : -1;
}

static void put_id(Out *o, const uint32_t *w, int64_t n, const Ctx *cx, uint32_t id, int inline_names)
{
    out_str(o, "%");
    if (inline_names && id < cx->bound && ctx_name_at(cx, id) >= 0) {
        int64_t p = ctx_name_at(cx, id);
        uint32_t c = w[p] >> 16;
        /* name = bytes from word 2 of the OpName up to its first NUL or its end */
        for (uint32_t i = 2; i < c && p + i < n; i++) {
            uint32_t x = w[p + i];
            int stop = 0;
            for (int b = 0; b < 4; b++) {
                unsigned ch = (x >> (8 * b)) & 0xffu;
                if (ch == 0) { stop = 1; break; }
                int keep = (ch >= '0' && ch <= '9') || (ch >= 'A' && ch <= 'Z') ||
                           (ch >= 'a' && ch <= 'z') || ch == '_';
                char cc = keep ? (char)ch : '_';
                out_bytes(o, &cc, 1);
            }
            if (stop) break;
        }
        out_str(o, "_");
    }
    out_fmt_u64(o, id);
}

static void put_string(Out *o, const uint32_t *w, uint32_t pos, uint32_t nwords)
{
    out_str(o, "\"");
    for (uint32_t i = 0; i < nwords; i++) {
        for (int b = 0; b < 4; b++) {
            unsigned ch = (w[pos + i] >> (8 * b)) & 0xffu;
            if (ch == 0) goto done;
            char t[8];
            if (ch == '"' || ch == '\\') { t[0] = '\\'; t[1] = (char)ch; out_bytes(o, t, 2); }
            else if (ch < 0x20 || ch > 0x7e) { snprintf(t, sizeof t, "\\x%02x", ch); out_str(o, t); }
            else { t[0] = (char)ch; out_bytes(o, t, 1); }
        }
    }
done:
    out_str(o, "\"");
}

static void put_enum(Out *o, const EnumKind *k, uint32_t v)
{
    if (!k->is_bits) {
        const Enumerant *e = find_enumerant(k, v);
        if (e) out_str(o, e->name); else out_fmt_u64(o, v);
        return;
    }
    if (v == 0) { out_str(o, "None"); return; }
    uint32_t known = 0;
    for (int i = 0; i < k->n; i++) known |= k->e[i].value;
    if (v & ~known) { out_fmt_u64(o, v); return; }
    int first = 1;
    for (int bit = 0; bit < 32; bit++) {
        if (!(v & (1u << bit))) continue;
        if (!first) out_str(o, "|");
        out_str(o, find_enumerant(k, 1u << bit)->name);
        first = 0;
    }
}

/* Float constants print as C99 hexadecimal floating point, exactly as glibc's
 * printf("%a") prints the value (a 32-bit float is widened to double first). */
static void put_float(Out *o, const uint32_t *w, uint32_t n)
{
    char t[64];
    if (n == 1) { float f; memcpy(&f, w, 4); snprintf(t, sizeof t, "%a", (double)f); }
    else { uint64_t b = (uint64_t)w[0] | ((uint64_t)w[1] << 32); double d; memcpy(&d, &b, 8); snprintf(t, sizeof t, "%a", d); }
    out_str(o, t);
}

static void put_raw(Out *o, const uint32_t *iw, uint32_t c)
{
    char t[16];
    for (uint32_t i = 1; i < c; i++) { snprintf(t, sizeof t, " 0x%08x", iw[i]); out_str(o, t); }
}

static void dis_row(Out *o, const uint32_t *w, int64_t n, int64_t p, const Ctx *cx, int inline_names, TokList *L)
{
    const uint32_t *iw = w + p;
    uint32_t c = iw[0] >> 16, opn = iw[0] & 0xffffu;
    const OpInfo *oi = find_op(opn);
    if (!oi) {
        char t[24]; snprintf(t, sizeof t, "Op%u", opn); out_str(o, t);
        put_raw(o, iw, c); out_str(o, "\n"); return;
    }
    if (walk_instruction(iw, c, oi, L)) {
        out_str(o, oi->name); put_raw(o, iw, c); out_str(o, "\n"); return;
    }
    int ti = 0;
    if (oi->rid) {
        /* the result id is the token after the result type (if any) */
        uint32_t rid_v = iw[1 + oi->rtype];
        put_id(o, w, n, cx, rid_v, inline_names);
        out_str(o, " = ");
    }
    out_str(o, oi->name);
    for (ti = 0; ti < L->n; ti++) {
        const Tok *t = &L->t[ti];
        if (oi->rid && t->pos == (uint32_t)(1 + oi->rtype) && t->type == TK_ID) continue;
        out_str(o, " ");
        switch (t->type) {
        case TK_ID: put_id(o, w, n, cx, iw[t->pos], inline_names); break;
        case TK_LIT: out_fmt_u64(o, iw[t->pos]); break;
        case TK_STR: put_string(o, iw, t->pos, t->n); break;
        case TK_ENUM: case TK_BITS: put_enum(o, t->kind, iw[t->pos]); break;
        case TK_CLIT: {
            uint32_t ty = iw[1];
            int is_float = ty < cx->bound && ctx_def_op(cx, ty) == 22;
            if (is_float && (t->n == 1 || t->n == 2)) put_float(o, iw + t->pos, t->n);
            else if (t->n == 1) out_fmt_u64(o, iw[t->pos]);
            else if (t->n == 2) out_fmt_u64(o, (uint64_t)iw[t->pos] | ((uint64_t)iw[t->pos + 1] << 32));
            else for (uint32_t i = 0; i < t->n; i++) { if (i) out_str(o, " "); out_fmt_u64(o, iw[t->pos + i]); }
            break;
        }
        }
    }
    out_str(o, "\n");
}

/* Disassemble a batch. text_off[m] .. text_off[m+1] is module m's text. A
 * module whose header is invalid has no text. Otherwise, with header set,
 * five comment lines (magic, version, generator, bound, schema) come first;
 * then one line per decoded row: "[%R = ]OpName[ operand]*\n" with the result
 * type as the first operand. Ids print as %<id>, or with inline names as
 * %<name>_<id> where name is the first OpName for that id with every byte
 * outside [A-Za-z0-9_] replaced by '_'. Literals print as unsigned decimal;
 * strings quoted with \" \\ and \xhh escapes; enums by name (decimal if
 * unknown, bit enums as A|B, 0 as None); OpConstant values of float type in
 * hexadecimal floating point, of other types as decimal (two words form one
 * 64-bit value, low word first). Rows whose opcode is unknown print as
 * Op<decimal>, and rows whose operands do not parse as their opcode name,
 * each followed by the instruction's remaining words as 0x%08x.
 * Returns the total number of bytes; text may be NULL to size. */
int64_t orc_disassemble(const uint32_t *words, const int64_t *mod_off, int32_t n_mod,
                        int inline_names, int header, char *text, int64_t cap, int64_t *text_off)
{
    Out o = {text, 0, cap};
    TokList *L = (TokList *)malloc(sizeof(TokList));
    for (int32_t m = 0; m < n_mod; m++) {
        const uint32_t *w = words + mod_off[m];
        int64_t n = mod_off[m + 1] - mod_off[m];
        text_off[m] = o.len;
        if (header_status(w, n) != ST_OK) continue;
        Ctx cx;
        cx.bound = w[3];
        idmap_init(&cx.name_at, n);
        idmap_init(&cx.def_op, n);
        /* first OpName per id, first definition per id (rows in order) */
        int64_t p = 5;
        while (p < n) {
            uint32_t c = w[p] >> 16;
            if (c == 0 || p + c > n) break;
            uint32_t opn = w[p] & 0xffffu;
            if (opn == 5 && c >= 2 && w[p + 1] < cx.bound) {
                int64_t *v = idmap_get(&cx.name_at, w[p + 1], 1);
                if (*v < 0) *v = p;
            }
            const OpInfo *oi = find_op(opn);
            if (oi && oi->rid && (uint32_t)(1 + oi->rtype) < c) {
                uint32_t id = w[p + 1 + oi->rtype];
                if (id < cx.bound) {
                    int64_t *v = idmap_get(&cx.def_op, id, 1);
                    if (*v < 0) *v = opn;
                }
            }
            p += c;
        }
        if (header) {
            char t[96];
            out_str(&o, "; SPIR-V\n");
            snprintf(t, sizeof t, "; Version: %u.%u\n", (w[1] >> 16) & 0xffu, (w[1] >> 8) & 0xffu); out_str(&o, t);
            snprintf(t, sizeof t, "; Generator: 0x%08x\n", w[2]); out_str(&o, t);
            snprintf(t, sizeof t, "; Bound: %u\n", w[3]); out_str(&o, t);
            snprintf(t, sizeof t, "; Schema: %u\n", w[4]); out_str(&o, t);
        }
        p = 5;
        while (p < n) {
            uint32_t c = w[p] >> 16;
            if (c == 0 || p + c > n) break;
            dis_row(&o, w, n, p, &cx, inline_names, L);
            p += c;
        }
        idmap_free(&cx.name_at); idmap_free(&cx.def_op);
    }
    text_off[n_mod] = o.len;
    free(L);
    return o.len;
}

/* ------------------------------------------------------------------ */
/* Assemble (text -> one module), section 3.4.4 "Dis/Assembler": the   */
/* text form the disassembler prints, read back into words, with the   */
/* map from id names to ids that the paper's assembler keeps in a hash */
/* table.                                                              */
/*                                                                     */
/* The text form, line by line ('\n' ends a line; a final '\n' does    */
/* not start another; lines are numbered from 1):                      */
/*  - an empty line is skipped;                                        */
/*  - a line starting with ';' is a comment; exactly                   */
/*    "; Version: A.B" (A, B <= 255), "; Generator: 0xH",              */
/*    "; Bound: N" and "; Schema: N" (values < 2^32, nothing after     */
/*    them) set the header words; the last such line wins;             */
/*  - any other line is one instruction: tokens split by spaces; a     */
/*    token that starts with '"' runs to the next '"' not escaped by   */
/*    '\' (an unclosed one is an error);                               */
/*    "[%r =] OpName operands" or "Op<decimal> 0xHHHHHHHH..." (raw).   */
/* Ids: "%<digits>" and "%<name>_<digits>" are the id <digits>         */
/* (< 2^32); any other "%<name>" is a named id: the distinct names get */
/* ids M+1, M+2, ... in order of first appearance in the module text,  */
/* M the largest explicit id of the module (0 if none).                */
/* Literals: decimal, < 2^32. Strings: "\xHH" is byte HH, '\' before   */
/* any other byte is that byte. OpConstant's value: two or more tokens */
/* are one word each; one token is a decimal integer (< 2^64) or a     */
/* float literal ([+-] then inf, nan, C99 hex or decimal), as wide as  */
/* the result type: the first OpTypeInt / OpTypeFloat of the module    */
/* that defines that id (a 32-bit integer if none). A float literal of */
/* a 32-bit type is rounded to double, then to float, both to nearest  */
/* even. Enumerants: the name, or decimal; bit enums also "None" and   */
/* "A|B". An instruction has at most 65535 words.                      */
/* Header: magic, version (default 1.2), generator (0), bound (the     */
/* Bound line, else the largest id + 1), schema (0).                   */
/* ------------------------------------------------------------------ */
typedef struct { const char *s; size_t n; int open; } Span;

static int is_raw_word(Span t)
{
    if (t.n != 10 || t.s[0] != '0' || t.s[1] != 'x') return 0;
    for (size_t i = 2; i < 10; i++) if (!isxdigit((unsigned char)t.s[i])) return 0;
    return 1;
}

/* decimal digits only, at least one, value <= max */
static int parse_dec(const char *s, size_t n, uint64_t max, uint64_t *v)
{
    if (n == 0) return -1;
    uint64_t a = 0;
    for (size_t i = 0; i < n; i++) {
        if (!isdigit((unsigned char)s[i])) return -1;
        uint64_t d = (uint64_t)(s[i] - '0');
        if (a > (max - d) / 10) return -1;
        a = a * 10 + d;
    }
    *v = a;
    return 0;
}

static int parse_u32(Span t, uint32_t *v)
{
    uint64_t u;
    if (parse_dec(t.s, t.n, 0xffffffffull, &u)) return -1;
    *v = (uint32_t)u;
    return 0;
}

/* Id token: 0 explicit (*id set), 1 named, -1 not an id. */
static int classify_id(Span t, uint32_t *id)
{
    if (t.n < 2 || t.s[0] != '%') return -1;
    size_t j = t.n;
    while (j > 1 && isdigit((unsigned char)t.s[j - 1])) j--;
    if (j == t.n || (j != 1 && t.s[j - 1] != '_')) return 1;
    uint64_t u;
    if (parse_dec(t.s + j, t.n - j, 0xffffffffull, &u)) return -1;
    *id = (uint32_t)u;
    return 0;
}

/* Float literal: the whole token must match
 *   [+-]? ( inf | nan | 0[xX] H* [. H*] [[pP] [+-]? D+] | D* [. D*] [[eE] [+-]? D+] )
 * with at least one digit in the mantissa. */
static int is_float_literal(Span t)
{
    size_t i = 0, n = t.n;
    const char *s = t.s;
    if (i < n && (s[i] == '+' || s[i] == '-')) i++;
    if (n - i == 3 && (strncmp(s + i, "inf", 3) == 0 || strncmp(s + i, "nan", 3) == 0)) return 1;
    int hex = (n - i >= 2 && s[i] == '0' && (s[i + 1] == 'x' || s[i + 1] == 'X'));
    if (hex) i += 2;
    size_t digits = 0;
    while (i < n && (hex ? isxdigit((unsigned char)s[i]) : isdigit((unsigned char)s[i]))) { i++; digits++; }
    if (i < n && s[i] == '.') {
        i++;
        while (i < n && (hex ? isxdigit((unsigned char)s[i]) : isdigit((unsigned char)s[i]))) { i++; digits++; }
    }
    if (digits == 0) return 0;
    if (i < n && (hex ? (s[i] == 'p' || s[i] == 'P') : (s[i] == 'e' || s[i] == 'E'))) {
        i++;
        if (i < n && (s[i] == '+' || s[i] == '-')) i++;
        size_t e = 0;
        while (i < n && isdigit((unsigned char)s[i])) { i++; e++; }
        if (e == 0) return 0;
    }
    return i == n;
}

static int tokenize(const char *s, size_t n, Span *toks)
{
    int k = 0;
    size_t i = 0;
    while (i < n) {
        while (i < n && s[i] == ' ') i++;
        if (i >= n) break;
        size_t b = i;
        int open = 0;
        if (s[i] == '"') {
            i++;
            while (i < n && s[i] != '"') i += (s[i] == '\\') ? 2 : 1;
            if (i >= n) { open = 1; i = n; }
            else i++;
        } else {
            while (i < n && s[i] != ' ') i++;
        }
        toks[k].s = s + b; toks[k].n = i - b; toks[k].open = open; k++;
    }
    return k;
}

typedef struct { uint32_t *out; int64_t n, cap; } Words;
static void put_word(Words *W, uint32_t v) { if (W->n < W->cap) W->out[W->n] = v; W->n++; }

static int hexval(int c)
{
    if (c >= '0' && c <= '9') return c - '0';
    if (c >= 'a' && c <= 'f') return c - 'a' + 10;
    if (c >= 'A' && c <= 'F') return c - 'A' + 10;
    return -1;
}

static int put_string_tok(Words *W, Span t)
{
    if (t.n < 2 || t.s[0] != '"' || t.open) return -1;
    const char *b = t.s + 1;
    size_t n = t.n - 2, i = 0;
    uint32_t acc = 0;
    int k = 0;
    while (i < n) {
        unsigned ch = (unsigned char)b[i];
        if (ch == '\\') {
            if (i + 3 < n && b[i + 1] == 'x' && hexval(b[i + 2]) >= 0 && hexval(b[i + 3]) >= 0) {
                ch = (unsigned)(hexval(b[i + 2]) * 16 + hexval(b[i + 3]));
                i += 4;
            } else {
                if (i + 1 >= n) return -1;
                ch = (unsigned char)b[i + 1];
                i += 2;
            }
        } else {
            i++;
        }
        acc |= (uint32_t)ch << (8 * k);
        if (++k == 4) { put_word(W, acc); acc = 0; k = 0; }
    }
    put_word(W, acc);            /* the NUL and the zero padding */
    return 0;
}

/* Named ids: an open-addressing hash map from name bytes to the index of
 * the name's first appearance. */
typedef struct { const char *s; size_t n; } Name;
typedef struct { Name *names; int n, cap; int *slot; int nslot; } NameMap;

static uint32_t name_hash(const char *s, size_t n)
{
    uint32_t h = 2166136261u;
    for (size_t i = 0; i < n; i++) { h ^= (unsigned char)s[i]; h *= 16777619u; }
    return h;
}

static int namemap_get(NameMap *M, Span t, int insert)
{
    if (M->nslot == 0 || (insert && 2 * (M->n + 1) > M->nslot)) {
        int ns = M->nslot ? 2 * M->nslot : 64;
        int *sl = (int *)malloc(sizeof(int) * ns);
        for (int i = 0; i < ns; i++) sl[i] = -1;
        for (int k = 0; k < M->n; k++) {
            uint32_t h = name_hash(M->names[k].s, M->names[k].n) % (uint32_t)ns;
            while (sl[h] >= 0) h = (h + 1) % (uint32_t)ns;
            sl[h] = k;
        }
        free(M->slot); M->slot = sl; M->nslot = ns;
    }
    uint32_t h = name_hash(t.s, t.n) % (uint32_t)M->nslot;
    while (M->slot[h] >= 0) {
        Name *q = &M->names[M->slot[h]];
        if (q->n == t.n && memcmp(q->s, t.s, t.n) == 0) return M->slot[h];
        h = (h + 1) % (uint32_t)M->nslot;
    }
    if (!insert) return -1;
    if (M->n == M->cap) {
        M->cap = M->cap ? 2 * M->cap : 64;
        M->names = (Name *)realloc(M->names, sizeof(Name) * M->cap);
    }
    M->names[M->n].s = t.s; M->names[M->n].n = t.n;
    M->slot[h] = M->n;
    return M->n++;
}

/* The first OpTypeInt / OpTypeFloat that defines each type id. */
typedef struct { uint32_t id; uint8_t is_float, width; } TypeDecl;

typedef struct {
    int pass;                    /* 0: named ids, largest explicit id; 1: type declarations; 2: words */
    Span *tk; int nt, ti;
    Words *W;
    NameMap names;
    uint64_t max_explicit;
    TypeDecl *types; int ntypes, captypes;
    uint32_t rtype;              /* result type of the instruction being assembled */
    uint64_t max_id;
} Asm;

/* Resolve an id token (pass 0 registers named ids). */
static int asm_id(Asm *A, Span t, uint32_t *out)
{
    uint32_t id;
    int c = classify_id(t, &id);
    if (c < 0) return -1;
    if (c == 0) {
        if (A->pass == 0 && id > A->max_explicit) A->max_explicit = id;
    } else {
        int k = namemap_get(&A->names, t, A->pass == 0);
        uint64_t fresh = A->max_explicit + 1 + (uint64_t)k;
        if (A->pass > 0 && fresh > 0xffffffffull) return -1;
        id = (uint32_t)fresh;
    }
    if (A->pass == 2 && id > A->max_id) A->max_id = id;
    *out = id;
    return 0;
}

static int parse_enum_tok(const EnumKind *k, Span t, uint32_t *v)
{
    if (parse_u32(t, v) == 0) return 0;
    if (!k->is_bits) {
        for (int i = 0; i < k->n; i++)
            if (strlen(k->e[i].name) == t.n && strncmp(k->e[i].name, t.s, t.n) == 0) { *v = k->e[i].value; return 0; }
        return -1;
    }
    if (t.n == 4 && strncmp(t.s, "None", 4) == 0) { *v = 0; return 0; }
    uint32_t acc = 0;
    size_t i = 0;
    for (;;) {
        size_t b = i;
        while (i < t.n && t.s[i] != '|') i++;
        int ok = 0;
        for (int j = 0; j < k->n; j++)
            if (strlen(k->e[j].name) == i - b && strncmp(k->e[j].name, t.s + b, i - b) == 0) { acc |= k->e[j].value; ok = 1; }
        if (!ok) return -1;
        if (i == t.n) break;
        i++;                     /* past '|': a name must follow */
    }
    *v = acc;
    return 0;
}

static int asm_spec(Asm *A, const char *spec);

static TypeDecl type_of(Asm *A, uint32_t id)
{
    for (int i = 0; i < A->ntypes; i++)
        if (A->types[i].id == id) return A->types[i];
    TypeDecl d = {id, 0, 32};
    return d;
}

static int asm_one(Asm *A, const char *tok, size_t len)
{
    Span t = A->tk[A->ti];
    if (len == 1 && tok[0] == 'I') {
        uint32_t id; if (asm_id(A, t, &id)) return -1;
        put_word(A->W, id); A->ti++; return 0;
    }
    if (len == 1 && tok[0] == 'L') { uint32_t v; if (parse_u32(t, &v)) return -1; put_word(A->W, v); A->ti++; return 0; }
    if (len == 1 && tok[0] == 'S') { if (put_string_tok(A->W, t)) return -1; A->ti++; return 0; }
    if (len == 1 && tok[0] == 'C') {
        if (A->nt - A->ti >= 2) {           /* three or more words print one per token */
            while (A->ti < A->nt) { uint32_t v; if (parse_u32(A->tk[A->ti], &v)) return -1; put_word(A->W, v); A->ti++; }
            return 0;
        }
        TypeDecl ty = type_of(A, A->rtype);
        uint64_t v;
        if (parse_dec(t.s, t.n, ~0ull, &v) == 0) {
            put_word(A->W, (uint32_t)v);
            if (ty.width == 64 || v > 0xffffffffull) put_word(A->W, (uint32_t)(v >> 32));
        } else {
            if (!is_float_literal(t)) return -1;
            char *b = (char *)malloc(t.n + 1);
            memcpy(b, t.s, t.n); b[t.n] = 0;
            double d = strtod(b, NULL);
            free(b);
            if (ty.width == 64) { uint64_t u; memcpy(&u, &d, 8); put_word(A->W, (uint32_t)u); put_word(A->W, (uint32_t)(u >> 32)); }
            else { float f = (float)d; uint32_t u; memcpy(&u, &f, 4); put_word(A->W, u); }
        }
        A->ti++;
        return 0;
    }
    if (len > 2 && (tok[0] == 'E' || tok[0] == 'B') && tok[1] == ':') {
        const EnumKind *k = find_kind(tok + 2, len - 2);
        uint32_t v;
        if (parse_enum_tok(k, t, &v)) return -1;
        put_word(A->W, v); A->ti++;
        if (!k->is_bits) {
            const Enumerant *e = find_enumerant(k, v);
            return asm_spec(A, (e && e->params) ? e->params : k->unknown_params);
        }
        for (int bit = 0; bit < 32; bit++) {
            if (!(v & (1u << bit))) continue;
            const Enumerant *e = find_enumerant(k, 1u << bit);
            if (e && e->params && e->params[0] && asm_spec(A, e->params)) return -1;
        }
        return 0;
    }
    return -1;
}

static int asm_spec(Asm *A, const char *spec)
{
    const char *s = spec;
    while (*s) {
        while (*s == ' ') s++;
        if (!*s) break;
        const char *b = s;
        while (*s && *s != ' ') s++;
        size_t len = (size_t)(s - b);
        int optional = 0, star = 0;
        if (b[0] == '?') { optional = 1; b++; len--; }
        if (len >= 1 && b[len - 1] == '*') { star = 1; len--; }
        if (star) {
            const char *one = (b[0] == 'L') ? "L" : "I";
            while (A->ti < A->nt) if (asm_one(A, one, 1)) return -1;
            continue;
        }
        if (A->ti >= A->nt) { if (optional) continue; return -1; }
        if (asm_one(A, b, len)) return -1;
    }
    return 0;
}

typedef struct { uint32_t version, generator, bound, schema; int have_bound; } AsmHeader;

/* digits of the given base from s[*i], at least one, value <= max */
static int scan_num(const char *s, size_t n, size_t *i, int base, uint64_t max, uint64_t *v)
{
    size_t b = *i;
    uint64_t a = 0;
    while (*i < n) {
        int d = hexval(s[*i]);
        if (d < 0 || d >= base) break;
        a = a * (uint64_t)base + (uint64_t)d;
        if (a > max) return -1;
        (*i)++;
    }
    if (*i == b) return -1;
    *v = a;
    return 0;
}

static int has_prefix(const char *s, size_t n, const char *p, size_t *i)
{
    size_t k = strlen(p);
    if (n < k || strncmp(s, p, k) != 0) return 0;
    *i = k;
    return 1;
}

static void header_comment(const char *s, size_t n, AsmHeader *H)
{
    size_t i;
    uint64_t a, c;
    if (has_prefix(s, n, "; Version: ", &i)) {
        if (scan_num(s, n, &i, 10, 255, &a) == 0 && i < n && s[i] == '.') {
            i++;
            if (scan_num(s, n, &i, 10, 255, &c) == 0 && i == n) H->version = (uint32_t)((a << 16) | (c << 8));
        }
    } else if (has_prefix(s, n, "; Generator: 0x", &i)) {
        if (scan_num(s, n, &i, 16, 0xffffffffull, &a) == 0 && i == n) H->generator = (uint32_t)a;
    } else if (has_prefix(s, n, "; Bound: ", &i)) {
        if (scan_num(s, n, &i, 10, 0xffffffffull, &a) == 0 && i == n) { H->bound = (uint32_t)a; H->have_bound = 1; }
    } else if (has_prefix(s, n, "; Schema: ", &i)) {
        if (scan_num(s, n, &i, 10, 0xffffffffull, &a) == 0 && i == n) H->schema = (uint32_t)a;
    }
}

/* One instruction line. Returns 0, or -1 when the line does not parse. */
static int asm_line(Asm *A, const char *s, size_t n, Span *toks)
{
    int nt = tokenize(s, n, toks);
    if (nt <= 0) return -1;
    int ti = 0;
    Span rid_tok = {0, 0, 0};
    int has_rid_tok = 0;
    if (nt >= 3 && toks[0].s[0] == '%' && toks[1].n == 1 && toks[1].s[0] == '=') {
        rid_tok = toks[0]; has_rid_tok = 1; ti = 2;
    }
    Span nm = toks[ti++];
    Words *W = A->W;
    int64_t start = W->n;
    put_word(W, 0);
    const OpInfo *oi = find_op_name(nm.s, nm.n);
    uint32_t opn;
    if (oi) opn = oi->op;
    else {
        uint64_t v;
        if (nm.n < 3 || strncmp(nm.s, "Op", 2) != 0 || parse_dec(nm.s + 2, nm.n - 2, 0xffff, &v)) return -1;
        opn = (uint32_t)v;
    }
    if (!oi || (ti < nt && is_raw_word(toks[ti]))) {
        if (has_rid_tok) return -1;
        for (; ti < nt; ti++) {
            if (!is_raw_word(toks[ti])) return -1;
            uint32_t v = 0;
            for (int k = 2; k < 10; k++) v = (v << 4) | (uint32_t)hexval(toks[ti].s[k]);
            put_word(W, v);
        }
    } else {
        A->tk = toks; A->nt = nt; A->ti = ti; A->rtype = 0;
        /* ids resolve in text order: the result id comes first */
        uint32_t rid = 0;
        if (has_rid_tok && asm_id(A, rid_tok, &rid)) return -1;
        if (oi->rtype) {
            uint32_t ty;
            if (A->ti >= nt || asm_id(A, toks[A->ti], &ty)) return -1;
            put_word(W, ty); A->rtype = ty; A->ti++;
        }
        if (oi->rid) { if (!has_rid_tok) return -1; put_word(W, rid); }
        else if (has_rid_tok) return -1;
        if (asm_spec(A, oi->operands)) return -1;
        if (A->ti != nt) return -1;
        if (A->pass == 1 && (oi->op == 21 || oi->op == 22)) {
            /* a type declaration: the first one of each id counts */
            int seen = 0;
            for (int i = 0; i < A->ntypes; i++) seen |= A->types[i].id == rid;
            uint32_t width;
            if (!seen && parse_u32(toks[A->nt - (oi->op == 21 ? 2 : 1)], &width) == 0) {
                if (A->ntypes == A->captypes) {
                    A->captypes = A->captypes ? 2 * A->captypes : 16;
                    A->types = (TypeDecl *)realloc(A->types, sizeof(TypeDecl) * A->captypes);
                }
                TypeDecl d = {rid, (uint8_t)(oi->op == 22), (uint8_t)(width == 64 ? 64 : 32)};
                A->types[A->ntypes++] = d;
            }
        }
    }
    if (W->n - start > 65535) return -1;
    if (start < W->cap) W->out[start] = ((uint32_t)(W->n - start) << 16) | opn;
    return 0;
}

/* Assemble text into out[] (cap words). Returns the number of words (which
 * may exceed cap: call again with a larger buffer), or -(line number) of the
 * first line that does not parse. */
int64_t orc_assemble(const char *text, int64_t len, uint32_t *out, int64_t cap)
{
    Words W = {out, 0, cap};
    uint32_t scratch;
    Words W0 = {&scratch, 0, 0};
    AsmHeader H = {0x00010200u, 0, 0, 0, 0};
    Span *toks = (Span *)malloc(sizeof(Span) * (size_t)(len / 2 + 2));
    Asm A;
    memset(&A, 0, sizeof A);
    int64_t result = 0;
    /* pass 0 registers the named ids in order of first appearance and finds
     * the largest explicit id; pass 1, with every id now final, records the
     * first type declaration of each id; pass 2 writes the words */
    for (int pass = 0; pass < 3 && result == 0; pass++) {
        A.pass = pass;
        W0.n = 0;
        A.W = pass == 2 ? &W : &W0;
        if (pass == 2) for (int i = 0; i < 5; i++) put_word(&W, 0);
        int64_t i = 0, line = 0;
        while (i < len) {
            int64_t b = i;
            while (i < len && text[i] != '\n') i++;
            const char *s = text + b;
            size_t n = (size_t)(i - b);
            i++; line++;
            if (n == 0) continue;
            if (s[0] == ';') {
                if (pass == 2) header_comment(s, n, &H);
                continue;
            }
            if (asm_line(&A, s, n, toks)) { result = -line; break; }
        }
    }
    if (result == 0) {
        result = W.n;
        if (5 <= W.cap) {
            out[0] = ORC_MAGIC; out[1] = H.version; out[2] = H.generator;
            out[3] = H.have_bound ? H.bound : (uint32_t)(A.max_id + 1);
            out[4] = H.schema;
        }
    }
    free(toks); free(A.names.names); free(A.names.slot); free(A.types);
    return result;
}

/* ------------------------------------------------------------------ */
/* Build modules from op lists, section 3.4.2 ("Enabling Function      */
/* Composition"): instructions are added in order and every one that   */
/* has a result takes a new id from the module, which alone hands ids  */
/* out (getNextId). Here a module is a list of rows: an opcode and its */
/* operands without the result id; an operand is a literal word or a   */
/* reference to another row of the module (its result id). The ids are */
/* handed out in row order: 1, 2, ... to the rows whose opcode has a   */
/* result id. For an opcode with a result type, the first operand is   */
/* the result type and the result id follows it. Checks, first bad row */
/* of the module, in this order within a row: an opcode with a result  */
/* type but no operand, or an instruction over 65535 words (BAD_ROW);  */
/* a reference outside the module or to a row without a result id      */
/* (BAD_REF). A module with a bad row has no words.                    */
/* ------------------------------------------------------------------ */
enum { BUILD_OK = 0, BUILD_BAD_REF = 1, BUILD_BAD_ROW = 2 };

int64_t orc_build(const uint16_t *op, const int64_t *opd_off, const uint32_t *opd, const uint8_t *opd_ref,
                  const int64_t *row_off, int32_t n_mod, uint32_t version, uint32_t generator,
                  uint32_t *out, int64_t cap, int64_t *word_off, uint32_t *status, int64_t *err_row, uint32_t *ids)
{
    int64_t n = 0;
    for (int32_t m = 0; m < n_mod; m++) {
        const int64_t r0 = row_off[m], r1 = row_off[m + 1];
        word_off[m] = n;
        /* getNextId, once per row with a result, in row order */
        uint32_t next = 1;
        for (int64_t r = r0; r < r1; r++) {
            const OpInfo *oi = find_op(op[r]);
            ids[r] = (oi && oi->rid) ? next++ : 0;
        }
        /* checks */
        uint32_t st = BUILD_OK;
        int64_t bad = -1;
        for (int64_t r = r0; r < r1 && st == BUILD_OK; r++) {
            const OpInfo *oi = find_op(op[r]);
            const int64_t nopd = opd_off[r + 1] - opd_off[r];
            if ((oi && oi->rtype && nopd == 0) || 1 + nopd + ((oi && oi->rid) ? 1 : 0) > 65535) {
                st = BUILD_BAD_ROW; bad = r - r0; break;
            }
            for (int64_t k = opd_off[r]; k < opd_off[r + 1]; k++) {
                if (!opd_ref[k]) continue;
                if ((int64_t)opd[k] >= r1 - r0 || ids[r0 + opd[k]] == 0) { st = BUILD_BAD_REF; bad = r - r0; break; }
            }
        }
        status[m] = st;
        err_row[m] = bad;
        if (st != BUILD_OK) continue;
        /* the words: header, then each row */
        const uint32_t head[5] = {ORC_MAGIC, version, generator, next, 0};
        for (int i = 0; i < 5; i++) { if (n < cap) out[n] = head[i]; n++; }
        for (int64_t r = r0; r < r1; r++) {
            const OpInfo *oi = find_op(op[r]);
            const int rt = oi && oi->rtype, rid = oi && oi->rid;
            const int64_t nopd = opd_off[r + 1] - opd_off[r];
            const uint32_t wc = (uint32_t)(1 + nopd + (rid ? 1 : 0));
            if (n < cap) out[n] = (wc << 16) | op[r];
            n++;
            for (int64_t j = 0; j <= nopd; j++) {
                /* the result id goes after the result type, or first */
                if (rid && j == (rt ? 1 : 0)) { if (n < cap) out[n] = ids[r]; n++; }
                if (j == nopd) break;
                const int64_t k = opd_off[r] + j;
                const uint32_t v = opd_ref[k] ? ids[r0 + opd[k]] : opd[k];
                if (n < cap) out[n] = v;
                n++;
            }
        }
    }
    word_off[n_mod] = n;
    return n;
}

/* ------------------------------------------------------------------ */
/* Table queries (for the test that cross-checks the two tables).      */
/* ------------------------------------------------------------------ */
int orc_op_info(uint32_t opn, int *has_rtype, int *has_rid, int *cap, const char **name)
{
    const OpInfo *oi = find_op(opn);
    if (!oi) return -1;
    *has_rtype = oi->rtype; *has_rid = oi->rid; *cap = oi->cap; *name = oi->name;
    return 0;
}

int orc_enum_name(const char *kind, uint32_t value, const char **name, int *cap)
{
    const EnumKind *k = find_kind(kind, strlen(kind));
    if (!k) return -1;
    const Enumerant *e = find_enumerant(k, value);
    if (!e) return -1;
    *name = e->name; *cap = e->cap;
    return 0;
}

int orc_num_ops(void) { return NE(OPS); }
uint32_t orc_op_at(int i) { return OPS[i].op; }
