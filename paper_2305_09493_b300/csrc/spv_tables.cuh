// spv_tables.cuh -- opcode and enumerant tables of the compute subset, built
// at compile time into dense arrays that device code indexes directly.
//
// The paper's library generates one class per instruction and per operand
// kind from the Khronos grammar (sections 3.2.1 and 3.3); here the same facts
// -- which opcodes carry a result type / result id, the operand list with its
// '?' / '*' quantifiers (section 3.2.1, "Parsing Instructions"), the operand
// kinds (Id, ValueEnum, BitEnum, Literal; "Parsing Operand Kinds") and the
// capability each instruction or enumerant requires (section 3.4.5) -- are a
// compact per-opcode operand program. Numbers are those of the public SPIR-V
// 1.2 specification.
#pragma once
#include <stdint.h>

namespace spvt {

// ---- operand program codes ------------------------------------------------
enum : uint8_t {
    A_END = 0,
    A_ID = 1,        // one <id>
    A_LIT = 2,       // one literal word
    A_STR = 3,       // literal string (NUL-terminated, zero-padded words)
    A_CTX = 4,       // context-dependent literal: all remaining words, at least one
    A_IDS = 5,       // <id>* to the end
    A_LITS = 6,      // literal* to the end
    A_IDPAIRS = 7,   // (<id>, <id>)* to the end; remaining words must be even
    A_ENUM = 8,      // + value-enum kind (8 .. 18)
    A_BITS = 24,     // + bit-enum kind (24 .. 27)
    A_OPT = 0x80     // flag: operand may be absent at the end of the instruction
};

// value-enum kinds
enum : uint8_t {
    K_SourceLanguage = 0, K_AddressingModel, K_MemoryModel, K_ExecutionModel, K_ExecutionMode,
    K_Capability, K_StorageClass, K_Decoration, K_BuiltIn, K_FuncParamAttr, K_LinkageType,
    NUM_VKINDS
};
// bit-enum kinds
enum : uint8_t { B_FunctionControl = 0, B_MemoryAccess, B_SelectionControl, B_LoopControl, NUM_BKINDS };

constexpr uint8_t E(uint8_t k) { return (uint8_t)(A_ENUM + k); }
constexpr uint8_t BI(uint8_t k) { return (uint8_t)(A_BITS + k); }
constexpr uint8_t OPT(uint8_t c) { return (uint8_t)(c | A_OPT); }

// capability numbers used by requirement rules
enum : int8_t {
    C_NONE = -1, C_Matrix = 0, C_Shader = 1, C_Geometry = 2, C_Tessellation = 3, C_Addresses = 4,
    C_Linkage = 5, C_Kernel = 6, C_Float16 = 9, C_Float64 = 10, C_Int64 = 11, C_AtomicStorage = 21,
    C_Int16 = 22, C_SampleRateShading = 35, C_GenericPointer = 38, C_Int8 = 39, C_InputAttachment = 40,
    C_TransformFeedback = 53, C_GeometryStreams = 54
};

// ---- sparse source lists ------------------------------------------------------
struct OpSrc { uint16_t op; const char *name; uint8_t rt, rid; int8_t cap; uint8_t p[5]; };
struct EnSrc { uint32_t v; const char *name; int8_t cap; uint8_t p[3]; };

constexpr uint8_t I = A_ID, L = A_LIT, S = A_STR;

constexpr OpSrc OP_LIST[] = {
    {0, "OpNop", 0, 0, C_NONE, {}},
    {1, "OpUndef", 1, 1, C_NONE, {}},
    {3, "OpSource", 0, 0, C_NONE, {E(K_SourceLanguage), L, OPT(I), OPT(S)}},
    {5, "OpName", 0, 0, C_NONE, {I, S}},
    {6, "OpMemberName", 0, 0, C_NONE, {I, L, S}},
    {7, "OpString", 0, 1, C_NONE, {S}},
    {10, "OpExtension", 0, 0, C_NONE, {S}},
    {11, "OpExtInstImport", 0, 1, C_NONE, {S}},
    {12, "OpExtInst", 1, 1, C_NONE, {I, L, A_IDS}},
    {14, "OpMemoryModel", 0, 0, C_NONE, {E(K_AddressingModel), E(K_MemoryModel)}},
    {15, "OpEntryPoint", 0, 0, C_NONE, {E(K_ExecutionModel), I, S, A_IDS}},
    {16, "OpExecutionMode", 0, 0, C_NONE, {I, E(K_ExecutionMode)}},
    {17, "OpCapability", 0, 0, C_NONE, {E(K_Capability)}},
    {19, "OpTypeVoid", 0, 1, C_NONE, {}},
    {20, "OpTypeBool", 0, 1, C_NONE, {}},
    {21, "OpTypeInt", 0, 1, C_NONE, {L, L}},
    {22, "OpTypeFloat", 0, 1, C_NONE, {L}},
    {23, "OpTypeVector", 0, 1, C_NONE, {I, L}},
    {28, "OpTypeArray", 0, 1, C_NONE, {I, I}},
    {30, "OpTypeStruct", 0, 1, C_NONE, {A_IDS}},
    {32, "OpTypePointer", 0, 1, C_NONE, {E(K_StorageClass), I}},
    {33, "OpTypeFunction", 0, 1, C_NONE, {I, A_IDS}},
    {41, "OpConstantTrue", 1, 1, C_NONE, {}},
    {42, "OpConstantFalse", 1, 1, C_NONE, {}},
    {43, "OpConstant", 1, 1, C_NONE, {A_CTX}},
    {44, "OpConstantComposite", 1, 1, C_NONE, {A_IDS}},
    {46, "OpConstantNull", 1, 1, C_NONE, {}},
    {54, "OpFunction", 1, 1, C_NONE, {BI(B_FunctionControl), I}},
    {55, "OpFunctionParameter", 1, 1, C_NONE, {}},
    {56, "OpFunctionEnd", 0, 0, C_NONE, {}},
    {57, "OpFunctionCall", 1, 1, C_NONE, {I, A_IDS}},
    {59, "OpVariable", 1, 1, C_NONE, {E(K_StorageClass), OPT(I)}},
    {61, "OpLoad", 1, 1, C_NONE, {I, OPT(BI(B_MemoryAccess))}},
    {62, "OpStore", 0, 0, C_NONE, {I, I, OPT(BI(B_MemoryAccess))}},
    {65, "OpAccessChain", 1, 1, C_NONE, {I, A_IDS}},
    {66, "OpInBoundsAccessChain", 1, 1, C_NONE, {I, A_IDS}},
    {67, "OpPtrAccessChain", 1, 1, C_Addresses, {I, I, A_IDS}},
    {70, "OpInBoundsPtrAccessChain", 1, 1, C_Addresses, {I, I, A_IDS}},
    {71, "OpDecorate", 0, 0, C_NONE, {I, E(K_Decoration)}},
    {80, "OpCompositeConstruct", 1, 1, C_NONE, {A_IDS}},
    {81, "OpCompositeExtract", 1, 1, C_NONE, {I, A_LITS}},
    {83, "OpCopyObject", 1, 1, C_NONE, {I}},
    {109, "OpConvertFToU", 1, 1, C_NONE, {I}},
    {110, "OpConvertFToS", 1, 1, C_NONE, {I}},
    {111, "OpConvertSToF", 1, 1, C_NONE, {I}},
    {112, "OpConvertUToF", 1, 1, C_NONE, {I}},
    {113, "OpUConvert", 1, 1, C_NONE, {I}},
    {114, "OpSConvert", 1, 1, C_NONE, {I}},
    {115, "OpFConvert", 1, 1, C_NONE, {I}},
    {117, "OpConvertPtrToU", 1, 1, C_Addresses, {I}},
    {120, "OpConvertUToPtr", 1, 1, C_Addresses, {I}},
    {121, "OpPtrCastToGeneric", 1, 1, C_Kernel, {I}},
    {122, "OpGenericCastToPtr", 1, 1, C_Kernel, {I}},
    {124, "OpBitcast", 1, 1, C_NONE, {I}},
    {126, "OpSNegate", 1, 1, C_NONE, {I}},
    {127, "OpFNegate", 1, 1, C_NONE, {I}},
    {128, "OpIAdd", 1, 1, C_NONE, {I, I}},
    {129, "OpFAdd", 1, 1, C_NONE, {I, I}},
    {130, "OpISub", 1, 1, C_NONE, {I, I}},
    {131, "OpFSub", 1, 1, C_NONE, {I, I}},
    {132, "OpIMul", 1, 1, C_NONE, {I, I}},
    {133, "OpFMul", 1, 1, C_NONE, {I, I}},
    {134, "OpUDiv", 1, 1, C_NONE, {I, I}},
    {135, "OpSDiv", 1, 1, C_NONE, {I, I}},
    {136, "OpFDiv", 1, 1, C_NONE, {I, I}},
    {137, "OpUMod", 1, 1, C_NONE, {I, I}},
    {138, "OpSRem", 1, 1, C_NONE, {I, I}},
    {139, "OpSMod", 1, 1, C_NONE, {I, I}},
    {140, "OpFRem", 1, 1, C_NONE, {I, I}},
    {141, "OpFMod", 1, 1, C_NONE, {I, I}},
    {164, "OpLogicalEqual", 1, 1, C_NONE, {I, I}},
    {165, "OpLogicalNotEqual", 1, 1, C_NONE, {I, I}},
    {166, "OpLogicalOr", 1, 1, C_NONE, {I, I}},
    {167, "OpLogicalAnd", 1, 1, C_NONE, {I, I}},
    {168, "OpLogicalNot", 1, 1, C_NONE, {I}},
    {169, "OpSelect", 1, 1, C_NONE, {I, I, I}},
    {170, "OpIEqual", 1, 1, C_NONE, {I, I}},
    {171, "OpINotEqual", 1, 1, C_NONE, {I, I}},
    {172, "OpUGreaterThan", 1, 1, C_NONE, {I, I}},
    {173, "OpSGreaterThan", 1, 1, C_NONE, {I, I}},
    {174, "OpUGreaterThanEqual", 1, 1, C_NONE, {I, I}},
    {175, "OpSGreaterThanEqual", 1, 1, C_NONE, {I, I}},
    {176, "OpULessThan", 1, 1, C_NONE, {I, I}},
    {177, "OpSLessThan", 1, 1, C_NONE, {I, I}},
    {178, "OpULessThanEqual", 1, 1, C_NONE, {I, I}},
    {179, "OpSLessThanEqual", 1, 1, C_NONE, {I, I}},
    {180, "OpFOrdEqual", 1, 1, C_NONE, {I, I}},
    {181, "OpFUnordEqual", 1, 1, C_NONE, {I, I}},
    {182, "OpFOrdNotEqual", 1, 1, C_NONE, {I, I}},
    {183, "OpFUnordNotEqual", 1, 1, C_NONE, {I, I}},
    {184, "OpFOrdLessThan", 1, 1, C_NONE, {I, I}},
    {185, "OpFUnordLessThan", 1, 1, C_NONE, {I, I}},
    {186, "OpFOrdGreaterThan", 1, 1, C_NONE, {I, I}},
    {187, "OpFUnordGreaterThan", 1, 1, C_NONE, {I, I}},
    {188, "OpFOrdLessThanEqual", 1, 1, C_NONE, {I, I}},
    {189, "OpFUnordLessThanEqual", 1, 1, C_NONE, {I, I}},
    {190, "OpFOrdGreaterThanEqual", 1, 1, C_NONE, {I, I}},
    {191, "OpFUnordGreaterThanEqual", 1, 1, C_NONE, {I, I}},
    {194, "OpShiftRightLogical", 1, 1, C_NONE, {I, I}},
    {195, "OpShiftRightArithmetic", 1, 1, C_NONE, {I, I}},
    {196, "OpShiftLeftLogical", 1, 1, C_NONE, {I, I}},
    {197, "OpBitwiseOr", 1, 1, C_NONE, {I, I}},
    {198, "OpBitwiseXor", 1, 1, C_NONE, {I, I}},
    {199, "OpBitwiseAnd", 1, 1, C_NONE, {I, I}},
    {200, "OpNot", 1, 1, C_NONE, {I}},
    {224, "OpControlBarrier", 0, 0, C_NONE, {I, I, I}},
    {225, "OpMemoryBarrier", 0, 0, C_NONE, {I, I}},
    {227, "OpAtomicLoad", 1, 1, C_NONE, {I, I, I}},
    {228, "OpAtomicStore", 0, 0, C_NONE, {I, I, I, I}},
    {229, "OpAtomicExchange", 1, 1, C_NONE, {I, I, I, I}},
    {234, "OpAtomicIAdd", 1, 1, C_NONE, {I, I, I, I}},
    {235, "OpAtomicISub", 1, 1, C_NONE, {I, I, I, I}},
    {245, "OpPhi", 1, 1, C_NONE, {A_IDPAIRS}},
    {246, "OpLoopMerge", 0, 0, C_NONE, {I, I, BI(B_LoopControl)}},
    {247, "OpSelectionMerge", 0, 0, C_NONE, {I, BI(B_SelectionControl)}},
    {248, "OpLabel", 0, 1, C_NONE, {}},
    {249, "OpBranch", 0, 0, C_NONE, {I}},
    {250, "OpBranchConditional", 0, 0, C_NONE, {I, I, I, A_LITS}},
    {253, "OpReturn", 0, 0, C_NONE, {}},
    {254, "OpReturnValue", 0, 0, C_NONE, {I}},
    {255, "OpUnreachable", 0, 0, C_NONE, {}},
};

constexpr EnSrc EN_SourceLanguage[] = {
    {0, "Unknown", C_NONE, {}}, {1, "ESSL", C_NONE, {}}, {2, "GLSL", C_NONE, {}},
    {3, "OpenCL_C", C_NONE, {}}, {4, "OpenCL_CPP", C_NONE, {}}, {5, "HLSL", C_NONE, {}}};
constexpr EnSrc EN_AddressingModel[] = {
    {0, "Logical", C_NONE, {}}, {1, "Physical32", C_Addresses, {}}, {2, "Physical64", C_Addresses, {}}};
constexpr EnSrc EN_MemoryModel[] = {
    {0, "Simple", C_Shader, {}}, {1, "GLSL450", C_Shader, {}}, {2, "OpenCL", C_Kernel, {}}};
constexpr EnSrc EN_ExecutionModel[] = {
    {0, "Vertex", C_Shader, {}}, {1, "TessellationControl", C_Tessellation, {}},
    {2, "TessellationEvaluation", C_Tessellation, {}}, {3, "Geometry", C_Geometry, {}},
    {4, "Fragment", C_Shader, {}}, {5, "GLCompute", C_Shader, {}}, {6, "Kernel", C_Kernel, {}}};
constexpr EnSrc EN_ExecutionMode[] = {
    {17, "LocalSize", C_NONE, {L, L, L}}, {18, "LocalSizeHint", C_Kernel, {L, L, L}},
    {30, "VecTypeHint", C_Kernel, {L}}, {31, "ContractionOff", C_Kernel, {}}};
constexpr EnSrc EN_Capability[] = {
    {0, "Matrix", C_NONE, {}}, {1, "Shader", C_NONE, {}}, {2, "Geometry", C_NONE, {}},
    {3, "Tessellation", C_NONE, {}}, {4, "Addresses", C_NONE, {}}, {5, "Linkage", C_NONE, {}},
    {6, "Kernel", C_NONE, {}}, {7, "Vector16", C_NONE, {}}, {8, "Float16Buffer", C_NONE, {}},
    {9, "Float16", C_NONE, {}}, {10, "Float64", C_NONE, {}}, {11, "Int64", C_NONE, {}},
    {12, "Int64Atomics", C_NONE, {}}, {13, "ImageBasic", C_NONE, {}}, {14, "ImageReadWrite", C_NONE, {}},
    {15, "ImageMipmap", C_NONE, {}}, {17, "Pipes", C_NONE, {}}, {18, "Groups", C_NONE, {}},
    {19, "DeviceEnqueue", C_NONE, {}}, {20, "LiteralSampler", C_NONE, {}},
    {21, "AtomicStorage", C_NONE, {}}, {22, "Int16", C_NONE, {}},
    {23, "TessellationPointSize", C_NONE, {}}, {24, "GeometryPointSize", C_NONE, {}},
    {25, "ImageGatherExtended", C_NONE, {}}, {27, "StorageImageMultisample", C_NONE, {}},
    {28, "UniformBufferArrayDynamicIndexing", C_NONE, {}},
    {29, "SampledImageArrayDynamicIndexing", C_NONE, {}},
    {30, "StorageBufferArrayDynamicIndexing", C_NONE, {}},
    {31, "StorageImageArrayDynamicIndexing", C_NONE, {}}, {32, "ClipDistance", C_NONE, {}},
    {33, "CullDistance", C_NONE, {}}, {34, "ImageCubeArray", C_NONE, {}},
    {35, "SampleRateShading", C_NONE, {}}, {36, "ImageRect", C_NONE, {}},
    {37, "SampledRect", C_NONE, {}}, {38, "GenericPointer", C_NONE, {}}, {39, "Int8", C_NONE, {}},
    {40, "InputAttachment", C_NONE, {}}, {41, "SparseResidency", C_NONE, {}},
    {42, "MinLod", C_NONE, {}}, {43, "Sampled1D", C_NONE, {}}, {44, "Image1D", C_NONE, {}},
    {45, "SampledCubeArray", C_NONE, {}}, {46, "SampledBuffer", C_NONE, {}},
    {47, "ImageBuffer", C_NONE, {}}, {48, "ImageMSArray", C_NONE, {}},
    {49, "StorageImageExtendedFormats", C_NONE, {}}, {50, "ImageQuery", C_NONE, {}},
    {51, "DerivativeControl", C_NONE, {}}, {52, "InterpolationFunction", C_NONE, {}},
    {53, "TransformFeedback", C_NONE, {}}, {54, "GeometryStreams", C_NONE, {}},
    {55, "StorageImageReadWithoutFormat", C_NONE, {}},
    {56, "StorageImageWriteWithoutFormat", C_NONE, {}}, {57, "MultiViewport", C_NONE, {}},
    {58, "SubgroupDispatch", C_NONE, {}}, {59, "NamedBarrier", C_NONE, {}},
    {60, "PipeStorage", C_NONE, {}}};
constexpr EnSrc EN_StorageClass[] = {
    {0, "UniformConstant", C_NONE, {}}, {1, "Input", C_NONE, {}}, {2, "Uniform", C_Shader, {}},
    {3, "Output", C_Shader, {}}, {4, "Workgroup", C_NONE, {}}, {5, "CrossWorkgroup", C_NONE, {}},
    {6, "Private", C_Shader, {}}, {7, "Function", C_NONE, {}}, {8, "Generic", C_GenericPointer, {}},
    {9, "PushConstant", C_Shader, {}}, {10, "AtomicCounter", C_AtomicStorage, {}},
    {11, "Image", C_NONE, {}}};
constexpr uint8_t LT = A_LITS;
constexpr EnSrc EN_Decoration[] = {
    {0, "RelaxedPrecision", C_Shader, {LT}}, {1, "SpecId", C_Shader, {LT}}, {2, "Block", C_Shader, {LT}},
    {3, "BufferBlock", C_Shader, {LT}}, {4, "RowMajor", C_Matrix, {LT}}, {5, "ColMajor", C_Matrix, {LT}},
    {6, "ArrayStride", C_Shader, {LT}}, {7, "MatrixStride", C_Matrix, {LT}},
    {8, "GLSLShared", C_Shader, {LT}}, {9, "GLSLPacked", C_Shader, {LT}}, {10, "CPacked", C_Kernel, {LT}},
    {11, "BuiltIn", C_NONE, {E(K_BuiltIn)}}, {13, "NoPerspective", C_Shader, {LT}},
    {14, "Flat", C_Shader, {LT}}, {15, "Patch", C_Tessellation, {LT}}, {16, "Centroid", C_Shader, {LT}},
    {17, "Sample", C_SampleRateShading, {LT}}, {18, "Invariant", C_Shader, {LT}},
    {19, "Restrict", C_NONE, {LT}}, {20, "Aliased", C_NONE, {LT}}, {21, "Volatile", C_NONE, {LT}},
    {22, "Constant", C_Kernel, {LT}}, {23, "Coherent", C_NONE, {LT}}, {24, "NonWritable", C_NONE, {LT}},
    {25, "NonReadable", C_NONE, {LT}}, {26, "Uniform", C_Shader, {LT}},
    {28, "SaturatedConversion", C_Kernel, {LT}}, {29, "Stream", C_GeometryStreams, {LT}},
    {30, "Location", C_Shader, {LT}}, {31, "Component", C_Shader, {LT}}, {32, "Index", C_Shader, {LT}},
    {33, "Binding", C_Shader, {LT}}, {34, "DescriptorSet", C_Shader, {LT}}, {35, "Offset", C_Shader, {LT}},
    {36, "XfbBuffer", C_TransformFeedback, {LT}}, {37, "XfbStride", C_TransformFeedback, {LT}},
    {38, "FuncParamAttr", C_Kernel, {E(K_FuncParamAttr)}}, {39, "FPRoundingMode", C_Kernel, {LT}},
    {40, "FPFastMathMode", C_Kernel, {LT}}, {41, "LinkageAttributes", C_Linkage, {S, E(K_LinkageType)}},
    {42, "NoContraction", C_Shader, {LT}}, {43, "InputAttachmentIndex", C_InputAttachment, {LT}},
    {44, "Alignment", C_Kernel, {L}}, {45, "MaxByteOffset", C_Addresses, {LT}},
    {46, "AlignmentId", C_Kernel, {I}}, {47, "MaxByteOffsetId", C_Addresses, {I}}};
constexpr EnSrc EN_BuiltIn[] = {
    {24, "NumWorkgroups", C_NONE, {}}, {25, "WorkgroupSize", C_NONE, {}}, {26, "WorkgroupId", C_NONE, {}},
    {27, "LocalInvocationId", C_NONE, {}}, {28, "GlobalInvocationId", C_NONE, {}},
    {29, "LocalInvocationIndex", C_NONE, {}}, {30, "WorkDim", C_Kernel, {}}, {31, "GlobalSize", C_Kernel, {}},
    {32, "EnqueuedWorkgroupSize", C_Kernel, {}}, {33, "GlobalOffset", C_Kernel, {}},
    {34, "GlobalLinearId", C_Kernel, {}}, {36, "SubgroupSize", C_Kernel, {}},
    {37, "SubgroupMaxSize", C_Kernel, {}}, {38, "NumSubgroups", C_Kernel, {}},
    {39, "NumEnqueuedSubgroups", C_Kernel, {}}, {40, "SubgroupId", C_Kernel, {}},
    {41, "SubgroupLocalInvocationId", C_Kernel, {}}};
constexpr EnSrc EN_FuncParamAttr[] = {
    {0, "Zext", C_NONE, {}}, {1, "Sext", C_NONE, {}}, {2, "ByVal", C_NONE, {}}, {3, "Sret", C_NONE, {}},
    {4, "NoAlias", C_NONE, {}}, {5, "NoCapture", C_NONE, {}}, {6, "NoWrite", C_NONE, {}},
    {7, "NoReadWrite", C_NONE, {}}};
constexpr EnSrc EN_LinkageType[] = {{0, "Export", C_NONE, {}}, {1, "Import", C_NONE, {}}};
// bit enums: value = the single bit
constexpr EnSrc BN_FunctionControl[] = {
    {0x1, "Inline", C_NONE, {}}, {0x2, "DontInline", C_NONE, {}}, {0x4, "Pure", C_NONE, {}},
    {0x8, "Const", C_NONE, {}}};
constexpr EnSrc BN_MemoryAccess[] = {
    {0x1, "Volatile", C_NONE, {}}, {0x2, "Aligned", C_NONE, {L}}, {0x4, "Nontemporal", C_NONE, {}}};
constexpr EnSrc BN_SelectionControl[] = {{0x1, "Flatten", C_NONE, {}}, {0x2, "DontFlatten", C_NONE, {}}};
constexpr EnSrc BN_LoopControl[] = {
    {0x1, "Unroll", C_NONE, {}}, {0x2, "DontUnroll", C_NONE, {}}, {0x4, "DependencyInfinite", C_NONE, {}},
    {0x8, "DependencyLength", C_NONE, {L}}};

// capability dependencies: declaring .a implicitly declares .b (section 3.4.5)
struct CapDep { uint8_t a, b; };
constexpr CapDep CAP_DEPS[] = {
    {1, 0}, {2, 1}, {3, 1}, {7, 6}, {8, 6}, {12, 11}, {13, 6}, {14, 13}, {15, 13}, {17, 6}, {19, 6},
    {20, 6}, {21, 1}, {23, 3}, {24, 2}, {25, 1}, {27, 1}, {28, 1}, {29, 1}, {30, 1}, {31, 1}, {32, 1},
    {33, 1}, {34, 45}, {35, 1}, {36, 37}, {37, 1}, {38, 4}, {40, 1}, {41, 1}, {42, 1}, {44, 43},
    {45, 1}, {47, 46}, {48, 1}, {49, 1}, {50, 1}, {51, 1}, {52, 1}, {53, 1}, {54, 2}, {55, 1}, {56, 1},
    {57, 2}, {58, 19}, {59, 6}, {60, 17}};

// ---- dense compiled tables ----------------------------------------------------
struct OpDesc {            // 16 bytes
    uint8_t flags;         // bit0 known, bit1 has result type, bit2 has result id, bit3 counted by validation
    int8_t cap;            // required capability or -1
    uint8_t nprog;
    uint8_t prog[5];
    uint16_t name_off;
    uint8_t name_len;
    // fast form, for operand lists made only of fixed ids / literals and an
    // optional tail: bit0 set when it applies, bits 1-3 the tail (0 none,
    // 1 ids, 2 literals, 3 id pairs, 4 one bit-enum word with its literal
    // parameters), bit4 set when that bit-enum word may be absent
    uint8_t fast;
    uint16_t id_mask;      // bit i: word i (1 <= i <= nfixed) is an id
    uint8_t nfixed;        // words after the first word before the tail
    uint8_t bkind;         // bit-enum kind of tail 4
};
struct EnDesc {            // 8 bytes
    uint8_t known;
    int8_t cap;
    uint8_t nparam;
    uint8_t param[3];
    uint8_t name_len;
    uint8_t name_hi;       // name offset = name_hi << 8 | name_lo
    uint8_t name_lo;
};

constexpr int NAME_POOL = 6144;
struct Tables {
    OpDesc ops[256];
    EnDesc venum[NUM_VKINDS][64];   // value enums, by value (< 64)
    EnDesc benum[NUM_BKINDS][32];   // bit enums, by bit index
    uint8_t vunknown[NUM_VKINDS];   // operand code used for the parameters of an unknown value (A_END: none)
    uint64_t cap_dep[64];           // bit b set in cap_dep[a]: declaring a declares b
    uint8_t shape[256];             // text shape class: opcodes with the same operand list share one (1 = unknown)
    uint8_t layout[256];            // layout class (low 4 bits, spv_layout_class) and module section (high 4 bits)
    char names[NAME_POOL];
    int name_used;
};

constexpr int cstrlen(const char *s) { int n = 0; while (s[n]) n++; return n; }

template <int N>
constexpr void fill_enum(Tables &t, EnDesc *dst, const EnSrc (&src)[N], bool bits)
{
    for (int i = 0; i < N; i++) {
        int idx = 0;
        if (bits) { while (!(src[i].v & (1u << idx))) idx++; }
        else idx = (int)src[i].v;
        EnDesc &d = dst[idx];
        d.known = 1;
        d.cap = src[i].cap;
        int np = 0;
        for (int k = 0; k < 3; k++) if (src[i].p[k]) { d.param[np++] = src[i].p[k]; }
        d.nparam = (uint8_t)np;
        int len = cstrlen(src[i].name);
        int off = t.name_used;
        for (int k = 0; k < len; k++) t.names[off + k] = src[i].name[k];
        t.name_used += len;
        d.name_len = (uint8_t)len;
        d.name_hi = (uint8_t)(off >> 8);
        d.name_lo = (uint8_t)(off & 0xff);
    }
}

// Layout classes of the opcodes that are not plain body instructions
// (section 3.4.1 scopes; sections in the SPIR-V specification's module
// order): {opcode, class, section}. Every other opcode of the table is a
// body instruction; opcodes outside the table are neutral.
struct LayoutSrc { uint16_t op; uint8_t cls, sec; };
enum : uint8_t { LCL_ANY = 0, LCL_SECTION = 1, LCL_MIXED = 2, LCL_FUNCTION = 3, LCL_PARAM = 4, LCL_FUNCEND = 5,
                 LCL_LABEL = 6, LCL_TERM = 7, LCL_BODY = 8 };
constexpr LayoutSrc LAYOUT_LIST[] = {
    {0, LCL_ANY, 0},                                                        // OpNop
    {17, LCL_SECTION, 1},                                                   // capabilities
    {10, LCL_SECTION, 2},                                                   // extensions
    {11, LCL_SECTION, 3},                                                   // extended-instruction imports
    {14, LCL_SECTION, 4},                                                   // memory model
    {15, LCL_SECTION, 5},                                                   // entry points
    {16, LCL_SECTION, 6},                                                   // execution modes
    {3, LCL_SECTION, 7}, {5, LCL_SECTION, 7}, {6, LCL_SECTION, 7}, {7, LCL_SECTION, 7},   // debug
    {71, LCL_SECTION, 8},                                                   // decorations
    {19, LCL_SECTION, 9}, {20, LCL_SECTION, 9}, {21, LCL_SECTION, 9}, {22, LCL_SECTION, 9},
    {23, LCL_SECTION, 9}, {28, LCL_SECTION, 9}, {30, LCL_SECTION, 9}, {32, LCL_SECTION, 9},
    {33, LCL_SECTION, 9},                                                   // types
    {41, LCL_SECTION, 9}, {42, LCL_SECTION, 9}, {43, LCL_SECTION, 9}, {44, LCL_SECTION, 9},
    {46, LCL_SECTION, 9},                                                   // constants
    {1, LCL_MIXED, 9}, {59, LCL_MIXED, 9},                                  // OpUndef, OpVariable
    {54, LCL_FUNCTION, 10}, {55, LCL_PARAM, 0}, {56, LCL_FUNCEND, 0},
    {248, LCL_LABEL, 0},
    {249, LCL_TERM, 0}, {250, LCL_TERM, 0}, {253, LCL_TERM, 0}, {254, LCL_TERM, 0}, {255, LCL_TERM, 0},
};

constexpr Tables build_tables()
{
    Tables t{};
    for (const OpSrc &o : OP_LIST) {
        OpDesc &d = t.ops[o.op];
        // bit 3: validation counts the instruction (capability, memory model,
        // entry point, function) or reads its width (integer and float types)
        const bool counted = o.op == 14 || o.op == 15 || o.op == 17 || o.op == 21 || o.op == 22 || o.op == 54;
        d.flags = (uint8_t)(1 | (o.rt ? 2 : 0) | (o.rid ? 4 : 0) | (counted ? 8 : 0));
        d.cap = o.cap;
        int np = 0;
        for (int k = 0; k < 5; k++) if (o.p[k]) d.prog[np++] = o.p[k];
        d.nprog = (uint8_t)np;
        // fast form
        {
            bool fast = true, opt = false;
            int nfixed = 0, tail = 0;
            uint8_t bkind = 0;
            uint16_t mask = 0;
            if (o.rt) { nfixed++; mask |= (uint16_t)(1u << nfixed); }
            if (o.rid) { nfixed++; mask |= (uint16_t)(1u << nfixed); }
            for (int k = 0; k < np; k++) {
                uint8_t c = d.prog[k];
                if (tail) { fast = false; break; }
                const uint8_t cb = (uint8_t)(c & 0x7f);
                if (c == A_ID) { nfixed++; mask |= (uint16_t)(1u << nfixed); }
                else if (c == A_LIT) { nfixed++; }
                else if (c == A_IDS) tail = 1;
                else if (c == A_LITS) tail = 2;
                else if (c == A_CTX) { nfixed++; tail = 2; }     // one literal word or more
                else if (c == A_IDPAIRS) tail = 3;
                else if (cb >= A_BITS && cb < A_BITS + NUM_BKINDS) {
                    tail = 4; opt = (c & A_OPT) != 0; bkind = (uint8_t)(cb - A_BITS);
                }
                else { fast = false; break; }
            }
            if (nfixed > 15) fast = false;
            d.fast = fast ? (uint8_t)(1 | (tail << 1) | (opt ? 16 : 0)) : 0;
            d.id_mask = fast ? mask : 0;
            d.nfixed = fast ? (uint8_t)nfixed : 0;
            d.bkind = fast ? bkind : 0;
        }
        t.layout[o.op] = LCL_BODY;
        int len = cstrlen(o.name);
        d.name_off = (uint16_t)t.name_used;
        d.name_len = (uint8_t)len;
        for (int k = 0; k < len; k++) t.names[t.name_used + k] = o.name[k];
        t.name_used += len;
    }
    fill_enum(t, t.venum[K_SourceLanguage], EN_SourceLanguage, false);
    fill_enum(t, t.venum[K_AddressingModel], EN_AddressingModel, false);
    fill_enum(t, t.venum[K_MemoryModel], EN_MemoryModel, false);
    fill_enum(t, t.venum[K_ExecutionModel], EN_ExecutionModel, false);
    fill_enum(t, t.venum[K_ExecutionMode], EN_ExecutionMode, false);
    fill_enum(t, t.venum[K_Capability], EN_Capability, false);
    fill_enum(t, t.venum[K_StorageClass], EN_StorageClass, false);
    fill_enum(t, t.venum[K_Decoration], EN_Decoration, false);
    fill_enum(t, t.venum[K_BuiltIn], EN_BuiltIn, false);
    fill_enum(t, t.venum[K_FuncParamAttr], EN_FuncParamAttr, false);
    fill_enum(t, t.venum[K_LinkageType], EN_LinkageType, false);
    fill_enum(t, t.benum[B_FunctionControl], BN_FunctionControl, true);
    fill_enum(t, t.benum[B_MemoryAccess], BN_MemoryAccess, true);
    fill_enum(t, t.benum[B_SelectionControl], BN_SelectionControl, true);
    fill_enum(t, t.benum[B_LoopControl], BN_LoopControl, true);
    t.vunknown[K_ExecutionMode] = A_LITS;
    t.vunknown[K_Decoration] = A_LITS;
    for (const CapDep &c : CAP_DEPS) t.cap_dep[c.a] |= 1ull << c.b;
    // shape classes: 0 is kept for module header lines, 1 for unknown opcodes
    int next_shape = 2;
    for (int o = 0; o < 256; o++) {
        t.shape[o] = 1;
        const OpDesc &d = t.ops[o];
        if (!(d.flags & 1)) continue;
        int found = -1;
        for (int q = 0; q < o && found < 0; q++) {
            const OpDesc &e = t.ops[q];
            if (!(e.flags & 1) || e.flags != d.flags || e.nprog != d.nprog) continue;
            bool same = true;
            for (int k = 0; k < d.nprog; k++) if (e.prog[k] != d.prog[k]) same = false;
            if (same) found = t.shape[q];
        }
        t.shape[o] = (uint8_t)(found >= 0 ? found : next_shape++);
    }
    for (const LayoutSrc &l : LAYOUT_LIST) t.layout[l.op] = (uint8_t)(l.cls | (l.sec << 4));
    return t;
}

}  // namespace spvt

// One copy for the host (queries) and one in device global memory, both
// initialised at compile time.
constexpr spvt::Tables SPV_TABLES_HOST = spvt::build_tables();
static __device__ const spvt::Tables g_spv_tables = spvt::build_tables();
