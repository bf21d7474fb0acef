// plan.h -- contraction-list parser and TTGT planner (host only).
//
// A statement of the list is one "Contraction" of arxiv 2409.06759 Sec. II C:
// a scalar factor, optional permutation operators on the output, at most two
// tensors (the binary-contraction constraint of Fig. algo:remove) and an
// output tensor.  The planner turns each statement into steps:
//   permutes of the operands into GEMM-ready layout (TTGT, Sec. I C),
//   one GEMM, and an antisymmetrising epilogue when P(..) operators are present.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.h"

namespace ccb {

enum class TKind { AMP, RES, INTEGRAL, INTERM };

struct Tensor {
    std::string name;
    TKind kind;
    std::vector<char> spaces;   // 'o' / 'v' per storage dim
    std::vector<int64_t> ext;
    std::vector<int64_t> str;   // element strides (row-major)
    int64_t elems = 0;
    int slot = 0;               // AMP/RES: rank/2 (1..3); INTEGRAL: block 0..5, 6 = packed vvvv
    int64_t ws_off = -1;        // INTERM: byte offset of its buffer in the workspace
    bool static_data = false;   // INTERM filled once per solve from integrals (packed blocks)
};

// Memory a step reads or writes, resolved at run time.
struct BufRef {
    enum Where { NONE, AMP, RES, INTEG, WS } where = NONE;
    int slot = 0;               // WS: 1 while the offset is relative to the scratch arena
    int64_t off = 0;            // WS: byte offset
};

// A tensor reference inside a statement, as a strided view.
struct View {
    int tensor = -1;
    std::vector<int> idx;       // letter id per storage dim of the tensor
    std::vector<int64_t> ext, str;
    double sign = 1.0;
    bool conj = false;
};

enum class StepKind { ZERO, ACCUM, GEMM, PACK, UNPACK };

// One contraction of a K-concatenated step: several statements that
// accumulate into the same output with the same split of its indices between
// their operands run as one pass over the output.  On the split route each
// member's operands fill its own K columns of the shared planes (its factor
// rides on the A split); on the narrow kernel a and b are its X and Y.  A
// member may stand for several statements whose shared operand multiplies the
// sum of their other operands.
struct KMember {
    int stmt = -1;
    BufRef a, b;
    SplitDesc split_a{}, split_b{};
    double flops = 0.0;
};

struct Step {
    StepKind kind;
    int stmt = -1;              // statement index (0-based)
    BufRef out, a, b;           // ACCUM: out, src=a; GEMM: C=out, A=a, B=b; ZERO: out
    BufRef c;                   // ACCUM with acc.has_add: the fused copy's source
    int64_t zero_elems = 0;
    AccumDesc acc{};
    GemmF64Desc gemm{};
    // split-bf16 tensor-core route of a GEMM
    bool mixed = false;
    SplitDesc split_a{}, split_b{};
    TcGemmDesc tc{};
    int64_t planes_a_off = 0, planes_b_off = 0;  // workspace byte offsets of the planes
    BufRef partials;                             // split-K partial sums (when splitk > 1)
    bool a_static = false, b_static = false;     // operand is an integral block (cacheable)
    bool static_src = false;                     // ACCUM permute of an integral block into the cache
    bool skip_a = false, skip_b = false;         // planes already split by an earlier step (same source version)
    std::vector<std::array<int, 3>> cands;       // autotuning candidates (tile width or 0, split-K, red epilogue)
    PackDesc pk{};                               // PACK: out = packed pairs of a
    UnpackDesc up{};                             // UNPACK: out (antisymmetric) from packed a
    bool rows = false;                           // narrow GEMM (one thread per row, operands in place)
    RowsGemmDesc rg{};
    bool nk = false;                             // long contraction, <= 8 columns, operands in place
    NarrowKDesc nkd{};
    std::vector<KMember> kcat;                   // K-concatenated members (a, b, split_a/b unused)
    std::vector<int> kstmts;                     // the statements a K-concatenated step carries
    RowsMultiDesc rm{};                          // K-concatenated on the narrow kernel (rows = true)
    double flops = 0.0;
    std::string note;
};

struct Plan {
    int o = 0, v = 0;
    int dtype = 0, precision = 0;
    std::vector<Tensor> tensors;
    std::vector<Step> steps;
    std::vector<std::string> stmt_text;
    bool res_used[4] = {false, false, false, false};
    bool amp_used[4] = {false, false, false, false};
    int64_t ws_bytes = 0;       // total workspace
    int64_t flags_off = 0;      // device status word of bounded waits (first 256 bytes)
    int64_t interm_bytes = 0;
    int64_t scratch_off = 0, scratch_bytes = 0;
    int64_t cache_off = 0, cache_bytes = 0;   // static split planes
    int64_t splits_off = 0, splits_bytes = 0; // per-iteration split planes shared between steps
    double flops = 0.0;
    double flops_mixed = 0.0;   // flops of steps on the split-bf16 route (fp64-equivalent)
    bool tuned = false;         // GEMM configurations picked by cc_plan_autotune
    bool packed_vvvv = false;   // packed <ab||ef> is an input (integral slot 6)
    bool integ_used[7] = {false, false, false, false, false, false, false};   // blocks some step reads
    int verbose = 0;
};

// Parses and plans; on failure returns false and sets err (with line number).
// precision >= 100 is a test hook: precision - 100, every GEMM on the split route.
// flags bit 0: packed <ab||ef> read from the vvvv_packed input (slot 6).
bool build_plan(const std::string &text, int o, int v, int dtype, int precision, Plan &plan,
                std::string &err, int flags = 0);

std::string describe_plan(const Plan &plan);

// Extents of the six canonical integral blocks (oooo, ooov, oovv, ovov, ovvv, vvvv).
void integral_block_dims(int o, int v, int block, int64_t ext[4]);

}  // namespace ccb
