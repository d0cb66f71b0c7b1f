// gemm_tc.h -- host interface of the tcgen05 tile GEMM (gemm_tc.cu).
//
// One launch processes a list of output blocks ("items") of BM x BN.  Each
// item accumulates, in a TMEM FP32 accumulator, the sum over its segments of
// A_seg * B_seg^T, where A_seg (BM x nb) and B_seg (BN x nb) are K-major
// operand blocks fetched by TMA (three BF16 split pieces per operand for the
// FP32 class, one TF32 copy for TF32, one BF16 piece for BF16, one FP8-E4M3
// copy for E4M3, whose per-tile scales the epilogue divides out), then
// applies the epilogue:
//   mode TC_SUB_F32: out32[off + r + c*ldo] -= acc   (trailing tile update)
//   mode TC_ADD_F64: out64[off + r + c*ldo] += acc   (sampling, r/c bounded)
//   mode TC_SUB_CLASS: out[off + r + c*ldo] -= acc in the working format of
//     the item's output class oc: FP32, or BF16 rounded to nearest (the BF16
//     class, and the E4M3 class before its tiles are solved): class-format
//     tile storage
#pragma once
#include <cuda.h>

#include "emu_internal.h"

namespace gemm_tc {

constexpr int BM = 128;   // rows of an output block (TMEM lanes)
constexpr int BN = 256;   // columns of an output block (TMEM columns)
constexpr int BK = 32;    // K per pipeline stage (BF16: 64 bytes, 64B swizzle)
constexpr int STAGES = 3;
constexpr int NPIECE = 3; // split pieces of an FP32-class operand

enum { TC_SUB_F32 = 0, TC_ADD_F64 = 1, TC_SUB_CLASS = 2 };

struct Seg {
  int ax, ay, ay_step;  // TMA coordinates of A piece 0 (x = K offset) and piece stride in rows
  int bx, by, by_step;  // same for B
  int cls;              // EMU_CLASS_FP32 (6 products), EMU_CLASS_TF32 (1, FP32 copies), EMU_CLASS_BF16 (1),
                        // EMU_CLASS_E4M3 (1, FP8 copies)
  int pad;
};

struct Item {
  int seg_begin, seg_end;
  long out_off;
  int rows_valid, cols_valid;  // TC_ADD_F64 only
  int sa, sb;                  // E4M3 items: tiles whose scales multiply A and B (else -1)
  int oc = EMU_CLASS_FP32;     // TC_SUB_CLASS: output class
  int pad2 = 0;
};

// Output arenas of a TC_SUB_CLASS launch (element offsets out_off in each):
// FP32 tiles, BF16 tiles, and the BF16 working tiles of the E4M3 class.
struct Outputs {
  float *f32;
  uint16_t *bf16;
  uint16_t *e8w;
};

// Operand sources of a launch: BF16 pieces (A box 128 x 32, B box 256 x 32,
// 64-byte swizzle), FP8-E4M3 copies (same boxes in bytes, 32-byte swizzle)
// with one power-of-two scale per tile, and TF32 copies (FP32 containers,
// same boxes, 128-byte swizzle).
struct Operands {
  CUtensorMap a16, b16, a8, b8, a32, b32;
  const float *scale8;
};

// 2-D BF16 tensor map over a row-major [rows x inner] array, box
// [box_rows x BK], 64-byte swizzle.
emu_status make_map_bf16(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner,
                         uint64_t rows, uint32_t box_rows);

// 2-D BF16 tensor map over a row-major [rows x inner] array, box
// [box_rows x 64] (128-byte rows), 128-byte swizzle.
emu_status make_map_bf16_sw128(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                               uint32_t box_rows);

// 2-D FP8 tensor map over a row-major [rows x inner] byte array, box
// [box_rows x 32], 32-byte swizzle.
emu_status make_map_e4m3(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner,
                         uint64_t rows, uint32_t box_rows);

// 2-D FP32 tensor map over a row-major [rows x inner] array (TF32 copies),
// box [box_rows x 32], 128-byte swizzle.
emu_status make_map_f32(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner,
                        uint64_t rows, uint32_t box_rows);

emu_status launch(emu_ctx *ctx, const Operands &ops, const Item *d_items, int nitems, const Seg *d_segs,
                  int ksteps, int mode, float *out32, double *out64, int ldo, int max_ctas);
// TC_SUB_CLASS: each item updates its tile in the format of its class.
emu_status launch_class(emu_ctx *ctx, const Operands &ops, const Item *d_items, int nitems, const Seg *d_segs,
                        int ksteps, const Outputs &outs, int ldo, int max_ctas);

}  // namespace gemm_tc
