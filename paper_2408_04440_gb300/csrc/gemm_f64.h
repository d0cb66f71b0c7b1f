// gemm_f64.h -- FP64-accurate tile update C -= A B^T on the BF16 tensor cores
// (gemm_f64.cu), for the FP64-class tiles of the mixed-precision factor.
//
// Ozaki scheme (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 2012), in fixed point: every row r of
// an operand tile is scaled by a power of two 2^-e_r so that its entries lie
// in (-1, 1), then written as NS digits of SLICE_BITS bits each,
//   x 2^-e_r = sum_p s_p 2^-(SLICE_BITS (p + 1)),   s_p integers, |s_p| <= 2^SLICE_BITS,
// every digit exact in BF16.  A product of two digits is an integer below
// 2^14; the sum of the (g + 1) products with p + q = g over K <= KCHUNK terms
// stays below 2^24, so the tensor cores accumulate each diagonal group g
// exactly in FP32.  The epilogue adds the groups, scaled by 2^-7(g+2), in
// FP64 (smallest first) every KCHUNK, and applies the row scales at the end.
// NS = 8 digits carry 57 bits, so the products with p + q < NS give the dot
// products to FP64 accuracy relative to the rows' largest entries.
#pragma once
#include <cuda.h>

#include "emu_internal.h"

namespace gemm64 {

constexpr int BM = 128;        // output rows of an item (TMEM lanes)
constexpr int BN = 64;         // output columns of an item; 8 groups x 64 = 512 TMEM columns
constexpr int BK = 32;         // K per pipeline stage
constexpr int STAGES = 2;
constexpr int NS = 8;          // digits per operand entry
constexpr int SLICE_BITS = 7;
constexpr int KCHUNK = 256;    // K accumulated exactly in FP32 between FP64 flushes

// One BM x BN output block.  The digit arena holds, per slot, NS digit
// planes of nb x nb (row-major: row r, K index c), plane p of slot s at rows
// (s * NS + p) * nb; `scales` holds 2^e_r for each row of each slot.
struct Item {
  long out_off;  // element offset of the block in the FP64 output
  int a_row;     // arena row of digit plane 0 of the A block (its first row)
  int b_row;     // same for the B block
  int a_sc;      // index in `scales` of the A block's first row
  int b_sc;      // same for the B block
  int pad[2];
};

// 2-D BF16 tensor map over the digit arena (inner = nb), box rows x 32.
emu_status make_map(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                    uint32_t box_rows);

// Digits and row scales of the listed tiles: jobs {tile, slot}; a tile is read
// from the FP64 arena when its class is FP64, else from the FP32 master.
emu_status launch_slice(emu_ctx *ctx, const double *t64, const float *t32, const unsigned char *cls,
                        const int2 *d_jobs, int njobs, int nb, uint16_t *digits, double *scales);

// out64[item block] -= A B^T for every item (K = nb, ldo = leading dimension
// of the output), on at most max_ctas persistent CTAs.
emu_status launch(emu_ctx *ctx, const CUtensorMap &a, const CUtensorMap &b, const Item *d_items, int nitems, int nb,
                  const double *scales, double *out64, int ldo, int max_ctas);

}  // namespace gemm64
