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
// exactly in FP32.  Every KCHUNK the epilogue folds the groups, scaled by
// 2^-7(g+2), in integer arithmetic and adds them in FP64; it applies the row
// scales at the end.
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

// One BM x BN output block: the sum over its segments of A_seg B_seg^T.
// Operand row r of digit plane p sits at arena row (row + p * plane); every
// entry of a row carries the scale 2^e of that row, read from an exponent
// array (A: a_exp[a_sc + r], B: b_exp[b_sc + c]), so all segments of an item
// share one scale per row and their digit products add exactly.
struct Seg {
  int a_row, b_row;  // arena rows of digit plane 0 of the A and B blocks
  int a_x, b_x;      // K offset of the segment in each arena
};
struct Item {
  long out_off;                // element offset of the block in the FP64 output
  int a_sc, b_sc;              // exponent indices of the block's first A row / B row
  int seg_begin, seg_end;      // segments [seg_begin, seg_end)
  int rows_valid, cols_valid;  // rows / columns of the block that exist (TC64_ADD)
};
enum { TC64_SUB = 0, TC64_ADD = 1 };  // out -= A B^T (factor) / out += A B^T (samples, bounded)

// 2-D BF16 tensor map over a digit arena of `inner` columns, box rows x 32.
emu_status make_map(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                    uint32_t box_rows);

// Exponent arrays hold e + kExpBias, so that a zeroed array (cudaMemset 0)
// holds the lowest exponent; readers clamp e at kExpMin, which only rows of
// zeros reach.
constexpr int kExpBias = 1024;
constexpr int kExpMin = -960;

// Row exponents of listed tiles: jobs {tile, -, exponent base}; a tile is read
// from the FP64 arena when its class is FP64, else from the FP32 master.  Row
// r gets exp[base + r] = max(exp[base + r], e) with max_c |x_rc| < 2^e, so
// tiles that share rows share the largest exponent.
emu_status launch_row_exponents(emu_ctx *ctx, const double *t64, const float *t32, const unsigned char *cls,
                                const int4 *d_jobs, int njobs, int nb, int *exps);
// Digit planes of listed tiles: jobs {tile, slot, exponent base}; plane p of
// slot s at rows (s * NS + p) * nb of a digit arena with nb columns.
emu_status launch_slice(emu_ctx *ctx, const double *t64, const float *t32, const unsigned char *cls,
                        const int4 *d_jobs, int njobs, int nb, const int *exps, uint16_t *digits);
// Digits of the columns of Z (samples) for each matrix block of rows
// [row0, row0 + nrows): plane p, row c (sample), column = row of Z; one
// exponent per (block, sample): exps[blk * s_pad + c].  blocks = {row0, nrows}.
emu_status launch_slice_z(emu_ctx *ctx, const double *Z, long ldz, int s, int s_pad, const int2 *d_blocks,
                          int nblocks, long zcols, int *exps, uint16_t *digits);

// Row exponents and digit planes of a dense column-major FP64 block
// X[0:nrows, col0:col0+ncols] (leading dimension ld): exps[r] for r < npad
// (zeroed first), plane p of row r at digits + (p * npad + r) * kpad, K-major,
// zero beyond nrows / ncols.  npad and kpad are multiples of 32.
emu_status launch_dense_digits(emu_ctx *ctx, const double *X, long ld, int nrows, long col0, long ncols, int npad,
                               long kpad, int *exps, uint16_t *digits);

// Blocked FP64-class panel TRSM X = A L_kk^{-T} (gemm_f64.cu): column block J
// (TW columns) of every listed tile is solved on the FP64 pipe against the
// TW x TW diagonal block of L_kk (launch_trsm_block), then its contribution to
// the later blocks, X_J L_{>J,J}^T, is subtracted as digit products on the
// tensor cores (launch, K = TW, output blocks of BN columns), so the FP64 pipe
// runs TW/nb of the nb^3 flops of a tile in nb/TW solve launches.
constexpr int TW = 128;
// Digits of L_kk's column blocks J < nb/TW - 1, rows r >= (J+1) TW (the rows
// the products read): exps[J nb + r] (biased), plane p of row r at arena row
// (J NS + p) nb + r of an arena with TW columns.  nb a multiple of BM.
emu_status launch_lkk_digits(emu_ctx *ctx, const double *Lkk, int nb, int *exps, uint16_t *digits);
// Column block J of the tiles d_tiles[0..ntiles) of t64 solved in place; Ls /
// rinvs are L_kk's pre-scaled 32 x 32 diagonal blocks and pivot reciprocals
// (launch_trsm64_prep).  With digits (not null), the solved block's row
// exponents and digits for the products: tile z in slot s = slot0 + z,
// exps[s nb + r], plane p of row r at arena row (s NS + p) nb + r (TW columns).
emu_status launch_trsm_block(emu_ctx *ctx, double *t64, int nb, const int *d_tiles, int ntiles, const double *Lkk,
                             int J, const double *Ls, const double *rinvs, int slot0, int *exps, uint16_t *digits);

// out64 (-= or +=) per item, K = nb per segment, on at most max_ctas persistent
// CTAs; a_plane / b_plane = arena rows between digit planes.
emu_status launch(emu_ctx *ctx, const CUtensorMap &a, const CUtensorMap &b, const Item *d_items, int nitems,
                  const Seg *d_segs, int nb, int a_plane, int b_plane, const int *a_exp, const int *b_exp, int mode,
                  double *out64, int ldo, int max_ctas);

}  // namespace gemm64
