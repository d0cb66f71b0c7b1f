// trsm_tc.h -- host interface of the FP32-class panel TRSM on the tensor
// cores (trsm_tc.cu): L_ik = A_ik L_kk^{-T} for the listed low-precision
// tiles of panel k of the mixed-precision tile Cholesky ("Mixed-Precision
// Computation Innovations": TRSM(r, c) tasks of column c).
//
// Blocked right-looking solve in 64-column blocks J, one CTA per 128 rows of
// a tile: the row block's trailing columns live in TMEM as FP32 accumulators;
// the 64 x 64 diagonal block of each J is solved in FP32 (SIMT, forward
// substitution), and the solved block X_J is subtracted from the trailing
// columns as X_J L_{>J,J}^T by tcgen05 MMAs of the three-piece BF16 split
// (the six products of the FP32 class, as in gemm_tc.cu).  The result is the
// FP32 master of the tile (column-major) and its three BF16 pieces
// (row-major), the same outputs as the SIMT panel TRSM.
#pragma once
#include <cuda.h>

#include "emu_internal.h"

namespace trsm_tc {

constexpr int RB = 128;  // rows of a CTA (TMEM lanes)
constexpr int W = 64;    // column block

// The tile sizes this kernel takes: nb a multiple of 128 whose trailing
// columns (nb - 64) fit in the 512 TMEM columns.
inline bool supports(int nb) { return nb % RB == 0 && nb - W <= 512; }

// FP32 copy (column-major) and three BF16 pieces (row-major, strict upper
// triangle zero) of the negated FP64 diagonal factor tiles -L of
// the arena t64 (nb x nb, column-major): entry z of the list, tile d_tiles[z]
// (or `tile` when d_tiles is null, n = 1), goes to slot z: L32 + z nb^2 and
// pieces + 3 z nb^2.
emu_status launch_prep(emu_ctx *ctx, const double *t64, long tile, const long *d_tiles, int n, float *L32,
                       uint16_t *pieces, int nb);

// 2-D tensor map over `nslots` piece sets (3 nb rows each) written by
// launch_prep, box 64 x 64, 128-byte swizzle.
emu_status make_map(emu_ctx *ctx, CUtensorMap *map, const uint16_t *pieces, int nb, int nslots);

// 2-D tensor map over the BF16 piece arena op (ntiles * 3 rows of nb x nb,
// row-major), box 128 rows x 64, 128-byte swizzle: the solved pieces are
// stored through it.
emu_status make_op_map(emu_ctx *ctx, CUtensorMap *map, const uint16_t *op, int nb, long ntiles);

// Solves the listed tiles in place: t32 holds the FP32 masters; the three
// BF16 pieces of each solved tile t go to the piece arena behind opmap (piece
// p at rows (t * 3 + p) nb, row-major).  Either d_rows (tile (rows[i], k) of
// an NT x NT tile matrix, L slot k & 1) or d_jobs ({tile index, L slot})
// lists the n tiles.  lkk0 / lmap: the FP32 copies and the pieces of the L
// slots (launch_prep).
emu_status launch(emu_ctx *ctx, const CUtensorMap &lmap, const CUtensorMap &opmap, const float *lkk0, float *t32,
                  int nb, int NT, int k, const int *d_rows, const int2 *d_jobs, int n);

}  // namespace trsm_tc
