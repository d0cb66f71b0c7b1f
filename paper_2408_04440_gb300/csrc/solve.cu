// solve.cu -- the triangular solves L L^T X = B with a mixed-precision factor
// in FP32-master storage: the preconditioner of iterative refinement (each
// correction is M^{-1} r with M = L L^T; the FP64 residual and update live in
// refine.cu).
//
// Arithmetic: FP32 products of the stored tiles (FP64 tiles rounded to FP32,
// FP32 masters as they are; the diagonal tiles from their FP64 factor),
// accumulated in FP32 per tile and added to the FP64 right-hand sides.
// Blocked by tile rows, right-looking:
//   forward  for k = 0..NT-1:   X_k <- L_kk^{-1} X_k;    X_i -= L_ik X_k   (i > k)
//   backward for k = NT-1..0:   X_k <- L_kk^{-T} X_k;    X_j -= L_kj^T X_k (j < k)
// The diagonal solve is one CTA (one thread per row, nb <= 1024) per group of
// right-hand sides, in 32-column blocks: one warp runs the 32-step chain of a
// block with shuffles while the other rows wait, then every later row
// subtracts the block.  The panel products run one CTA per (64-row slab of an
// output block, group of right-hand sides) with the operands staged in shared
// memory (coalesced tile reads), so a sweep reads each stored tile once.
#include "mixed.h"

namespace {

constexpr int SB = 32;  // column block of the diagonal solve
constexpr int PS = 64;  // output slab of the panel products
constexpr int PK = 32;  // K chunk of the panel products

__device__ inline bool failed(const int *st) { return *((volatile const int *)st) != DEV_OK; }

// X[0:nb, c0:c0+P] <- L^{-1} X (trans = 0) or L^{-T} X (trans = 1), L the
// nb x nb lower-triangular FP64 factor tile D (column-major).
template <int P>
__global__ void __launch_bounds__(1024) k_trsv_diag(const double *__restrict__ D, int nb, double *__restrict__ X,
                                                    long ld, int nrhs, int trans, const int *st) {
  if (failed(st)) return;
  __shared__ float Ld[SB][SB + 1];
  __shared__ float ys[SB][P + 1];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int c0 = blockIdx.x * P;
  const int p = min(P, nrhs - c0);
  float b[P];
#pragma unroll
  for (int q = 0; q < P; q++) b[q] = q < p ? (float)X[t + (size_t)(c0 + q) * ld] : 0.0f;
  const int nblk = nb / SB;
  for (int s = 0; s < nblk; s++) {
    const int cb = trans ? nblk - 1 - s : s;
    for (int e = t; e < SB * SB; e += blockDim.x) {
      const int r = e % SB, c = e / SB;
      Ld[r][c] = (float)D[(size_t)(cb * SB + r) + (size_t)(cb * SB + c) * nb];
    }
    __syncthreads();
    if (warp == cb) {
      if (!trans) {
        for (int c = 0; c < SB; c++) {
          const float rinv = 1.0f / Ld[c][c];
          const float lc = Ld[lane][c];
#pragma unroll
          for (int q = 0; q < P; q++) {
            const float y = __shfl_sync(0xffffffffu, b[q] * rinv, c);
            if (lane == c) b[q] = y;
            else if (lane > c) b[q] = fmaf(-lc, y, b[q]);
          }
        }
      } else {
        for (int c = SB - 1; c >= 0; c--) {
          const float rinv = 1.0f / Ld[c][c];
          const float lc = Ld[c][lane];  // row c, column lane: L^T(lane, c)
#pragma unroll
          for (int q = 0; q < P; q++) {
            const float y = __shfl_sync(0xffffffffu, b[q] * rinv, c);
            if (lane == c) b[q] = y;
            else if (lane < c) b[q] = fmaf(-lc, y, b[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < P; q++) ys[lane][q] = b[q];
    }
    __syncthreads();
    if (!trans && t >= (cb + 1) * SB) {
      // later rows: b_t -= sum_c L(t, cb*32 + c) y_c (column reads, coalesced over t)
      for (int c = 0; c < SB; c++) {
        const float l = (float)D[(size_t)t + (size_t)(cb * SB + c) * nb];
#pragma unroll
        for (int q = 0; q < P; q++) b[q] = fmaf(-l, ys[c][q], b[q]);
      }
    } else if (trans && t < cb * SB) {
      // earlier rows: b_t -= sum_c L(cb*32 + c, t) x_c (32 consecutive entries of column t)
      const double *col = D + (size_t)cb * SB + (size_t)t * nb;
      for (int c = 0; c < SB; c++) {
        const float l = (float)col[c];
#pragma unroll
        for (int q = 0; q < P; q++) b[q] = fmaf(-l, ys[c][q], b[q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < P; q++)
    if (q < p) X[t + (size_t)(c0 + q) * ld] = (double)b[q];
}

// One tile's entry (r, c) as FP32 from its storage.
__device__ inline float tile32(const double *t64, const float *t32, bool fp64, size_t o) {
  return fp64 ? (float)t64[o] : t32[o];
}

// forward: X_i -= L_ik X_k for the tiles (i, k), i = k+1 .. NT-1
// (blockIdx.x = slab of the rows k+1 .. NT-1 blocks); backward: X_j -= L_kj^T
// X_k for j = 0 .. k-1 (blockIdx.x = slab of the rows of blocks 0 .. k-1).
template <int P>
__global__ void __launch_bounds__(256) k_panel(const double *__restrict__ t64, const float *__restrict__ t32,
                                               const unsigned char *__restrict__ cls, int nb, int NT, int k,
                                               int backward, double *__restrict__ X, long ld, int nrhs,
                                               const int *st) {
  if (failed(st)) return;
  constexpr int NQ = P / 4;
  __shared__ float a[PK][PS + 1];
  __shared__ float x[PK][P + 1];
  const int per = nb / PS;
  const int blk = (int)(blockIdx.x / per) + (backward ? 0 : k + 1), m0 = (int)(blockIdx.x % per) * PS;
  const long t = backward ? tile_index(k, blk, NT) : tile_index(blk, k, NT);
  const bool fp64 = cls[t] == EMU_CLASS_FP64;
  const size_t tb = (size_t)t * nb * nb;
  const int c0 = blockIdx.y * P;
  const int p = min(P, nrhs - c0);
  const int tid = threadIdx.x, mm = tid & (PS - 1), q0 = tid >> 6;
  float acc[NQ];
#pragma unroll
  for (int w = 0; w < NQ; w++) acc[w] = 0.0f;
  for (int k0 = 0; k0 < nb; k0 += PK) {
    for (int e = tid; e < PK * PS; e += 256) {
      if (!backward) {
        const int m = e % PS, kk = e / PS;
        a[kk][m] = tile32(t64, t32, fp64, tb + (size_t)(m0 + m) + (size_t)(k0 + kk) * nb);
      } else {
        const int kk = e % PK, m = e / PK;
        a[kk][m] = tile32(t64, t32, fp64, tb + (size_t)(k0 + kk) + (size_t)(m0 + m) * nb);
      }
    }
    for (int e = tid; e < PK * P; e += 256) {
      const int kk = e % PK, q = e / PK;
      x[kk][q] = q < p ? (float)X[(size_t)k * nb + k0 + kk + (size_t)(c0 + q) * ld] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < PK; kk++) {
      const float av = a[kk][mm];
#pragma unroll
      for (int w = 0; w < NQ; w++) acc[w] = fmaf(av, x[kk][q0 + 4 * w], acc[w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int w = 0; w < NQ; w++) {
    const int q = q0 + 4 * w;
    if (q < p) X[(size_t)blk * nb + m0 + mm + (size_t)(c0 + q) * ld] -= (double)acc[w];
  }
}

template <int P>
emu_status solve_sweeps(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs) {
  const int nb = L->nb, NT = L->nt;
  const unsigned groups = (unsigned)((nrhs + P - 1) / P);
  const int *st = ctx->d_status;
  for (int k = 0; k < NT; k++) {
    const double *D = L->t64 + (size_t)tile_index(k, k, NT) * nb * nb;
    k_trsv_diag<P><<<groups, nb, 0, ctx->stream>>>(D, nb, X + (size_t)k * nb, ldx, nrhs, 0, st);
    EMU_LAUNCHED(ctx);
    if (k + 1 < NT) {
      k_panel<P><<<dim3((unsigned)((NT - k - 1) * (nb / PS)), groups), 256, 0, ctx->stream>>>(
          L->t64, L->t32, L->d_cls, nb, NT, k, 0, X, ldx, nrhs, st);
      EMU_LAUNCHED(ctx);
    }
  }
  for (int k = NT - 1; k >= 0; k--) {
    const double *D = L->t64 + (size_t)tile_index(k, k, NT) * nb * nb;
    k_trsv_diag<P><<<groups, nb, 0, ctx->stream>>>(D, nb, X + (size_t)k * nb, ldx, nrhs, 1, st);
    EMU_LAUNCHED(ctx);
    if (k > 0) {
      k_panel<P><<<dim3((unsigned)(k * (nb / PS)), groups), 256, 0, ctx->stream>>>(
          L->t64, L->t32, L->d_cls, nb, NT, k, 1, X, ldx, nrhs, st);
      EMU_LAUNCHED(ctx);
    }
  }
  return EMU_OK;
}

}  // namespace

bool mixed_potrs_blocked_supports(int nb) { return nb >= 64 && nb <= 1024 && nb % 64 == 0; }

emu_status mixed_potrs_blocked(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs) {
  if (!mixed_potrs_blocked_supports(L->nb)) return EMU_EINVAL;
  ProfScope ps(ctx, PROF_SOLVE, 2.0 * (double)L->n * L->n * nrhs, 4.0 * (double)L->n * L->n);
  return nrhs <= 16 ? solve_sweeps<16>(ctx, L, X, ldx, nrhs) : solve_sweeps<32>(ctx, L, X, ldx, nrhs);
}
