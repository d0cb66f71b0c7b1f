// fp64.cu -- FP64 kernels of the tile Cholesky ("Advancements in Dense Linear
// Algebra": POTRF on the diagonal tile, TRSM on the panel, SYRK/GEMM on the
// trailing tiles), the TRMM that draws emulations ("Generating Emulations",
// xi = V z) and the tile-blocked triangular solves.
//
// GB300 runs FP64 on the SIMT pipe at about 2 DFMA per clock per SM (the FP64
// MMA path measured slower), so these kernels are FP64-issue bound: the
// register/shared-memory blocking below only has to keep that pipe busy.
#include "emu_internal.h"

namespace {

constexpr int B = 32;  // inner block of the diagonal-tile POTRF and the TRSM

__device__ inline bool failed(const int *st) {
  return *((volatile const int *)st) != DEV_OK;
}

// ------------------------------------------------------------ POTRF (tile)
// The diagonal tile D (nb x nb, column-major) is factored right-looking in
// 32-wide steps s: leaf POTRF of block (s,s), TRSM of the blocks below it,
// SYRK/GEMM of the trailing lower blocks.

// Leaf: one warp factors the 32x32 block (s,s) in shared memory.
__global__ void __launch_bounds__(32)
    k_potrf_leaf(double *__restrict__ D, int nb, int s, int gcol0, int *st) {
  if (failed(st)) return;
  __shared__ double a[B][B + 1];
  int lane = threadIdx.x;
  double *blk = D + (size_t)s * B + (size_t)s * B * nb;
  for (int c = 0; c < B; c++) a[lane][c] = (lane >= c) ? blk[lane + (size_t)c * nb] : 0.0;
  __syncwarp();
  for (int j = 0; j < B; j++) {
    double d = a[j][j];
    if (!(d > 0.0)) {  // also catches NaN
      if (lane == 0) {
        st[ST_PIVOT] = gcol0 + s * B + j + 1;
        __threadfence();
        atomicExch(&st[ST_CODE], DEV_NOTPD);
      }
      return;
    }
    d = sqrt(d);
    __syncwarp();
    if (lane == j) a[j][j] = d;
    if (lane > j) a[lane][j] /= d;
    __syncwarp();
    if (lane > j) {
      double lj = a[lane][j];
      for (int c = j + 1; c <= lane; c++) a[lane][c] -= lj * a[c][j];
    }
    __syncwarp();
  }
  for (int c = 0; c <= lane; c++) blk[lane + (size_t)c * nb] = a[lane][c];
}

// Rows below block s inside the tile: X = D[rows, s] * L_ss^{-T}.  One warp
// per 32-row block; lane r solves row r by forward substitution.
__global__ void __launch_bounds__(32)
    k_potrf_inner_trsm(double *__restrict__ D, int nb, int s, const int *st) {
  if (failed(st)) return;
  __shared__ double l[B][B + 1];
  __shared__ double x[B][B + 1];
  int lane = threadIdx.x;
  int r0 = (s + 1 + blockIdx.x) * B;
  const double *ls = D + (size_t)s * B + (size_t)s * B * nb;
  double *xs = D + r0 + (size_t)s * B * nb;
  for (int c = 0; c < B; c++) {
    l[lane][c] = ls[lane + (size_t)c * nb];
    x[lane][c] = xs[lane + (size_t)c * nb];
  }
  __syncwarp();
  for (int c = 0; c < B; c++) {
    double v = x[lane][c];
    for (int p = 0; p < c; p++) v -= x[lane][p] * l[c][p];
    x[lane][c] = v / l[c][c];
  }
  __syncwarp();
  for (int c = 0; c < B; c++) xs[lane + (size_t)c * nb] = x[lane][c];
}

// Trailing lower blocks (bi >= bj) inside the tile:
// D[bi, bj] -= X_bi X_bj^T, X_b = D[block b rows, s-block columns].
__global__ void __launch_bounds__(256)
    k_potrf_inner_syrk(double *__restrict__ D, int nb, int s, const int *st) {
  int bi = s + 1 + blockIdx.x, bj = s + 1 + blockIdx.y;
  if (bi < bj || failed(st)) return;
  __shared__ double xi[B][B + 1];
  __shared__ double xj[B][B + 1];
  int t = threadIdx.x;
  int c = t % B, rr = t / B;  // rr in 0..7
  const double *pi = D + (size_t)bi * B + (size_t)s * B * nb;
  const double *pj = D + (size_t)bj * B + (size_t)s * B * nb;
  for (int q = 0; q < 4; q++) {
    int p = rr + 8 * q;  // column of the panel
    xi[c][p] = pi[c + (size_t)p * nb];
    xj[c][p] = pj[c + (size_t)p * nb];
  }
  __syncthreads();
  double acc[4] = {0, 0, 0, 0};
  for (int p = 0; p < B; p++) {
    double bjv = xj[c][p];
#pragma unroll
    for (int q = 0; q < 4; q++) acc[q] += xi[rr + 8 * q][p] * bjv;
  }
  double *cb = D + (size_t)bi * B + (size_t)bj * B * nb;
#pragma unroll
  for (int q = 0; q < 4; q++) cb[(rr + 8 * q) + (size_t)c * nb] -= acc[q];
}

// ------------------------------------------------------------ panel TRSM
// L_ik = A_ik L_kk^{-T} for every i > k.  One CTA per (32-row block, tile);
// column blocks cb left to right: subtract the already-solved blocks
// (GEMM part), then solve against the 32x32 diagonal block of L_kk.
__global__ void __launch_bounds__(256)
    k_trsm64_panel(double *__restrict__ t64, int nb, int NT, int k, const int *__restrict__ rows,
                   const int *st) {
  if (failed(st)) return;
  __shared__ double xp[B][B + 1];
  __shared__ double lc[B][B + 1];
  __shared__ double sx[B][B + 1];
  int i = rows ? rows[blockIdx.y] : k + 1 + blockIdx.y;
  int r0 = blockIdx.x * B;
  const double *Lkk = t64 + (size_t)tile_index(k, k, NT) * nb * nb;
  double *X = t64 + (size_t)tile_index(i, k, NT) * nb * nb + r0;  // row block
  int t = threadIdx.x;
  int c = t % B, rr = t / B;
  int nbb = nb / B;
  for (int cb = 0; cb < nbb; cb++) {
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; q++) acc[q] = X[(rr + 8 * q) + (size_t)(cb * B + c) * nb];
    for (int pb = 0; pb < cb; pb++) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; q++) {
        int p = rr + 8 * q;
        xp[c][p] = X[c + (size_t)(pb * B + p) * nb];                   // X[r=c][p]
        lc[c][p] = Lkk[(cb * B + c) + (size_t)(pb * B + p) * nb];      // L[cb row c][p]
      }
      __syncthreads();
      for (int p = 0; p < B; p++) {
        double lv = lc[c][p];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] -= xp[rr + 8 * q][p] * lv;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      sx[rr + 8 * q][c] = acc[q];
      int p = rr + 8 * q;
      lc[c][p] = Lkk[(cb * B + c) + (size_t)(cb * B + p) * nb];  // diagonal block
    }
    __syncthreads();
    if (t < B) {
      for (int cc = 0; cc < B; cc++) {
        double v = sx[t][cc];
        for (int p = 0; p < cc; p++) v -= sx[t][p] * lc[cc][p];
        sx[t][cc] = v / lc[cc][cc];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) X[(rr + 8 * q) + (size_t)(cb * B + c) * nb] = sx[rr + 8 * q][c];
    __syncthreads();
  }
}

// ------------------------------------------------------- trailing update
// C_ij -= L_ik L_jk^T for k < j <= i (SYRK when i == j: lower 64-blocks
// only).  One CTA per (tile pair, 64x64 block), 4x4 outputs per thread,
// K in slices of 16 through shared memory.
constexpr int GM = 64, GK = 16;

__device__ inline void trailing_pair(long q, int m, int *a, int *b) {
  // q-th lower pair (a >= b) of an m x m triangle, packed by column.
  int bb = 0;
  long base = 0;
  while (base + (m - bb) <= q) {
    base += m - bb;
    bb++;
  }
  *b = bb;
  *a = bb + (int)(q - base);
}

__global__ void __launch_bounds__(256)
    k_update64(double *__restrict__ t64, int nb, int NT, int k, const int *st) {
  if (failed(st)) return;
  int m = NT - k - 1;
  int a, b;
  trailing_pair(blockIdx.x, m, &a, &b);
  int i = k + 1 + a, j = k + 1 + b;
  int nsub = nb / GM;
  int bi = blockIdx.y % nsub, bj = blockIdx.y / nsub;
  if (i == j && bi < bj) return;
  const double *Ai = t64 + (size_t)tile_index(i, k, NT) * nb * nb + bi * GM;
  const double *Aj = t64 + (size_t)tile_index(j, k, NT) * nb * nb + bj * GM;
  double *C = t64 + (size_t)tile_index(i, j, NT) * nb * nb + bi * GM + (size_t)bj * GM * nb;
  __shared__ double as[GK][GM];
  __shared__ double bs[GK][GM];
  int t = threadIdx.x, tx = t % 16, ty = t / 16;
  int lc = t / 16, lr = (t % 16) * 4;  // loader: column lc of the slice, rows lr..lr+3
  double acc[4][4] = {};
  for (int p0 = 0; p0 < nb; p0 += GK) {
#pragma unroll
    for (int e = 0; e < 4; e++) {
      as[lc][lr + e] = Ai[(lr + e) + (size_t)(p0 + lc) * nb];
      bs[lc][lr + e] = Aj[(lr + e) + (size_t)(p0 + lc) * nb];
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < GK; p++) {
      double av[4], bv[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        av[e] = as[p][ty + 16 * e];
        bv[e] = bs[p][tx + 16 * e];
      }
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; x++)
#pragma unroll
    for (int y = 0; y < 4; y++) C[(ty + 16 * x) + (size_t)(tx + 16 * y) * nb] -= acc[x][y];
}

// Zero the strict upper triangle of every diagonal tile (they held the
// mirrored covariance), so factor tiles are exactly lower triangular.
__global__ void k_tril_diag(double *__restrict__ t64, int nb, int NT) {
  int k = blockIdx.y;
  double *D = t64 + (size_t)tile_index(k, k, NT) * nb * nb;
  int c = blockIdx.x;
  for (int r = threadIdx.x; r < c; r += blockDim.x) D[r + (size_t)c * nb] = 0.0;
}

// ---------------------------------------------------------------- TRMM
// Y[rows of tile i, samples] = sum_{k <= i} L_ik Z_k in a fixed k order.
// One CTA per (64 rows, 64 samples).
__global__ void __launch_bounds__(256)
    k_trmm64(const double *__restrict__ t64, int n, int nb, int NT,
             const double *__restrict__ Z, long ldz, int s, double *__restrict__ Y,
             long ldy, const unsigned char *__restrict__ cls) {
  int nsub = nb / GM;
  int i = blockIdx.x / nsub, bi = blockIdx.x % nsub;
  int c0 = blockIdx.y * GM;
  __shared__ double as[GK][GM];
  __shared__ double bs[GK][GM];
  int t = threadIdx.x, tx = t % 16, ty = t / 16;
  int lc = t / 16, lr = (t % 16) * 4;    // A loader
  int zc = t / 4, zp = (t % 4) * 4;      // Z loader: sample zc, rows zp..zp+3
  double acc[4][4] = {};
  for (int k = 0; k <= i; k++) {
    if (cls && cls[tile_index(i, k, NT)] != EMU_CLASS_FP64) continue;
    const double *Ai = t64 + (size_t)tile_index(i, k, NT) * nb * nb + bi * GM;
    for (int p0 = 0; p0 < nb; p0 += GK) {
#pragma unroll
      for (int e = 0; e < 4; e++) {
        as[lc][lr + e] = Ai[(lr + e) + (size_t)(p0 + lc) * nb];
        int col = c0 + zc;
        bs[zp + e][zc] = (col < s) ? Z[(size_t)k * nb + p0 + zp + e + (size_t)col * ldz] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < GK; p++) {
        double av[4], bv[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          av[e] = as[p][ty + 16 * e];
          bv[e] = bs[p][tx + 16 * e];
        }
#pragma unroll
        for (int x = 0; x < 4; x++)
#pragma unroll
          for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int x = 0; x < 4; x++) {
    long gi = (long)i * nb + bi * GM + ty + 16 * x;
    if (gi >= n) continue;
#pragma unroll
    for (int y = 0; y < 4; y++) {
      int col = c0 + tx + 16 * y;
      if (col < s) Y[gi + (size_t)col * ldy] = acc[x][y];
    }
  }
}

// -------------------------------------------------- triangular solves
// Block-row update of the forward solve: X_k -= sum_{j<k} L_kj X_j, and of
// the backward solve: X_k -= sum_{i>k} L_ik^T X_i.  One thread per (row,
// rhs); the sums run over tiles in a fixed order.
__global__ void k_solve_update(const double *__restrict__ t64, int nb, int NT, int k,
                               int backward, double *__restrict__ X, long ldx, int nrhs) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (r >= nb) return;
  double acc = 0.0;
  if (!backward) {
    for (int j = 0; j < k; j++) {
      const double *T = t64 + (size_t)tile_index(k, j, NT) * nb * nb;
      const double *xj = X + (size_t)j * nb + (size_t)c * ldx;
      for (int p = 0; p < nb; p++) acc += T[r + (size_t)p * nb] * xj[p];
    }
  } else {
    for (int i = k + 1; i < NT; i++) {
      const double *T = t64 + (size_t)tile_index(i, k, NT) * nb * nb;
      const double *xi = X + (size_t)i * nb + (size_t)c * ldx;
      for (int p = 0; p < nb; p++) acc += T[p + (size_t)r * nb] * xi[p];
    }
  }
  X[(size_t)k * nb + r + (size_t)c * ldx] -= acc;
}

// Solve with the diagonal tile: one CTA per right-hand side, one thread per
// row; column-oriented substitution (L x = b) or row-oriented (L^T x = b).
__global__ void k_solve_diag(const double *__restrict__ t64, int nb, int NT, int k,
                             int backward, double *__restrict__ X, long ldx) {
  extern __shared__ double xs[];
  int c = blockIdx.x;
  const double *D = t64 + (size_t)tile_index(k, k, NT) * nb * nb;
  double *x = X + (size_t)k * nb + (size_t)c * ldx;
  for (int r = threadIdx.x; r < nb; r += blockDim.x) xs[r] = x[r];
  __syncthreads();
  if (!backward) {
    for (int p = 0; p < nb; p++) {
      double xp = xs[p] / D[p + (size_t)p * nb];
      __syncthreads();
      if (threadIdx.x == 0) xs[p] = xp;
      for (int r = p + 1 + threadIdx.x; r < nb; r += blockDim.x)
        xs[r] -= D[r + (size_t)p * nb] * xp;
      __syncthreads();
    }
  } else {
    for (int p = nb - 1; p >= 0; p--) {
      // x_p = (y_p - sum_{r>p} L[r,p] x_r) / L[p,p]: reduce over r
      double part = 0.0;
      for (int r = p + 1 + threadIdx.x; r < nb; r += blockDim.x)
        part += D[r + (size_t)p * nb] * xs[r];
      __shared__ double red[32];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) sum += red[w];
        xs[p] = (xs[p] - sum) / D[p + (size_t)p * nb];
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < nb; r += blockDim.x) x[r] = xs[r];
}

}  // namespace

emu_status launch_potrf64_tile(emu_ctx *ctx, emu_mat *A, int k) {
  int nb = A->nb, NT = A->nt;
  double *D = A->t64 + (size_t)tile_index(k, k, NT) * nb * nb;
  int nbb = nb / B;
  ProfScope ps(ctx, PROF_POTRF, (double)nb * nb * nb / 3.0, 16.0 * nb * nb);
  for (int s = 0; s < nbb; s++) {
    k_potrf_leaf<<<1, 32, 0, ctx->stream>>>(D, nb, s, k * nb, ctx->d_status);
    EMU_LAUNCHED(ctx);
    int m = nbb - s - 1;
    if (m == 0) break;
    k_potrf_inner_trsm<<<m, 32, 0, ctx->stream>>>(D, nb, s, ctx->d_status);
    EMU_LAUNCHED(ctx);
    k_potrf_inner_syrk<<<dim3(m, m), 256, 0, ctx->stream>>>(D, nb, s, ctx->d_status);
    EMU_LAUNCHED(ctx);
  }
  return EMU_OK;
}

emu_status launch_trsm64_panel(emu_ctx *ctx, emu_mat *A, int k, const int *d_rows, int nrows) {
  int m = d_rows ? nrows : A->nt - k - 1;
  if (m <= 0) return EMU_OK;
  double nb3 = (double)A->nb * A->nb * A->nb;
  ProfScope ps(ctx, PROF_TRSM64, m * nb3, 16.0 * m * A->nb * A->nb);
  k_trsm64_panel<<<dim3(A->nb / B, m), 256, 0, ctx->stream>>>(A->t64, A->nb, A->nt, k, d_rows,
                                                             ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_update64(emu_ctx *ctx, emu_mat *A, int k) {
  int m = A->nt - k - 1;
  if (m <= 0) return EMU_OK;
  long pairs = (long)m * (m + 1) / 2;
  int nsub = A->nb / GM;
  double nb3 = (double)A->nb * A->nb * A->nb;
  ProfScope ps(ctx, PROF_UPDATE64, (double)m * m * nb3, 8.0 * A->nb * A->nb * (2.0 * pairs + 2.0 * m));
  k_update64<<<dim3((unsigned)pairs, nsub * nsub), 256, 0, ctx->stream>>>(
      A->t64, A->nb, A->nt, k, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_tril_diag(emu_ctx *ctx, emu_mat *A) {
  k_tril_diag<<<dim3(A->nb, A->nt), 128, 0, ctx->stream>>>(A->t64, A->nb, A->nt);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_trmm64(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz,
                         int s, double *Y, long ldy, const unsigned char *cls) {
  dim3 grid(L->nt * (L->nb / GM), (s + GM - 1) / GM);
  ProfScope ps(ctx, PROF_TRMM64, (double)L->n * L->n * s, 8.0 * tile_count(L->nt) * L->nb * L->nb);
  k_trmm64<<<grid, 256, 0, ctx->stream>>>(L->t64, L->n, L->nb, L->nt, Z, ldz, s, Y, ldy, cls);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

// X (npad x nrhs, ld ldx >= npad, padded rows zero) <- (L L^T)^{-1} X.
emu_status launch_potrs64(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs) {
  int nb = L->nb, NT = L->nt;
  int thr = 256;
  ProfScope ps(ctx, PROF_SOLVE, 2.0 * L->n * L->n * nrhs, 16.0 * tile_count(NT) * nb * nb);
  for (int k = 0; k < NT; k++) {
    if (k > 0) {
      k_solve_update<<<dim3((nb + thr - 1) / thr, nrhs), thr, 0, ctx->stream>>>(
          L->t64, nb, NT, k, 0, X, ldx, nrhs);
      EMU_LAUNCHED(ctx);
    }
    k_solve_diag<<<nrhs, 512, nb * sizeof(double), ctx->stream>>>(L->t64, nb, NT, k, 0, X, ldx);
    EMU_LAUNCHED(ctx);
  }
  for (int k = NT - 1; k >= 0; k--) {
    if (k < NT - 1) {
      k_solve_update<<<dim3((nb + thr - 1) / thr, nrhs), thr, 0, ctx->stream>>>(
          L->t64, nb, NT, k, 1, X, ldx, nrhs);
      EMU_LAUNCHED(ctx);
    }
    k_solve_diag<<<nrhs, 512, nb * sizeof(double), ctx->stream>>>(L->t64, nb, NT, k, 1, X, ldx);
    EMU_LAUNCHED(ctx);
  }
  return EMU_OK;
}
