// cov.cu -- covariance build / import into packed FP64 tiles, the fused
// per-tile Frobenius-norm pass, the precision map, and export to dense.
//
// Covariance: synthetic stand-in for U-hat ("Modeling the Temporal Dependence
// and Constructing a Covariance Matrix", equation for U-hat and the diagonal
// perturbation that keeps it positive definite).  The correlation exp(-d/beta)
// depends only on (l_i - l_j, m_i - m_j), so it is evaluated once per offset
// into a table; every entry is then s(l_i) * s(l_j) * rho(dl, dm) -- the same
// operations, in the same order, as evaluating the formula entry by entry.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "emu_internal.h"

namespace {

constexpr int kChunk = 32;     // columns of a tile handled by one CTA
constexpr int kThreads = 256;

// Degree l of coefficient row k (k = l^2 + l + m): floor(sqrt(k)), from a
// single-precision estimate corrected in integer arithmetic.
__device__ inline int degree_of(long k) {
  int l = (int)sqrtf((float)k);
  while ((long)l * l > k) l--;
  while ((long)(l + 1) * (l + 1) <= k) l++;
  return l;
}

// sigma[l] = (1 + l)^(-sexp); rho[(dl + L - 1) * W + (dm + 2L - 2)] =
// exp(-sqrt(dl^2 + dm^2) / beta), W = 4L - 3; out[0] = nugget added to
// the diagonal = nugget_rel * max_l sigma[l]^2.  Thread `tid` of `nthr`
// strides over the entries; `leader` computes the nugget.
__device__ inline void cov_tables_part(int L, double beta, double sexp, double nugget_rel, double *sigma,
                                       double *rho, double *nugget, long tid, long nthr, bool leader) {
  int W = 4 * L - 3;
  long total = (long)(2 * L - 1) * W;
  for (long t = tid; t < total; t += nthr) {
    int a = (int)(t / W), b = (int)(t % W);
    double dl = (double)(a - (L - 1)), dm = (double)(b - (2 * L - 2));
    double d = sqrt(dl * dl + dm * dm);
    rho[t] = exp(-d / beta);
  }
  for (long l = tid; l < L; l += nthr) sigma[l] = pow(1.0 + l, -sexp);
  if (leader) {
    // max_l sigma[l]^2 rho(0, 0): (1 + l)^(-sexp) is monotone in l, so the
    // largest square is at l = 0 or l = L - 1 (the same two pow values the
    // whole scan would compare; rho(0, 0) = exp(0) = 1)
    const double s0 = pow(1.0, -sexp), s1 = pow((double)L, -sexp);
    const double v0 = s0 * s0 * 1.0, v1 = s1 * s1 * 1.0;
    *nugget = nugget_rel * (v1 > v0 ? v1 : v0);
  }
}

__global__ void k_cov_tables(int L, double beta, double sexp, double nugget_rel,
                             double *sigma, double *rho, double *nugget) {
  cov_tables_part(L, beta, sexp, nugget_rel, sigma, rho, nugget, blockIdx.x * (long)blockDim.x + threadIdx.x,
                  (long)gridDim.x * blockDim.x, blockIdx.x == 0 && threadIdx.x == 0);
}

// Batch: blockIdx.y = matrix; its tables at tab_base (rho, then sigma, then
// the nugget).
__global__ void k_cov_tables_batch(const BatchInst *__restrict__ inst, double *tables) {
  BatchInst I = inst[blockIdx.y];
  double *rho = tables + I.tab_base;
  double *sigma = rho + (long)(2 * I.L - 1) * (4 * I.L - 3);
  cov_tables_part(I.L, I.beta, I.sigma_exp, I.nugget_rel, sigma, rho, sigma + I.L,
                  blockIdx.x * (long)blockDim.x + threadIdx.x, (long)gridDim.x * blockDim.x,
                  blockIdx.x == 0 && threadIdx.x == 0);
}

// Deterministic block reduction of one double per thread (fixed tree).
__device__ inline double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) r += sh[i];
  }
  __syncthreads();
  return r;
}

// One CTA per (tile, 32-column chunk): blockIdx.x = tile, blockIdx.y = chunk.  Writes the tile's chunk (padded
// entries: unit diagonal, zeros elsewhere) and the chunk's sum of squares
// over the real (unpadded) entries of the full symmetric tile.
// Chunk `chunk` (kChunk columns) of tile (ti, tj) of the covariance of
// bandlimit L; returns this thread's sum of squares of the real entries.
// `store(r, c, v)` receives every entry of the chunk (the padded ones too).
template <class Store>
__device__ inline double cov_tile_chunk_t(int L, int n, int nb, int ti, int tj, int chunk,
                                          const double *__restrict__ sigma, const double *__restrict__ rho,
                                          double nug, const Store &store) {
  const int W = 4 * L - 3;
  // this thread's rows (r = threadIdx.x + k blockDim.x): degree, order and
  // sigma once per row; rho's index is then rbase - (l_j W + m_j) per entry
  constexpr int kMaxRows = 8;  // nb <= 8 * kThreads
  int rbase[kMaxRows];
  double si[kMaxRows];
  bool real[kMaxRows];
#pragma unroll
  for (int k = 0; k < kMaxRows; k++) {
    const int r = threadIdx.x + k * blockDim.x;
    const long gi = (long)ti * nb + r;
    real[k] = r < nb && gi < n;
    rbase[k] = 0;
    si[k] = 0.0;
    if (real[k]) {
      const int li = degree_of(gi);
      const int mi = (int)(gi - (long)li * li - li);
      rbase[k] = (li + L - 1) * W + (mi + 2 * L - 2);
      si[k] = sigma[li];
    }
  }
  double ss = 0.0;
  for (int cc = 0; cc < kChunk; cc++) {
    const int c = chunk * kChunk + cc;
    const long gj = (long)tj * nb + c;
    int cbase = 0;
    double sj = 0.0;
    if (gj < n) {
      const int lj = degree_of(gj);
      const int mj = (int)(gj - (long)lj * lj - lj);
      cbase = lj * W + mj;
      sj = sigma[lj];
    }
#pragma unroll
    for (int k = 0; k < kMaxRows; k++) {
      const int r = threadIdx.x + k * blockDim.x;
      if (r >= nb) break;
      const long gi = (long)ti * nb + r;
      double v;
      if (real[k] && gj < n) {
        const double e = rho[rbase[k] - cbase];
        v = __dmul_rn(__dmul_rn(si[k], sj), e);  // (sigma_i sigma_j) rho, no FMA contraction
        if (gi == gj) v = __dadd_rn(v, nug);
        ss += v * v;
      } else {
        v = (gi == gj) ? 1.0 : 0.0;
      }
      store(r, c, v);
    }
  }
  return ss;
}

struct StoreF64 {
  double *tile;
  int nb;
  __device__ void operator()(int r, int c, double v) const { tile[r + (size_t)c * nb] = v; }
};
struct StoreNone {
  __device__ void operator()(int, int, double) const {}
};
// Class-format storage: the entry rounded to the tile's class (nearest);
// E4M3-class tiles hold BF16 working values until the factor solves them.
struct StoreClass {
  int cls, nb;
  size_t base;
  ClassArenas ar;
  __device__ void operator()(int r, int c, double v) const {
    const size_t e = base + r + (size_t)c * nb;
    if (cls == EMU_CLASS_FP64) ar.t64[e] = v;
    else if (cls == EMU_CLASS_FP32) ar.t32[e] = (float)v;
    else if (cls == EMU_CLASS_BF16) ar.t16[e] = __bfloat16_as_ushort(__double2bfloat16(v));
    else reinterpret_cast<uint16_t *>(ar.t8)[e] = __bfloat16_as_ushort(__double2bfloat16(v));
  }
};

__device__ inline double cov_tile_chunk(int L, int n, int nb, int ti, int tj, int chunk,
                                        const double *__restrict__ sigma, const double *__restrict__ rho,
                                        double nug, double *__restrict__ tile) {
  return cov_tile_chunk_t(L, n, nb, ti, tj, chunk, sigma, rho, nug, StoreF64{tile, nb});
}

__global__ void __launch_bounds__(kThreads)
    k_cov_build(int L, int n, int nb, int NT, const double *__restrict__ sigma,
                const double *__restrict__ rho, const double *__restrict__ nugget,
                double *__restrict__ t64, double *__restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  long t = blockIdx.x;
  int ti, tj;
  tile_coords(t, NT, &ti, &tj);
  double ss = cov_tile_chunk(L, n, nb, ti, tj, blockIdx.y, sigma, rho, *nugget, t64 + (size_t)t * nb * nb);
  double tot = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[t * gridDim.y + blockIdx.y] = tot;
}

// Class format, pass 1: the norm partials only.  Pass 2 (classes known):
// every tile stored in its class's arena.
__global__ void __launch_bounds__(kThreads)
    k_cov_norms(int L, int n, int nb, int NT, const double *__restrict__ sigma, const double *__restrict__ rho,
                const double *__restrict__ nugget, double *__restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  long t = blockIdx.x;
  int ti, tj;
  tile_coords(t, NT, &ti, &tj);
  double ss = cov_tile_chunk_t(L, n, nb, ti, tj, blockIdx.y, sigma, rho, *nugget, StoreNone{});
  double tot = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[t * gridDim.y + blockIdx.y] = tot;
}

__global__ void __launch_bounds__(kThreads)
    k_cov_store_class(int L, int n, int nb, int NT, const double *__restrict__ sigma,
                      const double *__restrict__ rho, const double *__restrict__ nugget, ClassArenas ar) {
  long t = blockIdx.x;
  int ti, tj;
  tile_coords(t, NT, &ti, &tj);
  const int c = ar.cls[t], sl = ar.slot[t];
  StoreClass st{c, nb, (size_t)sl * nb * nb, ar};
  (void)cov_tile_chunk_t(L, n, nb, ti, tj, blockIdx.y, sigma, rho, *nugget, st);
}

// Batch: blockIdx.x = tile of the batch arena, tile_inst = its matrix.
__global__ void __launch_bounds__(kThreads)
    k_cov_build_batch(const BatchInst *__restrict__ inst, const int *__restrict__ tile_inst, int nb,
                      const double *__restrict__ tables, double *__restrict__ t64, double *__restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  long g = blockIdx.x;
  BatchInst I = inst[tile_inst[g]];
  int ti, tj;
  tile_coords(g - I.tile_base, I.NT, &ti, &tj);
  const double *rho = tables + I.tab_base;
  const double *sigma = rho + (long)(2 * I.L - 1) * (4 * I.L - 3);
  double ss = cov_tile_chunk(I.L, I.n, nb, ti, tj, blockIdx.y, sigma, rho, sigma[I.L], t64 + (size_t)g * nb * nb);
  double tot = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[g * gridDim.y + blockIdx.y] = tot;
}

// Same layout from a dense, column-major, lower-triangle user matrix.
__global__ void __launch_bounds__(kThreads)
    k_import(int n, int nb, int NT, const double *__restrict__ A, long lda,
             double *__restrict__ t64, double *__restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  long t = blockIdx.x;
  int ti, tj;
  tile_coords(t, NT, &ti, &tj);
  double *tile = t64 + (size_t)t * nb * nb;
  double ss = 0.0;
  for (int cc = 0; cc < kChunk; cc++) {
    int c = blockIdx.y * kChunk + cc;
    long gj = (long)tj * nb + c;
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      long gi = (long)ti * nb + r;
      double v;
      if (gi < n && gj < n) {
        v = (gi >= gj) ? A[gi + gj * lda] : A[gj + gi * lda];
        ss += v * v;
      } else {
        v = (gi == gj) ? 1.0 : 0.0;
      }
      tile[r + (size_t)c * nb] = v;
    }
  }
  double tot = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[t * gridDim.y + blockIdx.y] = tot;
}

// Empirical covariance ("Modeling the Temporal Dependence": U-hat = the sum
// of xi xi^T over the residual vectors divided by their number m): the tiles
// hold the raw sums.  k_emp_maxdiag: max_k U-hat_kk as the bits of a
// non-negative double (atomicMax on the bits orders such doubles).
__global__ void k_emp_maxdiag(int n, int nb, int NT, const double *__restrict__ t64, double inv_m,
                              unsigned long long *__restrict__ maxbits) {
  unsigned long long best = 0;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const int tk = (int)(k / nb), r = (int)(k % nb);
    const double v = t64[(size_t)tile_index(tk, tk, NT) * nb * nb + r + (size_t)r * nb] * inv_m;
    best = max(best, (unsigned long long)__double_as_longlong(fmax(v, 0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, best);
}

// Scale the sums by 1/m, add nugget_rel * max diag to the diagonal (the
// paper's perturbation when there are fewer residual vectors than
// coefficients), set the padding (identity diagonal), and write the tile-norm
// partials as the covariance build does.
__global__ void __launch_bounds__(kThreads)
    k_emp_finish(int n, int nb, int NT, double inv_m, double nugget_rel,
                 const unsigned long long *__restrict__ maxbits, double *__restrict__ t64,
                 double *__restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  long t = blockIdx.x;
  int ti, tj;
  tile_coords(t, NT, &ti, &tj);
  double *tile = t64 + (size_t)t * nb * nb;
  const double nug = nugget_rel * __longlong_as_double((long long)*maxbits);
  double ss = 0.0;
  for (int cc = 0; cc < kChunk; cc++) {
    int c = blockIdx.y * kChunk + cc;
    long gj = (long)tj * nb + c;
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      long gi = (long)ti * nb + r;
      double v;
      if (gi < n && gj < n) {
        v = tile[r + (size_t)c * nb] * inv_m;
        if (gi == gj) v += nug;
        ss += v * v;
      } else {
        v = (gi == gj) ? 1.0 : 0.0;
      }
      tile[r + (size_t)c * nb] = v;
    }
  }
  double tot = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[t * gridDim.y + blockIdx.y] = tot;
}

// One tile column j from a staging block holding rows j*nb .. n-1 of
// columns j*nb .. j*nb+nb-1 (column-major, leading dimension ld).
__global__ void __launch_bounds__(kThreads)
    k_import_col(int n, int nb, int NT, int tj, const double *__restrict__ S, long ld,
                 double *__restrict__ t64, double *__restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  int ti = tj + blockIdx.x;
  long t = tile_index(ti, tj, NT);
  double *tile = t64 + (size_t)t * nb * nb;
  long base = (long)tj * nb;
  double ss = 0.0;
  for (int cc = 0; cc < kChunk; cc++) {
    int c = blockIdx.y * kChunk + cc;
    long gj = base + c;
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      long gi = (long)ti * nb + r;
      double v;
      if (gi < n && gj < n) {
        v = (gi >= gj) ? S[(gi - base) + (gj - base) * ld] : S[(gj - base) + (gi - base) * ld];
        ss += v * v;
      } else {
        v = (gi == gj) ? 1.0 : 0.0;
      }
      tile[r + (size_t)c * nb] = v;
    }
  }
  double tot = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[t * gridDim.y + blockIdx.y] = tot;
}

// Single CTA: tile norms from the partial sums (fixed order), ||S||_F, and
// the class of each tile under the rule t_ij * u[c] <= eps * ||S||_F / NT.
// Band maps of the paper's precision variants (EMU_MAP_*): the diagonal band
// FP64; DP/SP: the rest FP32; DP/HP: the rest BF16; DP/SP/HP: sub-diagonal
// bands 1 .. nsp FP32, the rest BF16.
__device__ inline int band_class(int band, int i, int j, int nsp) {
  const int d = i - j;
  if (d == 0) return EMU_CLASS_FP64;
  if (band == EMU_MAP_DP_SP) return EMU_CLASS_FP32;
  if (band == EMU_MAP_DP_HP) return EMU_CLASS_BF16;
  return d <= nsp ? EMU_CLASS_FP32 : EMU_CLASS_BF16;
}
// The fewest whole sub-diagonal bands (band d holds NT - d tiles) that hold
// at least frac of the NT (NT + 1) / 2 lower tiles.
__device__ inline int sp_bands(int NT, double frac) {
  if (!(frac > 0.0)) return 0;
  const double need = frac * 0.5 * (double)NT * (double)(NT + 1);
  long have = 0;
  int b = 0;
  while (b < NT - 1 && (double)have < need) {
    b++;
    have += NT - b;
  }
  return b;
}

__global__ void __launch_bounds__(1024)
    k_precision_map(int NT, long ntiles, int nchunk,
                    const double *__restrict__ partial, double *__restrict__ tnorm,
                    double *__restrict__ frob, unsigned char *__restrict__ cls,
                    double eps, double u1, double u2, double u3, double u4,
                    unsigned mask, int diag_fp64, int band, double sp_frac,
                    const BatchInst *__restrict__ inst) {
  __shared__ double sh[32];
  if (inst) {
    // batch: one CTA per matrix, its tiles at tile_base
    BatchInst I = inst[blockIdx.x];
    NT = I.NT;
    ntiles = (long)NT * (NT + 1) / 2;
    partial += I.tile_base * nchunk;
    tnorm += I.tile_base;
    frob += blockIdx.x;
    if (cls) cls += I.tile_base;
  }
  double acc = 0.0;
  for (long t = threadIdx.x; t < ntiles; t += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; c++) s += partial[t * nchunk + c];
    double tn = sqrt(s);
    tnorm[t] = tn;
    int i, j;
    tile_coords(t, NT, &i, &j);
    acc += (i == j ? 1.0 : 2.0) * tn * tn;
  }
  double tot = block_sum(acc, sh);
  __shared__ double s_frob;
  if (threadIdx.x == 0) {
    s_frob = sqrt(tot);
    *frob = s_frob;
  }
  __syncthreads();
  if (cls == nullptr) return;
  if (band != EMU_MAP_NORM) {
    const int nsp = sp_bands(NT, sp_frac);
    for (long t = threadIdx.x; t < ntiles; t += blockDim.x) {
      int i, j;
      tile_coords(t, NT, &i, &j);
      cls[t] = (unsigned char)band_class(band, i, j, nsp);
    }
    return;
  }
  double thr = eps * s_frob / (double)NT;
  const double uu[EMU_NCLASS] = {0.0, u1, u2, u3, u4};
  for (long t = threadIdx.x; t < ntiles; t += blockDim.x) {
    int i, j;
    tile_coords(t, NT, &i, &j);
    int c = 0;
    if (!(diag_fp64 && i == j)) {
      double tn = tnorm[t];
      for (int cc = EMU_NCLASS - 1; cc >= 1; cc--) {
        if (((mask >> cc) & 1u) && tn * uu[cc] <= thr) {
          c = cc;
          break;
        }
      }
    }
    cls[t] = (unsigned char)c;
  }
}

// Dense FP64 lower triangle from the tiles, chunk `chunk` of the tile pair
// (ti, tj): upper tiles and the strict upper part of diagonal tiles become 0.
// Low-precision off-diagonal tiles of a mixed factor come from the FP32
// master arena (t32 and cls given).
__device__ inline void export_chunk(int n, int nb, int NT, int ti, int tj, int chunk, const double *__restrict__ t64,
                                    const float *__restrict__ t32, const unsigned char *__restrict__ cls,
                                    double *__restrict__ out, long ld) {
  const double *tile = nullptr;
  const float *tile32 = nullptr;
  if (ti >= tj) {
    long t = tile_index(ti, tj, NT);
    if (t32 != nullptr && cls != nullptr && ti != tj && cls[t] != EMU_CLASS_FP64)
      tile32 = t32 + (size_t)t * nb * nb;
    else
      tile = t64 + (size_t)t * nb * nb;
  }
  for (int cc = 0; cc < kChunk; cc++) {
    int c = chunk * kChunk + cc;
    long gj = (long)tj * nb + c;
    if (gj >= n) break;
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      long gi = (long)ti * nb + r;
      if (gi >= n) break;
      double v = 0.0;
      if (gi >= gj) {
        if (tile32) v = (double)tile32[r + (size_t)c * nb];
        else if (tile) v = tile[r + (size_t)c * nb];
      }
      out[gi + gj * ld] = v;
    }
  }
}

// grid.x enumerates all NT*NT tile pairs.
__global__ void __launch_bounds__(kThreads)
    k_export(int n, int nb, int NT, const double *__restrict__ t64,
             const float *__restrict__ t32, const unsigned char *__restrict__ cls,
             double *__restrict__ out, long ld) {
  export_chunk(n, nb, NT, blockIdx.x % NT, blockIdx.x / NT, blockIdx.y, t64, t32, cls, out, ld);
}

// Batch: pairs[blockIdx.x] = {matrix, ti, tj}; matrix b goes to out[b]
// (n_b x n_b, leading dimension n_b).
__global__ void __launch_bounds__(kThreads)
    k_export_batch(const BatchInst *__restrict__ inst, const int4 *__restrict__ pairs, int nb,
                   const double *__restrict__ t64, const float *__restrict__ t32,
                   const unsigned char *__restrict__ cls, double *const *__restrict__ out) {
  int4 pr = pairs[blockIdx.x];
  BatchInst I = inst[pr.x];
  export_chunk(I.n, nb, I.NT, pr.y, pr.z, blockIdx.y, t64 + (size_t)I.tile_base * nb * nb,
               t32 ? t32 + (size_t)I.tile_base * nb * nb : nullptr, cls ? cls + I.tile_base : nullptr, out[pr.x],
               I.n);
}

}  // namespace

emu_status launch_cov_build(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p) {
  int L = p->L;
  size_t ntab = (size_t)(2 * L - 1) * (4 * L - 3);
  double *buf = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&buf, (ntab + L + 1) * sizeof(double), ctx->stream));
  double *rho = buf, *sigma = buf + ntab, *nug = buf + ntab + L;
  int blocks = (int)((ntab + 255) / 256);
  if (blocks > 4 * ctx->sm_count) blocks = 4 * ctx->sm_count;
  k_cov_tables<<<blocks, 256, 0, ctx->stream>>>(L, p->beta, p->sigma_exp, p->nugget_rel,
                                               sigma, rho, nug);
  EMU_LAUNCHED(ctx);
  dim3 grid((unsigned)A->ntiles, A->nb / kChunk);
  ProfScope ps(ctx, PROF_COV, 3.0 * A->ntiles * A->tile_elems, 8.0 * A->ntiles * A->tile_elems);
  k_cov_build<<<grid, kThreads, 0, ctx->stream>>>(L, A->n, A->nb, A->nt, sigma, rho, nug,
                                                 A->t64, A->d_partial);
  EMU_LAUNCHED(ctx);
  EMU_CUDA_TRY(ctx, cudaFreeAsync(buf, ctx->stream));
  return launch_precision_map(ctx, A, 0.0, nullptr, 0u, 0, EMU_MAP_NORM, 0.0);
}

emu_status launch_cov_tables(emu_ctx *ctx, const emu_cov_params *p, double *tables) {
  const int L = p->L;
  const size_t ntab = (size_t)(2 * L - 1) * (4 * L - 3);
  int blocks = (int)((ntab + 255) / 256);
  if (blocks > 4 * ctx->sm_count) blocks = 4 * ctx->sm_count;
  k_cov_tables<<<blocks, 256, 0, ctx->stream>>>(L, p->beta, p->sigma_exp, p->nugget_rel, tables + ntab, tables,
                                               tables + ntab + L);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_cov_norms(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p) {
  const int L = p->L;
  const size_t ntab = (size_t)(2 * L - 1) * (4 * L - 3);
  double *buf = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&buf, (ntab + L + 1) * sizeof(double), ctx->stream));
  emu_status s = launch_cov_tables(ctx, p, buf);
  if (s == EMU_OK) {
    dim3 grid((unsigned)A->ntiles, A->nb / kChunk);
    ProfScope ps(ctx, PROF_COV, 3.0 * A->ntiles * A->tile_elems, 0.0);
    k_cov_norms<<<grid, kThreads, 0, ctx->stream>>>(L, A->n, A->nb, A->nt, buf + ntab, buf, buf + ntab + L,
                                                   A->d_partial);
    EMU_LAUNCHED(ctx);
  }
  cudaFreeAsync(buf, ctx->stream);
  return s;
}

emu_status launch_cov_store_class(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p, const ClassArenas &ar) {
  const int L = p->L;
  const size_t ntab = (size_t)(2 * L - 1) * (4 * L - 3);
  double *buf = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&buf, (ntab + L + 1) * sizeof(double), ctx->stream));
  emu_status s = launch_cov_tables(ctx, p, buf);
  if (s == EMU_OK) {
    dim3 grid((unsigned)A->ntiles, A->nb / kChunk);
    ProfScope ps(ctx, PROF_COV, 3.0 * A->ntiles * A->tile_elems, 0.0);
    k_cov_store_class<<<grid, kThreads, 0, ctx->stream>>>(L, A->n, A->nb, A->nt, buf + ntab, buf, buf + ntab + L,
                                                         ar);
    EMU_LAUNCHED(ctx);
  }
  cudaFreeAsync(buf, ctx->stream);
  return s;
}

emu_status launch_import(emu_ctx *ctx, emu_mat *A, const double *dA, long lda) {
  dim3 grid((unsigned)A->ntiles, A->nb / kChunk);
  k_import<<<grid, kThreads, 0, ctx->stream>>>(A->n, A->nb, A->nt, dA, lda, A->t64,
                                              A->d_partial);
  EMU_LAUNCHED(ctx);
  return launch_precision_map(ctx, A, 0.0, nullptr, 0u, 0, EMU_MAP_NORM, 0.0);
}

emu_status launch_emp_finish(emu_ctx *ctx, emu_mat *A, long m, double nugget_rel, unsigned long long *d_maxbits) {
  const double inv_m = 1.0 / (double)m;
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(d_maxbits, 0, sizeof(unsigned long long), ctx->stream));
  k_emp_maxdiag<<<64, 256, 0, ctx->stream>>>(A->n, A->nb, A->nt, A->t64, inv_m, d_maxbits);
  EMU_LAUNCHED(ctx);
  dim3 grid((unsigned)A->ntiles, A->nb / kChunk);
  k_emp_finish<<<grid, kThreads, 0, ctx->stream>>>(A->n, A->nb, A->nt, inv_m, nugget_rel, d_maxbits, A->t64,
                                                  A->d_partial);
  EMU_LAUNCHED(ctx);
  return launch_precision_map(ctx, A, 0.0, nullptr, 0u, 0, EMU_MAP_NORM, 0.0);
}

emu_status launch_import_col(emu_ctx *ctx, emu_mat *A, int tj, const double *dS, long ld) {
  dim3 grid(A->nt - tj, A->nb / kChunk);
  k_import_col<<<grid, kThreads, 0, ctx->stream>>>(A->n, A->nb, A->nt, tj, dS, ld, A->t64, A->d_partial);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

// With u == nullptr only the norms and ||S||_F are (re)computed.
emu_status launch_precision_map(emu_ctx *ctx, emu_mat *A, double eps,
                                const double *u, unsigned mask, int diag_fp64, int band, double sp_frac) {
  ProfScope ps(ctx, PROF_MAP, 0.0, 8.0 * A->ntiles * (A->nchunk + 1));
  k_precision_map<<<1, 1024, 0, ctx->stream>>>(
      A->nt, A->ntiles, A->nchunk, A->d_partial, A->d_tnorm, A->d_frob,
      u ? A->d_cls : nullptr, eps, u ? u[1] : 0.0, u ? u[2] : 0.0,
      u ? u[3] : 0.0, u ? u[4] : 0.0, mask, diag_fp64, band, sp_frac, nullptr);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_cov_build_batch(emu_ctx *ctx, const BatchInst *d_inst, int count, int maxL, long ntab,
                                  const int *d_tile_inst, long ntiles, int nb, double *tables, double *t64,
                                  double *partial) {
  long per = (long)(2 * maxL - 1) * (4 * maxL - 3);
  int bx = (int)std::min<long>((per + 255) / 256, 64);
  k_cov_tables_batch<<<dim3(bx, count), 256, 0, ctx->stream>>>(d_inst, tables);
  EMU_LAUNCHED(ctx);
  (void)ntab;
  ProfScope ps(ctx, PROF_COV, 3.0 * ntiles * nb * nb, 8.0 * ntiles * nb * nb);
  k_cov_build_batch<<<dim3((unsigned)ntiles, nb / kChunk), kThreads, 0, ctx->stream>>>(d_inst, d_tile_inst, nb,
                                                                                       tables, t64, partial);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_precision_map_batch(emu_ctx *ctx, const BatchInst *d_inst, int count, int nb, double *partial,
                                      double *tnorm, double *frob, unsigned char *cls, double eps,
                                      const double *u, unsigned mask, int diag_fp64, int band, double sp_frac) {
  ProfScope ps(ctx, PROF_MAP, 0.0, 0.0);
  k_precision_map<<<count, 1024, 0, ctx->stream>>>(0, 0, nb / kChunk, partial, tnorm, frob, cls, eps,
                                                   u ? u[1] : 0.0, u ? u[2] : 0.0, u ? u[3] : 0.0,
                                                   u ? u[4] : 0.0, mask, diag_fp64, band, sp_frac, d_inst);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_export(emu_ctx *ctx, const emu_mat *A, double *dOut, long ld) {
  dim3 grid((unsigned)(A->nt * A->nt), A->nb / kChunk);
  bool mixed = A->state == MAT_FACTOR_MIXED;
  k_export<<<grid, kThreads, 0, ctx->stream>>>(A->n, A->nb, A->nt, A->t64,
                                              mixed ? A->t32 : nullptr,
                                              mixed ? A->d_cls : nullptr, dOut, ld);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_export_batch(emu_ctx *ctx, const BatchInst *d_inst, const int4 *d_pairs, long npairs, int nb,
                               const double *t64, const float *t32, const unsigned char *cls,
                               double *const *d_out) {
  if (npairs <= 0) return EMU_OK;
  k_export_batch<<<dim3((unsigned)npairs, nb / kChunk), kThreads, 0, ctx->stream>>>(d_inst, d_pairs, nb, t64, t32,
                                                                                    cls, d_out);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}
