// refine.cu -- iterative refinement for S X = B: the correction comes from the
// (possibly mixed-precision) factor, the residual R = B - S X and the update
// X += D are FP64 against the FP64 covariance tiles.  Stops when the normwise
// backward error ||r||_2 / (||S||_F ||x||_2 + ||b||_2) of every column is <= tol.
#include <math.h>

#include <vector>

#include "mixed.h"

namespace {

// R[:, c0:c0+P] = B - S X for S symmetric from its packed lower FP64 tiles,
// FP64 on the SIMT pipes: one CTA per (64-row slab of the padded matrix,
// group of P right-hand sides), a loop over every tile column j of the slab's
// block row i (tile (i, j) for j <= i, tile (j, i) read transposed for
// j > i), operands staged through shared memory in 32-wide K chunks so that
// every global read is coalesced.  Deterministic: one CTA owns each output.
constexpr int RS = 64, RK = 32;
template <int P>
__global__ void __launch_bounds__(256)
    k_symm_res(const double *__restrict__ t64, int nb, int NT, const double *__restrict__ X,
               const double *__restrict__ Bm, double *__restrict__ R, long ld, int nrhs) {
  constexpr int NQ = P / 4;  // right-hand sides per thread
  __shared__ double a[RK][RS + 1];
  __shared__ double x[RK][P + 1];
  const long g0 = (long)blockIdx.x * RS;
  const int i = (int)(g0 / nb), m0 = (int)(g0 % nb);
  const int c0 = blockIdx.y * P;
  const int p = min(P, nrhs - c0);
  const int tid = threadIdx.x, mm = tid & (RS - 1), q0 = tid >> 6;
  double acc[NQ];
#pragma unroll
  for (int w = 0; w < NQ; w++) acc[w] = 0.0;
  for (int j = 0; j < NT; j++) {
    const bool lower = j <= i;
    const double *T = t64 + (size_t)(lower ? tile_index(i, j, NT) : tile_index(j, i, NT)) * nb * nb;
    for (int k0 = 0; k0 < nb; k0 += RK) {
      for (int e = tid; e < RK * RS; e += 256) {
        if (lower) {
          const int m = e % RS, k = e / RS;
          a[k][m] = T[(size_t)(m0 + m) + (size_t)(k0 + k) * nb];
        } else {
          const int k = e % RK, m = e / RK;
          a[k][m] = T[(size_t)(k0 + k) + (size_t)(m0 + m) * nb];
        }
      }
      for (int e = tid; e < RK * P; e += 256) {
        const int k = e % RK, q = e / RK;
        x[k][q] = q < p ? X[(size_t)j * nb + k0 + k + (size_t)(c0 + q) * ld] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < RK; k++) {
        const double av = a[k][mm];
#pragma unroll
        for (int w = 0; w < NQ; w++) acc[w] = fma(av, x[k][q0 + 4 * w], acc[w]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int w = 0; w < NQ; w++) {
    const int q = q0 + 4 * w;
    if (q < p) {
      const size_t o = (size_t)(g0 + mm) + (size_t)(c0 + q) * ld;
      R[o] = Bm[o] - acc[w];
    }
  }
}

// Column sums of squares of R, X and B (one CTA per column, fixed order).
__global__ void k_col_norms(const double *__restrict__ R, const double *__restrict__ X,
                            const double *__restrict__ Bm, long n, long ld, double *__restrict__ out) {
  int c = blockIdx.x;
  double sr = 0, sx = 0, sb = 0;
  for (long r = threadIdx.x; r < n; r += blockDim.x) {
    double a = R[r + c * ld], b = X[r + c * ld], d = Bm[r + c * ld];
    sr += a * a;
    sx += b * b;
    sb += d * d;
  }
  __shared__ double sh[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    sx += __shfl_down_sync(0xffffffffu, sx, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
  }
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = sr;
    sh[1][w] = sx;
    sh[2][w] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, d = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
      a += sh[0][k];
      b += sh[1][k];
      d += sh[2][k];
    }
    out[3 * c] = a;
    out[3 * c + 1] = b;
    out[3 * c + 2] = d;
  }
}

__global__ void k_axpy(double *__restrict__ X, const double *__restrict__ D, long total) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x)
    X[q] += D[q];
}

}  // namespace

static emu_status solve_with_factor(emu_ctx *ctx, const emu_mat *L, double *X, long ld, int nrhs) {
  if (L->state == MAT_FACTOR64) return launch_potrs64(ctx, L, X, ld, nrhs);
  return mixed_potrs(ctx, L, X, ld, nrhs);
}

emu_status refine_solve(emu_ctx *ctx, const emu_mat *L, const emu_mat *S, const double *dB,
                        long ldb, double *dX, long ldx, int nrhs, double tol, int maxit,
                        emu_refine_info *info) {
  if (nrhs == 0) return EMU_OK;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  int NT = L->nt, nb = L->nb;
  long npad = (long)NT * nb;
  size_t blk = (size_t)npad * nrhs;
  double *buf = nullptr, *norms = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&buf, 4 * blk * sizeof(double), ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&norms, 3 * nrhs * sizeof(double), ctx->stream));
  double *Bp = buf, *X = buf + blk, *R = buf + 2 * blk, *D = buf + 3 * blk;
  std::vector<double> hn(3 * nrhs);
  double frobS = 0.0;
  emu_status s = EMU_OK;
  int it = 0;
  double eta = INFINITY;
  float ms = 0.f;
  cudaError_t e = cudaMemsetAsync(buf, 0, 4 * blk * sizeof(double), ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(Bp, npad * sizeof(double), dB, ldb * sizeof(double), (size_t)L->n * sizeof(double),
                          nrhs, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&frobS, S->d_frob, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev0, ctx->stream);
  if (e != cudaSuccess) s = emu_cuda_fail(ctx, e, "refine setup");
  // X0 = M^{-1} B
  if (s == EMU_OK) {
    e = cudaMemcpyAsync(X, Bp, blk * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
    s = (e == cudaSuccess) ? solve_with_factor(ctx, L, X, npad, nrhs) : emu_cuda_fail(ctx, e, "refine x0");
  }
  while (s == EMU_OK) {
    {
      ProfScope ps(ctx, PROF_SOLVE, 2.0 * (double)npad * npad * nrhs, 8.0 * (double)npad * npad);
      if (nrhs <= 16)
        k_symm_res<16><<<dim3((unsigned)(npad / RS), 1), 256, 0, ctx->stream>>>(S->t64, nb, NT, X, Bp, R, npad,
                                                                                nrhs);
      else
        k_symm_res<32><<<dim3((unsigned)(npad / RS), (nrhs + 31) / 32), 256, 0, ctx->stream>>>(S->t64, nb, NT, X,
                                                                                              Bp, R, npad, nrhs);
    }
    ctx->launches++;
    k_col_norms<<<nrhs, 256, 0, ctx->stream>>>(R, X, Bp, npad, npad, norms);
    ctx->launches++;
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hn.data(), norms, 3 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      s = emu_cuda_fail(ctx, e, "refine residual");
      break;
    }
    eta = 0.0;
    for (int c = 0; c < nrhs; c++) {
      double den = frobS * sqrt(hn[3 * c + 1]) + sqrt(hn[3 * c + 2]);
      double v = den > 0 ? sqrt(hn[3 * c]) / den : 0.0;
      if (!(v <= eta)) eta = v;  // NaN propagates
    }
    if (eta <= tol) break;
    if (it >= maxit) {
      s = EMU_ENOCONV;
      break;
    }
    e = cudaMemcpyAsync(D, R, blk * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) {
      s = emu_cuda_fail(ctx, e, "refine copy");
      break;
    }
    s = solve_with_factor(ctx, L, D, npad, nrhs);
    if (s != EMU_OK) break;
    k_axpy<<<4 * ctx->sm_count, 256, 0, ctx->stream>>>(X, D, (long)blk);
    ctx->launches++;
    it++;
  }
  cudaEventRecord(ctx->ev1, ctx->stream);
  if (s == EMU_OK || s == EMU_ENOCONV) {
    e = cudaMemcpy2DAsync(dX, ldx * sizeof(double), X, npad * sizeof(double), (size_t)L->n * sizeof(double),
                          nrhs, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) s = emu_cuda_fail(ctx, e, "refine copy-out");
  }
  cudaFreeAsync(buf, ctx->stream);
  cudaFreeAsync(norms, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  if (info) {
    info->iters = it;
    info->rel_resid = eta;
    info->ms = ms;
  }
  return s;
}
