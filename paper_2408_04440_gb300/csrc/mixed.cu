// mixed.cu -- adaptive per-tile precision tile Cholesky ("Mixed-Precision
// Computation Innovations"), its sampler and solves.
//
// Storage per tile (i,j) of class c (from the norm rule, precision_map):
//   c = FP64        : FP64 master in t64, updated by FP64 SIMT kernels.
//   c = FP32 / BF16 : FP32 master in t32, updated on the tensor cores
//                     (gemm_tc.cu) with FP32 accumulation.
// Diagonal tiles are factored by the FP64 POTRF whatever their class (their
// FP32 master is widened first); L_kk stays FP64 in t64.
// Sender-side conversion ("Performance of Mixed-Precision Cholesky on
// Summit"): the producer of a panel tile L_ik (the TRSM) writes it once as
// three BF16 pieces, row-major (K-major), in the operand arena `op`; every
// consumer reads the pieces its class needs (three for FP32, one for BF16).
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "gemm_tc.h"
#include "mixed.h"

namespace {

constexpr int B = 32;

__device__ inline bool failed(const int *st) { return *((volatile const int *)st) != DEV_OK; }

__device__ inline void split3(float x, uint16_t &p0, uint16_t &p1, uint16_t &p2) {
  __nv_bfloat16 b0 = __float2bfloat16_rn(x);
  float r1 = x - __bfloat162float(b0);
  __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  float r2 = r1 - __bfloat162float(b1);
  __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
  p0 = __bfloat16_as_ushort(b0);
  p1 = __bfloat16_as_ushort(b1);
  p2 = __bfloat16_as_ushort(b2);
}
__device__ inline void split3(double x, uint16_t &p0, uint16_t &p1, uint16_t &p2) {
  __nv_bfloat16 b0 = __double2bfloat16(x);
  double r1 = x - (double)__bfloat162float(b0);
  __nv_bfloat16 b1 = __double2bfloat16(r1);
  double r2 = r1 - (double)__bfloat162float(b1);
  __nv_bfloat16 b2 = __double2bfloat16(r2);
  p0 = __bfloat16_as_ushort(b0);
  p1 = __bfloat16_as_ushort(b1);
  p2 = __bfloat16_as_ushort(b2);
}

// FP32 masters of the low-precision tiles: t32 = (float) t64.
__global__ void k_to_f32(const double *__restrict__ t64, float *__restrict__ t32,
                         const unsigned char *__restrict__ cls, size_t tile_elems) {
  long t = blockIdx.y;
  if (cls[t] == EMU_CLASS_FP64) return;
  const double *s = t64 + (size_t)t * tile_elems;
  float *d = t32 + (size_t)t * tile_elems;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tile_elems;
       e += (size_t)gridDim.x * blockDim.x)
    d[e] = (float)s[e];
}

// Widen one FP32 master tile into the FP64 arena (before its POTRF).
__global__ void k_tile_to_f64(const float *__restrict__ s, double *__restrict__ d, size_t tile_elems,
                              const int *st) {
  if (failed(st)) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tile_elems;
       e += (size_t)gridDim.x * blockDim.x)
    d[e] = (double)s[e];
}

// FP32 copy of the FP64 diagonal factor tile L_kk for the FP32 panel TRSM
// (converted once here instead of by every TRSM CTA).
__global__ void k_diag_to_f32(const double *__restrict__ s, float *__restrict__ d, size_t tile_elems,
                              const int *st) {
  if (failed(st)) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tile_elems;
       e += (size_t)gridDim.x * blockDim.x)
    d[e] = (float)s[e];
}

// Three BF16 pieces, row-major, of whole tiles from their FP64 (or FP32)
// masters.  One CTA per (32x32 block, listed tile); lower_only zeroes the
// strict upper triangle (diagonal tiles).
template <typename T>
__global__ void k_split_tiles(const T *__restrict__ src, uint16_t *__restrict__ op, const int *__restrict__ tiles,
                              int nb, int lower_only, const int *st) {
  if (failed(st)) return;
  __shared__ T blk[B][B + 1];
  long t = tiles[blockIdx.y];
  int nbb = nb / B;
  int rb = blockIdx.x % nbb, cb = blockIdx.x / nbb;
  const T *s = src + (size_t)t * nb * nb;
  int tx = threadIdx.x % B, ty = threadIdx.x / B;  // 32 x 8
  for (int c = ty; c < B; c += 8) blk[tx][c] = s[(rb * B + tx) + (size_t)(cb * B + c) * nb];
  __syncthreads();
  size_t plane = (size_t)nb * nb;
  uint16_t *o = op + (size_t)t * 3 * plane;
  for (int r = ty; r < B; r += 8) {
    int gr = rb * B + r, gc = cb * B + tx;
    T x = blk[r][tx];
    if (lower_only && gr < gc) x = (T)0;
    uint16_t p0, p1, p2;
    split3(x, p0, p1, p2);
    size_t off = (size_t)gr * nb + gc;
    o[off] = p0;
    o[plane + off] = p1;
    o[2 * plane + off] = p2;
  }
}

// FP32 panel TRSM for the low-precision tiles of column k:
// L_ik = A_ik L_kk^{-T} from the FP32 master A_ik and the FP64 L_kk (read as
// FP32), written back to the master and, split, to the operand arena.
// One CTA per (32-row block, tile): the 32 rows stay in shared memory; for
// each 32-column block cb the already-solved columns are subtracted (a small
// GEMM against L_kk blocks staged in shared memory), then warp w solves rows
// 4w..4w+3 against the 32x32 diagonal block by forward substitution, one
// lane per column, with shuffles (no block-wide barrier inside the solve).
constexpr int TS_LD_PAD = 4;
constexpr int TS_STRIP = 512;  // columns of L_kk staged at once
__global__ void __launch_bounds__(256)
    k_trsm32_panel(const float *__restrict__ Lkk, float *__restrict__ t32, uint16_t *__restrict__ op, int nb,
                   int NT, int k, const int *__restrict__ rows, const int *st) {
  if (failed(st)) return;
  extern __shared__ float sm[];
  const int ldx = nb + TS_LD_PAD;
  const int lds = TS_STRIP + 1;
  float *X = sm;              // [32][ldx]: the CTA's rows of A_ik, solved in place
  float *S = X + 32 * ldx;    // [32][lds]: strip of L_kk rows cb*32 + lane, up to TS_STRIP columns
  int i = rows[blockIdx.y];
  int r0 = blockIdx.x * B;
  long ti = tile_index(i, k, NT);
  float *A = t32 + (size_t)ti * nb * nb + r0;
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int e = tid; e < 32 * nb; e += 256) {
    int r = e & 31, c = e >> 5;
    X[r * ldx + c] = A[r + (size_t)c * nb];
  }
  int nbb = nb / B;
  for (int cb = 0; cb < nbb; cb++) {
    const float *Lrow = Lkk + cb * B + lane;  // row cb*32 + lane of L_kk
    float ld[B];
#pragma unroll
    for (int p = 0; p < B; p++) ld[p] = (p <= lane) ? Lrow[(size_t)(cb * B + p) * nb] : 0.f;
    float acc[4];
    __syncthreads();  // X of the previous column blocks is complete
#pragma unroll
    for (int q = 0; q < 4; q++) acc[q] = X[(4 * w + q) * ldx + cb * B + lane];
    for (int p0 = 0; p0 < cb * B; p0 += TS_STRIP) {
      int pw = min(TS_STRIP, cb * B - p0);
      // the strip chunk: all loads issued together
      for (int p = w; p < pw; p += 8) S[lane * lds + p] = Lrow[(size_t)(p0 + p) * nb];
      __syncthreads();
#pragma unroll 4
      for (int p = 0; p < pw; p++) {
        float l = S[lane * lds + p];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] -= X[(4 * w + q) * ldx + p0 + p] * l;
      }
      __syncthreads();
    }
    float mydiag = ld[0];
#pragma unroll
    for (int p = 1; p < B; p++)
      if (p == lane) mydiag = ld[p];
    float myrinv = 1.0f / mydiag;
#pragma unroll
    for (int j = 0; j < B; j++) {
      float rj = __shfl_sync(0xffffffffu, myrinv, j);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        float xj = __shfl_sync(0xffffffffu, acc[q], j) * rj;
        if (lane == j) acc[q] = xj;
        if (lane > j) acc[q] -= xj * ld[j];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) X[(4 * w + q) * ldx + cb * B + lane] = acc[q];
  }
  __syncthreads();
  // FP32 master (column-major) and the sender-side BF16 pieces (row-major)
  for (int e = tid; e < 32 * nb; e += 256) {
    int r = e & 31, c = e >> 5;
    A[r + (size_t)c * nb] = X[r * ldx + c];
  }
  size_t plane = (size_t)nb * nb;
  uint16_t *P = op + (size_t)ti * 3 * plane + (size_t)r0 * nb;
  for (int e = tid; e < 32 * nb; e += 256) {
    int r = e / nb, c = e % nb;
    uint16_t p0, p1, p2;
    split3(X[r * ldx + c], p0, p1, p2);
    size_t off = (size_t)r * nb + c;
    P[off] = p0;
    P[plane + off] = p1;
    P[2 * plane + off] = p2;
  }
}

static size_t trsm32_smem(int nb) { return (size_t)(32 * (nb + TS_LD_PAD) + 32 * (TS_STRIP + 1)) * sizeof(float); }

// FP64-class trailing tiles: C_ij -= L_ik L_jk^T in FP64; each operand comes
// from the FP64 master or (widened) from the FP32 master, by its class.
constexpr int GM = 64, GK = 16;
__global__ void __launch_bounds__(256)
    k_update64_list(double *__restrict__ t64, const float *__restrict__ t32,
                    const unsigned char *__restrict__ cls, int nb, int NT, int k, const int2 *__restrict__ pairs,
                    const int *st) {
  if (failed(st)) return;
  int2 pr = pairs[blockIdx.x];
  int i = pr.x, j = pr.y;
  int nsub = nb / GM;
  int bi = blockIdx.y % nsub, bj = blockIdx.y / nsub;
  if (i == j && bi < bj) return;
  long tik = tile_index(i, k, NT), tjk = tile_index(j, k, NT);
  bool i64 = cls[tik] == EMU_CLASS_FP64, j64 = cls[tjk] == EMU_CLASS_FP64;
  size_t oi = (size_t)tik * nb * nb + bi * GM, oj = (size_t)tjk * nb * nb + bj * GM;
  double *C = t64 + (size_t)tile_index(i, j, NT) * nb * nb + bi * GM + (size_t)bj * GM * nb;
  __shared__ double as[GK][GM];
  __shared__ double bs[GK][GM];
  int t = threadIdx.x, tx = t % 16, ty = t / 16;
  int lc = t / 16, lr = (t % 16) * 4;
  double acc[4][4] = {};
  for (int p0 = 0; p0 < nb; p0 += GK) {
#pragma unroll
    for (int e = 0; e < 4; e++) {
      size_t o = (lr + e) + (size_t)(p0 + lc) * nb;
      as[lc][lr + e] = i64 ? t64[oi + o] : (double)t32[oi + o];
      bs[lc][lr + e] = j64 ? t64[oj + o] : (double)t32[oj + o];
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

// z pieces for the sampler: zp[q][n][k] = piece q of Z[k][n], n < s_pad
// (zero beyond s).
__global__ void k_split_z(const double *__restrict__ Z, long ldz, long npad, int s, int s_pad,
                          uint16_t *__restrict__ zp) {
  long total = npad * (long)s_pad;
  size_t plane = (size_t)s_pad * npad;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    long k = q % npad;
    int n = (int)(q / npad);
    double x = (n < s) ? Z[k + (size_t)n * ldz] : 0.0;
    uint16_t p0, p1, p2;
    split3(x, p0, p1, p2);
    zp[q] = p0;
    zp[plane + q] = p1;
    zp[2 * plane + q] = p2;
  }
}

// ---------------------------------------------- FP32 triangular solves
// Tile element (r, c) of a factor tile in FP32: diagonal and FP64-class tiles
// from t64, others from the FP32 master.
__device__ inline float ftile(const double *t64, const float *t32, const unsigned char *cls, long t, int nb,
                              int r, int c, bool diag) {
  size_t o = (size_t)t * nb * nb + r + (size_t)c * nb;
  return (diag || cls[t] == EMU_CLASS_FP64) ? (float)t64[o] : t32[o];
}

__global__ void k_solve32_update(const double *__restrict__ t64, const float *__restrict__ t32,
                                 const unsigned char *__restrict__ cls, int nb, int NT, int k, int backward,
                                 double *__restrict__ X, long ldx) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (r >= nb) return;
  float acc = 0.f;
  if (!backward) {
    for (int j = 0; j < k; j++) {
      long t = tile_index(k, j, NT);
      const double *xj = X + (size_t)j * nb + (size_t)c * ldx;
      for (int p = 0; p < nb; p++) acc += ftile(t64, t32, cls, t, nb, r, p, false) * (float)xj[p];
    }
  } else {
    for (int i = k + 1; i < NT; i++) {
      long t = tile_index(i, k, NT);
      const double *xi = X + (size_t)i * nb + (size_t)c * ldx;
      for (int p = 0; p < nb; p++) acc += ftile(t64, t32, cls, t, nb, p, r, false) * (float)xi[p];
    }
  }
  X[(size_t)k * nb + r + (size_t)c * ldx] -= (double)acc;
}

__global__ void k_solve32_diag(const double *__restrict__ t64, int nb, int NT, int k, int backward,
                               double *__restrict__ X, long ldx) {
  extern __shared__ float xs[];
  __shared__ float red[32];
  int c = blockIdx.x;
  const double *D = t64 + (size_t)tile_index(k, k, NT) * nb * nb;
  double *x = X + (size_t)k * nb + (size_t)c * ldx;
  for (int r = threadIdx.x; r < nb; r += blockDim.x) xs[r] = (float)x[r];
  __syncthreads();
  if (!backward) {
    for (int p = 0; p < nb; p++) {
      float xp = xs[p] / (float)D[p + (size_t)p * nb];
      __syncthreads();
      if (threadIdx.x == 0) xs[p] = xp;
      for (int r = p + 1 + threadIdx.x; r < nb; r += blockDim.x) xs[r] -= (float)D[r + (size_t)p * nb] * xp;
      __syncthreads();
    }
  } else {
    for (int p = nb - 1; p >= 0; p--) {
      float part = 0.f;
      for (int r = p + 1 + threadIdx.x; r < nb; r += blockDim.x) part += (float)D[r + (size_t)p * nb] * xs[r];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        float sum = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) sum += red[w];
        xs[p] = (xs[p] - sum) / (float)D[p + (size_t)p * nb];
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < nb; r += blockDim.x) x[r] = (double)xs[r];
}

}  // namespace

// ------------------------------------------------------------------ plan
struct MixedPlan {
  int NT = 0, nb = 0;
  std::vector<unsigned char> cls;  // packed by tile index
  // per step k: offsets into the concatenated device lists
  std::vector<int> off_t64rows, off_t32rows, off_pairs, off_items;
  std::vector<int> g1_pairs, g1_items;  // leading entries of a step that update column k+1
  std::vector<int> diag_low;       // class(k,k) != FP64
  std::vector<double> step_flops, step_mma;  // tensor-core work of each step
  int *d_rows64 = nullptr, *d_rows32 = nullptr;
  int2 *d_pairs = nullptr;
  gemm_tc::Item *d_items = nullptr;
  gemm_tc::Seg *d_segs = nullptr;
  int *d_tiles_fp64_panel = nullptr;  // FP64-class off-diagonal tiles (split after their TRSM)
  int *d_diag_tiles = nullptr;        // all diagonal tiles (split after the factor)
  float *d_lkk32 = nullptr;           // FP32 copy of the current L_kk
  CUtensorMap mapA, mapB;
  double update_flops[EMU_NCLASS] = {};
  int tiles[EMU_NCLASS] = {};
};

static void plan_free(MixedPlan *p) {
  if (!p) return;
  cudaFree(p->d_rows64);
  cudaFree(p->d_rows32);
  cudaFree(p->d_pairs);
  cudaFree(p->d_items);
  cudaFree(p->d_segs);
  cudaFree(p->d_tiles_fp64_panel);
  cudaFree(p->d_diag_tiles);
  cudaFree(p->d_lkk32);
  delete p;
}

void mixed_mat_release(emu_mat *A) {
  plan_free(static_cast<MixedPlan *>(A->plan));
  A->plan = nullptr;
}

template <typename T>
static emu_status upload(emu_ctx *ctx, T **dst, const std::vector<T> &v) {
  size_t n = v.empty() ? 1 : v.size();
  EMU_CUDA_TRY(ctx, cudaMalloc(dst, n * sizeof(T)));
  if (!v.empty()) EMU_CUDA_TRY(ctx, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return EMU_OK;
}

static emu_status build_plan(emu_ctx *ctx, emu_mat *A, MixedPlan *P) {
  int NT = A->nt, nb = A->nb;
  P->NT = NT;
  P->nb = nb;
  P->cls.assign(A->h_cls, A->h_cls + A->ntiles);
  auto C = [&](int i, int j) { return (int)P->cls[tile_index(i, j, NT)]; };
  std::vector<int> rows64, rows32, fp64panel, diag;
  std::vector<int2> pairs;
  std::vector<gemm_tc::Item> items;
  std::vector<gemm_tc::Seg> segs;
  double nb3 = (double)nb * nb * nb;
  for (int j = 0; j < NT; j++)
    for (int i = j; i < NT; i++) {
      int c = C(i, j);
      P->tiles[c]++;
      P->update_flops[c] += (i == j ? 1.0 : 2.0) * j * nb3 + (i > j ? nb3 : 0.0);
    }
  for (int k = 0; k < NT; k++) {
    diag.push_back((int)tile_index(k, k, NT));
    P->diag_low.push_back(C(k, k) != EMU_CLASS_FP64);
    P->off_t64rows.push_back((int)rows64.size());
    P->off_t32rows.push_back((int)rows32.size());
    P->off_pairs.push_back((int)pairs.size());
    P->off_items.push_back((int)items.size());
    double sf = 0.0, sm = 0.0;
    int g1p = 0, g1i = 0;
    for (int i = k + 1; i < NT; i++) {
      if (C(i, k) == EMU_CLASS_FP64) {
        rows64.push_back(i);
        fp64panel.push_back((int)tile_index(i, k, NT));
      } else {
        rows32.push_back(i);
      }
    }
    // trailing tiles, ordered by column j then row i
    for (int j = k + 1; j < NT; j++)
      for (int i = j; i < NT; i++) {
        int c = C(i, j);
        if (c == EMU_CLASS_FP64) {
          pairs.push_back(make_int2(i, j));
          if (j == k + 1) g1p++;
          continue;
        }
        int cc = (c == EMU_CLASS_FP32) ? EMU_CLASS_FP32 : EMU_CLASS_BF16;  // TF32/E4M3 fall back
        for (int nbk = 0; nbk < nb / gemm_tc::BN; nbk++)
          for (int mb = 0; mb < nb / gemm_tc::BM; mb++) {
            if (i == j && mb * gemm_tc::BM + gemm_tc::BM - 1 < nbk * gemm_tc::BN) continue;  // above diagonal
            gemm_tc::Seg s;
            s.ax = 0;
            s.ay = (int)(tile_index(i, k, NT) * 3 * nb + mb * gemm_tc::BM);
            s.ay_step = nb;
            s.bx = 0;
            s.by = (int)(tile_index(j, k, NT) * 3 * nb + nbk * gemm_tc::BN);
            s.by_step = nb;
            s.cls = cc;
            s.pad = 0;
            gemm_tc::Item it;
            it.seg_begin = (int)segs.size();
            segs.push_back(s);
            it.seg_end = (int)segs.size();
            it.out_off = tile_index(i, j, NT) * (long)nb * nb + mb * gemm_tc::BM + (long)nbk * gemm_tc::BN * nb;
            it.rows_valid = gemm_tc::BM;
            it.cols_valid = gemm_tc::BN;
            items.push_back(it);
            double f = 2.0 * gemm_tc::BM * gemm_tc::BN * nb;
            sf += f;
            sm += f * (cc == EMU_CLASS_FP32 ? 6.0 : 1.0);
            if (j == k + 1) g1i++;
          }
      }
    P->g1_pairs.push_back(g1p);
    P->g1_items.push_back(g1i);
    P->step_flops.push_back(sf);
    P->step_mma.push_back(sm);
  }
  P->off_t64rows.push_back((int)rows64.size());
  P->off_t32rows.push_back((int)rows32.size());
  P->off_pairs.push_back((int)pairs.size());
  P->off_items.push_back((int)items.size());
  emu_status s;
  if ((s = upload(ctx, &P->d_rows64, rows64)) != EMU_OK) return s;
  if ((s = upload(ctx, &P->d_rows32, rows32)) != EMU_OK) return s;
  if ((s = upload(ctx, &P->d_pairs, pairs)) != EMU_OK) return s;
  if ((s = upload(ctx, &P->d_items, items)) != EMU_OK) return s;
  if ((s = upload(ctx, &P->d_segs, segs)) != EMU_OK) return s;
  if ((s = upload(ctx, &P->d_tiles_fp64_panel, fp64panel)) != EMU_OK) return s;
  if ((s = upload(ctx, &P->d_diag_tiles, diag)) != EMU_OK) return s;
  EMU_CUDA_TRY(ctx, cudaMalloc(&P->d_lkk32, (size_t)nb * nb * sizeof(float)));
  uint64_t rows = (uint64_t)A->ntiles * 3 * nb;
  if ((s = gemm_tc::make_map_bf16(ctx, &P->mapA, A->op_bf16, nb, rows, gemm_tc::BM)) != EMU_OK) return s;
  if ((s = gemm_tc::make_map_bf16(ctx, &P->mapB, A->op_bf16, nb, rows, gemm_tc::BN)) != EMU_OK) return s;
  return EMU_OK;
}

// Internal streams of the mixed schedule (created once per context) and at
// least `nev` ordering events.
static emu_status sched_streams(emu_ctx *ctx, int nev) {
  if (!ctx->crit) {
    int least = 0, greatest = 0;
    EMU_CUDA_TRY(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    EMU_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&ctx->crit, cudaStreamNonBlocking, greatest));
    EMU_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&ctx->bulk, cudaStreamNonBlocking, least));
  }
  while ((int)ctx->sched_ev.size() < nev) {
    cudaEvent_t e;
    EMU_CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->sched_ev.push_back(e);
  }
  return EMU_OK;
}

emu_status factor_mixed(emu_ctx *ctx, emu_mat *A, const emu_mp_opts *o) {
  int NT = A->nt, nb = A->nb;
  if (nb % gemm_tc::BN != 0) {
    ctx->last_error = "the mixed-precision factor needs nb to be a multiple of 256";
    return EMU_EINVAL;
  }
  double u[EMU_NCLASS] = {0x1p-53, 0x1p-24, 0x1p-11, 0x1p-8, 0x1p-4};
  for (int c = 0; c < EMU_NCLASS; c++)
    if (o->u[c] > 0.0) u[c] = o->u[c];
  // TF32 and E4M3 classes are not built on the tensor cores yet: leave them out
  unsigned mask = (o->prec_mask | 1u) & ((1u << EMU_CLASS_FP32) | (1u << EMU_CLASS_BF16) | 1u);
  emu_status s = launch_precision_map(ctx, A, o->eps, u, mask, o->diag_fp64);
  if (s != EMU_OK) return s;
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(A->h_cls, A->d_cls, A->ntiles, cudaMemcpyDeviceToHost, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(&A->frob, A->d_frob, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  size_t te = A->tile_elems;
  if (!A->t32) EMU_CUDA_TRY(ctx, cudaMallocAsync(&A->t32, (size_t)A->ntiles * te * sizeof(float), ctx->stream));
  if (!A->op_bf16)
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&A->op_bf16, (size_t)A->ntiles * 3 * te * sizeof(uint16_t), ctx->stream));
  mixed_mat_release(A);
  MixedPlan *P = new MixedPlan();
  A->plan = P;
  if ((s = build_plan(ctx, A, P)) != EMU_OK) return s;

  int *st = ctx->d_status;
  double nb3 = (double)nb * nb * nb;
  {
    ProfScope ps(ctx, PROF_SPLIT, 0.0, 12.0 * A->ntiles * te);
    k_to_f32<<<dim3(64, (unsigned)A->ntiles), 256, 0, ctx->stream>>>(A->t64, A->t32, A->d_cls, te);
    EMU_LAUNCHED(ctx);
  }
  // Lookahead-1 schedule.  Critical stream: POTRF(k), TRSM(:,k), then the
  // update of column k+1 by panel k (G1), which feeds POTRF(k+1).  Bulk
  // stream: the update of columns >= k+2 by panel k (G2), overlapping the
  // next panel.  G1(k) must not overlap G2(k-1) (both write column k+1).
  cudaStream_t user = ctx->stream;
  if ((s = sched_streams(ctx, 2 * NT + 2)) != EMU_OK) return s;
  cudaEvent_t ev_start = ctx->sched_ev[2 * NT], ev_bulk_end = ctx->sched_ev[2 * NT + 1];
  EMU_CUDA_TRY(ctx, cudaEventRecord(ev_start, user));
  EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev_start, 0));
  EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->bulk, ev_start, 0));
  for (int k = 0; k < NT; k++) {
    cudaEvent_t ev_trsm = ctx->sched_ev[2 * k], ev_g2 = ctx->sched_ev[2 * k + 1];
    long tkk = tile_index(k, k, NT);
    ctx->stream = ctx->crit;
    if (P->diag_low[k]) {
      ProfScope ps(ctx, PROF_SPLIT, 0.0, 12.0 * te);
      k_tile_to_f64<<<64, 256, 0, ctx->stream>>>(A->t32 + tkk * te, A->t64 + tkk * te, te, st);
      EMU_LAUNCHED(ctx);
    }
    if ((s = launch_potrf64_tile(ctx, A, k)) != EMU_OK) break;
    int n64 = P->off_t64rows[k + 1] - P->off_t64rows[k];
    int n32 = P->off_t32rows[k + 1] - P->off_t32rows[k];
    if (n64 > 0) {
      if ((s = launch_trsm64_panel(ctx, A, k, P->d_rows64 + P->off_t64rows[k], n64)) != EMU_OK) break;
      ProfScope ps(ctx, PROF_SPLIT, 0.0, 14.0 * n64 * te);
      k_split_tiles<double><<<dim3((nb / B) * (nb / B), n64), 256, 0, ctx->stream>>>(
          A->t64, A->op_bf16, P->d_tiles_fp64_panel + P->off_t64rows[k], nb, 0, st);
      EMU_LAUNCHED(ctx);
    }
    if (n32 > 0) {
      ProfScope ps(ctx, PROF_TRSM32, n32 * nb3, 14.0 * n32 * te);
      k_diag_to_f32<<<2 * ctx->sm_count, 256, 0, ctx->stream>>>(A->t64 + tkk * te, P->d_lkk32, te, st);
      EMU_LAUNCHED(ctx);
      size_t sm = trsm32_smem(nb);
      EMU_CUDA_TRY(ctx, cudaFuncSetAttribute(k_trsm32_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_trsm32_panel<<<dim3(nb / B, n32), 256, sm, ctx->stream>>>(P->d_lkk32, A->t32, A->op_bf16, nb, NT, k,
                                                                  P->d_rows32 + P->off_t32rows[k], st);
      EMU_LAUNCHED(ctx);
    }
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev_trsm, ctx->crit));
    if (k > 0) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ctx->sched_ev[2 * (k - 1) + 1], 0));
    int p0 = P->off_pairs[k], np = P->off_pairs[k + 1] - p0, np1 = P->g1_pairs[k];
    int i0 = P->off_items[k], ni = P->off_items[k + 1] - i0, ni1 = P->g1_items[k];
    // G1 on the critical stream, G2 on the bulk stream
    for (int part = 0; part < 2 && s == EMU_OK; part++) {
      ctx->stream = part == 0 ? ctx->crit : ctx->bulk;
      if (part == 1) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->bulk, ev_trsm, 0));
      int pb = part == 0 ? p0 : p0 + np1, pn = part == 0 ? np1 : np - np1;
      int ib = part == 0 ? i0 : i0 + ni1, in = part == 0 ? ni1 : ni - ni1;
      if (pn > 0) {
        ProfScope ps(ctx, PROF_UPDATE64, 2.0 * pn * nb3, 24.0 * pn * te);
        k_update64_list<<<dim3(pn, (nb / GM) * (nb / GM)), 256, 0, ctx->stream>>>(A->t64, A->t32, A->d_cls, nb, NT,
                                                                                 k, P->d_pairs + pb, st);
        EMU_LAUNCHED(ctx);
      }
      if (in > 0) {
        double fr = (double)in / ni;
        ProfScope ps(ctx, PROF_TC_FACTOR, P->step_flops[k] * fr, 0.0, P->step_mma[k] * fr);
        // short-lived CTAs on the bulk stream (at most 4 items each) let the
        // critical stream's CTAs take SMs as they free up
        int ctas = part == 0 ? ctx->sm_count : std::max(1, (in + 3) / 4);
        s = gemm_tc::launch(ctx, P->mapA, P->mapB, P->d_items + ib, in, P->d_segs, nb / gemm_tc::BK,
                            gemm_tc::TC_SUB_F32, A->t32, nullptr, nb, ctas);
      }
    }
    if (s != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev_g2, ctx->bulk));
  }
  ctx->stream = user;
  if (s != EMU_OK) return s;
  EMU_CUDA_TRY(ctx, cudaEventRecord(ev_bulk_end, ctx->bulk));
  EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev_bulk_end, 0));
  EMU_CUDA_TRY(ctx, cudaEventRecord(ev_bulk_end, ctx->crit));
  EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(user, ev_bulk_end, 0));
  if ((s = launch_tril_diag(ctx, A)) != EMU_OK) return s;
  // pieces of the (lower-triangular) diagonal factor tiles, for the sampler
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 14.0 * NT * te);
  k_split_tiles<double><<<dim3((nb / B) * (nb / B), NT), 256, 0, ctx->stream>>>(A->t64, A->op_bf16,
                                                                               P->d_diag_tiles, nb, 1, st);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

void mixed_fill_info(const emu_mat *A, emu_factor_info *info) {
  const MixedPlan *P = static_cast<const MixedPlan *>(A->plan);
  info->frob = A->frob;
  if (!P) return;
  for (int c = 0; c < EMU_NCLASS; c++) {
    info->tiles[c] = P->tiles[c];
    info->update_flops[c] = P->update_flops[c];
  }
}

// Y = L Z: FP64-class tiles on the FP64 pipe (this also initialises Y), the
// FP32/BF16-class tiles on the tensor cores accumulated in FP32 per output
// block over k in a fixed order, then added to Y.
emu_status mixed_sample(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz, int s, double *Y, long ldy) {
  const MixedPlan *P = static_cast<const MixedPlan *>(L->plan);
  if (!P) return EMU_ESTATE;
  int NT = L->nt, nb = L->nb;
  long npad = (long)NT * nb;
  int s_pad = ((s + gemm_tc::BN - 1) / gemm_tc::BN) * gemm_tc::BN;
  emu_status st = launch_trmm64(ctx, L, Z, ldz, s, Y, ldy, L->d_cls);
  if (st != EMU_OK) return st;
  std::vector<gemm_tc::Item> items;
  std::vector<gemm_tc::Seg> segs;
  for (int i = 0; i < NT; i++)
    for (int nbk = 0; nbk < s_pad / gemm_tc::BN; nbk++)
      for (int mb = 0; mb < nb / gemm_tc::BM; mb++) {
        long row0 = (long)i * nb + mb * gemm_tc::BM;
        if (row0 >= L->n) continue;
        gemm_tc::Item it;
        it.seg_begin = (int)segs.size();
        for (int k = 0; k <= i; k++) {
          int c = P->cls[tile_index(i, k, NT)];
          if (c == EMU_CLASS_FP64) continue;
          gemm_tc::Seg sg;
          sg.ax = 0;
          sg.ay = (int)(tile_index(i, k, NT) * 3 * nb + mb * gemm_tc::BM);
          sg.ay_step = nb;
          sg.bx = k * nb;
          sg.by = nbk * gemm_tc::BN;
          sg.by_step = s_pad;
          sg.cls = (c == EMU_CLASS_FP32) ? EMU_CLASS_FP32 : EMU_CLASS_BF16;
          sg.pad = 0;
          segs.push_back(sg);
        }
        it.seg_end = (int)segs.size();
        if (it.seg_end == it.seg_begin) continue;
        it.out_off = row0 + (long)nbk * gemm_tc::BN * ldy;
        it.rows_valid = (int)std::min<long>(gemm_tc::BM, L->n - row0);
        it.cols_valid = s - nbk * gemm_tc::BN;
        items.push_back(it);
      }
  if (items.empty()) return EMU_OK;
  uint16_t *zp = nullptr;
  gemm_tc::Item *d_items = nullptr;
  gemm_tc::Seg *d_segs = nullptr;
  size_t zbytes = (size_t)3 * s_pad * npad * sizeof(uint16_t);
  size_t ibytes = items.size() * sizeof(gemm_tc::Item), sbytes = segs.size() * sizeof(gemm_tc::Seg);
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&zp, zbytes, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_items, ibytes, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_segs, sbytes, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_items, items.data(), ibytes, cudaMemcpyHostToDevice, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_segs, segs.data(), sbytes, cudaMemcpyHostToDevice, ctx->stream));
  {
    ProfScope ps(ctx, PROF_SPLIT, 0.0, 14.0 * npad * s_pad);
    k_split_z<<<8 * ctx->sm_count, 256, 0, ctx->stream>>>(Z, ldz, npad, s, s_pad, zp);
    EMU_LAUNCHED(ctx);
  }
  double tf = 0.0, tm = 0.0;
  for (const gemm_tc::Item &it : items)
    for (int q = it.seg_begin; q < it.seg_end; q++) {
      double f = 2.0 * gemm_tc::BM * gemm_tc::BN * nb;
      tf += f;
      tm += f * (segs[q].cls == EMU_CLASS_FP32 ? 6.0 : 1.0);
    }
  CUtensorMap mapB;
  st = gemm_tc::make_map_bf16(ctx, &mapB, zp, npad, (uint64_t)3 * s_pad, gemm_tc::BN);
  ProfScope ps(ctx, PROF_TC_SAMPLE, tf, 0.0, tm);
  if (st == EMU_OK)
    st = gemm_tc::launch(ctx, P->mapA, mapB, d_items, (int)items.size(), d_segs, nb / gemm_tc::BK,
                         gemm_tc::TC_ADD_F64, nullptr, Y, (int)ldy, ctx->sm_count);
  cudaFreeAsync(zp, ctx->stream);
  cudaFreeAsync(d_items, ctx->stream);
  cudaFreeAsync(d_segs, ctx->stream);
  // the host vectors above must outlive the asynchronous copies
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return st;
}

emu_status mixed_potrs(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs) {
  int nb = L->nb, NT = L->nt;
  int thr = 256;
  ProfScope ps(ctx, PROF_SOLVE, 2.0 * L->n * L->n * nrhs, 0.0);
  for (int k = 0; k < NT; k++) {
    if (k > 0) {
      k_solve32_update<<<dim3((nb + thr - 1) / thr, nrhs), thr, 0, ctx->stream>>>(L->t64, L->t32, L->d_cls, nb, NT,
                                                                                 k, 0, X, ldx);
      EMU_LAUNCHED(ctx);
    }
    k_solve32_diag<<<nrhs, 512, nb * sizeof(float), ctx->stream>>>(L->t64, nb, NT, k, 0, X, ldx);
    EMU_LAUNCHED(ctx);
  }
  for (int k = NT - 1; k >= 0; k--) {
    if (k < NT - 1) {
      k_solve32_update<<<dim3((nb + thr - 1) / thr, nrhs), thr, 0, ctx->stream>>>(L->t64, L->t32, L->d_cls, nb, NT,
                                                                                 k, 1, X, ldx);
      EMU_LAUNCHED(ctx);
    }
    k_solve32_diag<<<nrhs, 512, nb * sizeof(float), ctx->stream>>>(L->t64, nb, NT, k, 1, X, ldx);
    EMU_LAUNCHED(ctx);
  }
  return EMU_OK;
}

void mixed_ctx_release(emu_ctx *ctx) {
  for (cudaEvent_t e : ctx->sched_ev) cudaEventDestroy(e);
  ctx->sched_ev.clear();
  if (ctx->crit) cudaStreamDestroy(ctx->crit);
  if (ctx->bulk) cudaStreamDestroy(ctx->bulk);
  ctx->crit = ctx->bulk = nullptr;
}
