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
#include <cuda_fp8.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "gemm_f64.h"
#include "gemm_tc.h"
#include "mixed.h"
#include "trsm_tc.h"

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

// TF32 copies of listed panel tiles for the TF32-class updates: each
// element's FP32 value, rebuilt exactly from its three BF16 pieces (they split
// the FP32 master exactly), rounded to TF32 (cvt.rna: nearest, ties away from
// zero), row-major like the pieces.  blockIdx.y splits a tile into parts.
__global__ void k_tf32_copy(const uint16_t *__restrict__ op, float *__restrict__ op32, const int *__restrict__ tiles,
                            int nb, const int *st) {
  if (failed(st)) return;
  const long t = tiles[blockIdx.x];
  const size_t plane = (size_t)nb * nb, part = plane / gridDim.y;
  const uint16_t *p = op + (size_t)t * 3 * plane;
  float *q = op32 + (size_t)t * plane;
  for (size_t e = blockIdx.y * part + threadIdx.x; e < (blockIdx.y + 1) * part; e += blockDim.x) {
    const float x = (__bfloat162float(__ushort_as_bfloat16(p[2 * plane + e])) +
                     __bfloat162float(__ushort_as_bfloat16(p[plane + e]))) +
                    __bfloat162float(__ushort_as_bfloat16(p[e]));
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    q[e] = __uint_as_float(r);
  }
}

// FP8-E4M3 copies of whole panel tiles for E4M3-class consumers, from the
// leading BF16 piece (already row-major / K-major).  One CTA per listed tile:
// amax over the tile, power-of-two scale s = 2^floor(log2(448 / amax)) so
// that |x s| <= 448 (the largest finite E4M3), then a saturating,
// round-to-nearest conversion of x s.  Zero tiles get s = 1.
__global__ void __launch_bounds__(1024)
    k_quant_e4m3(const uint16_t *__restrict__ op, uint8_t *__restrict__ op8, float *__restrict__ scale,
                 const int *__restrict__ tiles, int nb, const int *st) {
  if (failed(st)) return;
  __shared__ float red[32];
  __shared__ float s_scale;
  long t = tiles[blockIdx.x];
  size_t plane = (size_t)nb * nb;
  const uint16_t *x0 = op + (size_t)t * 3 * plane;
  // 16-byte accesses (eight entries per thread and load), so that the
  // loads of a tile are in flight together
  const uint4 *x8 = reinterpret_cast<const uint4 *>(x0);
  const size_t n8 = plane / 8;
  float amax = 0.f;
  for (size_t e = threadIdx.x; e < n8; e += blockDim.x) {
    const uint4 v = __ldg(x8 + e);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int h = 0; h < 4; h++) {
      amax = fmaxf(amax, fabsf(__uint_as_float(w[h] << 16)));
      amax = fmaxf(amax, fabsf(__uint_as_float(w[h] & 0xffff0000u)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_down_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, red[w]);
    // 448 / m = f 2^e with f in [0.5, 1): the largest power of two not above it is 2^(e-1)
    int e = 1;
    if (m > 0.f) frexpf(448.f / m, &e);
    s_scale = ldexpf(1.f, e - 1);
    scale[t] = s_scale;
  }
  __syncthreads();
  float s = s_scale;
  uint2 *q8 = reinterpret_cast<uint2 *>(op8 + (size_t)t * plane);
  for (size_t e = threadIdx.x; e < n8; e += blockDim.x) {
    const uint4 v = __ldg(x8 + e);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t o[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 4; h++) {
      // a BF16 value is the high half of the FP32 with the same bits
      const uint32_t lo = __nv_cvt_float_to_fp8(__uint_as_float(w[h] << 16) * s, __NV_SATFINITE, __NV_E4M3);
      const uint32_t hi = __nv_cvt_float_to_fp8(__uint_as_float(w[h] & 0xffff0000u) * s, __NV_SATFINITE, __NV_E4M3);
      o[h >> 1] |= (lo | (hi << 8)) << (16 * (h & 1));
    }
    q8[e] = make_uint2(o[0], o[1]);
  }
}

// SIMT FP32 panel TRSM for the low-precision tiles of column k, used where
// trsm_tc::supports(nb) is false (nb not a multiple of the tensor-core
// TRSM's 128-row block, or nb - 64 > 512 TMEM columns): L_ik = A_ik L_kk^{-T} from the FP32 master A_ik and an FP32 copy
// of the FP64 L_kk, written back to the master and, split, to the operand
// arena.
// One CTA per (row block, tile); warp w owns rows w + NW*q, a lane owns one
// column of the current 32-column block cb.  L_kk streams through shared
// memory as 32x32 chunks (rows of block cb, columns of block c <= cb) in a
// ring of NBUF buffers filled by cp.async several chunks ahead, the same
// sequence for every CTA: a chunk c < cb is subtracted from the block's
// columns (four independent partial sums per row), the diagonal chunk c = cb
// is solved by forward substitution with shuffles.  One barrier per chunk.
constexpr int TS_LD_PAD = 4;
constexpr int TS_CHUNK = B * B;  // floats per chunk, column-major (32 columns x 32 rows)
constexpr int TS_NBUF_CRIT = 8;   // chunk buffers, single critical-path tile (1 CTA per SM)
constexpr int TS_NBUF_PANEL = 4;  // panel launches (4 CTAs per SM hide each other's latency)

__device__ inline void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// NW warps, RPW rows per warp, NBUF chunk buffers: 16-row CTAs (8 warps x 2)
// for throughput on the panel, 4-row CTAs (4 warps x 1, deeper ring) for the
// single tile on the critical path, where more CTAs in parallel mean less
// latency.
template <int NW, int RPW, int NBUF, bool JOBS = false>
__global__ void __launch_bounds__(NW * 32)
    k_trsm32_panel(const float *__restrict__ Lkk0, float *__restrict__ t32, uint16_t *__restrict__ op, int nb,
                   int NT, int k, const int *__restrict__ rows, const int *st,
                   const int2 *__restrict__ jobs = nullptr) {
  constexpr int ROWS = NW * RPW, NTH = NW * 32;
  if (failed(st)) return;
  extern __shared__ __align__(16) float sm[];
  const int ldx = nb + TS_LD_PAD;
  float *S = sm;                     // [NBUF][32][32]: chunk ring, S[p * 32 + r] = L_kk(cb*32 + r, c*32 + p)
  float *X = sm + NBUF * TS_CHUNK;   // [ROWS][ldx]: the CTA's rows of A_ik, solved in place
  int r0 = blockIdx.x * ROWS;
  // tile (i, k) of one matrix, or (batched) an explicit tile index and the
  // slot of its L_kk copy
  long ti;
  const float *Lkk = Lkk0;
  if (JOBS) {
    int2 jb = jobs[blockIdx.y];
    ti = jb.x;
    Lkk = Lkk0 + (size_t)jb.y * nb * nb;
  } else {
    ti = tile_index(rows[blockIdx.y], k, NT);
  }
  float *A = t32 + (size_t)ti * nb * nb + r0;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nbc = nb / B, nchunks = nbc * (nbc + 1) / 2;
  // chunk i = (cb, c) with i = cb (cb + 1) / 2 + c, c <= cb
  int ic_cb = 0, ic_c = 0;  // the next chunk to issue
  auto issue = [&]() {
    const int i = ic_cb * (ic_cb + 1) / 2 + ic_c;
    if (i < nchunks) {
      float *dst = S + (i % NBUF) * TS_CHUNK;
      const float *src = Lkk + (size_t)(ic_c * B) * nb + ic_cb * B;
      for (int e = tid; e < TS_CHUNK / 4; e += NTH) {
        const int pc = e >> 3, q = (e & 7) * 4;  // chunk column pc, rows q .. q+3
        cp_async16(dst + pc * B + q, src + (size_t)pc * nb + q);
      }
      if (++ic_c > ic_cb) {
        ic_cb++;
        ic_c = 0;
      }
    }
    cp_async_commit();  // an empty group at the tail keeps the count uniform
  };
  for (int u = 0; u < NBUF - 1; u++) issue();
#pragma unroll 8
  for (int e = tid; e < ROWS * nb; e += NTH) {
    int r = e % ROWS, c = e / ROWS;
    X[r * ldx + c] = A[r + (size_t)c * nb];
  }
  int i = 0;
  for (int cb = 0; cb < nbc; cb++) {
    float a0[RPW], a1[RPW], a2[RPW], a3[RPW];
    for (int c = 0; c <= cb; c++, i++) {
      cp_async_wait<NBUF - 2>();  // this thread's copies of chunk i have landed
      __syncthreads();            // everyone's; and chunk i-1's buffer is free
      issue();
      const float *Sc = S + (i % NBUF) * TS_CHUNK;
      if (c == 0) {
#pragma unroll
        for (int q = 0; q < RPW; q++) {
          a0[q] = X[(w + NW * q) * ldx + cb * B + lane];
          a1[q] = a2[q] = a3[q] = 0.f;
        }
      }
      if (c < cb) {
#pragma unroll
        for (int q = 0; q < RPW; q++) {
          const float4 *xq = reinterpret_cast<const float4 *>(X + (w + NW * q) * ldx + c * B);
#pragma unroll
          for (int p4 = 0; p4 < B / 4; p4++) {
            const float4 xv = xq[p4];
            a0[q] -= xv.x * Sc[(4 * p4 + 0) * B + lane];
            a1[q] -= xv.y * Sc[(4 * p4 + 1) * B + lane];
            a2[q] -= xv.z * Sc[(4 * p4 + 2) * B + lane];
            a3[q] -= xv.w * Sc[(4 * p4 + 3) * B + lane];
          }
        }
      } else {
        // diagonal chunk: ld[p] = L_kk(cb*32 + lane, cb*32 + p) for p <= lane
        float ld[B];
#pragma unroll
        for (int p = 0; p < B; p++) ld[p] = (p <= lane) ? Sc[p * B + lane] : 0.f;
        float mydiag = ld[0];
#pragma unroll
        for (int p = 1; p < B; p++)
          if (p == lane) mydiag = ld[p];
        const float myrinv = 1.0f / mydiag;
        float a[RPW];
#pragma unroll
        for (int q = 0; q < RPW; q++) a[q] = (a0[q] + a1[q]) + (a2[q] + a3[q]);
#pragma unroll
        for (int j = 0; j < B; j++) {
          float rj = __shfl_sync(0xffffffffu, myrinv, j);
#pragma unroll
          for (int q = 0; q < RPW; q++) {
            float xj = __shfl_sync(0xffffffffu, a[q], j) * rj;
            if (lane == j) a[q] = xj;
            if (lane > j) a[q] -= xj * ld[j];
          }
        }
#pragma unroll
        for (int q = 0; q < RPW; q++) X[(w + NW * q) * ldx + cb * B + lane] = a[q];
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // FP32 master (column-major) and the sender-side BF16 pieces (row-major)
#pragma unroll 8
  for (int e = tid; e < ROWS * nb; e += NTH) {
    int r = e % ROWS, c = e / ROWS;
    A[r + (size_t)c * nb] = X[r * ldx + c];
  }
  size_t plane = (size_t)nb * nb;
  uint16_t *P = op + (size_t)ti * 3 * plane + (size_t)r0 * nb;
  for (int e = tid; e < ROWS * nb; e += NTH) {
    int r = e / nb, c = e % nb;
    uint16_t p0, p1, p2;
    split3(X[r * ldx + c], p0, p1, p2);
    size_t off = (size_t)r * nb + c;
    P[off] = p0;
    P[plane + off] = p1;
    P[2 * plane + off] = p2;
  }
}

static size_t trsm32_smem(int nb, int rows, int nbuf) {
  return (size_t)(nbuf * TS_CHUNK + rows * (nb + TS_LD_PAD)) * sizeof(float);
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
// Work of panel step k, split so that the critical chain
// POTRF(k) -> TRSM(k+1,k) -> SYRK(k+1,k+1) -> POTRF(k+1) carries as little
// as possible.  Groups: T1 = TRSM of row k+1, TR = TRSM of rows >= k+2,
// S = update of tile (k+1,k+1), G1 = updates of (i, k+1), i >= k+2,
// G2A = updates of column k+2, G2 = updates of columns >= k+3.  Each group has FP64 entries (rows / pairs
// for the SIMT kernels) and tensor-core items.
enum { GR_S = 0, GR_G1 = 1, GR_G2A = 2, GR_G2 = 3, GR_N = 4 };
struct StepPlan {
  int r64_1 = 0, n64_1 = 0, r32_1 = 0, n32_1 = 0;  // T1 (offset, count) in rows64 / rows32
  int r64_r = 0, n64_r = 0, r32_r = 0, n32_r = 0;  // TR
  int q_1 = 0, nq_1 = 0, q_r = 0, nq_r = 0;        // panel tiles to quantize to E4M3 (row k+1 / rest)
  int t_1 = 0, nt_1 = 0, t_r = 0, nt_r = 0;        // panel tiles copied to TF32 (row k+1 / rest)
  int p_off[GR_N] = {}, p_n[GR_N] = {};            // FP64-class tensor-core items per update group
  double p_flops[GR_N] = {};
  int z1_off = 0, z1_n = 0, zr_off = 0, zr_n = 0;  // panel tiles digit-sliced for them (row k+1 / rest)
  int i_off[GR_N] = {}, i_n[GR_N] = {};            // tensor-core items per update group
  double flops[GR_N] = {}, mma[GR_N] = {};
  bool diag_low = false;
  bool fp64_panel = false;  // FP64-class TRSM or SYRK on the critical or panel stream
  int b_off1 = 0, b_offr = 0;  // blocked FP64 TRSM: first product item of T1 / TR in items_tr
};

struct MixedPlan {
  int NT = 0, nb = 0;
  std::vector<unsigned char> cls;  // packed by tile index
  std::vector<StepPlan> steps;
  int *d_rows64 = nullptr, *d_rows32 = nullptr;
  gemm64::Item *d_items64 = nullptr;  // FP64-class updates on the tensor cores (digit products)
  gemm64::Seg *d_segs64 = nullptr;
  int4 *d_zjobs = nullptr;            // {tile, slot, exponent base} of the panel tiles sliced for them
  int nslots = 0;
  uint16_t *d_digits = nullptr;       // nslots * NS digit planes of nb x nb
  int *d_exp64 = nullptr;             // nslots * nb row exponents (biased)
  // the sampler's FP64-class tiles (sliced on the first draw after the factor)
  bool samp_ready = false;
  int nslots_s = 0;
  uint16_t *d_dig_s = nullptr;
  int *d_exp_s = nullptr;             // row exponents per row of the padded matrix
  std::vector<int> slot_s;            // tile -> sampler slot (-1: not FP64 class)
  CUtensorMap map_s;
  CUtensorMap map64a, map64b;
  gemm_tc::Item *d_items = nullptr;
  gemm_tc::Seg *d_segs = nullptr;
  int *d_tiles64 = nullptr;           // tile index of every entry of rows64 (split after its TRSM)
  int *d_qtiles = nullptr;            // panel tiles quantized to E4M3, per step (see StepPlan)
  bool any_e4m3 = false;
  int *d_ttiles = nullptr;            // panel tiles copied to TF32, per step (see StepPlan)
  bool any_tf32 = false;
  gemm_tc::Operands ops;
  int *d_diag_tiles = nullptr;        // all diagonal tiles (split after the factor)
  float *d_lkk32 = nullptr;           // FP32 copies of L_kk, double-buffered by step parity
  uint16_t *d_lkkp = nullptr;         // three BF16 pieces of L_kk (row-major), same slots (tensor-core TRSM)
  double *d_ls64 = nullptr;           // pre-scaled diagonal blocks of L_kk for the FP64 TRSM (nb x 32), same slots
  double *d_rinv64 = nullptr;         // 1 / L_kk(c, c), same slots
  // blocked FP64-class TRSM (gemm64::launch_trsm_block): products X_J L_{>J,J}^T
  bool blk64 = false;
  int nslots_x = 0;                   // digit slots of solved blocks: 0 = row k+1, 1.. = rows >= k+2
  gemm64::Item *d_items_tr = nullptr;
  gemm64::Seg *d_segs_tr = nullptr;
  uint16_t *d_xdig = nullptr;         // nslots_x * NS planes of nb x TW
  int *d_xexp = nullptr;              // nslots_x * nb
  uint16_t *d_ldig = nullptr;         // L_kk's column blocks, double-buffered by step parity
  int *d_lexp = nullptr;
  CUtensorMap map_xa, map_lb[2];
  CUtensorMap lmap;                   // over d_lkkp
  CUtensorMap opmap;                  // over the piece arena (the TRSM's tile stores)
  bool tc_trsm = false;               // FP32-class panel TRSMs on the tensor cores (trsm_tc.cu)
  CUtensorMap mapA, mapB;
  double update_flops[EMU_NCLASS] = {};
  int tiles[EMU_NCLASS] = {};
  // every device list above lives in one stream-ordered allocation, filled by
  // one copy from `host_blob` (kept until the factor's stream work is done)
  void *d_blob = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<char> host_blob;
};

static void plan_free(MixedPlan *p) {
  if (!p) return;
  if (p->d_blob) cudaFreeAsync(p->d_blob, p->stream);
  for (void *q : {(void *)p->d_digits, (void *)p->d_exp64, (void *)p->d_dig_s, (void *)p->d_exp_s,
                  (void *)p->d_xdig, (void *)p->d_xexp, (void *)p->d_ldig, (void *)p->d_lexp})
    if (q) cudaFreeAsync(q, p->stream);
  delete p;
}

void mixed_mat_release(emu_mat *A) {
  plan_free(static_cast<MixedPlan *>(A->plan));
  A->plan = nullptr;
}

static emu_status build_plan(emu_ctx *ctx, emu_mat *A, MixedPlan *P) {
  int NT = A->nt, nb = A->nb;
  P->NT = NT;
  P->nb = nb;
  P->cls.assign(A->h_cls, A->h_cls + A->ntiles);
  auto C = [&](int i, int j) { return (int)P->cls[tile_index(i, j, NT)]; };
  std::vector<int> rows64, rows32, tiles64, diag, qtiles, ttiles;
  std::vector<gemm64::Item> items64;
  std::vector<gemm64::Seg> segs64;
  std::vector<int4> zjobs, z1_step, zr_step;
  std::vector<int> slot_of_tile(A->ntiles, -1);
  std::vector<gemm_tc::Item> items;
  std::vector<gemm_tc::Seg> segs;
  double nb3 = (double)nb * nb * nb;
  for (int j = 0; j < NT; j++)
    for (int i = j; i < NT; i++) {
      int c = C(i, j);
      P->tiles[c]++;
      P->update_flops[c] += (i == j ? 1.0 : 2.0) * j * nb3 + (i > j ? nb3 : 0.0);
    }
  // digit slot of panel tile (r, k), sliced after its TRSM
  auto slot_of = [&](int k, int r) {
    long t = tile_index(r, k, NT);
    if (slot_of_tile[t] < 0) {
      slot_of_tile[t] = P->nslots++;
      (r == k + 1 ? z1_step : zr_step)
          .push_back(make_int4((int)t, slot_of_tile[t], slot_of_tile[t] * nb, 0));
    }
    return slot_of_tile[t];
  };
  auto add_tile_update = [&](StepPlan &sp, int g, int k, int i, int j) {
    int c = C(i, j);
    if (c == EMU_CLASS_FP64) {
      // FP64 accuracy on the tensor cores: digit products of panel tiles (i, k), (j, k)
      int si = slot_of(k, i), sj = slot_of(k, j);
      for (int nbk = 0; nbk < nb / gemm64::BN; nbk++)
        for (int mb = 0; mb < nb / gemm64::BM; mb++) {
          if (i == j && mb * gemm64::BM + gemm64::BM - 1 < nbk * gemm64::BN) continue;  // above the diagonal
          gemm64::Seg sg;
          sg.a_row = si * gemm64::NS * nb + mb * gemm64::BM;
          sg.b_row = sj * gemm64::NS * nb + nbk * gemm64::BN;
          sg.a_x = sg.b_x = 0;
          gemm64::Item it;
          it.out_off = tile_index(i, j, NT) * (long)nb * nb + mb * gemm64::BM + (long)nbk * gemm64::BN * nb;
          it.a_sc = si * nb + mb * gemm64::BM;
          it.b_sc = sj * nb + nbk * gemm64::BN;
          it.seg_begin = (int)segs64.size();
          segs64.push_back(sg);
          it.seg_end = (int)segs64.size();
          it.rows_valid = gemm64::BM;
          it.cols_valid = gemm64::BN;
          items64.push_back(it);
          sp.p_n[g]++;
        }
      sp.p_flops[g] += 2.0 * nb3;
      return;
    }
    int cc = (c == EMU_CLASS_FP32 || c == EMU_CLASS_TF32 || c == EMU_CLASS_E4M3) ? c : EMU_CLASS_BF16;
    bool f8 = cc == EMU_CLASS_E4M3, t32 = cc == EMU_CLASS_TF32;
    if (f8) P->any_e4m3 = true;
    if (t32) P->any_tf32 = true;
    long tik = tile_index(i, k, NT), tjk = tile_index(j, k, NT);
    for (int nbk = 0; nbk < nb / gemm_tc::BN; nbk++)
      for (int mb = 0; mb < nb / gemm_tc::BM; mb++) {
        if (i == j && mb * gemm_tc::BM + gemm_tc::BM - 1 < nbk * gemm_tc::BN) continue;  // above the diagonal
        // BF16 pieces: row (tile*3 + piece)*nb + r; FP8 and TF32 copies: row tile*nb + r
        const int rows_per_tile = (f8 || t32) ? 1 : 3;
        gemm_tc::Seg s;
        s.ax = 0;
        s.ay = (int)(tik * rows_per_tile * nb + mb * gemm_tc::BM);
        s.ay_step = nb;
        s.bx = 0;
        s.by = (int)(tjk * rows_per_tile * nb + nbk * gemm_tc::BN);
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
        it.sa = f8 ? (int)tik : -1;
        it.sb = f8 ? (int)tjk : -1;
        items.push_back(it);
        double f = 2.0 * gemm_tc::BM * gemm_tc::BN * nb;
        sp.i_n[g]++;
        sp.flops[g] += f;
        // in BF16-product units: a TF32 product runs at half the BF16 rate,
        // an E4M3 product (kind::f8f6f4) at twice it
        sp.mma[g] += f * (cc == EMU_CLASS_FP32 ? 6.0 : t32 ? 2.0 : f8 ? 0.5 : 1.0);
      }
  };
  auto add_row = [&](int k, int i, int &n64, int &n32) {
    if (C(i, k) == EMU_CLASS_FP64) {
      rows64.push_back(i);
      tiles64.push_back((int)tile_index(i, k, NT));
      n64++;
    } else {
      rows32.push_back(i);
      n32++;
    }
  };
  for (int k = 0; k < NT; k++) {
    StepPlan sp;
    diag.push_back((int)tile_index(k, k, NT));
    sp.diag_low = C(k, k) != EMU_CLASS_FP64;
    sp.r64_1 = (int)rows64.size();
    sp.r32_1 = (int)rows32.size();
    if (k + 1 < NT) add_row(k, k + 1, sp.n64_1, sp.n32_1);
    sp.r64_r = (int)rows64.size();
    sp.r32_r = (int)rows32.size();
    for (int i = k + 2; i < NT; i++) add_row(k, i, sp.n64_r, sp.n32_r);
    for (int g = 0; g < GR_N; g++) {
      sp.p_off[g] = (int)items64.size();
      sp.i_off[g] = (int)items.size();
      if (g == GR_S) {
        if (k + 1 < NT) add_tile_update(sp, g, k, k + 1, k + 1);
      } else if (g == GR_G1) {
        for (int i = k + 2; i < NT; i++) add_tile_update(sp, g, k, i, k + 1);
      } else if (g == GR_G2A) {
        for (int i = k + 2; i < NT; i++) add_tile_update(sp, g, k, i, k + 2);
      } else {
        for (int j = k + 3; j < NT; j++)
          for (int i = j; i < NT; i++) add_tile_update(sp, g, k, i, j);
      }
    }
    // E4M3 consumers read FP8 copies of the panel tiles: quantize them all
    // when the step has any E4M3 update
    bool step_f8 = false;
    for (int g = 0; g < GR_N; g++)
      for (int q = sp.i_off[g]; q < sp.i_off[g] + sp.i_n[g]; q++)
        if (items[q].sa >= 0) step_f8 = true;
    sp.q_1 = (int)qtiles.size();
    if (step_f8 && k + 1 < NT) {
      qtiles.push_back((int)tile_index(k + 1, k, NT));
      sp.nq_1 = 1;
    }
    sp.q_r = (int)qtiles.size();
    if (step_f8)
      for (int i = k + 2; i < NT; i++) {
        qtiles.push_back((int)tile_index(i, k, NT));
        sp.nq_r++;
      }
    // TF32 consumers read TF32 copies of the panel tiles: copy them all when
    // the step has any TF32 update
    bool step_t32 = false;
    for (int g = 0; g < GR_N; g++)
      for (int q = sp.i_off[g]; q < sp.i_off[g] + sp.i_n[g]; q++)
        if (segs[items[q].seg_begin].cls == EMU_CLASS_TF32) step_t32 = true;
    sp.t_1 = (int)ttiles.size();
    if (step_t32 && k + 1 < NT) {
      ttiles.push_back((int)tile_index(k + 1, k, NT));
      sp.nt_1 = 1;
    }
    sp.t_r = (int)ttiles.size();
    if (step_t32)
      for (int i = k + 2; i < NT; i++) {
        ttiles.push_back((int)tile_index(i, k, NT));
        sp.nt_r++;
      }
    sp.fp64_panel = sp.n64_1 > 0 || sp.n64_r > 0 || sp.p_n[GR_S] > 0;
    sp.z1_off = (int)zjobs.size();
    zjobs.insert(zjobs.end(), z1_step.begin(), z1_step.end());
    sp.z1_n = (int)z1_step.size();
    sp.zr_off = (int)zjobs.size();
    zjobs.insert(zjobs.end(), zr_step.begin(), zr_step.end());
    sp.zr_n = (int)zr_step.size();
    z1_step.clear();
    zr_step.clear();
    P->steps.push_back(sp);
  }
  // blocked FP64-class TRSM: per step and list (row k+1 in slot 0, rows >= k+2
  // in slots 1..), for each column block J < nJ - 1 the products of every
  // listed tile's (BM-row block, BN-column block right of block J) pairs,
  // J-major
  std::vector<gemm64::Item> items_tr;
  std::vector<gemm64::Seg> segs_tr;
  const int nJ = nb / gemm64::TW;
  P->blk64 = nb % gemm64::TW == 0 && nb % gemm64::BM == 0 && nJ >= 2;
  if (P->blk64) {
    int max_r = 0;
    for (StepPlan &sp : P->steps) {
      max_r = std::max(max_r, sp.n64_r);
      for (int list = 0; list < 2; list++) {
        const int r0 = list ? sp.r64_r : sp.r64_1, n = list ? sp.n64_r : sp.n64_1, slot0 = list;
        (list ? sp.b_offr : sp.b_off1) = (int)items_tr.size();
        for (int J = 0; J + 1 < nJ; J++)
          for (int z = 0; z < n; z++)
            for (int rb = 0; rb < nb / gemm64::BM; rb++)
              for (int cb = (J + 1) * (gemm64::TW / gemm64::BN); cb < nb / gemm64::BN; cb++) {
                gemm64::Seg sg;
                sg.a_row = (slot0 + z) * gemm64::NS * nb + rb * gemm64::BM;
                sg.b_row = J * gemm64::NS * nb + cb * gemm64::BN;
                sg.a_x = sg.b_x = 0;
                gemm64::Item it;
                it.out_off = (long)tiles64[r0 + z] * nb * nb + rb * gemm64::BM + (long)cb * gemm64::BN * nb;
                it.a_sc = (slot0 + z) * nb + rb * gemm64::BM;
                it.b_sc = J * nb + cb * gemm64::BN;
                it.seg_begin = (int)segs_tr.size();
                segs_tr.push_back(sg);
                it.seg_end = (int)segs_tr.size();
                it.rows_valid = gemm64::BM;
                it.cols_valid = gemm64::BN;
                items_tr.push_back(it);
              }
      }
    }
    P->nslots_x = 1 + max_r;
    if (items_tr.empty()) P->blk64 = false;
  }
  // one allocation and one copy for all lists (256-byte aligned parts)
  size_t off = 0;
  auto part = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  auto vbytes = [](const auto &v) { return v.size() * sizeof(v[0]); };
  size_t o_r64 = part(vbytes(rows64)), o_r32 = part(vbytes(rows32)), o_i64 = part(vbytes(items64)),
         o_s64 = part(vbytes(segs64)), o_z = part(vbytes(zjobs)),
         o_items = part(vbytes(items)), o_segs = part(vbytes(segs)), o_t64 = part(vbytes(tiles64)),
         o_diag = part(vbytes(diag)), o_q = part(vbytes(qtiles)), o_tt = part(vbytes(ttiles)),
         o_itr = part(vbytes(items_tr)), o_str = part(vbytes(segs_tr)),
         o_lkk = part(2 * (size_t)nb * nb * sizeof(float)), o_lkkp = part(2 * 3 * (size_t)nb * nb * sizeof(uint16_t)),
         o_ls64 = part(2 * (size_t)nb * 32 * sizeof(double)), o_rinv64 = part(2 * (size_t)nb * sizeof(double));
  size_t copy_bytes = o_lkk;  // everything before the L_kk buffers comes from the host
  P->host_blob.assign(copy_bytes, 0);
  auto put = [&](size_t o, const auto &v) {
    if (!v.empty()) memcpy(P->host_blob.data() + o, v.data(), vbytes(v));
  };
  put(o_r64, rows64);
  put(o_r32, rows32);
  put(o_i64, items64);
  put(o_s64, segs64);
  put(o_z, zjobs);
  put(o_items, items);
  put(o_segs, segs);
  put(o_t64, tiles64);
  put(o_diag, diag);
  put(o_q, qtiles);
  put(o_tt, ttiles);
  put(o_itr, items_tr);
  put(o_str, segs_tr);
  P->stream = ctx->stream;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_blob, off, ctx->stream));
  char *b = static_cast<char *>(P->d_blob);
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(b, P->host_blob.data(), copy_bytes, cudaMemcpyHostToDevice, ctx->stream));
  P->d_rows64 = reinterpret_cast<int *>(b + o_r64);
  P->d_rows32 = reinterpret_cast<int *>(b + o_r32);
  P->d_items64 = reinterpret_cast<gemm64::Item *>(b + o_i64);
  P->d_segs64 = reinterpret_cast<gemm64::Seg *>(b + o_s64);
  P->d_zjobs = reinterpret_cast<int4 *>(b + o_z);
  P->d_items = reinterpret_cast<gemm_tc::Item *>(b + o_items);
  P->d_segs = reinterpret_cast<gemm_tc::Seg *>(b + o_segs);
  P->d_tiles64 = reinterpret_cast<int *>(b + o_t64);
  P->d_diag_tiles = reinterpret_cast<int *>(b + o_diag);
  P->d_qtiles = reinterpret_cast<int *>(b + o_q);
  P->d_ttiles = reinterpret_cast<int *>(b + o_tt);
  P->d_items_tr = reinterpret_cast<gemm64::Item *>(b + o_itr);
  P->d_segs_tr = reinterpret_cast<gemm64::Seg *>(b + o_str);
  P->d_lkk32 = reinterpret_cast<float *>(b + o_lkk);
  P->d_lkkp = reinterpret_cast<uint16_t *>(b + o_lkkp);
  P->d_ls64 = reinterpret_cast<double *>(b + o_ls64);
  P->d_rinv64 = reinterpret_cast<double *>(b + o_rinv64);
  emu_status s;
  uint64_t rows = (uint64_t)A->ntiles * 3 * nb;
  if ((s = gemm_tc::make_map_bf16(ctx, &P->mapA, A->op_bf16, nb, rows, gemm_tc::BM)) != EMU_OK) return s;
  if ((s = gemm_tc::make_map_bf16(ctx, &P->mapB, A->op_bf16, nb, rows, gemm_tc::BN)) != EMU_OK) return s;
  P->ops.a16 = P->mapA;
  P->ops.b16 = P->mapB;
  P->ops.a8 = P->mapA;  // valid maps even when no FP8 or TF32 copies exist (then never used)
  P->ops.b8 = P->mapB;
  P->ops.a32 = P->mapA;
  P->ops.b32 = P->mapB;
  P->ops.scale8 = nullptr;
  P->tc_trsm = trsm_tc::supports(nb);
  if (P->tc_trsm && ((s = trsm_tc::make_map(ctx, &P->lmap, P->d_lkkp, nb, 2)) != EMU_OK ||
                     (s = trsm_tc::make_op_map(ctx, &P->opmap, A->op_bf16, nb, A->ntiles)) != EMU_OK))
    return s;
  if (P->nslots > 0) {
    size_t te = (size_t)nb * nb;
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_digits, (size_t)P->nslots * gemm64::NS * te * sizeof(uint16_t),
                                      ctx->stream));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_exp64, (size_t)P->nslots * nb * sizeof(int), ctx->stream));
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(P->d_exp64, 0, (size_t)P->nslots * nb * sizeof(int), ctx->stream));
    uint64_t drows = (uint64_t)P->nslots * gemm64::NS * nb;
    if ((s = gemm64::make_map(ctx, &P->map64a, P->d_digits, nb, drows, gemm64::BM)) != EMU_OK) return s;
    if ((s = gemm64::make_map(ctx, &P->map64b, P->d_digits, nb, drows, gemm64::BN)) != EMU_OK) return s;
  }
  if (P->blk64) {
    const size_t xplane = (size_t)nb * gemm64::TW, lbuf = (size_t)(nJ - 1) * gemm64::NS * xplane;
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_xdig, (size_t)P->nslots_x * gemm64::NS * xplane * sizeof(uint16_t),
                                      ctx->stream));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_xexp, (size_t)P->nslots_x * nb * sizeof(int), ctx->stream));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_ldig, 2 * lbuf * sizeof(uint16_t), ctx->stream));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_lexp, 2 * (size_t)(nJ - 1) * nb * sizeof(int), ctx->stream));
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(P->d_lexp, 0, 2 * (size_t)(nJ - 1) * nb * sizeof(int), ctx->stream));
    if ((s = gemm64::make_map(ctx, &P->map_xa, P->d_xdig, gemm64::TW, (uint64_t)P->nslots_x * gemm64::NS * nb,
                              gemm64::BM)) != EMU_OK)
      return s;
    for (int q = 0; q < 2; q++)
      if ((s = gemm64::make_map(ctx, &P->map_lb[q], P->d_ldig + q * lbuf, gemm64::TW,
                                (uint64_t)(nJ - 1) * gemm64::NS * nb, gemm64::BN)) != EMU_OK)
        return s;
  }
  if (P->any_e4m3) {
    size_t te = (size_t)nb * nb;
    if (!A->op_e4m3) EMU_CUDA_TRY(ctx, cudaMallocAsync(&A->op_e4m3, (size_t)A->ntiles * te, ctx->stream));
    if (!A->scale_e4m3)
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&A->scale_e4m3, (size_t)A->ntiles * sizeof(float), ctx->stream));
    uint64_t rows8 = (uint64_t)A->ntiles * nb;
    if ((s = gemm_tc::make_map_e4m3(ctx, &P->ops.a8, A->op_e4m3, nb, rows8, gemm_tc::BM)) != EMU_OK) return s;
    if ((s = gemm_tc::make_map_e4m3(ctx, &P->ops.b8, A->op_e4m3, nb, rows8, gemm_tc::BN)) != EMU_OK) return s;
    P->ops.scale8 = A->scale_e4m3;
  }
  if (P->any_tf32) {
    size_t te = (size_t)nb * nb;
    if (!A->op_tf32)
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&A->op_tf32, (size_t)A->ntiles * te * sizeof(float), ctx->stream));
    uint64_t rows32 = (uint64_t)A->ntiles * nb;
    if ((s = gemm_tc::make_map_f32(ctx, &P->ops.a32, A->op_tf32, nb, rows32, gemm_tc::BM)) != EMU_OK) return s;
    if ((s = gemm_tc::make_map_f32(ctx, &P->ops.b32, A->op_tf32, nb, rows32, gemm_tc::BN)) != EMU_OK) return s;
  }
  return EMU_OK;
}

// SMs the bulk trailing update leaves to the critical-path and panel
// kernels.  The persistent bulk GEMM holds about 217 KB of shared memory per
// SM, so the panel TRSMs and the FP64-class SYRK (more shared memory than is
// left beside it) run only on these.  While FP64-class TRSMs or SYRKs are
// near (the first panels of a covariance) they bound the factor and get more
// SMs; afterwards the bulk update is the bound and keeps them.
constexpr int kReservedSMs = 16;
constexpr int kReservedSMsFP64 = 32;

// Internal streams of the mixed schedule (created once per context) and at
// least `nev` ordering events.
int mixed_reserved_sms(bool fp64_near) { return fp64_near ? kReservedSMsFP64 : kReservedSMs; }

emu_status mixed_sched_streams(emu_ctx *ctx, int nev) {
  if (!ctx->crit) {
    int least = 0, greatest = 0;
    EMU_CUDA_TRY(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    EMU_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&ctx->crit, cudaStreamNonBlocking, greatest));
    EMU_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&ctx->mid, cudaStreamNonBlocking, (greatest + least) / 2));
    EMU_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&ctx->bulk, cudaStreamNonBlocking, least));
  }
  while ((int)ctx->sched_ev.size() < nev) {
    cudaEvent_t e;
    EMU_CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->sched_ev.push_back(e);
  }
  return EMU_OK;
}

// ------------------------------------------- graph replay and schedule tuning
// After the precision map (one host round trip) the factor's launches depend
// only on the map, the tiling and the arenas' addresses.  They are recorded
// once into a CUDA graph over the four streams and replayed while those are
// unchanged (one host launch per factor).  The tuner times the reserved-SM
// choices below on the first factors of each (NT, nb, class map) and keeps
// the fastest; every choice gives the same result bit for bit (it only moves
// CTAs between SMs).
static emu_status factor_mixed_record(emu_ctx *ctx, emu_mat *A, MixedPlan *P, int R, int R64);
struct MixedCtx;
static emu_status factor_mixed_launch(emu_ctx *ctx, emu_mat *A, MixedPlan *P, MixedCtx *M, int R, int R64);
constexpr int kTuneR[][2] = {{kReservedSMs, kReservedSMsFP64}, {8, 16}, {24, 48}, {32, 64}};
constexpr int kTuneN = 4;
struct TuneEntry {
  std::vector<char> sig;
  float ms[kTuneN] = {};
  int tried = 0, best = 0;
};
struct MixedCtx {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<char> key;
  uint64_t graph_launches = 0;
  std::vector<TuneEntry> tune;
  int pending = -1, pending_cand = 0;  // tuning entry and choice of the factor in flight
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;  // around the factor's launches
  bool use_graphs = true, tuning = true;
};
static MixedCtx *mctx(emu_ctx *ctx) {
  if (!ctx->mixed) ctx->mixed = new MixedCtx();
  return static_cast<MixedCtx *>(ctx->mixed);
}
template <typename T>
static void key_put(std::vector<char> &k, const T &v) {
  const char *b = reinterpret_cast<const char *>(&v);
  k.insert(k.end(), b, b + sizeof(T));
}

void mixed_set_schedule(emu_ctx *ctx, int use_graphs, int tuning) {
  MixedCtx *M = mctx(ctx);
  M->use_graphs = use_graphs != 0;
  M->tuning = tuning != 0;
}

void mixed_tune_record(emu_ctx *ctx, bool ok) {
  MixedCtx *M = static_cast<MixedCtx *>(ctx->mixed);
  if (!M || M->pending < 0) return;
  float ms = 0.f;
  if (!ok || cudaEventElapsedTime(&ms, M->ev_a, M->ev_b) != cudaSuccess) {
    cudaGetLastError();
    M->pending = -1;
    return;
  }
  TuneEntry &t = M->tune[M->pending];
  if (M->pending_cand == t.tried && t.tried < kTuneN) {
    t.ms[t.tried++] = ms;
    if (t.tried == kTuneN) {
      t.best = 0;
      for (int c = 1; c < kTuneN; c++)
        if (t.ms[c] < t.ms[t.best]) t.best = c;
    }
  }
  M->pending = -1;
}

int mixed_tuned_choice(emu_ctx *ctx, int *tried, int *R, int *R64) {
  MixedCtx *M = static_cast<MixedCtx *>(ctx->mixed);
  if (!M || M->tune.empty()) return -1;
  const TuneEntry &t = M->tune.back();
  if (tried) *tried = t.tried;
  const int c = t.tried < kTuneN ? t.tried : t.best;
  if (R) *R = kTuneR[c][0];
  if (R64) *R64 = kTuneR[c][1];
  return c;
}

static emu_status factor_mixed_run(emu_ctx *ctx, emu_mat *A, MixedPlan *P) {
  MixedCtx *M = mctx(ctx);
  // schedule choice: the next untimed candidate of this signature, else the best
  std::vector<char> sig;
  key_put(sig, A->nt);
  key_put(sig, A->nb);
  sig.insert(sig.end(), P->cls.begin(), P->cls.end());
  int cand = 0;
  M->pending = -1;
  if (M->tuning) {
    int e = -1;
    for (int i = 0; i < (int)M->tune.size(); i++)
      if (M->tune[i].sig == sig) e = i;
    if (e < 0) {
      if (M->tune.size() >= 16) M->tune.erase(M->tune.begin());
      M->tune.push_back(TuneEntry{sig});
      e = (int)M->tune.size() - 1;
    }
    TuneEntry &t = M->tune[e];
    cand = t.tried < kTuneN ? t.tried : t.best;
    M->pending = e;
    M->pending_cand = cand;
  }
  const int R = kTuneR[cand][0], R64 = kTuneR[cand][1];
  emu_status s = potrf_dag_prepare(ctx, A->nb);
  if (s != EMU_OK) return s;
  if (!M->ev_a) {
    EMU_CUDA_TRY(ctx, cudaEventCreate(&M->ev_a));
    EMU_CUDA_TRY(ctx, cudaEventCreate(&M->ev_b));
  }
  EMU_CUDA_TRY(ctx, cudaEventRecord(M->ev_a, ctx->stream));
  s = factor_mixed_launch(ctx, A, P, M, R, R64);
  if (s == EMU_OK) EMU_CUDA_TRY(ctx, cudaEventRecord(M->ev_b, ctx->stream));
  return s;
}

static emu_status factor_mixed_launch(emu_ctx *ctx, emu_mat *A, MixedPlan *P, MixedCtx *M, int R, int R64) {
  emu_status s = EMU_OK;
  if (!M->use_graphs || ctx->prof || ctx->trace_on) return factor_mixed_record(ctx, A, P, R, R64);
  std::vector<char> sig;
  key_put(sig, A->nt);
  key_put(sig, A->nb);
  sig.insert(sig.end(), P->cls.begin(), P->cls.end());
  // everything a replay depends on
  std::vector<char> key = sig;
  for (const void *q : {(const void *)A->t64, (const void *)A->t32, (const void *)A->op_bf16, (const void *)A->op_e4m3,
                        (const void *)A->scale_e4m3, (const void *)A->op_tf32, (const void *)A->d_cls,
                        (const void *)P->d_blob, (const void *)P->d_digits, (const void *)P->d_exp64,
                        (const void *)ctx->dag_ws, (const void *)ctx->dag_tasks, (const void *)ctx->d_status})
    key_put(key, q);
  key_put(key, R);
  key_put(key, R64);
  key_put(key, ctx->sm_count);
  cudaStream_t user = ctx->stream;
  if (M->exec && M->key == key) {
    EMU_CUDA_TRY(ctx, cudaGraphLaunch(M->exec, user));
    ctx->launches += M->graph_launches;
    ctx->host_launches++;
    return EMU_OK;
  }
  if (!M->cap) EMU_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&M->cap, cudaStreamNonBlocking));
  const uint64_t l0 = ctx->launches, h0 = ctx->host_launches;
  ctx->stream = M->cap;
  // relaxed: the launchers set kernel attributes while the streams are captured
  cudaError_t e = cudaStreamBeginCapture(M->cap, cudaStreamCaptureModeRelaxed);
  s = (e == cudaSuccess) ? factor_mixed_record(ctx, A, P, R, R64) : emu_cuda_fail(ctx, e, "begin capture");
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) e = cudaStreamEndCapture(M->cap, &g);
  ctx->stream = user;
  const uint64_t nl = ctx->launches - l0;
  ctx->launches = l0;
  ctx->host_launches = h0;
  if (s != EMU_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    M->key.clear();
    return s != EMU_OK ? s : emu_cuda_fail(ctx, e, "end capture");
  }
  bool ok = false;
  if (M->exec) {
    cudaGraphExecUpdateResultInfo info;
    ok = cudaGraphExecUpdate(M->exec, g, &info) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();  // the update error is not a launch error
      cudaGraphExecDestroy(M->exec);
      M->exec = nullptr;
    }
  }
  if (!ok) e = cudaGraphInstantiate(&M->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    M->exec = nullptr;
    M->key.clear();
    return emu_cuda_fail(ctx, e, "graph instantiate");
  }
  M->key = key;
  M->graph_launches = nl;
  EMU_CUDA_TRY(ctx, cudaGraphLaunch(M->exec, user));
  ctx->launches += nl;
  ctx->host_launches++;
  return EMU_OK;
}

emu_status factor_mixed(emu_ctx *ctx, emu_mat *A, const emu_mp_opts *o) {
  int NT = A->nt, nb = A->nb;
  if (nb % gemm_tc::BN != 0) {
    ctx->last_error = "the mixed-precision factor needs nb to be a multiple of 256";
    return EMU_EINVAL;
  }
  // Default unit roundoffs.  The FP32 class takes the FP32 accumulation of
  // an nb-term update into account: its error in tile (i,j) is bounded by
  // 2^-24 sum_k ||L_ik||_F ||L_jk||_F, which on the diagonal tiles reaches
  // sqrt(nb) 2^-24 ||S_ii||_F (trace against Frobenius norm), the same factor
  // as the probabilistic bound on an nb-term FP32 sum.  For BF16 and E4M3 the
  // operand rounding (2^-8, 2^-4) is far larger than that and stays the bound.
  double u[EMU_NCLASS] = {0x1p-53, 0x1p-24 * sqrt((double)nb), 0x1p-11, 0x1p-8, 0x1p-4};
  for (int c = 0; c < EMU_NCLASS; c++)
    if (o->u[c] > 0.0) u[c] = o->u[c];
  unsigned mask = (o->prec_mask | 1u) & ((1u << EMU_NCLASS) - 1u);
  emu_status s = launch_precision_map(ctx, A, o->eps, u, mask, o->diag_fp64, o->band, band_sp_frac(o));
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
  return factor_mixed_run(ctx, A, P);
}

// The launches of the factor after its plan: on ctx->stream (the context
// stream, or a capture stream when the factor is recorded into a graph) and
// the three internal streams joined to it.  R / R64: SMs the bulk GEMM leaves
// free, without / with FP64-class panel work near.
static emu_status factor_mixed_record(emu_ctx *ctx, emu_mat *A, MixedPlan *P, int R, int R64) {
  const int NT = A->nt, nb = A->nb;
  const size_t te = A->tile_elems;
  emu_status s = EMU_OK;
  int *st = ctx->d_status;
  double nb3 = (double)nb * nb * nb;
  {
    ProfScope ps(ctx, PROF_SPLIT, 0.0, 12.0 * A->ntiles * te);
    k_to_f32<<<dim3(64, (unsigned)A->ntiles), 256, 0, ctx->stream>>>(A->t64, A->t32, A->d_cls, te);
    EMU_LAUNCHED(ctx);
  }
  // Lookahead schedule on three priority streams (see StepPlan):
  //   crit: POTRF(k) -> TRSM(k+1,k) -> S(k) = SYRK of tile (k+1,k+1)
  //   mid : TRSM(i>=k+2, k) -> G1(k) = update of column k+1 below the diagonal
  //   bulk: G2A(k) = update of column k+2, then G2(k) = columns >= k+3
  // Two launches that write the same tiles never overlap: S(k) and G1(k)
  // wait for G2A(k-1) (the last other writer of column k+1), and the bulk
  // stream runs G2A(k-1), G2(k-1), G2A(k), G2(k) in order.  TRSM(k+1,k) waits
  // for G1(k-1), which finished the update of its tile.
  cudaStream_t user = ctx->stream;
  const int EV = 5;  // per step: POTRF done, TRSM(k+1) done, TRSM rest done, G1 done, G2 done
  if ((s = mixed_sched_streams(ctx, EV * NT + 2)) != EMU_OK) return s;
  auto ev = [&](int k, int w) { return ctx->sched_ev[EV * k + w]; };
  enum { E_P = 0, E_T1 = 1, E_T = 2, E_G1 = 3, E_G2 = 4 };
  cudaEvent_t ev_start = ctx->sched_ev[EV * NT], ev_end = ctx->sched_ev[EV * NT + 1];
  EMU_CUDA_TRY(ctx, cudaEventRecord(ev_start, user));
  for (cudaStream_t q : {ctx->crit, ctx->mid, ctx->bulk}) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(q, ev_start, 0));
  size_t tsm16 = trsm32_smem(nb, 16, TS_NBUF_PANEL), tsm4 = trsm32_smem(nb, 4, TS_NBUF_CRIT);
  EMU_CUDA_TRY(ctx, cudaFuncSetAttribute(k_trsm32_panel<8, 2, TS_NBUF_PANEL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm16));
  EMU_CUDA_TRY(ctx, cudaFuncSetAttribute(k_trsm32_panel<4, 1, TS_NBUF_CRIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm4));

  // TRSM of the listed rows of panel k: FP64 rows on the FP64 pipe, then split;
  // low-class rows on the tensor cores (trsm_tc.cu), else the SIMT kernel
  auto quantize = [&](int q0, int nq) -> emu_status {
    if (nq <= 0) return EMU_OK;
    ProfScope ps(ctx, PROF_SPLIT, 0.0, 3.0 * nq * te);
    k_quant_e4m3<<<nq, 1024, 0, ctx->stream>>>(A->op_bf16, A->op_e4m3, A->scale_e4m3, P->d_qtiles + q0, nb, st);
    EMU_LAUNCHED(ctx);
    return EMU_OK;
  };
  auto tf32copy = [&](int t0, int nt) -> emu_status {
    if (nt <= 0) return EMU_OK;
    ProfScope ps(ctx, PROF_SPLIT, 0.0, 10.0 * nt * te);
    k_tf32_copy<<<dim3(nt, 32), 256, 0, ctx->stream>>>(A->op_bf16, A->op_tf32, P->d_ttiles + t0, nb, st);
    EMU_LAUNCHED(ctx);
    return EMU_OK;
  };
  auto slice64 = [&](int z0, int nz) -> emu_status {
    emu_status e = gemm64::launch_row_exponents(ctx, A->t64, A->t32, A->d_cls, P->d_zjobs + z0, nz, nb, P->d_exp64);
    if (e != EMU_OK) return e;
    return gemm64::launch_slice(ctx, A->t64, A->t32, A->d_cls, P->d_zjobs + z0, nz, nb, P->d_exp64, P->d_digits);
  };
  const int nJ = nb / gemm64::TW;
  const size_t lbuf = (size_t)(nJ - 1) * gemm64::NS * nb * gemm64::TW;
  // blocked FP64-class TRSM of n64 listed tiles: per column block J, the
  // block solve on the FP64 pipe, then X_J L_{>J,J}^T off the later blocks
  // as digit products (items J-major from b_off)
  auto trsm64_blocked = [&](int k, int r64, int n64, int slot0, int b_off) -> emu_status {
    ProfScope ps(ctx, PROF_TRSM64, n64 * nb3, 16.0 * n64 * te, 36.0 * n64 * nb3 * (nJ - 1) / nJ);
    const double *Lkk = A->t64 + tile_index(k, k, NT) * te;
    const double *Ls = P->d_ls64 + (size_t)(k & 1) * nb * 32, *ri = P->d_rinv64 + (size_t)(k & 1) * nb;
    const int per_pair = n64 * (nb / gemm64::BM);
    int off = b_off;
    for (int J = 0; J < nJ; J++) {
      const bool last = J + 1 == nJ;
      emu_status e = gemm64::launch_trsm_block(ctx, A->t64, nb, P->d_tiles64 + r64, n64, Lkk, J, Ls, ri, slot0,
                                               P->d_xexp, last ? nullptr : P->d_xdig);
      if (e != EMU_OK || last) return e;
      const int cnt = per_pair * (nJ - 1 - J) * (gemm64::TW / gemm64::BN);
      if ((e = gemm64::launch(ctx, P->map_xa, P->map_lb[k & 1], P->d_items_tr + off, cnt, P->d_segs_tr,
                              gemm64::TW, nb, nb, P->d_xexp, P->d_lexp + (size_t)(k & 1) * (nJ - 1) * nb,
                              gemm64::TC64_SUB, A->t64, nb, ctx->sm_count)) != EMU_OK)
        return e;
      off += cnt;
    }
    return EMU_OK;
  };
  // BF16 pieces of n64 listed FP64-class tiles (the low-class updates' operands)
  auto split64 = [&](int r64, int n64) -> emu_status {
    if (n64 <= 0) return EMU_OK;
    ProfScope ps(ctx, PROF_SPLIT, 0.0, 14.0 * n64 * te);
    k_split_tiles<double><<<dim3((nb / B) * (nb / B), n64), 256, 0, ctx->stream>>>(A->t64, A->op_bf16,
                                                                                  P->d_tiles64 + r64, nb, 0, st);
    EMU_LAUNCHED(ctx);
    return EMU_OK;
  };
  // FP32 copy and BF16 pieces of L_kk for the low-class TRSMs of panel k
  auto prep32 = [&](int k) -> emu_status {
    const long tkk = tile_index(k, k, NT);
    if (P->tc_trsm)
      return trsm_tc::launch_prep(ctx, A->t64, tkk, nullptr, 1, P->d_lkk32 + (size_t)(k & 1) * te,
                                  P->d_lkkp + (size_t)(k & 1) * 3 * te, nb);
    k_diag_to_f32<<<2 * ctx->sm_count, 256, 0, ctx->stream>>>(A->t64 + tkk * te, P->d_lkk32 + (size_t)(k & 1) * te,
                                                             te, st);
    EMU_LAUNCHED(ctx);
    return EMU_OK;
  };
  auto trsm_rows = [&](int k, int r64, int n64, int r32, int n32, bool critical, bool split = true) -> emu_status {
    emu_status e = EMU_OK;
    if (n64 > 0) {
      const StepPlan &sp = P->steps[k];
      if (P->blk64)
        e = trsm64_blocked(k, r64, n64, critical ? 0 : 1, critical ? sp.b_off1 : sp.b_offr);
      else
        e = launch_trsm64_panel(ctx, A, k, P->d_rows64 + r64, n64, P->d_ls64 + (size_t)(k & 1) * nb * 32,
                                P->d_rinv64 + (size_t)(k & 1) * nb);
      if (e != EMU_OK) return e;
      if (split && (e = split64(r64, n64)) != EMU_OK) return e;
    }
    if (n32 > 0 && P->tc_trsm)
      return trsm_tc::launch(ctx, P->lmap, P->opmap, P->d_lkk32, A->t32, nb, NT, k, P->d_rows32 + r32, nullptr, n32);
    if (n32 > 0) {
      ProfScope ps(ctx, PROF_TRSM32, n32 * nb3, 14.0 * n32 * te);
      const float *lkk = P->d_lkk32 + (size_t)(k & 1) * te;
      if (critical)
        k_trsm32_panel<4, 1, TS_NBUF_CRIT><<<dim3(nb / 4, n32), 128, tsm4, ctx->stream>>>(
            lkk, A->t32, A->op_bf16, nb, NT, k, P->d_rows32 + r32, st);
      else
        k_trsm32_panel<8, 2, TS_NBUF_PANEL><<<dim3(nb / 16, n32), 256, tsm16, ctx->stream>>>(
            lkk, A->t32, A->op_bf16, nb, NT, k, P->d_rows32 + r32, st);
      EMU_LAUNCHED(ctx);
    }
    return e;
  };
  // updates of group g of panel k on at most `max_ctas` persistent CTAs
  auto update_group = [&](int k, int g, int max_ctas) -> emu_status {
    const StepPlan &sp = P->steps[k];
    if (sp.p_n[g] > 0) {
      // FP64-class tiles: 36 digit products per K step on the BF16 tensor cores
      ProfScope ps(ctx, PROF_UPDATE64, sp.p_flops[g], 24.0 * sp.p_flops[g] / (2.0 * nb), 36.0 * sp.p_flops[g]);
      emu_status e = gemm64::launch(ctx, P->map64a, P->map64b, P->d_items64 + sp.p_off[g], sp.p_n[g], P->d_segs64,
                                    nb, nb, nb, P->d_exp64, P->d_exp64, gemm64::TC64_SUB, A->t64, nb,
                                    std::max(1, max_ctas));
      if (e != EMU_OK) return e;
    }
    if (sp.i_n[g] > 0) {
      ProfScope ps(ctx, PROF_TC_FACTOR, sp.flops[g], 0.0, sp.mma[g]);
      int in = sp.i_n[g];
      int ctas = std::max(1, max_ctas);
      return gemm_tc::launch(ctx, P->ops, P->d_items + sp.i_off[g], in, P->d_segs, nb / gemm_tc::BK,
                             gemm_tc::TC_SUB_F32, A->t32, nullptr, nb, ctas);
    }
    return EMU_OK;
  };

  for (int k = 0; k < NT && s == EMU_OK; k++) {
    const StepPlan &sp = P->steps[k];
    long tkk = tile_index(k, k, NT);
    // ---- critical stream
    ctx->stream = ctx->crit;
    if (sp.diag_low) {
      ProfScope ps(ctx, PROF_SPLIT, 0.0, 12.0 * te);
      // one element per thread: the widening sits on the critical stream
      k_tile_to_f64<<<(unsigned)((te + 255) / 256), 256, 0, ctx->stream>>>(A->t32 + tkk * te, A->t64 + tkk * te,
                                                                          te, st);
      EMU_LAUNCHED(ctx);
    }
    if ((s = launch_potrf64_tile(ctx, A, k)) != EMU_OK) break;
    // L_kk's FP32 copy and pieces are made on the critical stream only if its
    // own TRSM needs them, else on the panel stream before its TRSMs
    if (sp.n32_1 > 0 && (s = prep32(k)) != EMU_OK) break;
    if (sp.n64_1 + sp.n64_r > 0 &&
        (s = launch_trsm64_prep(ctx, A->t64 + tkk * te, nb, P->d_ls64 + (size_t)(k & 1) * nb * 32,
                                P->d_rinv64 + (size_t)(k & 1) * nb)) != EMU_OK)
      break;
    if (sp.n64_1 + sp.n64_r > 0 && P->blk64 &&
        (s = gemm64::launch_lkk_digits(ctx, A->t64 + tkk * te, nb, P->d_lexp + (size_t)(k & 1) * (nJ - 1) * nb,
                                       P->d_ldig + (k & 1) * lbuf)) != EMU_OK)
      break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_P), ctx->crit));
    if (k > 0) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev(k - 1, E_G1), 0));
    // the BF16 pieces of an FP64-class row k+1 feed only the panel stream's
    // G1(k), unless the critical SYRK or this row's E4M3 / TF32 copies read
    // them: then they are made here, else on the panel stream before G1(k)
    const bool split1_here = sp.i_n[GR_S] > 0 || sp.nq_1 > 0 || sp.nt_1 > 0;
    if ((s = trsm_rows(k, sp.r64_1, sp.n64_1, sp.r32_1, sp.n32_1, true, split1_here)) != EMU_OK) break;
    if ((s = quantize(sp.q_1, sp.nq_1)) != EMU_OK) break;
    if ((s = tf32copy(sp.t_1, sp.nt_1)) != EMU_OK) break;
    if ((s = slice64(sp.z1_off, sp.z1_n)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_T1), ctx->crit));
    if (k > 0) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev(k - 1, E_G2), 0));  // G2A(k-1)
    if ((s = update_group(k, GR_S, ctx->sm_count)) != EMU_OK) break;
    // ---- mid stream
    ctx->stream = ctx->mid;
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->mid, ev(k, E_P), 0));
    if (sp.n32_1 == 0 && sp.n32_r > 0 && (s = prep32(k)) != EMU_OK) break;
    if ((s = trsm_rows(k, sp.r64_r, sp.n64_r, sp.r32_r, sp.n32_r, false)) != EMU_OK) break;
    if ((s = quantize(sp.q_r, sp.nq_r)) != EMU_OK) break;
    if ((s = tf32copy(sp.t_r, sp.nt_r)) != EMU_OK) break;
    if ((s = slice64(sp.zr_off, sp.zr_n)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_T), ctx->mid));
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->mid, ev(k, E_T1), 0));
    if (!split1_here && (s = split64(sp.r64_1, sp.n64_1)) != EMU_OK) break;
    if (k > 0) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->mid, ev(k - 1, E_G2), 0));
    if ((s = update_group(k, GR_G1, ctx->sm_count)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_G1), ctx->mid));
    // ---- bulk stream: persistent on all but kReservedSMs SMs, which stay
    // free for the critical and panel streams' kernels
    ctx->stream = ctx->bulk;
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->bulk, ev(k, E_T), 0));
    // the bulk GEMMs of step k run beside the critical and panel work of
    // steps k and k+1: while that has FP64-class TRSMs or SYRKs (FP64-pipe
    // bound, too much shared memory to fit beside the GEMM) more SMs stay free
    const bool fp64_near = sp.fp64_panel || (k + 1 < NT && P->steps[k + 1].fp64_panel);
    int bulk_ctas = std::max(1, ctx->sm_count - (fp64_near ? R64 : R));
    if ((s = update_group(k, GR_G2A, bulk_ctas)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_G2), ctx->bulk));
    if ((s = update_group(k, GR_G2, bulk_ctas)) != EMU_OK) break;
  }
  ctx->stream = user;
  if (s != EMU_OK) return s;
  for (cudaStream_t q : {ctx->mid, ctx->bulk}) {
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev_end, q));
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev_end, 0));
  }
  EMU_CUDA_TRY(ctx, cudaEventRecord(ev_end, ctx->crit));
  EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(user, ev_end, 0));
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
// Digit slices of the factor's FP64-class tiles for the sampler, with one
// exponent per row of the matrix (shared by the row's FP64 tiles), made once
// after the factor.
static emu_status sampler_slices(emu_ctx *ctx, const emu_mat *L, MixedPlan *P) {
  if (P->samp_ready) return EMU_OK;
  int NT = L->nt, nb = L->nb;
  long npad = (long)NT * nb;
  P->slot_s.assign(L->ntiles, -1);
  std::vector<int4> jobs;
  for (int j = 0; j < NT; j++)
    for (int i = j; i < NT; i++) {
      long t = tile_index(i, j, NT);
      if (P->cls[t] != EMU_CLASS_FP64) continue;
      P->slot_s[t] = P->nslots_s++;
      jobs.push_back(make_int4((int)t, P->slot_s[t], i * nb, 0));
    }
  P->samp_ready = true;
  if (jobs.empty()) return EMU_OK;
  size_t te = (size_t)nb * nb;
  int4 *d_jobs = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_dig_s, (size_t)P->nslots_s * gemm64::NS * te * sizeof(uint16_t), ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_exp_s, npad * sizeof(int), ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_jobs, jobs.size() * sizeof(int4), ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(P->d_exp_s, 0, npad * sizeof(int), ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    ctx->stream));
  emu_status s = gemm64::launch_row_exponents(ctx, L->t64, L->t32, L->d_cls, d_jobs, (int)jobs.size(), nb, P->d_exp_s);
  if (s == EMU_OK)
    s = gemm64::launch_slice(ctx, L->t64, L->t32, L->d_cls, d_jobs, (int)jobs.size(), nb, P->d_exp_s, P->d_dig_s);
  cudaFreeAsync(d_jobs, ctx->stream);
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the host job list must outlive its copy
  if (s != EMU_OK) return s;
  return gemm64::make_map(ctx, &P->map_s, P->d_dig_s, nb, (uint64_t)P->nslots_s * gemm64::NS * nb, gemm64::BM);
}

emu_status mixed_sample(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz, int s, double *Y, long ldy) {
  MixedPlan *P = static_cast<MixedPlan *>(L->plan);
  if (!P) return EMU_ESTATE;
  int NT = L->nt, nb = L->nb;
  long npad = (long)NT * nb;
  int s_pad = ((s + gemm_tc::BN - 1) / gemm_tc::BN) * gemm_tc::BN;
  // Y = 0, then the FP64-class tiles (digit products, FP64 accurate) and the
  // low-precision tiles are added on the tensor cores
  EMU_CUDA_TRY(ctx, cudaMemset2DAsync(Y, ldy * sizeof(double), 0, (size_t)L->n * sizeof(double), s, ctx->stream));
  emu_status st = sampler_slices(ctx, L, P);
  if (st != EMU_OK) return st;
  if (P->nslots_s > 0 && s > 0) {
    std::vector<gemm64::Item> it64;
    std::vector<gemm64::Seg> sg64;
    double f64 = 0.0;
    for (int i = 0; i < NT; i++)
      for (int nbk = 0; nbk < s_pad / gemm64::BN; nbk++)
        for (int mb = 0; mb < nb / gemm64::BM; mb++) {
          long row0 = (long)i * nb + mb * gemm64::BM;
          int cols = std::min(gemm64::BN, s - nbk * gemm64::BN);
          if (row0 >= L->n || cols <= 0) continue;
          gemm64::Item it;
          it.seg_begin = (int)sg64.size();
          for (int k = 0; k <= i; k++) {
            int sl = P->slot_s[tile_index(i, k, NT)];
            if (sl < 0) continue;
            gemm64::Seg sg;
            sg.a_row = sl * gemm64::NS * nb + mb * gemm64::BM;
            sg.b_row = nbk * gemm64::BN;
            sg.a_x = 0;
            sg.b_x = k * nb;
            sg64.push_back(sg);
            f64 += 2.0 * gemm64::BM * gemm64::BN * nb;
          }
          it.seg_end = (int)sg64.size();
          if (it.seg_end == it.seg_begin) continue;
          it.out_off = row0 + (long)nbk * gemm64::BN * ldy;
          it.a_sc = (int)row0;
          it.b_sc = nbk * gemm64::BN;
          it.rows_valid = (int)std::min<long>(gemm64::BM, L->n - row0);
          it.cols_valid = cols;
          it64.push_back(it);
        }
    if (!it64.empty()) {
      uint16_t *zd = nullptr;
      int *ze = nullptr;
      int2 *blk = nullptr;
      gemm64::Item *d_it = nullptr;
      gemm64::Seg *d_sg = nullptr;
      int2 hblk = make_int2(0, (int)npad);
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&zd, (size_t)gemm64::NS * s_pad * npad * sizeof(uint16_t), ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&ze, s_pad * sizeof(int) + 16, ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&blk, sizeof(int2), ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_it, it64.size() * sizeof(gemm64::Item), ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_sg, sg64.size() * sizeof(gemm64::Seg), ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMemcpyAsync(blk, &hblk, sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_it, it64.data(), it64.size() * sizeof(gemm64::Item),
                                        cudaMemcpyHostToDevice, ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_sg, sg64.data(), sg64.size() * sizeof(gemm64::Seg), cudaMemcpyHostToDevice,
                                        ctx->stream));
      CUtensorMap zmap;
      st = gemm64::launch_slice_z(ctx, Z, ldz, s, s_pad, blk, 1, npad, ze, zd);
      if (st == EMU_OK) st = gemm64::make_map(ctx, &zmap, zd, npad, (uint64_t)gemm64::NS * s_pad, gemm64::BN);
      if (st == EMU_OK) {
        ProfScope ps(ctx, PROF_TRMM64, f64, 0.0, 36.0 * f64);
        st = gemm64::launch(ctx, P->map_s, zmap, d_it, (int)it64.size(), d_sg, nb, nb, s_pad, P->d_exp_s, ze,
                            gemm64::TC64_ADD, Y, (int)ldy, ctx->sm_count);
      }
      for (void *q : {(void *)zd, (void *)ze, (void *)blk, (void *)d_it, (void *)d_sg}) cudaFreeAsync(q, ctx->stream);
      // the host item lists must outlive their copies
      EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      if (st != EMU_OK) return st;
    }
  }
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
          // the sampler reads E4M3-class tiles through their leading BF16 piece
          // TF32-class tiles are drawn on the FP32 path (their three BF16 pieces exist)
          sg.cls = (c == EMU_CLASS_FP32 || c == EMU_CLASS_TF32) ? EMU_CLASS_FP32 : EMU_CLASS_BF16;
          sg.pad = 0;
          segs.push_back(sg);
        }
        it.seg_end = (int)segs.size();
        if (it.seg_end == it.seg_begin) continue;
        it.out_off = row0 + (long)nbk * gemm_tc::BN * ldy;
        it.rows_valid = (int)std::min<long>(gemm_tc::BM, L->n - row0);
        it.cols_valid = s - nbk * gemm_tc::BN;
        it.sa = it.sb = -1;
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
  gemm_tc::Operands ops = P->ops;
  st = gemm_tc::make_map_bf16(ctx, &ops.b16, zp, npad, (uint64_t)3 * s_pad, gemm_tc::BN);
  ProfScope ps(ctx, PROF_TC_SAMPLE, tf, 0.0, tm);
  if (st == EMU_OK)
    st = gemm_tc::launch(ctx, ops, d_items, (int)items.size(), d_segs, nb / gemm_tc::BK,
                         gemm_tc::TC_ADD_F64, nullptr, Y, (int)ldy, ctx->sm_count);
  cudaFreeAsync(zp, ctx->stream);
  cudaFreeAsync(d_items, ctx->stream);
  cudaFreeAsync(d_segs, ctx->stream);
  // the host vectors above must outlive the asynchronous copies
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return st;
}

emu_status mixed_potrs(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs) {
  if (mixed_potrs_blocked_supports(L->nb)) return mixed_potrs_blocked(ctx, L, X, ldx, nrhs);
  // nb > 1024: one thread per row and right-hand side
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
  if (MixedCtx *M = static_cast<MixedCtx *>(ctx->mixed)) {
    if (M->exec) cudaGraphExecDestroy(M->exec);
    if (M->cap) cudaStreamDestroy(M->cap);
    if (M->ev_a) cudaEventDestroy(M->ev_a);
    if (M->ev_b) cudaEventDestroy(M->ev_b);
    delete M;
    ctx->mixed = nullptr;
  }
  for (cudaEvent_t e : ctx->sched_ev) cudaEventDestroy(e);
  ctx->sched_ev.clear();
  if (ctx->crit) cudaStreamDestroy(ctx->crit);
  if (ctx->mid) cudaStreamDestroy(ctx->mid);
  if (ctx->bulk) cudaStreamDestroy(ctx->bulk);
  ctx->crit = ctx->mid = ctx->bulk = nullptr;
}

// ------------------------------------------------ batched factor launchers
// The batched factor (batch.cu) runs the same kernels over explicit tile
// indices of one shared arena: lists of tiles or jobs instead of (k, NT).
namespace {

// FP32 -> FP64 of listed whole tiles (low-precision diagonal tiles before
// their FP64 POTRF).
__global__ void k_tiles_to_f64(const float *__restrict__ t32, double *__restrict__ t64, const long *__restrict__ tiles,
                               size_t te, const int *st) {
  if (failed(st)) return;
  size_t base = (size_t)tiles[blockIdx.y] * te;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < te; e += (size_t)gridDim.x * blockDim.x)
    t64[base + e] = (double)t32[base + e];
}

// FP32 copies of listed FP64 diagonal factor tiles into consecutive slots.
__global__ void k_diag_to_f32_slots(const double *__restrict__ t64, float *__restrict__ slots,
                                    const long *__restrict__ tiles, size_t te, const int *st) {
  if (failed(st)) return;
  size_t base = (size_t)tiles[blockIdx.y] * te;
  float *d = slots + (size_t)blockIdx.y * te;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < te; e += (size_t)gridDim.x * blockDim.x)
    d[e] = (float)t64[base + e];
}

}  // namespace

emu_status launch_to_f32_tiles(emu_ctx *ctx, const double *t64, float *t32, const unsigned char *cls, long ntiles,
                               size_t te) {
  if (ntiles <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 12.0 * ntiles * te);
  k_to_f32<<<dim3(16, (unsigned)ntiles), 256, 0, ctx->stream>>>(t64, t32, cls, te);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_tiles_to_f64(emu_ctx *ctx, const float *t32, double *t64, const long *d_tiles, int n, size_t te) {
  if (n <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 12.0 * n * te);
  k_tiles_to_f64<<<dim3(16, n), 256, 0, ctx->stream>>>(t32, t64, d_tiles, te, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_diag_to_f32_slots(emu_ctx *ctx, const double *t64, float *slots, const long *d_tiles, int n,
                                    size_t te) {
  if (n <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 12.0 * n * te);
  k_diag_to_f32_slots<<<dim3(16, n), 256, 0, ctx->stream>>>(t64, slots, d_tiles, te, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_trsm32_jobs(emu_ctx *ctx, const float *slots, float *t32, uint16_t *op, int nb, const int2 *d_jobs,
                              int njobs) {
  if (njobs <= 0) return EMU_OK;
  size_t sm = trsm32_smem(nb, 16, TS_NBUF_PANEL);
  EMU_CUDA_TRY(ctx, cudaFuncSetAttribute(k_trsm32_panel<8, 2, TS_NBUF_PANEL, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  double nb3 = (double)nb * nb * nb;
  ProfScope ps(ctx, PROF_TRSM32, njobs * nb3, 14.0 * njobs * nb * nb);
  k_trsm32_panel<8, 2, TS_NBUF_PANEL, true><<<dim3(nb / 16, njobs), 256, sm, ctx->stream>>>(
      slots, t32, op, nb, 0, 0, nullptr, ctx->d_status, d_jobs);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_split_tiles64(emu_ctx *ctx, const double *t64, uint16_t *op, const int *d_tiles, int n, int nb,
                                int lower_only) {
  if (n <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 14.0 * n * (double)nb * nb);
  k_split_tiles<double><<<dim3((nb / B) * (nb / B), n), 256, 0, ctx->stream>>>(t64, op, d_tiles, nb, lower_only,
                                                                            ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_quant_e4m3(emu_ctx *ctx, const uint16_t *op, uint8_t *op8, float *scales, const int *d_tiles, int n,
                             int nb) {
  if (n <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 3.0 * n * (double)nb * nb);
  k_quant_e4m3<<<n, 1024, 0, ctx->stream>>>(op, op8, scales, d_tiles, nb, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_split_z(emu_ctx *ctx, const double *Z, long ldz, long npad, int s, int s_pad, uint16_t *zp) {
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 14.0 * npad * s_pad);
  k_split_z<<<8 * ctx->sm_count, 256, 0, ctx->stream>>>(Z, ldz, npad, s, s_pad, zp);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}
