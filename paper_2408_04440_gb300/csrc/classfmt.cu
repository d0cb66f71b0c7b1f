// classfmt.cu -- class-format tile storage for covariances whose FP64 lower
// triangle does not fit the device ("Mixed-Precision Computation
// Innovations": tiles are allocated at the size of their precision, and a
// producer converts a tile once into the precision its consumers need;
// "Performance Results": the problem size grows with L).
//
// Every lower tile lives in the format of its class, column-major nb x nb:
//   FP64 (every diagonal tile, and the FP64-class tiles)  8 bytes / entry
//   FP32 class                                            4 bytes
//   BF16 class                                            2 bytes
//   E4M3 class: BF16 while the tile is a trailing (Schur complement) tile,
//     then, once solved, codes q of the value q / s with a power-of-two s per
//     tile (1 byte, in the first half of the tile's 2-byte slot)
// and is re-rounded to its working format after every trailing update (the
// tensor cores accumulate each update in FP32 in TMEM).  Re-rounding trailing
// tiles to E4M3 itself after each update made factors of these covariances
// lose positive definiteness (at eps = 1e-4, L = 40); BF16 working storage
// keeps the backward error within eps.  Panel k is decoded into
// FP32 / FP64 panel buffers (a ring of three panels), solved by the same
// TRSM kernels as the FP32-master factor, rounded back to its storage format,
// and the panel's operand copies (three BF16 pieces, FP8 copies, FP64 digit
// slices) are made from the rounded values, so every later update uses the
// stored factor tiles exactly.
// The sampler converts the stored tiles of a group of tile columns into
// K-major BF16 operand planes and accumulates Y = L Z on the tensor cores
// (FP64-class tiles as exact digit products).
// The backward error of a factor is estimated without Sigma in memory:
// ||(L L^T - S) G||_F / sqrt(p) over p Gaussian probes (Hutchinson), with
// S G regenerated from the covariance's parameters.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "emu_internal.h"
#include "gemm_f64.h"
#include "gemm_tc.h"
#include "mixed.h"
#include "rng.cuh"
#include "trsm_tc.h"

namespace {

constexpr int RING = 3;  // panels whose buffers are live at once
constexpr int TB = 32;   // transpose block

__device__ inline bool failed(const int *st) { return *((volatile const int *)st) != DEV_OK; }

__device__ inline float e4m3_to_float(uint8_t q) {
  return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3)));
}
__device__ inline uint8_t float_to_e4m3(float x) {
  return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// Decode panel tiles from their storage into the panel buffers: jobs
// {panel index, slot, class, -}; FP64 tiles to P64, the others to P32 (as
// FP32, exactly: every storage value is an FP32 number).
__global__ void k_decode(const int4 *__restrict__ jobs, size_t te, const double *__restrict__ t64,
                         const float *__restrict__ t32, const uint16_t *__restrict__ t16,
                         const uint8_t *__restrict__ t8, const float *__restrict__ sc8, double *__restrict__ P64,
                         float *__restrict__ P32, const int *st) {
  if (failed(st)) return;
  const int4 j = jobs[blockIdx.y];
  const size_t o = (size_t)j.y * te, p = (size_t)j.x * te;
  const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
  if (j.z == EMU_CLASS_FP64) {
    for (size_t e = i0; e < te; e += step) P64[p + e] = t64[o + e];
  } else if (j.z == EMU_CLASS_FP32) {
    for (size_t e = i0; e < te; e += step) P32[p + e] = t32[o + e];
  } else if (j.z == EMU_CLASS_BF16) {
    for (size_t e = i0; e < te; e += step) P32[p + e] = __bfloat162float(__ushort_as_bfloat16(t16[o + e]));
  } else {
    // an E4M3-class tile before its panel step: its BF16 working values
    const uint16_t *w = reinterpret_cast<const uint16_t *>(t8);
    for (size_t e = i0; e < te; e += step) P32[p + e] = __bfloat162float(__ushort_as_bfloat16(w[o + e]));
  }
}

// Round solved panel tiles to their storage format and store them: jobs
// {panel index, slot, class, -} for the FP64, FP32 and BF16 classes.  BF16
// tiles: the stored value bf16(x) also replaces x in the FP32 panel buffer,
// and the operand pieces become (bf16(x), 0, 0) (piece 0 already is bf16(x)).
__global__ void k_encode(const int4 *__restrict__ jobs, int nb, double *__restrict__ t64, float *__restrict__ t32,
                         uint16_t *__restrict__ t16, const double *__restrict__ P64, float *__restrict__ P32,
                         uint16_t *__restrict__ Pop, const int *st) {
  if (failed(st)) return;
  const int4 j = jobs[blockIdx.y];
  const size_t te = (size_t)nb * nb;
  const size_t o = (size_t)j.y * te, p = (size_t)j.x * te;
  const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
  if (j.z == EMU_CLASS_FP64) {
    for (size_t e = i0; e < te; e += step) t64[o + e] = P64[p + e];
  } else if (j.z == EMU_CLASS_FP32) {
    for (size_t e = i0; e < te; e += step) t32[o + e] = P32[p + e];
  } else {
    uint16_t *p1 = Pop + ((size_t)j.x * 3 + 1) * te;
    for (size_t e = i0; e < te; e += step) {
      const __nv_bfloat16 b = __float2bfloat16_rn(P32[p + e]);
      t16[o + e] = __bfloat16_as_ushort(b);
      P32[p + e] = __bfloat162float(b);
      p1[e] = 0;
      p1[e + te] = 0;
    }
  }
}

// E4M3-class panel tiles, jobs {panel index, slot, -, -}: the tile's amax
// (k_amax_tiles: partial maxima of 64 CTAs per tile folded by an integer
// atomicMax on the bits, which order non-negative floats), then
// (k_encode_e4m3, one CTA per 32 x 32 block and tile) the scale
// s = 2^floor(log2(448 / amax)) (1 for a zero tile), the codes q = e4m3(x s)
// (saturating, nearest) into the first half of the slot (column-major; the
// slot's BF16 working values are no longer needed) and, transposed, into the
// panel's FP8 operand copy (row-major) with scale s; the value q / s replaces
// x in the FP32 panel buffer, and the operand pieces become (bf16(q / s), 0, 0)
// (exact: an E4M3 value fits BF16).
__global__ void __launch_bounds__(256) k_amax_tiles(const int4 *__restrict__ jobs, int nb,
                                                    const float *__restrict__ P32, unsigned *__restrict__ amax_bits,
                                                    const int *st) {
  if (failed(st)) return;
  const int4 j = jobs[blockIdx.y];
  const size_t te = (size_t)nb * nb;
  const float4 *x = reinterpret_cast<const float4 *>(P32 + (size_t)j.x * te);
  float m = 0.0f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < te / 4; e += (size_t)gridDim.x * blockDim.x) {
    const float4 v = x[e];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&amax_bits[j.x], __float_as_uint(m));
}

__device__ inline float e4m3_scale(float m) {
  if (!(m > 0.0f)) return 1.0f;
  // 448 / m = f 2^e with f in [0.5, 1): the largest power of two not above it is 2^(e-1)
  int e = 1;
  frexpf(448.0f / m, &e);
  return ldexpf(1.0f, e - 1);
}

__global__ void __launch_bounds__(256) k_encode_e4m3(const int4 *__restrict__ jobs, int nb, uint8_t *__restrict__ t8,
                                                     float *__restrict__ sc8, float *__restrict__ P32,
                                                     uint16_t *__restrict__ Pop, uint8_t *__restrict__ P8,
                                                     float *__restrict__ Psc8, const unsigned *__restrict__ amax_bits,
                                                     const int *st) {
  if (failed(st)) return;
  __shared__ float blk[TB][TB + 1];
  const int4 j = jobs[blockIdx.y];
  const size_t te = (size_t)nb * nb;
  const float s = e4m3_scale(__uint_as_float(amax_bits[j.x])), inv = 1.0f / s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc8[j.y] = s;
    Psc8[j.x] = s;
  }
  const int nbb = nb / TB;
  const int rb = blockIdx.x % nbb, cb = blockIdx.x / nbb;
  const int tx = threadIdx.x & (TB - 1), ty = threadIdx.x >> 5;  // 32 x 8
  float *x = P32 + (size_t)j.x * te;
  uint8_t *q8 = t8 + (size_t)j.y * 2 * te;
  uint8_t *p8 = P8 + (size_t)j.x * te;
  uint16_t *p0 = Pop + (size_t)j.x * 3 * te;
  for (int yy = ty; yy < TB; yy += 8) {
    // element (r, c) = (rb*32 + tx, cb*32 + yy): column-major, coalesced over tx
    const size_t e = (size_t)(rb * TB + tx) + (size_t)(cb * TB + yy) * nb;
    const uint8_t q = float_to_e4m3(x[e] * s);
    q8[e] = q;
    const float v = e4m3_to_float(q) * inv;
    x[e] = v;
    blk[yy][tx] = v;
  }
  __syncthreads();
  for (int yy = ty; yy < TB; yy += 8) {
    // transposed: row r = rb*32 + yy, column c = cb*32 + tx (row-major, coalesced over tx)
    const float w = blk[tx][yy];
    const size_t f = (size_t)(rb * TB + yy) * nb + (cb * TB + tx);
    p8[f] = float_to_e4m3(w * s);
    p0[f] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
    p0[f + te] = 0;
    p0[f + 2 * te] = 0;
  }
}

// Zero the strict upper triangle of listed FP64 slots (diagonal factor tiles).
__global__ void k_tril_slots(const int *__restrict__ slots, int nb, double *__restrict__ t64) {
  double *T = t64 + (size_t)slots[blockIdx.y] * nb * nb;
  const int c = blockIdx.x;
  for (int r = threadIdx.x; r < c; r += blockDim.x) T[r + (size_t)c * nb] = 0.0;
}

// Sampler operand planes, K-major BF16, from stored tiles: jobs {slot,
// class, first plane, -}; FP32 tiles give three planes (the exact split
// x = p0 + p1 + p2), BF16 and E4M3 tiles one (E4M3 values fit BF16 exactly).
// One CTA of 32 x 8 threads per (32 x 32 block, job).
__global__ void k_samp_planes(const int4 *__restrict__ jobs, int nb, const float *__restrict__ t32,
                              const uint16_t *__restrict__ t16, const uint8_t *__restrict__ t8,
                              const float *__restrict__ sc8, uint16_t *__restrict__ planes) {
  __shared__ float blk[TB][TB + 1];
  const int4 j = jobs[blockIdx.y];
  const size_t te = (size_t)nb * nb;
  const int nbb = nb / TB;
  const int rb = blockIdx.x % nbb, cb = blockIdx.x / nbb;
  const int tx = threadIdx.x & (TB - 1), ty = threadIdx.x >> 5;
  const size_t o = (size_t)j.x * te;
  const float inv8 = (j.y == EMU_CLASS_E4M3) ? 1.0f / sc8[j.x] : 1.0f;
  for (int yy = ty; yy < TB; yy += 8) {
    const size_t e = (size_t)(rb * TB + tx) + (size_t)(cb * TB + yy) * nb;  // within the tile
    float v;
    if (j.y == EMU_CLASS_FP32) v = t32[o + e];
    else if (j.y == EMU_CLASS_BF16) v = __bfloat162float(__ushort_as_bfloat16(t16[o + e]));
    else v = e4m3_to_float(t8[2 * o + e]) * inv8;  // a solved E4M3 tile: codes in its slot's first half
    blk[yy][tx] = v;
  }
  __syncthreads();
  for (int yy = ty; yy < TB; yy += 8) {
    const float x = blk[tx][yy];  // element (rb*32 + yy, cb*32 + tx)
    const size_t f = (size_t)(rb * TB + yy) * nb + (cb * TB + tx);
    uint16_t *pl = planes + (size_t)j.z * te;
    const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
    pl[f] = __bfloat16_as_ushort(b0);
    if (j.y == EMU_CLASS_FP32) {
      const float r1 = x - __bfloat162float(b0);
      const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
      const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
      pl[f + te] = __bfloat16_as_ushort(b1);
      pl[f + 2 * te] = __bfloat16_as_ushort(b2);
    }
  }
}

// Tile (i, j)'s entry (r, c) from its storage, as FP64.
struct TileSrc {
  const unsigned char *cls;  // per tile
  const int *slot;           // per tile
  const double *t64;
  const float *t32;
  const uint16_t *t16;
  const uint8_t *t8;
  const float *sc8;
  int nb, NT;
  int master;      // FP32-master storage: every non-FP64 tile is an FP32 master
  int e4m3_final;  // class format: E4M3 tiles hold their codes (factor), else BF16 working values
};
__device__ inline double tile_at(const TileSrc &S, long t, size_t e, int c, int sl) {
  const size_t o = (size_t)sl * S.nb * S.nb + e;
  if (c == EMU_CLASS_FP64) return S.t64[o];
  if (S.master) return (double)S.t32[o];
  if (c == EMU_CLASS_FP32 || c == EMU_CLASS_TF32) return (double)S.t32[o];
  if (c == EMU_CLASS_BF16) return (double)__bfloat162float(__ushort_as_bfloat16(S.t16[o]));
  if (!S.e4m3_final) return (double)__bfloat162float(__ushort_as_bfloat16(reinterpret_cast<const uint16_t *>(S.t8)[o]));
  return (double)e4m3_to_float(S.t8[(size_t)sl * S.nb * S.nb + o]) / (double)S.sc8[sl];
}

// Dense lower triangle of a stored matrix (export): one CTA per (tile, column).
__global__ void k_export_class(TileSrc S, int n, double *__restrict__ out, long ld) {
  const long t = blockIdx.x;
  int ti, tj;
  tile_coords(t, S.NT, &ti, &tj);
  const int c = blockIdx.y, cl = S.cls[t], sl = S.slot[t];
  const long gc = (long)tj * S.nb + c;
  if (gc >= n) return;
  for (int r = threadIdx.x; r < S.nb; r += blockDim.x) {
    const long gr = (long)ti * S.nb + r;
    if (gr >= n) break;
    const double v = (gr >= gc) ? tile_at(S, t, (size_t)r + (size_t)c * S.nb, cl, sl) : 0.0;
    out[gr + gc * ld] = v;
  }
}

// ---------------------------------------------------- backward-error estimate
// Block products with the stored factor, FP64 on the SIMT pipes, p <= 32
// probe columns (column-major n_pad x p arrays, leading dimension ldx):
//   trans = 0: Y[rows of i] += L_ij X[rows of j]
//   trans = 1: Y[rows of j] += L_ij^T X[rows of i]
// One CTA per (tile, 64-row output slab); atomics add the tiles' parts.
constexpr int HS = 64;  // output slab
constexpr int HK = 32;  // inner chunk
__global__ void __launch_bounds__(256) k_hutch_apply(TileSrc S, int trans, int p, const double *__restrict__ X,
                                                     double *__restrict__ Y, long ldx) {
  __shared__ double a[HK][HS + 1];  // a[k][m]: operand entry for output m, inner k
  __shared__ double x[HK][33];      // x[k][q]
  const long t = blockIdx.x;
  int ti, tj;
  tile_coords(t, S.NT, &ti, &tj);
  const bool diag = ti == tj;
  // the diagonal factor tiles of FP32-master storage are FP64 whatever their class
  const int cl = (S.master && diag) ? EMU_CLASS_FP64 : S.cls[t], sl = S.slot[t], nb = S.nb;
  const int m0 = blockIdx.y * HS;
  const int out_blk = trans ? tj : ti, in_blk = trans ? ti : tj;
  const int tid = threadIdx.x;
  // thread: outputs m = tid % 64 (+0), probes q = tid / 64 + 4 w, w < 8
  const int mm = tid & (HS - 1), q0 = tid >> 6;
  double acc[8];
#pragma unroll
  for (int w = 0; w < 8; w++) acc[w] = 0.0;
  for (int k0 = 0; k0 < nb; k0 += HK) {
    // operand: trans = 0: L(m0 + m, k0 + k); trans = 1: L(k0 + k, m0 + m)
    for (int e = tid; e < HK * HS; e += 256) {
      int k, m;
      size_t idx;
      bool lower;
      if (!trans) {
        m = e % HS;
        k = e / HS;
        idx = (size_t)(m0 + m) + (size_t)(k0 + k) * nb;  // column-major: consecutive m coalesced
        lower = !diag || (m0 + m) >= (k0 + k);
      } else {
        k = e % HK;
        m = e / HK;
        idx = (size_t)(k0 + k) + (size_t)(m0 + m) * nb;
        lower = !diag || (k0 + k) >= (m0 + m);
      }
      a[k][m] = lower ? tile_at(S, t, idx, cl, sl) : 0.0;
    }
    for (int e = tid; e < HK * 32; e += 256) {
      const int k = e % HK, q = e / HK;
      x[k][q] = q < p ? X[(size_t)in_blk * nb + k0 + k + (size_t)q * ldx] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < HK; k++) {
      const double av = a[k][mm];
#pragma unroll
      for (int w = 0; w < 8; w++) acc[w] = fma(av, x[k][q0 + 4 * w], acc[w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int w = 0; w < 8; w++) {
    const int q = q0 + 4 * w;
    if (q < p) atomicAdd(&Y[(size_t)out_blk * nb + m0 + mm + (size_t)q * ldx], acc[w]);
  }
}

// W = S X with S regenerated from its parameters (the synthetic covariance of
// the library: sigma_l sigma_l' rho(dl, dm), nugget on the diagonal) for both
// triangles: one CTA per (tile row block i, tile column block j, 64-row slab
// of block i), over all NT x NT blocks.  Same tables and operation order as the builder.
__global__ void __launch_bounds__(256) k_sigma_apply(int L, int n, int nb, const double *__restrict__ sigma,
                                                     const double *__restrict__ rho, const double *__restrict__ nugget,
                                                     int p, const double *__restrict__ X, double *__restrict__ Y,
                                                     long ldx) {
  __shared__ double a[HK][HS + 1];
  __shared__ double x[HK][33];
  const int bi = blockIdx.x, bj = blockIdx.y, slab = blockIdx.z;
  const int m0 = slab * HS;
  if (m0 >= nb) return;
  const int W = 4 * L - 3;
  const double nug = *nugget;
  const int tid = threadIdx.x, mm = tid & (HS - 1), q0 = tid >> 6;
  double acc[8];
#pragma unroll
  for (int w = 0; w < 8; w++) acc[w] = 0.0;
  for (int k0 = 0; k0 < nb; k0 += HK) {
    for (int e = tid; e < HK * HS; e += 256) {
      const int m = e % HS, k = e / HS;
      const long gi = (long)bi * nb + m0 + m, gj = (long)bj * nb + k0 + k;
      double v = 0.0;
      if (gi < n && gj < n) {
        int li = (int)sqrtf((float)gi);
        while ((long)li * li > gi) li--;
        while ((long)(li + 1) * (li + 1) <= gi) li++;
        int lj = (int)sqrtf((float)gj);
        while ((long)lj * lj > gj) lj--;
        while ((long)(lj + 1) * (lj + 1) <= gj) lj++;
        const int mi = (int)(gi - (long)li * li - li), mj = (int)(gj - (long)lj * lj - lj);
        const double r = rho[(long)(li - lj + L - 1) * W + (mi - mj + 2 * L - 2)];
        v = __dmul_rn(__dmul_rn(sigma[li], sigma[lj]), r);
        if (gi == gj) v = __dadd_rn(v, nug);
      }
      a[k][m] = v;
    }
    for (int e = tid; e < HK * 32; e += 256) {
      const int k = e % HK, q = e / HK;
      x[k][q] = q < p ? X[(size_t)bj * nb + k0 + k + (size_t)q * ldx] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < HK; k++) {
      const double av = a[k][mm];
#pragma unroll
      for (int w = 0; w < 8; w++) acc[w] = fma(av, x[k][q0 + 4 * w], acc[w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int w = 0; w < 8; w++) {
    const int q = q0 + 4 * w;
    if (q < p) atomicAdd(&Y[(size_t)bi * nb + m0 + mm + (size_t)q * ldx], acc[w]);
  }
}

// Gaussian probes G (n_pad x p, zero beyond n) from the library's normals.
__global__ void k_probes(uint64_t seed, int n, long npad, int p, double *__restrict__ G, long ldg) {
  const long npairs = (npad + 1) / 2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < npairs * p; q += (long)gridDim.x * blockDim.x) {
    const long pr = q % npairs;
    const int col = (int)(q / npairs);
    double z[2] = {0.0, 0.0};
    normal_pair(seed, 7u, pr, col, (int)npad, z);
    for (int u = 0; u < 2; u++) {
      const long r = 2 * pr + u;
      if (r < npad) G[r + (size_t)col * ldg] = r < n ? z[u] : 0.0;
    }
  }
}

// sum over the first n rows of each of p columns of (V - W)^2, one double.
__global__ void k_diff_sq(int n, int p, const double *__restrict__ V, const double *__restrict__ Wm, long ld,
                          double *__restrict__ out) {
  double s = 0.0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * p; e += (long)gridDim.x * blockDim.x) {
    const long r = e % n, q = e / n;
    const double d = V[r + q * ld] - Wm[r + q * ld];
    s += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

}  // namespace

// ====================================================================== host
namespace {

// Factor schedule of a class-format matrix: per panel step, job lists for
// the critical row (k + 1) and the other rows (>= k + 2), and the update
// groups of mixed.cu's lookahead schedule (S, G1, G2A, G2).
enum { CG_S = 0, CG_G1 = 1, CG_G2A = 2, CG_G2 = 3, CG_N = 4 };
struct Range {
  int off = 0, n = 0;
};
struct CPart {       // the panel tiles of one stream in one step
  Range dec;         // decode jobs (int4 {pi, slot, cls, -})
  Range t64;         // FP64 TRSM jobs (int2 {pi, pi of L_kk}); the same pi in `pis`
  Range t32;         // low-class TRSM jobs (int2 {pi, L slot})
  Range enc;         // encode jobs FP64 / FP32 / BF16 (int4)
  Range enc8;        // E4M3 encode jobs (int4)
  Range split;       // panel indices of the FP64 rows, split into BF16 pieces after their TRSM (int)
  Range quant;       // panel indices quantized to FP8 for E4M3 consumers (int)
  Range slice;       // digit-slice jobs (int4 {pi, pi, pi * nb, 0})
};
struct CStep {
  CPart crit, mid;
  Range tc[CG_N], g64[CG_N];
  double flops[CG_N] = {}, mma[CG_N] = {}, f64[CG_N] = {};
  bool fp64_panel = false;
  bool low_panel = false;
};

struct ClassPlan {
  int NT = 0, nb = 0;
  std::vector<CStep> steps;
  // device lists, one allocation
  void *d_blob = nullptr;
  int4 *d_j4 = nullptr;        // decode / encode / slice jobs
  int2 *d_j2 = nullptr;        // TRSM jobs
  int *d_i1 = nullptr;         // panel-index lists (split, quantize) and L slots of FP64 TRSM jobs
  long *d_kk = nullptr;        // per step: FP64 slot of L_kk (for the FP32 copy of L_kk)
  unsigned char *d_pcls = nullptr;  // per step: 3 NT classes by panel index
  gemm_tc::Item *d_items = nullptr;
  gemm_tc::Seg *d_segs = nullptr;
  gemm64::Item *d_items64 = nullptr;
  gemm64::Seg *d_segs64 = nullptr;
  int *d_jslot = nullptr;      // FP64 TRSM jobs: pre-scaled L_kk slot (k & 1)
  // panel ring
  double *P64 = nullptr;
  float *P32 = nullptr;
  uint16_t *Pop = nullptr;
  uint8_t *P8 = nullptr;
  float *Psc8 = nullptr;
  uint16_t *digits = nullptr;
  int *exps = nullptr;
  unsigned *amax = nullptr;    // per panel index: amax bits of the E4M3-class tiles being encoded
  float *lkk32 = nullptr;      // FP32 copies of L_kk (two slots)
  uint16_t *lkkp = nullptr;    // their pieces (tensor-core TRSM)
  double *ls64 = nullptr, *rinv64 = nullptr;  // pre-scaled L_kk blocks for the FP64 TRSM
  gemm_tc::Operands ops;
  CUtensorMap map64a, map64b, lmap, opmap;
  bool tc_trsm = false;
  double update_flops[EMU_NCLASS] = {};
  int tiles[EMU_NCLASS] = {};
  std::vector<char> host;
  cudaStream_t stream = nullptr;
};

void cplan_free(ClassPlan *P) {
  if (!P) return;
  for (void *q : {(void *)P->d_blob, (void *)P->P64, (void *)P->P32, (void *)P->Pop, (void *)P->P8,
                  (void *)P->Psc8, (void *)P->digits, (void *)P->exps, (void *)P->amax, (void *)P->lkk32,
                  (void *)P->lkkp, (void *)P->ls64, (void *)P->rinv64})
    if (q) cudaFreeAsync(q, P->stream);
  delete P;
}

emu_status fail_status(emu_ctx *ctx, emu_status s, const char *msg) {
  ctx->last_error = msg;
  return s;
}

}  // namespace

void classfmt_release(emu_mat *A) {
  ClassStore *cs = A->cs;
  if (!cs) return;
  cudaStream_t s = A->ctx ? A->ctx->stream : nullptr;
  cplan_free(static_cast<ClassPlan *>(cs->work));
  for (void *q : {(void *)cs->d_slot, (void *)cs->t64, (void *)cs->t32, (void *)cs->t16, (void *)cs->t8,
                  (void *)cs->sc8, (void *)cs->samp_dig, (void *)cs->samp_exp})
    if (q) cudaFreeAsync(q, s);
  delete cs;
  A->cs = nullptr;
}

// ----------------------------------------------------------------- build
// The covariance straight into class format: a norm pass (no stores), the
// precision map, then every tile computed again and stored in its class.
// Diagonal tiles are FP64 (their POTRF is FP64 and they stay FP64 in the
// factor); TF32 is not a storage class.
emu_status classfmt_build(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p, const emu_mp_opts *o) {
  const int NT = A->nt, nb = A->nb;
  const size_t te = A->tile_elems;
  emu_status s = launch_cov_norms(ctx, A, p);
  if (s != EMU_OK) return s;
  double u[EMU_NCLASS] = {0x1p-53, 0x1p-24 * sqrt((double)nb), 0x1p-11, 0x1p-8, 0x1p-4};
  for (int c = 0; c < EMU_NCLASS; c++)
    if (o->u[c] > 0.0) u[c] = o->u[c];
  unsigned mask = (o->prec_mask | 1u) & ((1u << EMU_NCLASS) - 1u) & ~(1u << EMU_CLASS_TF32);
  if (o->band == EMU_MAP_NORM && !(o->eps > 0.0)) mask = 1u;  // eps <= 0: every tile FP64
  if ((s = launch_precision_map(ctx, A, o->eps > 0.0 ? o->eps : 0.0, u, mask, 1, o->band, band_sp_frac(o))) !=
      EMU_OK)
    return s;
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(A->h_cls, A->d_cls, A->ntiles, cudaMemcpyDeviceToHost, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(&A->frob, A->d_frob, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  ClassStore *cs = new ClassStore();
  A->cs = cs;
  cs->cls.assign(A->h_cls, A->h_cls + A->ntiles);
  cs->slot.assign(A->ntiles, -1);
  for (long t = 0; t < A->ntiles; t++) {
    int c = cs->cls[t];
    if (c == EMU_CLASS_TF32) c = cs->cls[t] = EMU_CLASS_FP32;
    cs->slot[t] = cs->nslot[c]++;
  }
  // E4M3 scales are set when each tile is solved (its final codes)
  std::vector<float> sc8(std::max(1, cs->nslot[EMU_CLASS_E4M3]), 1.0f);
  cudaStream_t st = ctx->stream;
  auto alloc = [&](void **q, size_t bytes) -> cudaError_t {
    return bytes ? cudaMallocAsync(q, bytes, st) : cudaSuccess;
  };
  cudaError_t e = alloc((void **)&cs->d_slot, A->ntiles * sizeof(int));
  if (e == cudaSuccess) e = alloc((void **)&cs->t64, cs->nslot[EMU_CLASS_FP64] * te * sizeof(double));
  if (e == cudaSuccess) e = alloc((void **)&cs->t32, cs->nslot[EMU_CLASS_FP32] * te * sizeof(float));
  if (e == cudaSuccess) e = alloc((void **)&cs->t16, cs->nslot[EMU_CLASS_BF16] * te * sizeof(uint16_t));
  if (e == cudaSuccess) e = alloc((void **)&cs->t8, cs->nslot[EMU_CLASS_E4M3] * te * 2);  // BF16 working values
  if (e == cudaSuccess) e = alloc((void **)&cs->sc8, sc8.size() * sizeof(float));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? EMU_ENOMEM : emu_cuda_fail(ctx, e, "class arenas");
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(cs->d_slot, cs->slot.data(), A->ntiles * sizeof(int), cudaMemcpyHostToDevice, st));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(A->d_cls, cs->cls.data(), A->ntiles, cudaMemcpyHostToDevice, st));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(cs->sc8, sc8.data(), sc8.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  ClassArenas ar{cs->d_slot, A->d_cls, cs->t64, cs->t32, cs->t16, cs->t8, cs->sc8};
  s = launch_cov_store_class(ctx, A, p, ar);
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));  // host vectors above
  memcpy(A->h_cls, cs->cls.data(), A->ntiles);
  return s;
}

// ----------------------------------------------------------------- factor
namespace {

emu_status build_cplan(emu_ctx *ctx, emu_mat *A, ClassPlan *P) {
  ClassStore *cs = A->cs;
  const int NT = A->nt, nb = A->nb;
  const size_t te = A->tile_elems;
  P->NT = NT;
  P->nb = nb;
  P->stream = ctx->stream;
  auto C = [&](int i, int j) { return (int)cs->cls[tile_index(i, j, NT)]; };
  auto SL = [&](int i, int j) { return cs->slot[tile_index(i, j, NT)]; };
  auto PI = [&](int k, int i) { return (k % RING) * NT + (i - k); };
  std::vector<int4> j4;
  std::vector<int2> j2;
  std::vector<int> i1, jslot;
  std::vector<gemm_tc::Item> items;
  std::vector<gemm_tc::Seg> segs;
  std::vector<gemm64::Item> items64;
  std::vector<gemm64::Seg> segs64;
  std::vector<long> kk(NT);
  std::vector<unsigned char> pcls((size_t)NT * RING * NT, 0);
  const double nb3 = (double)nb * nb * nb;
  for (int j = 0; j < NT; j++)
    for (int i = j; i < NT; i++) {
      int c = C(i, j);
      P->tiles[c]++;
      P->update_flops[c] += (i == j ? 1.0 : 2.0) * j * nb3 + (i > j ? nb3 : 0.0);
    }
  P->tc_trsm = trsm_tc::supports(nb);
  for (int k = 0; k < NT; k++) {
    CStep sp;
    kk[k] = SL(k, k);
    for (int i = k + 1; i < NT; i++) pcls[(size_t)k * RING * NT + PI(k, i)] = (unsigned char)C(i, k);
    std::vector<char> need_dig(NT - k, 0);
    bool step_f8 = false;
    auto add_update = [&](int g, int i, int j) {
      const int c = C(i, j);
      const int pi = PI(k, i), pj = PI(k, j);
      if (c == EMU_CLASS_FP64) {
        need_dig[i - k] = need_dig[j - k] = 1;
        for (int nbk = 0; nbk < nb / gemm64::BN; nbk++)
          for (int mb = 0; mb < nb / gemm64::BM; mb++) {
            if (i == j && mb * gemm64::BM + gemm64::BM - 1 < nbk * gemm64::BN) continue;  // above the diagonal
            gemm64::Seg sg;
            sg.a_row = pi * gemm64::NS * nb + mb * gemm64::BM;
            sg.b_row = pj * gemm64::NS * nb + nbk * gemm64::BN;
            sg.a_x = sg.b_x = 0;
            gemm64::Item it;
            it.out_off = (long)SL(i, j) * (long)te + mb * gemm64::BM + (long)nbk * gemm64::BN * nb;
            it.a_sc = pi * nb + mb * gemm64::BM;
            it.b_sc = pj * nb + nbk * gemm64::BN;
            it.seg_begin = (int)segs64.size();
            segs64.push_back(sg);
            it.seg_end = (int)segs64.size();
            it.rows_valid = gemm64::BM;
            it.cols_valid = gemm64::BN;
            items64.push_back(it);
            sp.g64[g].n++;
          }
        sp.f64[g] += (i == j ? 1.0 : 2.0) * nb3;
        return;
      }
      const bool f8 = c == EMU_CLASS_E4M3;
      if (f8) step_f8 = true;
      const int rpt = f8 ? 1 : 3;
      for (int nbk = 0; nbk < nb / gemm_tc::BN; nbk++)
        for (int mb = 0; mb < nb / gemm_tc::BM; mb++) {
          if (i == j && mb * gemm_tc::BM + gemm_tc::BM - 1 < nbk * gemm_tc::BN) continue;
          gemm_tc::Seg s;
          s.ax = 0;
          s.ay = pi * rpt * nb + mb * gemm_tc::BM;
          s.ay_step = nb;
          s.bx = 0;
          s.by = pj * rpt * nb + nbk * gemm_tc::BN;
          s.by_step = nb;
          s.cls = c;
          s.pad = 0;
          gemm_tc::Item it;
          it.seg_begin = (int)segs.size();
          segs.push_back(s);
          it.seg_end = (int)segs.size();
          it.out_off = (long)SL(i, j) * (long)te + mb * gemm_tc::BM + (long)nbk * gemm_tc::BN * nb;
          it.rows_valid = gemm_tc::BM;
          it.cols_valid = gemm_tc::BN;
          it.sa = f8 ? pi : -1;
          it.sb = f8 ? pj : -1;
          it.oc = c;
          items.push_back(it);
          const double f = 2.0 * gemm_tc::BM * gemm_tc::BN * nb;
          sp.tc[g].n++;
          sp.flops[g] += f;
          sp.mma[g] += f * (c == EMU_CLASS_FP32 ? 6.0 : f8 ? 0.5 : 1.0);
        }
    };
    for (int g = 0; g < CG_N; g++) {
      sp.tc[g].off = (int)items.size();
      sp.g64[g].off = (int)items64.size();
      if (g == CG_S) {
        if (k + 1 < NT) add_update(g, k + 1, k + 1);
      } else if (g == CG_G1) {
        for (int i = k + 2; i < NT; i++) add_update(g, i, k + 1);
      } else if (g == CG_G2A) {
        for (int i = k + 2; i < NT; i++) add_update(g, i, k + 2);
      } else {
        for (int j = k + 3; j < NT; j++)
          for (int i = j; i < NT; i++) add_update(g, i, j);
      }
    }
    auto fill = [&](CPart &pt, int r0, int r1) {
      pt.dec.off = (int)j4.size();
      for (int i = r0; i < r1; i++) j4.push_back(make_int4(PI(k, i), SL(i, k), C(i, k), 0));
      pt.dec.n = (int)j4.size() - pt.dec.off;
      pt.t64.off = (int)j2.size();
      for (int i = r0; i < r1; i++)
        if (C(i, k) == EMU_CLASS_FP64) {
          j2.push_back(make_int2(PI(k, i), PI(k, k)));
          jslot.push_back(k & 1);
        }
      pt.t64.n = (int)j2.size() - pt.t64.off;
      pt.t32.off = (int)j2.size();
      for (int i = r0; i < r1; i++)
        if (C(i, k) != EMU_CLASS_FP64) {
          j2.push_back(make_int2(PI(k, i), k & 1));
          jslot.push_back(0);
        }
      pt.t32.n = (int)j2.size() - pt.t32.off;
      pt.enc.off = (int)j4.size();
      for (int i = r0; i < r1; i++)
        if (C(i, k) != EMU_CLASS_E4M3) j4.push_back(make_int4(PI(k, i), SL(i, k), C(i, k), 0));
      pt.enc.n = (int)j4.size() - pt.enc.off;
      pt.enc8.off = (int)j4.size();
      for (int i = r0; i < r1; i++)
        if (C(i, k) == EMU_CLASS_E4M3) j4.push_back(make_int4(PI(k, i), SL(i, k), C(i, k), 0));
      pt.enc8.n = (int)j4.size() - pt.enc8.off;
      // FP64 rows: their pieces are split from P64 after their TRSM
      pt.split.off = (int)i1.size();
      for (int i = r0; i < r1; i++)
        if (C(i, k) == EMU_CLASS_FP64) i1.push_back(PI(k, i));
      pt.split.n = (int)i1.size() - pt.split.off;
      // panel tiles quantized for the step's E4M3 consumers (the E4M3 rows
      // have their FP8 copies from the encode)
      pt.quant.off = (int)i1.size();
      for (int i = r0; i < r1; i++)
        if (step_f8 && C(i, k) != EMU_CLASS_E4M3) i1.push_back(PI(k, i));
      pt.quant.n = (int)i1.size() - pt.quant.off;
      pt.slice.off = (int)j4.size();
      for (int i = r0; i < r1; i++)
        if (need_dig[i - k]) j4.push_back(make_int4(PI(k, i), PI(k, i), PI(k, i) * nb, 0));
      pt.slice.n = (int)j4.size() - pt.slice.off;
    };
    if (k + 1 < NT) fill(sp.crit, k + 1, k + 2);
    fill(sp.mid, k + 2, NT);
    sp.fp64_panel = sp.crit.t64.n + sp.mid.t64.n > 0;
    sp.low_panel = sp.crit.t32.n + sp.mid.t32.n > 0;
    P->steps.push_back(sp);
  }
  // one allocation for the lists and the panel ring
  size_t off = 0;
  auto part = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  auto vb = [](const auto &v) { return v.size() * sizeof(v[0]); };
  const size_t o4 = part(vb(j4)), o2 = part(vb(j2)), o1 = part(vb(i1)), ojs = part(vb(jslot)), okk = part(vb(kk)),
               opc = part(vb(pcls)), oit = part(vb(items)), osg = part(vb(segs)), oi64 = part(vb(items64)),
               os64 = part(vb(segs64));
  P->host.assign(off, 0);
  auto put = [&](size_t o, const auto &v) {
    if (!v.empty()) memcpy(P->host.data() + o, v.data(), vb(v));
  };
  put(o4, j4);
  put(o2, j2);
  put(o1, i1);
  put(ojs, jslot);
  put(okk, kk);
  put(opc, pcls);
  put(oit, items);
  put(osg, segs);
  put(oi64, items64);
  put(os64, segs64);
  cudaStream_t st = ctx->stream;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&P->d_blob, off, st));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(P->d_blob, P->host.data(), off, cudaMemcpyHostToDevice, st));
  char *b = static_cast<char *>(P->d_blob);
  P->d_j4 = (int4 *)(b + o4);
  P->d_j2 = (int2 *)(b + o2);
  P->d_i1 = (int *)(b + o1);
  P->d_jslot = (int *)(b + ojs);
  P->d_kk = (long *)(b + okk);
  P->d_pcls = (unsigned char *)(b + opc);
  P->d_items = (gemm_tc::Item *)(b + oit);
  P->d_segs = (gemm_tc::Seg *)(b + osg);
  P->d_items64 = (gemm64::Item *)(b + oi64);
  P->d_segs64 = (gemm64::Seg *)(b + os64);
  const size_t np = (size_t)RING * NT;
  auto alloc = [&](void **q, size_t bytes) -> emu_status {
    cudaError_t e = cudaMallocAsync(q, bytes, st);
    if (e == cudaErrorMemoryAllocation) return EMU_ENOMEM;
    if (e != cudaSuccess) return emu_cuda_fail(ctx, e, "panel buffers");
    return EMU_OK;
  };
  emu_status s = EMU_OK;
  bool any64 = false;
  for (const CStep &q : P->steps) any64 = any64 || q.fp64_panel;
  if (s == EMU_OK && any64) s = alloc((void **)&P->P64, np * te * sizeof(double));
  if (s == EMU_OK) s = alloc((void **)&P->P32, np * te * sizeof(float));
  if (s == EMU_OK) s = alloc((void **)&P->Pop, np * 3 * te * sizeof(uint16_t));
  if (s == EMU_OK) s = alloc((void **)&P->P8, np * te);
  if (s == EMU_OK) s = alloc((void **)&P->Psc8, np * sizeof(float));
  if (s == EMU_OK) s = alloc((void **)&P->digits, np * gemm64::NS * te * sizeof(uint16_t));
  if (s == EMU_OK) s = alloc((void **)&P->exps, np * nb * sizeof(int));
  if (s == EMU_OK) s = alloc((void **)&P->amax, np * sizeof(unsigned));
  if (s == EMU_OK) s = alloc((void **)&P->lkk32, 2 * te * sizeof(float));
  if (s == EMU_OK) s = alloc((void **)&P->lkkp, 2 * 3 * te * sizeof(uint16_t));
  if (s == EMU_OK) s = alloc((void **)&P->ls64, 2 * (size_t)nb * 32 * sizeof(double));
  if (s == EMU_OK) s = alloc((void **)&P->rinv64, 2 * (size_t)nb * sizeof(double));
  if (s != EMU_OK) return s;
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(P->Pop, 0, np * 3 * te * sizeof(uint16_t), st));
  const uint64_t prow = (uint64_t)np * 3 * nb;
  if ((s = gemm_tc::make_map_bf16(ctx, &P->ops.a16, P->Pop, nb, prow, gemm_tc::BM)) != EMU_OK) return s;
  if ((s = gemm_tc::make_map_bf16(ctx, &P->ops.b16, P->Pop, nb, prow, gemm_tc::BN)) != EMU_OK) return s;
  if ((s = gemm_tc::make_map_e4m3(ctx, &P->ops.a8, P->P8, nb, (uint64_t)np * nb, gemm_tc::BM)) != EMU_OK) return s;
  if ((s = gemm_tc::make_map_e4m3(ctx, &P->ops.b8, P->P8, nb, (uint64_t)np * nb, gemm_tc::BN)) != EMU_OK) return s;
  P->ops.a32 = P->ops.a16;  // no TF32 class in class-format storage
  P->ops.b32 = P->ops.b16;
  P->ops.scale8 = P->Psc8;
  const uint64_t drow = (uint64_t)np * gemm64::NS * nb;
  if ((s = gemm64::make_map(ctx, &P->map64a, P->digits, nb, drow, gemm64::BM)) != EMU_OK) return s;
  if ((s = gemm64::make_map(ctx, &P->map64b, P->digits, nb, drow, gemm64::BN)) != EMU_OK) return s;
  if (P->tc_trsm) {
    if ((s = trsm_tc::make_map(ctx, &P->lmap, P->lkkp, nb, 2)) != EMU_OK) return s;
    if ((s = trsm_tc::make_op_map(ctx, &P->opmap, P->Pop, nb, (long)np)) != EMU_OK) return s;
  }
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));  // the host lists must outlive their copy
  return EMU_OK;
}

}  // namespace

// The factor of a class-format matrix in place: the lookahead schedule of the
// FP32-master factor (critical / panel / bulk streams, the bulk GEMM on all
// but a few SMs), with each panel decoded before and encoded after its TRSM.
emu_status classfmt_factor(emu_ctx *ctx, emu_mat *A) {
  ClassStore *cs = A->cs;
  const int NT = A->nt, nb = A->nb;
  const size_t te = A->tile_elems;
  cplan_free(static_cast<ClassPlan *>(cs->work));
  ClassPlan *P = new ClassPlan();
  cs->work = P;
  emu_status s = build_cplan(ctx, A, P);
  if (s != EMU_OK) return s;
  const int *st = ctx->d_status;
  cudaStream_t user = ctx->stream;
  const int EV = 6;  // per step: POTRF, TRSM row k+1, TRSM rest, G1, G2A, G2 done
  if ((s = mixed_sched_streams(ctx, EV * NT + 2)) != EMU_OK) return s;
  auto ev = [&](int k, int w) { return ctx->sched_ev[EV * k + w]; };
  enum { E_P = 0, E_T1 = 1, E_T = 2, E_G1 = 3, E_G2 = 4, E_END = 5 };
  cudaEvent_t ev_start = ctx->sched_ev[EV * NT], ev_end = ctx->sched_ev[EV * NT + 1];
  EMU_CUDA_TRY(ctx, cudaEventRecord(ev_start, user));
  for (cudaStream_t q : {ctx->crit, ctx->mid, ctx->bulk}) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(q, ev_start, 0));
  const size_t np = (size_t)RING * NT;
  // the panel of step k: decode, TRSM, encode, pieces, FP8 copies, digits
  auto panel = [&](int k, const CPart &pt) -> emu_status {
    emu_status e = EMU_OK;
    const unsigned char *pcls = P->d_pcls + (size_t)k * np;
    if (pt.dec.n > 0) {
      ProfScope ps(ctx, PROF_SPLIT, 0.0, 8.0 * pt.dec.n * te);
      k_decode<<<dim3(64, pt.dec.n), 256, 0, ctx->stream>>>(P->d_j4 + pt.dec.off, te, cs->t64, cs->t32, cs->t16,
                                                           cs->t8, cs->sc8, P->P64, P->P32, st);
      EMU_LAUNCHED(ctx);
    }
    if (pt.t64.n > 0) {
      if ((e = launch_trsm64_jobs(ctx, P->P64, nb, P->d_j2 + pt.t64.off, pt.t64.n, P->ls64, P->rinv64,
                                  P->d_jslot + pt.t64.off)) != EMU_OK)
        return e;
      if ((e = launch_split_tiles64(ctx, P->P64, P->Pop, P->d_i1 + pt.split.off, pt.split.n, nb, 0)) != EMU_OK)
        return e;
    }
    if (pt.t32.n > 0) {
      if (P->tc_trsm)
        e = trsm_tc::launch(ctx, P->lmap, P->opmap, P->lkk32, P->P32, nb, NT, k, nullptr, P->d_j2 + pt.t32.off,
                            pt.t32.n);
      else
        e = launch_trsm32_jobs(ctx, P->lkk32, P->P32, P->Pop, nb, P->d_j2 + pt.t32.off, pt.t32.n);
      if (e != EMU_OK) return e;
    }
    if (pt.enc.n > 0) {
      ProfScope ps(ctx, PROF_SPLIT, 0.0, 10.0 * pt.enc.n * te);
      k_encode<<<dim3(64, pt.enc.n), 256, 0, ctx->stream>>>(P->d_j4 + pt.enc.off, nb, cs->t64, cs->t32, cs->t16,
                                                           P->P64, P->P32, P->Pop, st);
      EMU_LAUNCHED(ctx);
    }
    if (pt.enc8.n > 0) {
      ProfScope ps(ctx, PROF_SPLIT, 0.0, 19.0 * pt.enc8.n * te);
      k_amax_tiles<<<dim3(64, pt.enc8.n), 256, 0, ctx->stream>>>(P->d_j4 + pt.enc8.off, nb, P->P32, P->amax, st);
      EMU_LAUNCHED(ctx);
      k_encode_e4m3<<<dim3((nb / TB) * (nb / TB), pt.enc8.n), 256, 0, ctx->stream>>>(
          P->d_j4 + pt.enc8.off, nb, cs->t8, cs->sc8, P->P32, P->Pop, P->P8, P->Psc8, P->amax, st);
      EMU_LAUNCHED(ctx);
    }
    if (pt.quant.n > 0 &&
        (e = launch_quant_e4m3(ctx, P->Pop, P->P8, P->Psc8, P->d_i1 + pt.quant.off, pt.quant.n, nb)) != EMU_OK)
      return e;
    if (pt.slice.n > 0) {
      e = gemm64::launch_row_exponents(ctx, P->P64, P->P32, pcls, P->d_j4 + pt.slice.off, pt.slice.n, nb, P->exps);
      if (e == EMU_OK)
        e = gemm64::launch_slice(ctx, P->P64, P->P32, pcls, P->d_j4 + pt.slice.off, pt.slice.n, nb, P->exps,
                                 P->digits);
    }
    return e;
  };
  gemm_tc::Outputs outs{cs->t32, cs->t16, reinterpret_cast<uint16_t *>(cs->t8)};
  auto update_group = [&](int k, int g, int max_ctas) -> emu_status {
    const CStep &sp = P->steps[k];
    if (sp.g64[g].n > 0) {
      ProfScope ps(ctx, PROF_UPDATE64, sp.f64[g], 24.0 * sp.f64[g] / (2.0 * nb), 36.0 * sp.f64[g]);
      emu_status e = gemm64::launch(ctx, P->map64a, P->map64b, P->d_items64 + sp.g64[g].off, sp.g64[g].n,
                                    P->d_segs64, nb, nb, nb, P->exps, P->exps, gemm64::TC64_SUB, cs->t64, nb,
                                    std::max(1, max_ctas));
      if (e != EMU_OK) return e;
    }
    if (sp.tc[g].n > 0) {
      ProfScope ps(ctx, PROF_TC_FACTOR, sp.flops[g], 0.0, sp.mma[g]);
      return gemm_tc::launch_class(ctx, P->ops, P->d_items + sp.tc[g].off, sp.tc[g].n, P->d_segs, nb / gemm_tc::BK,
                                   outs, nb, std::max(1, max_ctas));
    }
    return EMU_OK;
  };
  for (int k = 0; k < NT && s == EMU_OK; k++) {
    const CStep &sp = P->steps[k];
    const int ps_ = k % RING;
    double *Lkk = cs->t64 + (size_t)cs->slot[tile_index(k, k, NT)] * te;
    // ---- critical stream
    ctx->stream = ctx->crit;
    if (k >= RING) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev(k - RING, E_END), 0));  // ring slot free
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(P->exps + (size_t)ps_ * NT * nb, 0, (size_t)NT * nb * sizeof(int), ctx->crit));
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(P->amax + (size_t)ps_ * NT, 0, (size_t)NT * sizeof(unsigned), ctx->crit));
    if ((s = launch_potrf64_ptr(ctx, Lkk, nb, k)) != EMU_OK) break;
    if (sp.low_panel) {
      if (P->tc_trsm) {
        if ((s = trsm_tc::launch_prep(ctx, cs->t64, cs->slot[tile_index(k, k, NT)], nullptr, 1,
                                      P->lkk32 + (size_t)(k & 1) * te, P->lkkp + (size_t)(k & 1) * 3 * te, nb)) !=
            EMU_OK)
          break;
      } else if ((s = launch_diag_to_f32_slots(ctx, cs->t64, P->lkk32 + (size_t)(k & 1) * te, P->d_kk + k, 1, te)) !=
                 EMU_OK) {
        break;
      }
    }
    if (sp.fp64_panel) {
      // L_kk beside the panel's FP64 tiles (the FP64 TRSM reads both from P64)
      EMU_CUDA_TRY(ctx, cudaMemcpyAsync(P->P64 + (size_t)ps_ * NT * te, Lkk, te * sizeof(double),
                                        cudaMemcpyDeviceToDevice, ctx->crit));
      if ((s = launch_trsm64_prep(ctx, Lkk, nb, P->ls64 + (size_t)(k & 1) * nb * 32,
                                  P->rinv64 + (size_t)(k & 1) * nb)) != EMU_OK)
        break;
    }
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_P), ctx->crit));
    if (k > 0) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev(k - 1, E_G1), 0));
    if ((s = panel(k, sp.crit)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_T1), ctx->crit));
    if (k > 0) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev(k - 1, E_G2), 0));  // G2A(k-1)
    if ((s = update_group(k, CG_S, ctx->sm_count)) != EMU_OK) break;
    // ---- panel stream
    ctx->stream = ctx->mid;
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->mid, ev(k, E_P), 0));
    if ((s = panel(k, sp.mid)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_T), ctx->mid));
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->mid, ev(k, E_T1), 0));
    if (k > 0) EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->mid, ev(k - 1, E_G2), 0));
    if ((s = update_group(k, CG_G1, ctx->sm_count)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_G1), ctx->mid));
    // ---- bulk stream
    ctx->stream = ctx->bulk;
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->bulk, ev(k, E_T), 0));
    const bool fp64_near = sp.fp64_panel || (k + 1 < NT && P->steps[k + 1].fp64_panel);
    const int bulk_ctas = std::max(1, ctx->sm_count - mixed_reserved_sms(fp64_near));
    if ((s = update_group(k, CG_G2A, bulk_ctas)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_G2), ctx->bulk));
    if ((s = update_group(k, CG_G2, bulk_ctas)) != EMU_OK) break;
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev(k, E_END), ctx->bulk));
  }
  ctx->stream = user;
  if (s != EMU_OK) return s;
  for (cudaStream_t q : {ctx->mid, ctx->bulk}) {
    EMU_CUDA_TRY(ctx, cudaEventRecord(ev_end, q));
    EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->crit, ev_end, 0));
  }
  EMU_CUDA_TRY(ctx, cudaEventRecord(ev_end, ctx->crit));
  EMU_CUDA_TRY(ctx, cudaStreamWaitEvent(user, ev_end, 0));
  // strict upper triangles of the diagonal factor tiles
  std::vector<int> dslots(NT);
  for (int k = 0; k < NT; k++) dslots[k] = cs->slot[tile_index(k, k, NT)];
  int *d_ds = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_ds, NT * sizeof(int), user));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_ds, dslots.data(), NT * sizeof(int), cudaMemcpyHostToDevice, user));
  k_tril_slots<<<dim3(nb, NT), 128, 0, user>>>(d_ds, nb, cs->t64);
  EMU_LAUNCHED(ctx);
  cudaFreeAsync(d_ds, user);
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(user));  // dslots
  // the panel ring is no longer needed; the plan's counts stay for info
  for (void **q : {(void **)&P->P64, (void **)&P->P32, (void **)&P->Pop, (void **)&P->P8, (void **)&P->Psc8,
                   (void **)&P->digits, (void **)&P->exps, (void **)&P->amax, (void **)&P->lkk32, (void **)&P->lkkp,
                   (void **)&P->ls64, (void **)&P->rinv64, (void **)&P->d_blob}) {
    if (*q) cudaFreeAsync(*q, user);
    *q = nullptr;
  }
  return EMU_OK;
}

void classfmt_fill_info(const emu_mat *A, emu_factor_info *info) {
  info->frob = A->frob;
  const ClassStore *cs = A->cs;
  if (!cs) return;
  const ClassPlan *P = static_cast<const ClassPlan *>(cs->work);
  for (int c = 0; c < EMU_NCLASS; c++) {
    info->tiles[c] = P ? P->tiles[c] : 0;
    info->update_flops[c] = P ? P->update_flops[c] : 0.0;
  }
}

// ---------------------------------------------------------------- sampling
// Y = L Z for a class-format factor: the FP64 tiles as exact digit products
// (one exponent per matrix row), the other tiles on the tensor cores in
// their class (FP32: three BF16 pieces against three pieces of z; BF16 and
// E4M3: one BF16 plane against bf16(z)), accumulated in FP32 over a group of
// tile columns and added to the FP64 Y.
emu_status classfmt_sample(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz, int s, double *Y, long ldy) {
  ClassStore *cs = L->cs;
  const int NT = L->nt, nb = L->nb;
  const size_t te = L->tile_elems;
  const long npad = (long)NT * nb;
  const int s_pad = ((s + gemm_tc::BN - 1) / gemm_tc::BN) * gemm_tc::BN;
  cudaStream_t st = ctx->stream;
  EMU_CUDA_TRY(ctx, cudaMemset2DAsync(Y, ldy * sizeof(double), 0, (size_t)L->n * sizeof(double), s, st));
  if (s <= 0) return EMU_OK;
  emu_status e = EMU_OK;
  // ---- FP64 tiles: digit slices made once per factor
  const int n64 = cs->nslot[EMU_CLASS_FP64];
  if (!cs->samp_ready && n64 > 0) {
    std::vector<int4> jobs;
    for (int j = 0; j < NT; j++)
      for (int i = j; i < NT; i++) {
        long t = tile_index(i, j, NT);
        if (cs->cls[t] == EMU_CLASS_FP64) jobs.push_back(make_int4(cs->slot[t], cs->slot[t], i * nb, 0));
      }
    int4 *d_jobs = nullptr;
    unsigned char *zc = nullptr;
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&cs->samp_dig, (size_t)n64 * gemm64::NS * te * sizeof(uint16_t), st));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&cs->samp_exp, npad * sizeof(int), st));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_jobs, jobs.size() * sizeof(int4), st));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&zc, n64, st));
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(zc, EMU_CLASS_FP64, n64, st));
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(cs->samp_exp, 0, npad * sizeof(int), st));
    EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    e = gemm64::launch_row_exponents(ctx, cs->t64, nullptr, zc, d_jobs, (int)jobs.size(), nb, cs->samp_exp);
    if (e == EMU_OK)
      e = gemm64::launch_slice(ctx, cs->t64, nullptr, zc, d_jobs, (int)jobs.size(), nb, cs->samp_exp, cs->samp_dig);
    cudaFreeAsync(d_jobs, st);
    cudaFreeAsync(zc, st);
    EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (e != EMU_OK) return e;
    cs->samp_ready = true;
  }
  if (n64 > 0) {
    CUtensorMap amap, zmap;
    std::vector<gemm64::Item> it64;
    std::vector<gemm64::Seg> sg64;
    double f64 = 0.0;
    for (int i = 0; i < NT; i++)
      for (int nbk = 0; nbk < s_pad / gemm64::BN; nbk++)
        for (int mb = 0; mb < nb / gemm64::BM; mb++) {
          const long row0 = (long)i * nb + mb * gemm64::BM;
          const int cols = std::min(gemm64::BN, s - nbk * gemm64::BN);
          if (row0 >= L->n || cols <= 0) continue;
          gemm64::Item it;
          it.seg_begin = (int)sg64.size();
          for (int k = 0; k <= i; k++) {
            const long t = tile_index(i, k, NT);
            if (cs->cls[t] != EMU_CLASS_FP64) continue;
            gemm64::Seg sg;
            sg.a_row = cs->slot[t] * gemm64::NS * nb + mb * gemm64::BM;
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
    uint16_t *zd = nullptr;
    int *ze = nullptr;
    int2 *blk = nullptr;
    gemm64::Item *d_it = nullptr;
    gemm64::Seg *d_sg = nullptr;
    const int2 hblk = make_int2(0, (int)npad);
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&zd, (size_t)gemm64::NS * s_pad * npad * sizeof(uint16_t), st));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&ze, s_pad * sizeof(int) + 16, st));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&blk, sizeof(int2), st));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_it, it64.size() * sizeof(gemm64::Item), st));
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_sg, sg64.size() * sizeof(gemm64::Seg), st));
    EMU_CUDA_TRY(ctx, cudaMemcpyAsync(blk, &hblk, sizeof(int2), cudaMemcpyHostToDevice, st));
    EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_it, it64.data(), it64.size() * sizeof(gemm64::Item), cudaMemcpyHostToDevice, st));
    EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_sg, sg64.data(), sg64.size() * sizeof(gemm64::Seg), cudaMemcpyHostToDevice, st));
    e = gemm64::launch_slice_z(ctx, Z, ldz, s, s_pad, blk, 1, npad, ze, zd);
    if (e == EMU_OK) e = gemm64::make_map(ctx, &zmap, zd, npad, (uint64_t)gemm64::NS * s_pad, gemm64::BN);
    if (e == EMU_OK) e = gemm64::make_map(ctx, &amap, cs->samp_dig, nb, (uint64_t)n64 * gemm64::NS * nb, gemm64::BM);
    if (e == EMU_OK) {
      ProfScope ps(ctx, PROF_TRMM64, f64, 0.0, 36.0 * f64);
      e = gemm64::launch(ctx, amap, zmap, d_it, (int)it64.size(), d_sg, nb, nb, s_pad, cs->samp_exp, ze,
                         gemm64::TC64_ADD, Y, (int)ldy, ctx->sm_count);
    }
    for (void *q : {(void *)zd, (void *)ze, (void *)blk, (void *)d_it, (void *)d_sg}) cudaFreeAsync(q, st);
    EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));  // host lists
    if (e != EMU_OK) return e;
  }
  // ---- the other tiles, a group of tile columns at a time
  const long kMaxPlanes = std::max<long>(3, (4096l << 20) / (long)(te * sizeof(uint16_t)));  // 4 GB of planes
  uint16_t *zp = nullptr, *planes = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&zp, (size_t)3 * s_pad * npad * sizeof(uint16_t), st));
  e = launch_split_z(ctx, Z, ldz, npad, s, s_pad, zp);
  long need = 0;
  for (long t = 0; t < L->ntiles; t++) {
    const int c = cs->cls[t];
    need += c == EMU_CLASS_FP64 ? 0 : c == EMU_CLASS_FP32 ? 3 : 1;
  }
  const long cap = std::min(need, kMaxPlanes);
  if (e == EMU_OK && cap > 0) {
    cudaError_t ce = cudaMallocAsync(&planes, (size_t)cap * te * sizeof(uint16_t), st);
    if (ce != cudaSuccess) e = ce == cudaErrorMemoryAllocation ? EMU_ENOMEM : emu_cuda_fail(ctx, ce, "sampler planes");
  }
  gemm_tc::Operands ops{};
  if (e == EMU_OK && cap > 0) e = gemm_tc::make_map_bf16(ctx, &ops.a16, planes, nb, (uint64_t)cap * nb, gemm_tc::BM);
  if (e == EMU_OK && cap > 0) e = gemm_tc::make_map_bf16(ctx, &ops.b16, zp, npad, (uint64_t)3 * s_pad, gemm_tc::BN);
  ops.a8 = ops.a32 = ops.a16;
  ops.b8 = ops.b32 = ops.b16;
  ops.scale8 = nullptr;
  int c0 = 0;
  while (e == EMU_OK && cap > 0 && c0 < NT) {
    // columns [c0, c1) whose planes fit the scratch
    std::vector<int4> jobs;
    std::vector<int> plane_of(0);
    long used = 0;
    int c1 = c0;
    std::vector<long> pl((size_t)NT * NT, -1);
    while (c1 < NT) {
      long col = 0;
      for (int i = c1; i < NT; i++) {
        const int c = cs->cls[tile_index(i, c1, NT)];
        col += c == EMU_CLASS_FP64 ? 0 : c == EMU_CLASS_FP32 ? 3 : 1;
      }
      if (used + col > cap && c1 > c0) break;
      if (used + col > cap) {  // one column larger than the scratch: cannot happen with 4 GB and nb <= 2048
        e = fail_status(ctx, EMU_ENOMEM, "sampler planes: one tile column exceeds the scratch");
        break;
      }
      for (int i = c1; i < NT; i++) {
        const long t = tile_index(i, c1, NT);
        const int c = cs->cls[t];
        if (c == EMU_CLASS_FP64) continue;
        pl[(size_t)i * NT + c1] = used;
        jobs.push_back(make_int4(cs->slot[t], c, (int)used, 0));
        used += c == EMU_CLASS_FP32 ? 3 : 1;
      }
      c1++;
    }
    if (e != EMU_OK) break;
    std::vector<gemm_tc::Item> items;
    std::vector<gemm_tc::Seg> segs;
    double tf = 0.0, tm = 0.0;
    for (int i = c0; i < NT; i++)
      for (int nbk = 0; nbk < s_pad / gemm_tc::BN; nbk++)
        for (int mb = 0; mb < nb / gemm_tc::BM; mb++) {
          const long row0 = (long)i * nb + mb * gemm_tc::BM;
          if (row0 >= L->n) continue;
          gemm_tc::Item it;
          it.seg_begin = (int)segs.size();
          for (int k = c0; k < std::min(c1, i + 1); k++) {
            const long p0 = pl[(size_t)i * NT + k];
            if (p0 < 0) continue;
            const int c = cs->cls[tile_index(i, k, NT)];
            gemm_tc::Seg sg;
            sg.ax = 0;
            sg.ay = (int)(p0 * nb + mb * gemm_tc::BM);
            sg.ay_step = nb;
            sg.bx = k * nb;
            sg.by = nbk * gemm_tc::BN;
            sg.by_step = s_pad;
            sg.cls = c == EMU_CLASS_FP32 ? EMU_CLASS_FP32 : EMU_CLASS_BF16;
            sg.pad = 0;
            segs.push_back(sg);
            const double f = 2.0 * gemm_tc::BM * gemm_tc::BN * nb;
            tf += f;
            tm += f * (sg.cls == EMU_CLASS_FP32 ? 6.0 : 1.0);
          }
          it.seg_end = (int)segs.size();
          if (it.seg_end == it.seg_begin) continue;
          it.out_off = row0 + (long)nbk * gemm_tc::BN * ldy;
          it.rows_valid = (int)std::min<long>(gemm_tc::BM, L->n - row0);
          it.cols_valid = s - nbk * gemm_tc::BN;
          it.sa = it.sb = -1;
          it.oc = EMU_CLASS_FP64;
          items.push_back(it);
        }
    int4 *d_jobs = nullptr;
    gemm_tc::Item *d_items = nullptr;
    gemm_tc::Seg *d_segs = nullptr;
    if (!jobs.empty()) {
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_jobs, jobs.size() * sizeof(int4), st));
      EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
      ProfScope ps(ctx, PROF_SPLIT, 0.0, 8.0 * used * te);
      k_samp_planes<<<dim3((nb / TB) * (nb / TB), (unsigned)jobs.size()), 256, 0, st>>>(d_jobs, nb, cs->t32, cs->t16,
                                                                                       cs->t8, cs->sc8, planes);
      EMU_LAUNCHED(ctx);
    }
    if (!items.empty()) {
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_items, items.size() * sizeof(gemm_tc::Item), st));
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&d_segs, segs.size() * sizeof(gemm_tc::Seg), st));
      EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(gemm_tc::Item),
                                        cudaMemcpyHostToDevice, st));
      EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(gemm_tc::Seg),
                                        cudaMemcpyHostToDevice, st));
      ProfScope ps(ctx, PROF_TC_SAMPLE, tf, 0.0, tm);
      e = gemm_tc::launch(ctx, ops, d_items, (int)items.size(), d_segs, nb / gemm_tc::BK, gemm_tc::TC_ADD_F64,
                          nullptr, Y, (int)ldy, ctx->sm_count);
    }
    for (void *q : {(void *)d_jobs, (void *)d_items, (void *)d_segs})
      if (q) cudaFreeAsync(q, st);
    EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));  // host lists of this group
    c0 = c1;
  }
  if (planes) cudaFreeAsync(planes, st);
  cudaFreeAsync(zp, st);
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return e;
}

// ------------------------------------------------------------------ export
emu_status classfmt_export(emu_ctx *ctx, const emu_mat *A, double *dOut, long ld) {
  const ClassStore *cs = A->cs;
  TileSrc S{A->d_cls, cs->d_slot, cs->t64, cs->t32, cs->t16, cs->t8, cs->sc8, A->nb, A->nt, 0,
            A->state != MAT_COV};
  EMU_CUDA_TRY(ctx, cudaMemset2DAsync(dOut, ld * sizeof(double), 0, (size_t)A->n * sizeof(double), A->n, ctx->stream));
  k_export_class<<<dim3((unsigned)A->ntiles, A->nb), 128, 0, ctx->stream>>>(S, A->n, dOut, ld);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

// ------------------------------------------------- backward-error estimate
// sqrt(sum over probes of ||(L L^T - S) g||^2 / p) / ||S||_F with S
// regenerated from p (the covariance the factor was built from).  Works for
// every storage: FP64 factor, FP32-master mixed factor, class format.
emu_status factor_backward_error_est(emu_ctx *ctx, const emu_mat *A, const emu_cov_params *cp, int nprobes,
                                     uint64_t seed, double *est) {
  const int NT = A->nt, nb = A->nb, n = A->n;
  const long npad = (long)NT * nb;
  cudaStream_t st = ctx->stream;
  TileSrc S{};
  int *ident = nullptr;
  if (A->cs) {
    S = TileSrc{A->d_cls, A->cs->d_slot, A->cs->t64, A->cs->t32, A->cs->t16, A->cs->t8, A->cs->sc8, nb, NT, 0, 1};
  } else {
    std::vector<int> id(A->ntiles);
    for (long t = 0; t < A->ntiles; t++) id[t] = (int)t;
    EMU_CUDA_TRY(ctx, cudaMallocAsync(&ident, A->ntiles * sizeof(int), st));
    EMU_CUDA_TRY(ctx, cudaMemcpyAsync(ident, id.data(), A->ntiles * sizeof(int), cudaMemcpyHostToDevice, st));
    EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    S = TileSrc{A->d_cls, ident, A->t64, A->t32, nullptr, nullptr, nullptr, nb, NT, 1, 0};
    if (A->state == MAT_FACTOR64) {
      // every tile of a plain FP64 factor is in the FP64 arena
      unsigned char *z = nullptr;
      EMU_CUDA_TRY(ctx, cudaMallocAsync(&z, A->ntiles, st));
      EMU_CUDA_TRY(ctx, cudaMemsetAsync(z, EMU_CLASS_FP64, A->ntiles, st));
      S.cls = z;
    }
  }
  const int L = cp->L;
  const size_t ntab = (size_t)(2 * L - 1) * (4 * L - 3);
  double *tab = nullptr, *G = nullptr, *U = nullptr, *V = nullptr, *W = nullptr, *acc = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&tab, (ntab + L + 1) * sizeof(double), st));
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&G, 4 * (size_t)npad * 32 * sizeof(double) + sizeof(double), st));
  U = G + (size_t)npad * 32;
  V = U + (size_t)npad * 32;
  W = V + (size_t)npad * 32;
  acc = W + (size_t)npad * 32;
  emu_status s = launch_cov_tables(ctx, cp, tab);
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, sizeof(double), st));
  const double frob = A->frob > 0.0 ? A->frob : 0.0;
  double fro = frob;
  if (!(fro > 0.0)) EMU_CUDA_TRY(ctx, cudaMemcpyAsync(&fro, A->d_frob, sizeof(double), cudaMemcpyDeviceToHost, st));
  for (int q0 = 0; q0 < nprobes && s == EMU_OK; q0 += 32) {
    const int p = std::min(32, nprobes - q0);
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(U, 0, 3 * (size_t)npad * 32 * sizeof(double), st));
    k_probes<<<8 * ctx->sm_count, 256, 0, st>>>(seed + (uint64_t)q0, n, npad, p, G, npad);
    EMU_LAUNCHED(ctx);
    {
      ProfScope ps(ctx, PROF_SOLVE, 4.0 * (double)A->ntiles * nb * nb * p, 0.0);
      k_hutch_apply<<<dim3((unsigned)A->ntiles, nb / HS), 256, 0, st>>>(S, 1, p, G, U, npad);
      EMU_LAUNCHED(ctx);
      k_hutch_apply<<<dim3((unsigned)A->ntiles, nb / HS), 256, 0, st>>>(S, 0, p, U, V, npad);
      EMU_LAUNCHED(ctx);
    }
    {
      ProfScope ps(ctx, PROF_COV, 2.0 * (double)npad * npad * p, 0.0);
      k_sigma_apply<<<dim3(NT, NT, nb / HS), 256, 0, st>>>(L, n, nb, tab + ntab, tab, tab + ntab + L, p, G, W, npad);
      EMU_LAUNCHED(ctx);
    }
    k_diff_sq<<<4 * ctx->sm_count, 256, 0, st>>>(n, p, V, W, npad, acc);
    EMU_LAUNCHED(ctx);
  }
  double sum = 0.0;
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(&sum, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  cudaFreeAsync(tab, st);
  cudaFreeAsync(G, st);
  if (ident) cudaFreeAsync(ident, st);
  if (!A->cs && A->state == MAT_FACTOR64) cudaFreeAsync((void *)S.cls, st);
  if (s != EMU_OK) return s;
  *est = (fro > 0.0 && nprobes > 0) ? sqrt(sum / nprobes) / fro : 0.0;
  return EMU_OK;
}
