// gemm_f64.cu -- FP64-accurate tile update on the BF16 tensor cores for the
// FP64-class tiles of the mixed-precision factor (see gemm_f64.h for the
// digit scheme and why every tensor-core sum is exact).
//
// Warp roles (192 threads, one CTA per SM, persistent over the item list):
//   warp 0      TMA producer: per K stage the NS digit planes of the A block
//               (128 x 32) and of the B block (64 x 32), 96 KB.
//   warp 1      TMEM allocator + MMA issuer: per 16-deep K step the 36 digit
//               products with p + q < NS, product (p, q) into the group
//               accumulator g = p + q (TMEM columns g * 64 .. g * 64 + 63).
//   warps 2..3  idle (registers come in groups of four warps)
//   warps 4..11 epilogue (two warps per TMEM lane quarter, 32 columns each):
//               every KCHUNK of K, the 8 group accumulators are folded in
//               integer arithmetic into exact fixed-point accumulators
//               (fold_groups), converted to FP64 once per item;
//               after the last chunk the row scales are applied and the block
//               is subtracted from the FP64 output.
// The 8 accumulators fill TMEM, so the MMA warp waits for the epilogue to
// drain them before the next chunk.
#include <cuda_bf16.h>

#include <algorithm>

#include "gemm_f64.h"
#include "gemm_tc.h"
#include "tc.cuh"

namespace gemm64 {
namespace {

constexpr int A_SL = BM * BK * 2;                     // one A digit plane: 8 KB
constexpr int B_SL = BN * BK * 2;                     // one B digit plane: 4 KB
constexpr int STAGE_BYTES = NS * (A_SL + B_SL);       // 96 KB
constexpr int RING_BYTES = STAGES * STAGE_BYTES;
constexpr int BAR_BYTES = 128;
constexpr int SMEM_BYTES = RING_BYTES + BAR_BYTES + 1024;  // + alignment slack
// 12 warps: registers are granted per group of four warps, so a 10-warp
// CTA would be charged for 12 at the same per-thread count.
constexpr int NTHREADS = 384;
constexpr int EPI_WARP0 = 4;                                // warps 4..11: epilogue
constexpr int EPI_THREADS = NTHREADS - 32 * EPI_WARP0;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t IDESC = tc::idesc_f32acc(1u /*BF16*/, BM, BN);
constexpr int CHUNK_STAGES = KCHUNK / BK;
static_assert(NS * BN <= (int)TMEM_COLS, "group accumulators must fit in TMEM");

struct Shared {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull;
  uint64_t tempty;
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(Shared) <= BAR_BYTES, "barrier block");

// Adds the chunk's sum_g G_g 2^-7(g+2), for the group sums G_g of one output
// (column x of r[g]), to the exact fixed-point accumulator (hi, lo) of value
// hi 2^-31 + lo 2^-63 (lo unsigned, below 2^32).  Each G_g is an integer held
// exactly in FP32 (below 2^24, see the header), so the chunk's sum is formed
// in integer arithmetic: groups 2..7 by Horner in 64 bits, T = sum_{g>=2}
// G_g 2^(7(7-g)), |T| < 2^59 (|G_g| < 2^23.4 for g >= 1 with KCHUNK = 256:
// at most two products of a leading digit, |d_0| <= 128, and g - 1 of
// trailing digits, |d_p| <= 64, per K term), and groups 0..1 as Q = 2^7 G_0
// + G_1, |Q| < 2^30 (|G_0| <= 2^22).  The chunk's value is Q 2^-21 + T 2^-63
// = (2^10 Q + floor(T / 2^32)) 2^-31 + (T mod 2^32) 2^-63; the low word's
// carry moves into hi, which grows by less than 2^41 per chunk.  No FP64
// instruction runs per chunk: the FP64 pipe, GB300's slowest unit, is used
// once per output at the end of the item (fixed_to_double).
static_assert(NS == 8 && SLICE_BITS == 7 && KCHUNK <= 256, "fold_groups is written for 8 digits of 7 bits");
__device__ __forceinline__ void fold_groups(const uint32_t (&r)[NS][2], int x, long long &hi, unsigned &lo) {
  int gi[NS];
#pragma unroll
  for (int g = 0; g < NS; g++) gi[g] = __float2int_rn(__uint_as_float(r[g][x]));  // exact: integers below 2^24
  long long t = gi[2];
#pragma unroll
  for (int g = 3; g < NS; g++) t = t * 128 + gi[g];
  const long long q = gi[0] * 128 + gi[1];
  const unsigned l = lo + (unsigned)t;  // low 32 bits of T, modulo 2^32
  hi += q * 1024 + (t >> 32) + (l < lo ? 1 : 0);  // arithmetic shift: floor; carry of the low word
  lo = l;
}
__device__ __forceinline__ double fixed_to_double(long long hi, unsigned lo) {
  return fma((double)hi, 0x1p-31, (double)lo * 0x1p-63);
}

__device__ inline bool failed(const int *st) { return *((volatile const int *)st) != DEV_OK; }

__device__ inline void raise_timeout(Shared *sh, int *status) {
  sh->abort = 1;
  if (atomicCAS(&status[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) status[ST_AUX] = 4;
}

// ------------------------------------------------------------- digits
// 2^e for integer e in the normal range (exact).
__device__ inline double exp2i(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
__device__ inline int exp_of(const int *exps, long i) { return max(exps[i] - kExpBias, kExpMin); }

// The NS digits of v (|v| < 1) written d[0], d[plane], ...: v is rounded to
// X = v 2^56 (an integer below 2^56; the unit of the last digit is 2^-56),
// then the digits are peeled off from the top in integer arithmetic, each
// rounded to nearest, so |digit 0| <= 128 and |digit p| <= 64 for p >= 1 and
// sum_p digit_p 2^(7 (NS - 1 - p)) = X exactly.
__device__ inline void write_digits(double v, uint16_t *d, size_t plane) {
  long long X = __double2ll_rn(v * 0x1p56);
#pragma unroll
  for (int p = 0; p < NS; p++) {
    const int sh = SLICE_BITS * (NS - 1 - p);
    long long dg = (sh > 0) ? ((X + (1LL << (sh > 0 ? sh - 1 : 0))) >> sh) : X;
    X -= dg << sh;
    d[p * plane] = __bfloat16_as_ushort(__float2bfloat16_rn((float)(int)dg));  // small integer: exact
  }
}

// Row exponents: one CTA per (32 rows, listed tile, stripe of the columns):
// lane = row, warps stride the stripe's columns; exp[base + r] =
// max(exp[base + r], e_r) with every |x_rc| < 2^e_r (the stripes combine
// through the atomic maximum).
__global__ void __launch_bounds__(256)
    k_rowexp64(const double *__restrict__ t64, const float *__restrict__ t32, const unsigned char *__restrict__ cls,
               const int4 *__restrict__ jobs, int nb, int *__restrict__ exps, const int *st) {
  if (failed(st)) return;
  __shared__ double red[8][33];
  int4 jb = jobs[blockIdx.y];
  size_t base = (size_t)jb.x * nb * nb;
  bool f64 = cls[jb.x] == EMU_CLASS_FP64;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int r = blockIdx.x * 32 + lane;
  double m = 0.0;
  for (int c = blockIdx.z * 8 + w; c < nb; c += 8 * gridDim.z) {
    size_t o = base + r + (size_t)c * nb;
    double x = f64 ? t64[o] : (double)t32[o];
    m = fmax(m, fabs(x));
  }
  red[w][lane] = m;
  __syncthreads();
  if (w == 0) {
    for (int q = 1; q < 8; q++) m = fmax(m, red[q][lane]);
    if (m > 0.0) {
      int e;
      frexp(m, &e);  // m = f 2^e, f in [0.5, 1): every |x| < 2^e
      atomicMax(&exps[jb.z + r], e + kExpBias);
    }
  }
}

// The NS digit planes of each listed tile.  One CTA per (32 x 32 block,
// tile): the block is read column by column (coalesced in the column-major
// tile), transposed in shared memory, and each digit plane is written row by
// row (coalesced in the row-major plane).
__global__ void __launch_bounds__(256)
    k_slice64(const double *__restrict__ t64, const float *__restrict__ t32, const unsigned char *__restrict__ cls,
              const int4 *__restrict__ jobs, int nb, const int *__restrict__ exps, uint16_t *__restrict__ digits,
              const int *st) {
  if (failed(st)) return;
  __shared__ double blk[32][33];
  int4 jb = jobs[blockIdx.y];
  size_t base = (size_t)jb.x * nb * nb;
  bool f64 = cls[jb.x] == EMU_CLASS_FP64;
  int nbb = nb / 32;
  int r0 = (blockIdx.x % nbb) * 32, c0 = (blockIdx.x / nbb) * 32;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = w; c < 32; c += 8) {
    size_t o = base + (r0 + lane) + (size_t)(c0 + c) * nb;
    blk[lane][c] = f64 ? t64[o] : (double)t32[o];
  }
  __syncthreads();
  size_t plane = (size_t)nb * nb;
  for (int q = 0; q < 4; q++) {
    int rr = w + 8 * q;
    int r = r0 + rr;
    double v = blk[rr][lane] * exp2i(-exp_of(exps, (long)jb.z + r));  // exact: |v| < 1
    write_digits(v, digits + (size_t)jb.y * NS * plane + (size_t)r * nb + c0 + lane, plane);
  }
}

// Row exponents of a dense column-major block X[0:nrows, col0:col0+ncols]
// (the residuals of the empirical covariance): one CTA per (32 rows, column
// stripe), lane = row, warps stride columns; exps[r] = max(exps[r], e) with
// every |x| < 2^e.
__global__ void __launch_bounds__(256)
    k_rowexp_dense(const double *__restrict__ X, long ld, int nrows, long col0, long ncols, int *__restrict__ exps,
                   const int *st) {
  if (failed(st)) return;
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  double m = 0.0;
  if (r < nrows)
    for (long c = (long)blockIdx.y * 8 + w; c < ncols; c += 8L * gridDim.y) m = fmax(m, fabs(X[r + (col0 + c) * ld]));
  red[w][lane] = m;
  __syncthreads();
  if (w == 0 && r < nrows) {
    for (int q = 1; q < 8; q++) m = fmax(m, red[q][lane]);
    if (m > 0.0) {
      int e;
      frexp(m, &e);
      atomicMax(&exps[r], e + kExpBias);
    }
  }
}

// Digit planes of that block, K-major: plane p, row r (< npad), column c
// (< kpad); rows >= nrows and columns >= ncols are zero.  One CTA per 32x32
// block, transposed through shared memory.
__global__ void __launch_bounds__(256)
    k_slice_dense(const double *__restrict__ X, long ld, int nrows, long col0, long ncols, int npad, long kpad,
                  const int *__restrict__ exps, uint16_t *__restrict__ digits, const int *st) {
  if (failed(st)) return;
  __shared__ double blk[32][33];
  const long c0 = (long)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int cc = w; cc < 32; cc += 8) {
    const int r = r0 + lane;
    const long c = c0 + cc;
    blk[lane][cc] = (r < nrows && c < ncols) ? X[r + (col0 + c) * ld] : 0.0;
  }
  __syncthreads();
  const size_t plane = (size_t)npad * kpad;
  for (int q = 0; q < 4; q++) {
    const int rr = w + 8 * q, r = r0 + rr;
    const double v = blk[rr][lane] * exp2i(-exp_of(exps, r));  // exact: |v| < 1
    write_digits(v, digits + (size_t)r * kpad + c0 + lane, plane);
  }
}

// Digits of Z columns per matrix block: one CTA per (sample c < s_pad, block).
// The exponent covers the block's rows of column c; samples c >= s are zero.
__global__ void __launch_bounds__(256)
    k_slicez64(const double *__restrict__ Z, long ldz, int s, int s_pad, const int2 *__restrict__ blocks, long zcols,
               int *__restrict__ exps, uint16_t *__restrict__ digits, const int *st) {
  if (failed(st)) return;
  __shared__ double red[8];
  __shared__ int s_e;
  int c = blockIdx.x, b = blockIdx.y;
  int2 blk = blocks[b];
  const double *z = Z + blk.x + (size_t)c * ldz;
  double m = 0.0;
  if (c < s)
    for (int r = threadIdx.x; r < blk.y; r += blockDim.x) m = fmax(m, fabs(z[r]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); q++) m = fmax(m, red[q]);
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    s_e = e;
    exps[(long)b * s_pad + c] = e + kExpBias;
  }
  __syncthreads();
  const double inv = exp2i(-s_e);
  size_t plane = (size_t)s_pad * zcols;
  for (int r = threadIdx.x; r < blk.y; r += blockDim.x)
    write_digits((c < s) ? z[r] * inv : 0.0, digits + (size_t)c * zcols + blk.x + r, plane);
}

// ------------------------------------------------------- blocked TRSM
constexpr int NQ = TW / 32;  // 32-column quarters of a block
static_assert(TW % 32 == 0 && TW % BN == 0, "block width");

// Row exponent (as the readers clamp it) and digits of one row of a
// TW-column block held NQ values per lane (columns lane + 32 q): the exponent
// is written to *e_out by lane 0 (0 for a row of zeros), plane p of column c
// at d[c + p plane].
__device__ inline void row_digits_tw(const double (&x)[NQ], int *e_out, uint16_t *d, size_t plane) {
  const int lane = threadIdx.x & 31;
  double m = 0.0;
#pragma unroll
  for (int q = 0; q < NQ; q++) m = fmax(m, fabs(x[q]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  int e = 0;
  if (m > 0.0) frexp(m, &e);  // every |x| < 2^e
  if (lane == 0) *e_out = (m > 0.0) ? e + kExpBias : 0;
  const double sc = exp2i(-((m > 0.0) ? max(e, kExpMin) : kExpMin));  // exact: |x sc| < 1
#pragma unroll
  for (int q = 0; q < NQ; q++) write_digits(x[q] * sc, d + 32 * q + lane, plane);
}

// Digits of L_kk's column blocks: one CTA per (32 rows, block J), warp w
// rows 4w..4w+3 of the 32, lane = columns lane + 32 q of the block.
__global__ void __launch_bounds__(256)
    k_lkk_digits(const double *__restrict__ L, int nb, int *__restrict__ exps, uint16_t *__restrict__ digits,
                 const int *st) {
  if (failed(st)) return;
  const int J = blockIdx.y, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c0 = J * TW;
  for (int i = 0; i < 4; i++) {
    const int r = blockIdx.x * 32 + w * 4 + i;
    if (r < (J + 1) * TW) continue;  // warp-uniform: rows no product reads
    double x[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) x[q] = L[(size_t)r + (size_t)(c0 + 32 * q + lane) * nb];
    row_digits_tw(x, exps + (size_t)J * nb + r, digits + ((size_t)J * NS * nb + r) * TW, (size_t)nb * TW);
  }
}

// Column block J of X = A L_kk^{-T} for every listed tile, in place: the
// earlier blocks' contributions have been subtracted (digit products), so
// only L_kk's TW x TW diagonal block enters.  One CTA per (4 rows, tile),
// warp = row, lane = column of each 32-column quarter q: the earlier
// quarters' contribution is subtracted (L_kk's entries read from L2, a
// warp's 32 rows of one column at a time), then forward substitution against
// the pre-scaled diagonal 32 x 32 block.
__global__ void __launch_bounds__(128)
    k_trsm64_block(double *__restrict__ t64, int nb, const int *__restrict__ tiles, const double *__restrict__ Lkk,
                   int J, const double *__restrict__ Ls, const double *__restrict__ rinvs, int slot0,
                   int *__restrict__ exps, uint16_t *__restrict__ digits, const int *st) {
  if (failed(st)) return;
  const int z = blockIdx.y, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c0 = J * TW, r = blockIdx.x * 4 + w;
  double *X = t64 + (size_t)tiles[z] * nb * nb + r;
  double a[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) a[q] = X[(size_t)(c0 + 32 * q + lane) * nb];
#pragma unroll
  for (int q = 0; q < NQ; q++) {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int qq = 0; qq < q; qq++) {
      const double *lq = Lkk + (size_t)(c0 + 32 * q + lane) + (size_t)(c0 + 32 * qq) * nb;
#pragma unroll 8
      for (int p = 0; p < 32; p += 2) {
        s0 = fma(__shfl_sync(0xffffffffu, a[qq], p), __ldg(lq + (size_t)p * nb), s0);
        s1 = fma(__shfl_sync(0xffffffffu, a[qq], p + 1), __ldg(lq + (size_t)(p + 1) * nb), s1);
      }
    }
    // Ls(p, l) = L(l, p) / L(p, p): a_l -= a_p Ls(p, l) on the unscaled a_p
    const int cb = J * NQ + q;
    double v = a[q] - (s0 + s1);
    double ld[32];
#pragma unroll
    for (int p = 0; p < 32; p++) ld[p] = (p < lane) ? Ls[(size_t)(cb * 32 + p) * 32 + lane] : 0.0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
      const double vj = __shfl_sync(0xffffffffu, v, j);
      if (lane > j) v = fma(-vj, ld[j], v);
    }
    a[q] = v * rinvs[cb * 32 + lane];
  }
#pragma unroll
  for (int q = 0; q < NQ; q++) X[(size_t)(c0 + 32 * q + lane) * nb] = a[q];
  if (digits) {
    const size_t slot = (size_t)slot0 + z;
    row_digits_tw(a, exps + slot * nb + r, digits + (slot * NS * nb + r) * TW, (size_t)nb * TW);
  }
}

// ------------------------------------------------------------- GEMM
template <int MODE>
__global__ void __maxnreg__(168)
    k_tc_gemm64(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                const Item *__restrict__ items, int nitems, const Seg *__restrict__ segs, int nb, int a_plane,
                int b_plane, const int *__restrict__ a_exp, const int *__restrict__ b_exp,
                double *__restrict__ out, int ldo, int *status) {
  extern __shared__ uint8_t smem_raw[];
  uint32_t raw_addr = tc::smem_u32(smem_raw);
  uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
  uint8_t *ring = smem_raw + pad;
  Shared *sh = reinterpret_cast<Shared *>(ring + RING_BYTES);
  const uint32_t ring_addr = raw_addr + pad;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kstages = nb / BK;  // stages per segment

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      tc::mbar_init(&sh->full[s], 1);
      tc::mbar_init(&sh->empty[s], 1);
    }
    tc::mbar_init(&sh->tfull, 1);
    tc::mbar_init(&sh->tempty, EPI_THREADS);
    tc::mbar_init(&sh->done, 1);
    // one reading of the status word for all roles: an earlier failure skips the work
    sh->abort = failed(status) ? 1 : 0;
    tc::fence_barrier_init();
    tc::tma_prefetch_desc(&amap);
    tc::tma_prefetch_desc(&bmap);
  }
  if (warp == 1) {
    tc::tmem_alloc(&sh->tmem_base, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sh->tmem_base;
  volatile int *abort = &sh->abort;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = *abort == 0;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        Item item = items[it];
        for (int sg = item.seg_begin; sg < item.seg_end && ok; sg++) {
          Seg sd = segs[sg];
          for (int kc = 0; kc < kstages; kc++) {
            if (!tc::mbar_wait(&sh->empty[stage], phase ^ 1u, abort)) {
              raise_timeout(sh, status);
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&sh->full[stage], (uint32_t)STAGE_BYTES);
            uint8_t *st = ring + stage * STAGE_BYTES;
            for (int p = 0; p < NS; p++)
              tc::tma_load_2d(st + p * A_SL, &amap, &sh->full[stage], sd.a_x + kc * BK, sd.a_row + p * a_plane);
            for (int q = 0; q < NS; q++)
              tc::tma_load_2d(st + NS * A_SL + q * B_SL, &bmap, &sh->full[stage], sd.b_x + kc * BK,
                              sd.b_row + q * b_plane);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // every stage's last load must have landed before the CTA exits
      for (int s = 0; s < STAGES; s++) {
        uint32_t par = (s < stage) ? phase : (phase ^ 1u);
        tc::mbar_wait_inflight(&sh->full[s], par);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t chunk = 0;
      uint32_t started = 0;
      bool ok = *abort == 0;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        Item item = items[it];
        const int total = (item.seg_end - item.seg_begin) * kstages;  // K stages of the item
        for (int ks_i = 0; ks_i < total && ok; ks_i++) {
          if (ks_i % CHUNK_STAGES == 0) {
            // the epilogue has read the previous chunk's accumulators
            if (!tc::mbar_wait(&sh->tempty, (chunk & 1u) ^ 1u, abort)) {
              raise_timeout(sh, status);
              ok = false;
              break;
            }
            tc::fence_after_sync();
            started = 0;
          }
          if (!tc::mbar_wait(&sh->full[stage], phase, abort)) {
            raise_timeout(sh, status);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          uint32_t st = ring_addr + stage * STAGE_BYTES;
          const uint64_t a0 = tc::smem_desc(st, 16, 512, tc::kSwizzle64B);
          const uint64_t b0 = tc::smem_desc(st + NS * A_SL, 16, 512, tc::kSwizzle64B);
#pragma unroll
          for (int ks = 0; ks < BK / 16; ks++) {
#pragma unroll
            for (int p = 0; p < NS; p++) {
              const uint64_t ad = tc::desc_add(a0, p * A_SL + ks * 32);
#pragma unroll
              for (int q = 0; q < NS - p; q++) {
                const int g = p + q;
                const uint64_t bd = tc::desc_add(b0, q * B_SL + ks * 32);
                tc::mma_f16(tmem + (uint32_t)(g * BN), ad, bd, IDESC, (started >> g) & 1u);
                started |= 1u << g;
              }
            }
          }
          tc::mma_commit(&sh->empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
          if (ks_i % CHUNK_STAGES == CHUNK_STAGES - 1 || ks_i == total - 1) {
            tc::mma_commit(&sh->tfull);
            chunk++;
          }
        }
      }
      tc::mma_commit(&sh->done);
      tc::mbar_wait_inflight(&sh->done, 0);
    }
  } else if (warp >= EPI_WARP0) {
    // ------------------------------------------------------------ epilogue
    // warps 4..11: TMEM lane quarter warp % 4 (the lanes a warp may access),
    // columns [half * 32, half * 32 + 32) of the block
    const int quarter = warp & 3;
    const int half = (warp - EPI_WARP0) >> 2;
    const int row = quarter * 32 + lane;
    const int col0 = half * 32;
    const uint32_t tlane = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
    uint32_t chunk = 0;
    bool ok = *abort == 0;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      Item item = items[it];
      const int total = (item.seg_end - item.seg_begin) * kstages;
      const int nchunks = (total + CHUNK_STAGES - 1) / CHUNK_STAGES;
      long long hi[32];
      unsigned lo[32];
#pragma unroll
      for (int x = 0; x < 32; x++) {
        hi[x] = 0;
        lo[x] = 0u;
      }
      for (int c = 0; c < nchunks; c++) {
        if (!tc::mbar_wait(&sh->tfull, chunk & 1u, abort)) {
          raise_timeout(sh, status);
          ok = false;
          break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int h = 0; h < 16; h++) {
          uint32_t r[NS][2];
#pragma unroll
          for (int g = 0; g < NS; g++) tc::tmem_ld_32x32b_x2(tlane + (uint32_t)(g * BN + h * 2), r[g]);
          tc::tmem_ld_wait();
#pragma unroll
          for (int x = 0; x < 2; x++) fold_groups(r, x, hi[h * 2 + x], lo[h * 2 + x]);
        }
        tc::fence_before_sync();
        tc::mbar_arrive(&sh->tempty);
        chunk++;
      }
      if (!ok) break;
      // scales 2^(e_row + e_col), exact; then the output block
      const int ea = exp_of(a_exp, (long)item.a_sc + row);
      double *o = out + item.out_off + row;
      // in groups of 8 columns: 8 loads in flight, then 8 stores
      if (MODE == TC64_SUB || row < item.rows_valid) {
#pragma unroll
        for (int x0 = 0; x0 < 32; x0 += 8) {
          double cv[8];
#pragma unroll
          for (int x = 0; x < 8; x++) {
            const int cx = col0 + x0 + x;
            cv[x] = (MODE == TC64_SUB || cx < item.cols_valid) ? __ldcg(o + (long)cx * ldo) : 0.0;
          }
#pragma unroll
          for (int x = 0; x < 8; x++) {
            const int cx = col0 + x0 + x;
            double v = fixed_to_double(hi[x0 + x], lo[x0 + x]) * exp2i(ea + exp_of(b_exp, (long)item.b_sc + cx));
            if (MODE == TC64_SUB)
              __stcg(o + (long)cx * ldo, cv[x] - v);
            else if (cx < item.cols_valid)
              __stcg(o + (long)cx * ldo, cv[x] + v);
          }
        }
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace

emu_status make_map(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                    uint32_t box_rows) {
  return gemm_tc::make_map_bf16(ctx, map, base, inner, rows, box_rows);
}

emu_status launch_row_exponents(emu_ctx *ctx, const double *t64, const float *t32, const unsigned char *cls,
                                const int4 *d_jobs, int njobs, int nb, int *exps) {
  if (njobs <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 8.0 * njobs * (double)nb * nb);
  k_rowexp64<<<dim3(nb / 32, njobs, 8), 256, 0, ctx->stream>>>(t64, t32, cls, d_jobs, nb, exps, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_slice(emu_ctx *ctx, const double *t64, const float *t32, const unsigned char *cls,
                        const int4 *d_jobs, int njobs, int nb, const int *exps, uint16_t *digits) {
  if (njobs <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, (8.0 + 2.0 * NS) * njobs * (double)nb * nb);
  k_slice64<<<dim3((nb / 32) * (nb / 32), njobs), 256, 0, ctx->stream>>>(t64, t32, cls, d_jobs, nb, exps, digits,
                                                                         ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_slice_z(emu_ctx *ctx, const double *Z, long ldz, int s, int s_pad, const int2 *d_blocks,
                          int nblocks, long zcols, int *exps, uint16_t *digits) {
  if (nblocks <= 0 || s_pad <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, (8.0 + 2.0 * NS) * (double)s_pad * zcols);
  k_slicez64<<<dim3(s_pad, nblocks), 256, 0, ctx->stream>>>(Z, ldz, s, s_pad, d_blocks, zcols, exps, digits,
                                                            ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_dense_digits(emu_ctx *ctx, const double *X, long ld, int nrows, long col0, long ncols, int npad,
                               long kpad, int *exps, uint16_t *digits) {
  if (npad % 32 != 0 || kpad % 32 != 0 || nrows > npad || ncols > kpad) return EMU_EINVAL;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, (16.0 + 2.0 * NS) * (double)npad * kpad);
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(exps, 0, (size_t)npad * sizeof(int), ctx->stream));
  const int ystripes = (int)std::min<long>(64, (ncols + 7) / 8);
  k_rowexp_dense<<<dim3(npad / 32, std::max(ystripes, 1)), 256, 0, ctx->stream>>>(X, ld, nrows, col0, ncols, exps,
                                                                                  ctx->d_status);
  EMU_LAUNCHED(ctx);
  k_slice_dense<<<dim3((unsigned)(kpad / 32), npad / 32), 256, 0, ctx->stream>>>(X, ld, nrows, col0, ncols, npad,
                                                                                 kpad, exps, digits, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_lkk_digits(emu_ctx *ctx, const double *Lkk, int nb, int *exps, uint16_t *digits) {
  if (nb % BM != 0) return EMU_EINVAL;
  const int nJ = nb / TW;
  if (nJ < 2) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, (8.0 + 2.0 * NS) * (double)nb * TW * (nJ - 1));
  k_lkk_digits<<<dim3(nb / 32, nJ - 1), 256, 0, ctx->stream>>>(Lkk, nb, exps, digits, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_trsm_block(emu_ctx *ctx, double *t64, int nb, const int *d_tiles, int ntiles, const double *Lkk,
                             int J, const double *Ls, const double *rinvs, int slot0, int *exps, uint16_t *digits) {
  if (nb % TW != 0 || J < 0 || J >= nb / TW) return EMU_EINVAL;
  if (ntiles <= 0) return EMU_OK;
  k_trsm64_block<<<dim3(nb / 4, ntiles), 128, 0, ctx->stream>>>(t64, nb, d_tiles, Lkk, J, Ls, rinvs, slot0, exps,
                                                                digits, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch(emu_ctx *ctx, const CUtensorMap &a, const CUtensorMap &b, const Item *d_items, int nitems,
                  const Seg *d_segs, int nb, int a_plane, int b_plane, const int *a_exp, const int *b_exp, int mode,
                  double *out64, int ldo, int max_ctas) {
  if (nitems <= 0) return EMU_OK;
  if (nb % BK != 0) return EMU_EINVAL;
  static std::atomic<uint64_t> attr_sub{0}, attr_add{0};
  EMU_CUDA_TRY(ctx, smem_limit_once(attr_sub, ctx->device, (const void *)k_tc_gemm64<TC64_SUB>, SMEM_BYTES));
  EMU_CUDA_TRY(ctx, smem_limit_once(attr_add, ctx->device, (const void *)k_tc_gemm64<TC64_ADD>, SMEM_BYTES));
  int grid = nitems < max_ctas ? nitems : max_ctas;
  if (mode == TC64_SUB)
    k_tc_gemm64<TC64_SUB><<<grid, NTHREADS, SMEM_BYTES, ctx->stream>>>(a, b, d_items, nitems, d_segs, nb, a_plane,
                                                                       b_plane, a_exp, b_exp, out64, ldo,
                                                                       ctx->d_status);
  else
    k_tc_gemm64<TC64_ADD><<<grid, NTHREADS, SMEM_BYTES, ctx->stream>>>(a, b, d_items, nitems, d_segs, nb, a_plane,
                                                                       b_plane, a_exp, b_exp, out64, ldo,
                                                                       ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

}  // namespace gemm64
