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
//   warps 2..5  epilogue: every KCHUNK of K, the 8 group accumulators are
//               added in FP64 into per-thread registers, smallest group first;
//               after the last chunk the row scales are applied and the block
//               is subtracted from the FP64 output.
// The 8 accumulators fill TMEM, so the MMA warp waits for the epilogue to
// drain them before the next chunk.
#include <cuda_bf16.h>

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
constexpr int NTHREADS = 192;
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

// Weight 2^-7(g+2) of the digit products of group g = p + q.
__constant__ double kGroupWeight[NS] = {0x1p-14, 0x1p-21, 0x1p-28, 0x1p-35, 0x1p-42, 0x1p-49, 0x1p-56, 0x1p-63};
static_assert(NS == 8 && SLICE_BITS == 7, "kGroupWeight is written for 8 digits of 7 bits");

__device__ inline bool failed(const int *st) { return *((volatile const int *)st) != DEV_OK; }

__device__ inline void raise_timeout(Shared *sh, int *status) {
  sh->abort = 1;
  if (atomicCAS(&status[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) status[ST_AUX] = 4;
}

// ------------------------------------------------------------- digits
// 2^e_r per row r of each listed tile, with max_c |x_rc| < 2^e_r (1 for a
// zero row).  One CTA per (32 rows, tile): lane = row, warps stride columns.
__global__ void __launch_bounds__(256)
    k_rowscale64(const double *__restrict__ t64, const float *__restrict__ t32, const unsigned char *__restrict__ cls,
                 const int2 *__restrict__ jobs, int nb, double *__restrict__ scales, const int *st) {
  if (failed(st)) return;
  __shared__ double red[8][33];
  int2 jb = jobs[blockIdx.y];
  size_t base = (size_t)jb.x * nb * nb;
  bool f64 = cls[jb.x] == EMU_CLASS_FP64;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int r = blockIdx.x * 32 + lane;
  double m = 0.0;
  for (int c = w; c < nb; c += 8) {
    size_t o = base + r + (size_t)c * nb;
    double x = f64 ? t64[o] : (double)t32[o];
    m = fmax(m, fabs(x));
  }
  red[w][lane] = m;
  __syncthreads();
  if (w == 0) {
    for (int q = 1; q < 8; q++) m = fmax(m, red[q][lane]);
    int e = 0;
    if (m > 0.0) frexp(m, &e);  // m = f 2^e, f in [0.5, 1): every |x| < 2^e
    scales[(size_t)jb.y * nb + r] = ldexp(1.0, e);
  }
}

// The NS digit planes of each listed tile.  One CTA per (32 x 32 block,
// tile): the block is read column by column (coalesced in the column-major
// tile), transposed in shared memory, and each digit plane is written row by
// row (coalesced in the row-major plane).
__global__ void __launch_bounds__(256)
    k_slice64(const double *__restrict__ t64, const float *__restrict__ t32, const unsigned char *__restrict__ cls,
              const int2 *__restrict__ jobs, int nb, const double *__restrict__ scales, uint16_t *__restrict__ digits,
              const int *st) {
  if (failed(st)) return;
  __shared__ double blk[32][33];
  int2 jb = jobs[blockIdx.y];
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
  const double radix = (double)(1 << SLICE_BITS);
  for (int q = 0; q < 4; q++) {
    int rr = w + 8 * q;
    int r = r0 + rr;
    double v = blk[rr][lane] * (1.0 / scales[(size_t)jb.y * nb + r]);  // powers of two: exact, |v| < 1
    size_t plane = (size_t)nb * nb;
    uint16_t *d = digits + (size_t)jb.y * NS * plane + (size_t)r * nb + c0 + lane;
#pragma unroll
    for (int p = 0; p < NS; p++) {
      v *= radix;                 // exact
      double s = rint(v);         // digit p, |s| <= 2^SLICE_BITS
      v -= s;                     // exact, |v| <= 1/2
      d[p * plane] = __bfloat16_as_ushort(__double2bfloat16(s));  // small integer: exact
    }
  }
}

// ------------------------------------------------------------- GEMM
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm64(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                const Item *__restrict__ items, int nitems, int nb, const double *__restrict__ scales,
                double *__restrict__ out, int ldo, int *status) {
  extern __shared__ uint8_t smem_raw[];
  uint32_t raw_addr = tc::smem_u32(smem_raw);
  uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
  uint8_t *ring = smem_raw + pad;
  Shared *sh = reinterpret_cast<Shared *>(ring + RING_BYTES);
  const uint32_t ring_addr = raw_addr + pad;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kstages = nb / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      tc::mbar_init(&sh->full[s], 1);
      tc::mbar_init(&sh->empty[s], 1);
    }
    tc::mbar_init(&sh->tfull, 1);
    tc::mbar_init(&sh->tempty, 128);
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
        for (int kc = 0; kc < kstages; kc++) {
          if (!tc::mbar_wait(&sh->empty[stage], phase ^ 1u, abort)) {
            raise_timeout(sh, status);
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&sh->full[stage], (uint32_t)STAGE_BYTES);
          uint8_t *st = ring + stage * STAGE_BYTES;
          for (int p = 0; p < NS; p++)
            tc::tma_load_2d(st + p * A_SL, &amap, &sh->full[stage], kc * BK, item.a_row + p * nb);
          for (int q = 0; q < NS; q++)
            tc::tma_load_2d(st + NS * A_SL + q * B_SL, &bmap, &sh->full[stage], kc * BK, item.b_row + q * nb);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // every stage's last load must have landed before the CTA exits
      for (int s = 0; s < STAGES; s++) {
        uint32_t par = (s < stage) ? phase : (phase ^ 1u);
        tc::mbar_wait(&sh->full[s], par, abort);
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
        for (int kc = 0; kc < kstages && ok; kc++) {
          if (kc % CHUNK_STAGES == 0) {
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
#pragma unroll
          for (int ks = 0; ks < BK / 16; ks++) {
#pragma unroll
            for (int p = 0; p < NS; p++) {
              uint64_t ad = tc::smem_desc(st + p * A_SL + ks * 32, 16, 512, tc::kSwizzle64B);
#pragma unroll
              for (int q = 0; q < NS - p; q++) {
                const int g = p + q;
                uint64_t bd = tc::smem_desc(st + NS * A_SL + q * B_SL + ks * 32, 16, 512, tc::kSwizzle64B);
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
          if (kc % CHUNK_STAGES == CHUNK_STAGES - 1 || kc == kstages - 1) {
            tc::mma_commit(&sh->tfull);
            chunk++;
          }
        }
      }
      tc::mma_commit(&sh->done);
      tc::mbar_wait(&sh->done, 0, abort);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;  // TMEM lanes this warp may access
    const int row = quarter * 32 + lane;
    const uint32_t tlane = tmem + ((uint32_t)(quarter * 32) << 16);
    const int nchunks = (kstages + CHUNK_STAGES - 1) / CHUNK_STAGES;
    uint32_t chunk = 0;
    bool ok = *abort == 0;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      double acc[BN];
#pragma unroll
      for (int x = 0; x < BN; x++) acc[x] = 0.0;
      for (int c = 0; c < nchunks; c++) {
        if (!tc::mbar_wait(&sh->tfull, chunk & 1u, abort)) {
          raise_timeout(sh, status);
          ok = false;
          break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int h = 0; h < BN / 32; h++) {
#pragma unroll
          for (int g = NS - 1; g >= 0; g--) {
            uint32_t r[32];
            tc::tmem_ld_32x32b_x32(tlane + (uint32_t)(g * BN + h * 32), r);
            tc::tmem_ld_wait();
            const double wg = kGroupWeight[g];
#pragma unroll
            for (int x = 0; x < 32; x++) acc[h * 32 + x] = fma((double)__uint_as_float(r[x]), wg, acc[h * 32 + x]);
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(&sh->tempty);
        chunk++;
      }
      if (!ok) break;
      Item item = items[it];
      const double sa = scales[item.a_sc + row];
      double *o = out + item.out_off + row;
#pragma unroll
      for (int h = 0; h < BN / 32; h++) {
        double cv[32];
#pragma unroll
        for (int x = 0; x < 32; x++) cv[x] = __ldcg(o + (long)(h * 32 + x) * ldo);
#pragma unroll
        for (int x = 0; x < 32; x++)
          __stcg(o + (long)(h * 32 + x) * ldo, cv[x] - acc[h * 32 + x] * (sa * scales[item.b_sc + h * 32 + x]));
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

emu_status launch_slice(emu_ctx *ctx, const double *t64, const float *t32, const unsigned char *cls,
                        const int2 *d_jobs, int njobs, int nb, uint16_t *digits, double *scales) {
  if (njobs <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, (8.0 + 2.0 * NS) * njobs * (double)nb * nb);
  k_rowscale64<<<dim3(nb / 32, njobs), 256, 0, ctx->stream>>>(t64, t32, cls, d_jobs, nb, scales, ctx->d_status);
  EMU_LAUNCHED(ctx);
  k_slice64<<<dim3((nb / 32) * (nb / 32), njobs), 256, 0, ctx->stream>>>(t64, t32, cls, d_jobs, nb, scales, digits,
                                                                         ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch(emu_ctx *ctx, const CUtensorMap &a, const CUtensorMap &b, const Item *d_items, int nitems, int nb,
                  const double *scales, double *out64, int ldo, int max_ctas) {
  if (nitems <= 0) return EMU_OK;
  if (nb % BK != 0) return EMU_EINVAL;
  static bool attr_done = false;
  if (!attr_done) {
    EMU_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_gemm64, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr_done = true;
  }
  int grid = nitems < max_ctas ? nitems : max_ctas;
  k_tc_gemm64<<<grid, NTHREADS, SMEM_BYTES, ctx->stream>>>(a, b, d_items, nitems, nb, scales, out64, ldo,
                                                           ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

}  // namespace gemm64
