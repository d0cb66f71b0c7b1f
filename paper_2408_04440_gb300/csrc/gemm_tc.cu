// gemm_tc.cu -- tcgen05 tile GEMM with TMEM accumulators and TMA operand
// loads: the trailing SYRK/GEMM updates of the mixed-precision tile Cholesky
// ("Mixed-Precision Computation Innovations") and the low-precision part of
// drawing emulations ("Generating Emulations", xi = V z).
//
// Precision classes on the tensor cores (FP32 accumulation):
//   E4M3 class: one kind::f8f6f4 product of FP8-E4M3 copies carrying a
//     power-of-two scale per tile; the epilogue divides the scales out.
//   TF32 class: one kind::tf32 product of copies rounded to TF32 (nearest),
//     K = 8 per instruction, at half the BF16 rate.
//   BF16 class: one kind::f16 product a0 b0 of the round-to-nearest BF16 operands.
//   FP32 class: each FP32 operand is split into three BF16 pieces
//     x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1))
//     and the six products with i + j <= 2 are accumulated, smallest first:
//     a1b1, a0b2, a2b0, a0b1, a1b0, a0b0.  The dropped terms are below
//     2^-24 relative, so the result carries FP32-level accuracy.
//
// Warp roles (192 threads, one CTA per SM, persistent over the item list):
//   warp 0      TMA producer (one lane): STAGES-deep ring of operand stages.
//   warp 1      TMEM allocator + MMA issuer (one lane).
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (one TMEM lane per
//               thread), read-modify-write of the output.
// Two 256-column accumulators let the epilogue of one block overlap the MMAs
// of the next.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "gemm_tc.h"
#include "tc.cuh"

namespace gemm_tc {
namespace {

constexpr int A_PIECE = BM * BK * 2;  // 8 KB
constexpr int B_PIECE = BN * BK * 2;  // 16 KB
constexpr int STAGE_BYTES = NPIECE * (A_PIECE + B_PIECE);
constexpr int RING_BYTES = STAGES * STAGE_BYTES;
constexpr int BAR_BYTES = 128;
constexpr int SMEM_BYTES = RING_BYTES + BAR_BYTES + 1024;  // + alignment slack
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t IDESC = tc::idesc_f32acc(1u /*BF16*/, BM, BN);
constexpr uint32_t IDESC8 = tc::idesc_f32acc(0u /*E4M3*/, BM, BN);
constexpr uint32_t IDESC32 = tc::idesc_f32acc(2u /*TF32*/, BM, BN);
constexpr int A8_BYTES = BM * BK;  // FP8: BK elements = BK bytes per row
constexpr int B8_BYTES = BN * BK;
constexpr int A32_BYTES = BM * BK * 4;  // TF32: 128 bytes per row (128-byte swizzle)
constexpr int B32_BYTES = BN * BK * 4;
static_assert(A32_BYTES <= NPIECE * A_PIECE && B32_BYTES <= NPIECE * B_PIECE, "TF32 operands fit a stage");

struct Shared {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(Shared) <= BAR_BYTES, "barrier block");

__device__ inline void raise_timeout(Shared *sh, int *status) {
  sh->abort = 1;
  if (atomicCAS(&status[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) status[ST_AUX] = 1;
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm(const __grid_constant__ Operands ops, const Item *__restrict__ items, int nitems,
              const Seg *__restrict__ segs, int ksteps, int mode, float *__restrict__ out32,
              double *__restrict__ out64, const __grid_constant__ Outputs outs, int ldo, int *status) {
  extern __shared__ uint8_t smem_raw[];
  uint32_t raw_addr = tc::smem_u32(smem_raw);
  uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
  uint8_t *ring = smem_raw + pad;
  Shared *sh = reinterpret_cast<Shared *>(ring + RING_BYTES);
  const uint32_t ring_addr = raw_addr + pad;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      tc::mbar_init(&sh->full[s], 1);
      tc::mbar_init(&sh->empty[s], 1);
    }
    for (int a = 0; a < 2; a++) {
      tc::mbar_init(&sh->tfull[a], 1);
      tc::mbar_init(&sh->tempty[a], 128);
    }
    tc::mbar_init(&sh->done, 1);
    sh->abort = 0;
    tc::fence_barrier_init();
    tc::tma_prefetch_desc(&ops.a16);
    tc::tma_prefetch_desc(&ops.b16);
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
      bool ok = true;
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        Item item = items[it];
        for (int sg = item.seg_begin; sg < item.seg_end && ok; sg++) {
          Seg s = segs[sg];
          bool f8 = s.cls == EMU_CLASS_E4M3, t32 = s.cls == EMU_CLASS_TF32;
          int np = (s.cls == EMU_CLASS_FP32) ? NPIECE : 1;
          uint32_t bytes = f8    ? (uint32_t)(A8_BYTES + B8_BYTES)
                           : t32 ? (uint32_t)(A32_BYTES + B32_BYTES)
                                 : (uint32_t)np * (A_PIECE + B_PIECE);
          for (int kc = 0; kc < ksteps; kc++) {
            if (!tc::mbar_wait(&sh->empty[stage], phase ^ 1u, abort)) {
              raise_timeout(sh, status);
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&sh->full[stage], bytes);
            uint8_t *st = ring + stage * STAGE_BYTES;
            if (f8) {
              tc::tma_load_2d(st, &ops.a8, &sh->full[stage], s.ax + kc * BK, s.ay);
              tc::tma_load_2d(st + NPIECE * A_PIECE, &ops.b8, &sh->full[stage], s.bx + kc * BK, s.by);
            } else if (t32) {
              tc::tma_load_2d(st, &ops.a32, &sh->full[stage], s.ax + kc * BK, s.ay);
              tc::tma_load_2d(st + NPIECE * A_PIECE, &ops.b32, &sh->full[stage], s.bx + kc * BK, s.by);
            } else {
              for (int q = 0; q < np; q++) {
                tc::tma_load_2d(st + q * A_PIECE, &ops.a16, &sh->full[stage], s.ax + kc * BK,
                                s.ay + q * s.ay_step);
                tc::tma_load_2d(st + NPIECE * A_PIECE + q * B_PIECE, &ops.b16, &sh->full[stage], s.bx + kc * BK,
                                s.by + q * s.by_step);
              }
            }
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // Drain: every stage's last load must have landed before the CTA exits.
      for (int s = 0; s < STAGES; s++) {
        // the most recent use of stage s completed phase (phase ^ (s >= stage))
        uint32_t par = (s < stage) ? phase : (phase ^ 1u);
        tc::mbar_wait_inflight(&sh->full[s], par);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      // products (qa, qb), smallest magnitude first
      const int pa[6] = {1, 0, 2, 0, 1, 0};
      const int pb[6] = {1, 2, 0, 1, 0, 0};
      for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        if (!tc::mbar_wait(&sh->tempty[acc], acc_phase ^ 1u, abort)) {
          raise_timeout(sh, status);
          break;
        }
        tc::fence_after_sync();
        uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
        Item item = items[it];
        uint32_t accumulate = 0;
        for (int sg = item.seg_begin; sg < item.seg_end && ok; sg++) {
          int cls = segs[sg].cls;
          int p0 = (cls == EMU_CLASS_FP32) ? 0 : 5;
          for (int kc = 0; kc < ksteps; kc++) {
            if (!tc::mbar_wait(&sh->full[stage], phase, abort)) {
              raise_timeout(sh, status);
              ok = false;
              break;
            }
            tc::fence_after_sync();
            uint32_t st = ring_addr + stage * STAGE_BYTES;
            if (cls == EMU_CLASS_E4M3) {
              // one K = 32 product of the FP8 copies (rows of 32 bytes, 32-byte swizzle)
              uint64_t ad = tc::smem_desc(st, 16, 256, tc::kSwizzle32B);
              uint64_t bd = tc::smem_desc(st + NPIECE * A_PIECE, 16, 256, tc::kSwizzle32B);
              tc::mma_f8(d_tmem, ad, bd, IDESC8, accumulate);
              accumulate = 1;
            } else if (cls == EMU_CLASS_TF32) {
              // four K = 8 products of the TF32 copies (rows of 128 bytes, 128-byte swizzle)
#pragma unroll
              for (int ks = 0; ks < BK / 8; ks++) {
                uint64_t ad = tc::smem_desc(st + ks * 32, 16, 1024, tc::kSwizzle128B);
                uint64_t bd = tc::smem_desc(st + NPIECE * A_PIECE + ks * 32, 16, 1024, tc::kSwizzle128B);
                tc::mma_tf32(d_tmem, ad, bd, IDESC32, accumulate);
                accumulate = 1;
              }
            } else {
              const uint64_t a0 = tc::smem_desc(st, 16, 512, tc::kSwizzle64B);
              const uint64_t b0 = tc::smem_desc(st + NPIECE * A_PIECE, 16, 512, tc::kSwizzle64B);
#pragma unroll
              for (int ks = 0; ks < BK / 16; ks++) {
                for (int p = p0; p < 6; p++) {
                  const uint64_t ad = tc::desc_add(a0, pa[p] * A_PIECE + ks * 32);
                  const uint64_t bd = tc::desc_add(b0, pb[p] * B_PIECE + ks * 32);
                  tc::mma_f16(d_tmem, ad, bd, IDESC, accumulate);
                  accumulate = 1;
                }
              }
            }
            tc::mma_commit(&sh->empty[stage]);  // frees the stage once these MMAs complete
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        tc::mma_commit(&sh->tfull[acc]);
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1u;
      }
      // all issued MMAs complete before TMEM is released
      tc::mma_commit(&sh->done);
      tc::mbar_wait_inflight(&sh->done, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    int quarter = warp & 3;  // TMEM lanes this warp may access
    int row = quarter * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
      const Item item = items[it];
      // FP32 or BF16 output tiles: the output's columns are loaded one
      // 32-column chunk ahead, the first chunk before the accumulator is
      // ready (the MMAs do not write the output), so that two chunks of
      // loads are in flight per warp
      const bool o32 = mode == TC_SUB_F32 || (mode == TC_SUB_CLASS && item.oc == EMU_CLASS_FP32);
      const bool o16 = mode == TC_SUB_CLASS && (item.oc == EMU_CLASS_BF16 || item.oc == EMU_CLASS_E4M3);
      float *p32 = o32 ? (mode == TC_SUB_F32 ? out32 : outs.f32) + item.out_off + row : nullptr;
      uint16_t *p16 = o16 ? (item.oc == EMU_CLASS_BF16 ? outs.bf16 : outs.e8w) + item.out_off + row : nullptr;
      // E4M3 items: undo the operands' power-of-two scales (exact)
      const float sc = (item.sa >= 0) ? 1.0f / (ops.scale8[item.sa] * ops.scale8[item.sb]) : 1.0f;
      float nf[32];  // the next chunk's output values (BF16 outputs widened on load)
      if (o32) {
#pragma unroll
        for (int x = 0; x < 32; x++) nf[x] = __ldcg(p32 + (long)x * ldo);
      } else if (o16) {
#pragma unroll
        for (int x = 0; x < 32; x++)
          nf[x] = __bfloat162float(__ushort_as_bfloat16(__ldcg((const unsigned short *)(p16 + (long)x * ldo))));
      }
      if (!tc::mbar_wait(&sh->tfull[acc], acc_phase, abort)) {
        raise_timeout(sh, status);
        break;
      }
      tc::fence_after_sync();
      uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
      for (int ch = 0; ch < BN / 32; ch++) {
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tbase + ch * 32, r);
        const bool more = ch + 1 < BN / 32;
        if (o32) {
          float c[32];
#pragma unroll
          for (int x = 0; x < 32; x++) c[x] = nf[x];
          if (more) {
            const float *q = p32 + (long)((ch + 1) * 32) * ldo;
#pragma unroll
            for (int x = 0; x < 32; x++) nf[x] = __ldcg(q + (long)x * ldo);
          }
          tc::tmem_ld_wait();
          float *o = p32 + (long)(ch * 32) * ldo;
#pragma unroll
          for (int x = 0; x < 32; x++) __stcg(o + (long)x * ldo, c[x] - __uint_as_float(r[x]) * sc);
        } else if (o16) {
          // BF16 storage (the E4M3 class's working tiles too): c - acc rounded to nearest BF16
          float c[32];
#pragma unroll
          for (int x = 0; x < 32; x++) c[x] = nf[x];
          if (more) {
            const uint16_t *q = p16 + (long)((ch + 1) * 32) * ldo;
#pragma unroll
            for (int x = 0; x < 32; x++)
              nf[x] = __bfloat162float(__ushort_as_bfloat16(__ldcg((const unsigned short *)(q + (long)x * ldo))));
          }
          tc::tmem_ld_wait();
          uint16_t *o = p16 + (long)(ch * 32) * ldo;
#pragma unroll
          for (int x = 0; x < 32; x++) {
            const float v = c[x] - __uint_as_float(r[x]) * sc;
            __stcg((unsigned short *)(o + (long)x * ldo), __bfloat16_as_ushort(__float2bfloat16_rn(v)));
          }
        } else {
          tc::tmem_ld_wait();
          if (row < item.rows_valid) {
            double *o = out64 + item.out_off + row + (long)(ch * 32) * ldo;
            int nval = item.cols_valid - ch * 32;
            double c[32];
#pragma unroll
            for (int x = 0; x < 32; x++) c[x] = (x < nval) ? __ldcg(o + (long)x * ldo) : 0.0;
#pragma unroll
            for (int x = 0; x < 32; x++)
              if (x < nval) __stcg(o + (long)x * ldo, c[x] + (double)__uint_as_float(r[x]));
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&sh->tempty[acc]);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

emu_status make_map_bf16(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                         uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    ctx->last_error = "cuTensorMapEncodeTiled unavailable";
    return EMU_ECUDA;
  }
  if (((uintptr_t)base & 15u) != 0 || (inner * 2) % 16 != 0 || inner % BK != 0) {
    ctx->last_error = "TMA operand base/stride not 16-byte aligned";
    return EMU_EINVAL;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    ctx->last_error = "cuTensorMapEncodeTiled failed";
    return EMU_ECUDA;
  }
  return EMU_OK;
}

emu_status make_map_bf16_sw128(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                               uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    ctx->last_error = "cuTensorMapEncodeTiled unavailable";
    return EMU_ECUDA;
  }
  if (((uintptr_t)base & 15u) != 0 || inner % 64 != 0) {
    ctx->last_error = "TMA operand base/stride not 16-byte aligned";
    return EMU_EINVAL;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {64u, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    ctx->last_error = "cuTensorMapEncodeTiled failed";
    return EMU_ECUDA;
  }
  return EMU_OK;
}

emu_status make_map_e4m3(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                         uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    ctx->last_error = "cuTensorMapEncodeTiled unavailable";
    return EMU_ECUDA;
  }
  if (((uintptr_t)base & 15u) != 0 || inner % 16 != 0 || inner % BK != 0) {
    ctx->last_error = "TMA operand base/stride not 16-byte aligned";
    return EMU_EINVAL;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    ctx->last_error = "cuTensorMapEncodeTiled failed";
    return EMU_ECUDA;
  }
  return EMU_OK;
}

emu_status make_map_f32(emu_ctx *ctx, CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows,
                        uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    ctx->last_error = "cuTensorMapEncodeTiled unavailable";
    return EMU_ECUDA;
  }
  if (((uintptr_t)base & 15u) != 0 || (inner * 4) % 16 != 0 || inner % BK != 0) {
    ctx->last_error = "TMA operand base/stride not 16-byte aligned";
    return EMU_EINVAL;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 4};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    ctx->last_error = "cuTensorMapEncodeTiled failed";
    return EMU_ECUDA;
  }
  return EMU_OK;
}

emu_status launch(emu_ctx *ctx, const Operands &ops, const Item *d_items, int nitems, const Seg *d_segs,
                  int ksteps, int mode, float *out32, double *out64, int ldo, int max_ctas) {
  if (nitems <= 0) return EMU_OK;
  static std::atomic<uint64_t> attr_done{0};
  EMU_CUDA_TRY(ctx, smem_limit_once(attr_done, ctx->device, (const void *)k_tc_gemm, SMEM_BYTES));
  int grid = nitems < max_ctas ? nitems : max_ctas;
  const Outputs none{nullptr, nullptr, nullptr};
  k_tc_gemm<<<grid, NTHREADS, SMEM_BYTES, ctx->stream>>>(ops, d_items, nitems, d_segs, ksteps, mode, out32,
                                                         out64, none, ldo, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_class(emu_ctx *ctx, const Operands &ops, const Item *d_items, int nitems, const Seg *d_segs,
                        int ksteps, const Outputs &outs, int ldo, int max_ctas) {
  if (nitems <= 0) return EMU_OK;
  static std::atomic<uint64_t> attr_done{0};
  EMU_CUDA_TRY(ctx, smem_limit_once(attr_done, ctx->device, (const void *)k_tc_gemm, SMEM_BYTES));
  int grid = nitems < max_ctas ? nitems : max_ctas;
  k_tc_gemm<<<grid, NTHREADS, SMEM_BYTES, ctx->stream>>>(ops, d_items, nitems, d_segs, ksteps, TC_SUB_CLASS,
                                                         nullptr, nullptr, outs, ldo, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

}  // namespace gemm_tc
