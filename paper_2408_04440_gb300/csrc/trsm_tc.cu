// trsm_tc.cu -- FP32-class panel TRSM on the tensor cores (see trsm_tc.h).
//
// One CTA per (128-row block, listed tile), 192 threads, persistent over the
// tile's 64-column blocks J = 0 .. nb/64 - 1:
//   warp 0      TMA producer (one lane): the three BF16 pieces of L_{n,J}
//               (rows of column block n > J, columns of block J, 64 x 64)
//               through a STAGES-deep ring.
//   warp 1      TMEM allocator + MMA issuer (one lane): for each n > J the
//               six products of X_J pieces (A, 128 x 64) and -L_{n,J} pieces
//               (B, 64 x 64) accumulate into the TMEM columns of block n.
//   warps 2..5  the leaf, one thread per row (TMEM lane): TMEM <- A_ik's
//               columns 64.., then per J the block's current values (from
//               TMEM once an update has reached them), forward substitution
//               against L_JJ in FP32, X_J to the FP32 master, and X_J's
//               pieces into shared memory: the MMAs' A operand, and the source
//               of three TMA tile stores into the piece arena.
// The MMAs of block n = J + 1 are issued first and committed on their own,
// so the leaf of J + 1 starts while those of the later blocks run; the X_J
// operand is double-buffered.  Every wait is bounded (DEV_TIMEOUT).
#include <cuda_bf16.h>

#include "gemm_tc.h"
#include "tc.cuh"
#include "trsm_tc.h"

namespace trsm_tc {
namespace {

constexpr int NPIECE = 3;
constexpr int A_PIECE = RB * W * 2;         // 16 KB: one piece of -X_J, 128 rows of 128 bytes
constexpr int A_BYTES = NPIECE * A_PIECE;   // 48 KB
constexpr int B_PIECE = W * W * 2;          // 8 KB
constexpr int B_STAGE = NPIECE * B_PIECE;   // 24 KB
constexpr int STAGES = 3;
constexpr int OFF_A = 0;                            // two -X_J buffers
constexpr int OFF_B = 2 * A_BYTES;                  // ring of L pieces
constexpr int OFF_L = OFF_B + STAGES * B_STAGE;     // two L_JJ buffers, FP32 column-major
constexpr int OFF_R = OFF_L + 2 * W * W * 4;        // two rows of 1 / L_JJ(c, c)
constexpr int OFF_BAR = OFF_R + 2 * W * 4;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = OFF_BAR + BAR_BYTES + 1024;  // + alignment slack
constexpr int NTHREADS = 192;
constexpr int LEAF0 = 64;                           // first leaf thread
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t IDESC = tc::idesc_f32acc(1u /*BF16*/, RB, W);
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");

struct Shared {
  uint64_t bfull[STAGES], bempty[STAGES];
  uint64_t afull[2], aempty[2];
  uint64_t colready;  // the MMAs of block J + 1 by X_J are complete
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(Shared) <= BAR_BYTES, "barrier block");

__device__ inline bool failed(const int *st) { return *((volatile const int *)st) != DEV_OK; }

__device__ inline void raise_timeout(Shared *sh, int *status) {
  sh->abort = 1;
  if (atomicCAS(&status[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) status[ST_AUX] = 6;
}

// x = p0 + p1 + p2 (each BF16, round to nearest): the operand split of the
// FP32 class.
template <typename T>
__device__ inline void split3(T x, uint16_t &p0, uint16_t &p1, uint16_t &p2) {
  const __nv_bfloat16 b0 = __float2bfloat16_rn((float)x);
  const T r1 = x - (T)__bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn((float)r1);
  const T r2 = r1 - (T)__bfloat162float(b1);
  const __nv_bfloat16 b2 = __float2bfloat16_rn((float)r2);
  p0 = __bfloat16_as_ushort(b0);
  p1 = __bfloat16_as_ushort(b1);
  p2 = __bfloat16_as_ushort(b2);
}

// The three pieces of x0 and x1, packed two per word (x0 in the low half):
// the same values as split3 on each, with paired conversions.
__device__ inline void split3_pair(float x0, float x1, uint32_t &w0, uint32_t &w1, uint32_t &w2) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float r0 = x0 - __low2float(h), r1 = x1 - __high2float(h);
  const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
  const float s0 = r0 - __low2float(m), s1 = r1 - __high2float(m);
  const __nv_bfloat162 l = __floats2bfloat162_rn(s0, s1);
  w0 = *reinterpret_cast<const uint32_t *>(&h);
  w1 = *reinterpret_cast<const uint32_t *>(&m);
  w2 = *reinterpret_cast<const uint32_t *>(&l);
}

// Two floats in one 64-bit register pair (lo in the low half), and the
// packed FP32 FMA of sm_100 (two lanes per instruction, each rounded as fmaf).
__device__ __forceinline__ unsigned long long pk(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float pk_lo(unsigned long long p) { return __uint_as_float((unsigned)p); }
__device__ __forceinline__ float pk_hi(unsigned long long p) { return __uint_as_float((unsigned)(p >> 32)); }
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// All 128 leaf threads: barrier 1, and whether every one of them is still ok.
__device__ inline bool leaf_all(bool ok) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.and.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((unsigned)ok)
      : "memory");
  return r != 0;
}
__device__ inline void leaf_sync() { asm volatile("barrier.cta.sync 1, 128;" ::: "memory"); }

__device__ inline void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// blockIdx.z = list entry z: diagonal tile tiles[z] (or tile0) of the FP64
// arena t64; outputs at slot z of L32 (nb^2 floats) and pieces (3 nb^2), both
// of -L: the MMAs and the leaf subtract X L^T by accumulating.
__global__ void k_lkk_prep(const double *__restrict__ t64, const long *__restrict__ tiles, long tile0,
                           float *__restrict__ L32, uint16_t *__restrict__ pieces, int nb, const int *st) {
  if (failed(st)) return;
  __shared__ double blk[32][33];
  const size_t plane = (size_t)nb * nb;
  const int z = blockIdx.z;
  const double *L = t64 + (size_t)(tiles ? tiles[z] : tile0) * plane;
  float *L32z = L32 + (size_t)z * plane;
  uint16_t *Pz = pieces + (size_t)z * 3 * plane;
  const int rb = blockIdx.x, cb = blockIdx.y;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int c = ty; c < 32; c += 8) {
    const size_t o = (size_t)(rb * 32 + tx) + (size_t)(cb * 32 + c) * nb;
    const double x = L[o];
    L32z[o] = (float)-x;
    blk[tx][c] = x;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int row = rb * 32 + r, col = cb * 32 + tx;
    uint16_t p0, p1, p2;
    split3(col > row ? 0.0 : -blk[r][tx], p0, p1, p2);  // pieces of -L
    const size_t o = (size_t)row * nb + col;
    Pz[o] = p0;
    Pz[plane + o] = p1;
    Pz[2 * plane + o] = p2;
  }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_trsm32_tc(const __grid_constant__ CUtensorMap lmap, const __grid_constant__ CUtensorMap opmap,
                const float *__restrict__ lkk0, float *__restrict__ t32, int nb, int NT, int k,
                const int *__restrict__ rows,
                const int2 *__restrict__ jobs, int *status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = tc::smem_u32(smem_raw);
  const uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
  uint8_t *base = smem_raw + pad;
  const uint32_t base_addr = raw_addr + pad;
  float *LJJ = reinterpret_cast<float *>(base + OFF_L);
  float *rinv = reinterpret_cast<float *>(base + OFF_R);
  Shared *sh = reinterpret_cast<Shared *>(base + OFF_BAR);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NJ = nb / W;
  long ti;
  int lslot;
  if (jobs) {
    const int2 jb = jobs[blockIdx.y];
    ti = jb.x;
    lslot = jb.y;
  } else {
    ti = tile_index(rows[blockIdx.y], k, NT);
    lslot = k & 1;
  }
  const float *Lkk = lkk0 + (size_t)lslot * nb * nb;
  const int lrow0 = lslot * NPIECE * nb;  // tensor-map row of piece 0 of this L_kk
  const int r0 = blockIdx.x * RB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      tc::mbar_init(&sh->bfull[s], 1);
      tc::mbar_init(&sh->bempty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&sh->afull[b], RB);
      tc::mbar_init(&sh->aempty[b], 1);
    }
    tc::mbar_init(&sh->colready, 1);
    tc::mbar_init(&sh->done, 1);
    sh->abort = failed(status) ? 1 : 0;
    tc::fence_barrier_init();
    tc::tma_prefetch_desc(&lmap);
    tc::tma_prefetch_desc(&opmap);
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
      for (int J = 0; J + 1 < NJ && ok; J++) {
        for (int n = J + 1; n < NJ; n++) {
          if (!tc::mbar_wait(&sh->bempty[stage], phase ^ 1u, abort)) {
            raise_timeout(sh, status);
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&sh->bfull[stage], (uint32_t)B_STAGE);
          uint8_t *dst = base + OFF_B + stage * B_STAGE;
          for (int p = 0; p < NPIECE; p++)
            tc::tma_load_2d(dst + p * B_PIECE, &lmap, &sh->bfull[stage], J * W, lrow0 + p * nb + n * W);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // every stage's last load has landed before the CTA exits
      for (int s = 0; s < STAGES; s++) {
        const uint32_t par = (s < stage) ? phase : (phase ^ 1u);
        tc::mbar_wait_inflight(&sh->bfull[s], par);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = *abort == 0;
      // products (pa, pb) of the pieces, smallest magnitude first
      const int pa[6] = {1, 0, 2, 0, 1, 0};
      const int pb[6] = {1, 2, 0, 1, 0, 0};
      for (int J = 0; J + 1 < NJ && ok; J++) {
        const int b = J & 1;
        if (!tc::mbar_wait(&sh->afull[b], (uint32_t)((J >> 1) & 1), abort)) {
          raise_timeout(sh, status);
          break;
        }
        tc::fence_after_sync();
        const uint32_t a_addr = base_addr + OFF_A + b * A_BYTES;
        for (int n = J + 1; n < NJ; n++) {
          if (!tc::mbar_wait(&sh->bfull[stage], phase, abort)) {
            raise_timeout(sh, status);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t b_addr = base_addr + OFF_B + stage * B_STAGE;
          const uint32_t d = tmem + (uint32_t)(n * W - W);
          const uint64_t a0 = tc::smem_desc(a_addr, 16, 1024, tc::kSwizzle128B);
          const uint64_t b0 = tc::smem_desc(b_addr, 16, 1024, tc::kSwizzle128B);
#pragma unroll
          for (int ks = 0; ks < W / 16; ks++) {
#pragma unroll
            for (int p = 0; p < 6; p++) {
              const uint64_t ad = tc::desc_add(a0, pa[p] * A_PIECE + ks * 32);
              const uint64_t bd = tc::desc_add(b0, pb[p] * B_PIECE + ks * 32);
              tc::mma_f16(d, ad, bd, IDESC, 1u);
            }
          }
          tc::mma_commit(&sh->bempty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
          if (n == J + 1) tc::mma_commit(&sh->colready);
        }
        if (ok) tc::mma_commit(&sh->aempty[b]);
      }
      tc::mma_commit(&sh->done);
      tc::mbar_wait_inflight(&sh->done, 0);
    }
  } else {
    // ---------------------------------------------------------------- leaf
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    const int lt = threadIdx.x - LEAF0;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    const size_t plane = (size_t)nb * nb;
    float *Ab = t32 + (size_t)ti * plane + r0 + row;  // (row, c) at Ab[c * nb]
    const int oprow0 = (int)(ti * NPIECE * nb) + r0;  // op tensor-map row of piece 0, row r0
    bool ok = *abort == 0;
    // L_JJ of block J into buffer J & 1 (one cp.async group per block; an
    // empty group past the last block keeps the count uniform)
    auto prefetch = [&](int J) {
      if (J < NJ) {
        float *dst = LJJ + (J & 1) * W * W;
        for (int e = lt; e < W * W / 4; e += RB) {
          const int j = e >> 4, i4 = (e & 15) * 4;  // column j, rows i4 .. i4+3
          cp_async16(dst + j * W + i4, Lkk + (size_t)(J * W + j) * nb + J * W + i4);
        }
      }
      cp_async_commit();
    };
    prefetch(0);
    if (ok) {
      // the trailing columns 64 .. nb-1 of the row block into TMEM, four
      // 32-column chunks of loads in flight at a time
      for (int c0 = W; c0 < nb; c0 += 128) {
        uint32_t v[4][32];
#pragma unroll
        for (int h = 0; h < 4; h++)
          if (c0 + 32 * h < nb) {
#pragma unroll
            for (int x = 0; x < 32; x++) v[h][x] = __float_as_uint(__ldcg(Ab + (size_t)(c0 + 32 * h + x) * nb));
          }
#pragma unroll
        for (int h = 0; h < 4; h++)
          if (c0 + 32 * h < nb) tc::tmem_st_32x32b_x32(tl + (uint32_t)(c0 + 32 * h - W), v[h]);
      }
      tc::tmem_st_wait();
    }
    for (int J = 0; J < NJ; J++) {
      // the piece stores of block J - 2 have read their buffer
      if (lt == 0) tc::bulk_wait_read<1>();
      // every leaf thread is past block J - 1 (its L_JJ buffer may be
      // refilled) and ok
      ok = leaf_all(ok && *abort == 0);
      if (!ok) break;
      prefetch(J + 1);
      cp_async_wait1();  // this thread's copies of block J have landed
      leaf_sync();       // everyone's
      const float *LJ = LJJ + (J & 1) * W * W;
      float *rinvJ = rinv + (J & 1) * W;
      if (lt < W) rinvJ[lt] = -1.0f / LJ[lt * W + lt];  // LJ holds -L_JJ
      leaf_sync();
      unsigned long long vp[W / 2];  // the row's block J, two columns per register pair
      if (J == 0) {
#pragma unroll
        for (int j = 0; j < W / 2; j++) vp[j] = pk(__ldcg(Ab + (size_t)(2 * j) * nb), __ldcg(Ab + (size_t)(2 * j + 1) * nb));
      } else {
        // every wait's outcome is agreed by all leaf threads at once, so that
        // they all take the same path through barrier 1
        const bool got = tc::mbar_wait(&sh->colready, (uint32_t)((J - 1) & 1), abort);
        if (!got) raise_timeout(sh, status);
        if (!leaf_all(got)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tl + (uint32_t)(J * W - W), r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; j++) vp[j] = pk(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
        tc::tmem_ld_32x32b_x32(tl + (uint32_t)(J * W - W + 32), r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; j++) vp[16 + j] = pk(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
      }
      // forward substitution: x_c = (v_c - sum_{c' < c} x_c' L(c, c')) / L(c, c),
      // the updates of later columns by x_c two at a time (LJ = -L_JJ,
      // column-major, read in 16-byte loads)
#pragma unroll
      for (int c = 0; c < W; c++) {
        const int j0 = c >> 1;
        const float *Lc = LJ + c * W;
        float x;
        if (c & 1) {
          x = pk_hi(vp[j0]) * rinvJ[c];
          vp[j0] = pk(pk_lo(vp[j0]), x);
        } else {
          x = pk_lo(vp[j0]) * rinvJ[c];
          vp[j0] = pk(x, fmaf(x, Lc[c + 1], pk_hi(vp[j0])));  // the partner column c + 1
        }
        const unsigned long long xx = pk(x, x);
        const float4 *Lc4 = reinterpret_cast<const float4 *>(Lc);
#pragma unroll
        for (int g = (j0 + 1) / 2; g < W / 4; g++) {
          const float4 l = Lc4[g];
          if (2 * g >= j0 + 1) vp[2 * g] = ffma2(xx, pk(l.x, l.y), vp[2 * g]);
          if (2 * g + 1 >= j0 + 1) vp[2 * g + 1] = ffma2(xx, pk(l.z, l.w), vp[2 * g + 1]);
        }
      }
      float v[W];
#pragma unroll
      for (int j = 0; j < W / 2; j++) {
        v[2 * j] = pk_lo(vp[j]);
        v[2 * j + 1] = pk_hi(vp[j]);
      }
#pragma unroll
      for (int c = 0; c < W; c++) Ab[(size_t)(J * W + c) * nb] = v[c];
      const bool feed = J + 1 < NJ;  // the last block updates nothing
      // the MMAs of block J - 2 have read this buffer (outcome agreed as above)
      const bool got = tc::mbar_wait(&sh->aempty[J & 1], (uint32_t)(((J >> 1) & 1) ^ 1), abort);
      if (!got) raise_timeout(sh, status);
      if (!leaf_all(got)) {
        ok = false;
        break;
      }
      // X_J's pieces, K-major with the 128-byte swizzle (16-byte chunk ch of
      // row `row` at chunk position ch ^ (row & 7)): the A operand of the
      // MMAs and the source of the tile stores into the piece arena
      uint8_t *As = base + OFF_A + (J & 1) * A_BYTES;
#pragma unroll
      for (int ch = 0; ch < W / 8; ch++) {
        uint32_t w[NPIECE][4];
#pragma unroll
        for (int e = 0; e < 4; e++) split3_pair(v[ch * 8 + 2 * e], v[ch * 8 + 2 * e + 1], w[0][e], w[1][e], w[2][e]);
        const uint32_t off = (uint32_t)row * 128u + (uint32_t)((ch ^ (row & 7)) << 4);
#pragma unroll
        for (int p = 0; p < NPIECE; p++)
          *reinterpret_cast<uint4 *>(As + p * A_PIECE + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      }
      tc::fence_proxy_async_smem();
      if (feed) {
        tc::fence_before_sync();
        tc::mbar_arrive(&sh->afull[J & 1]);
      }
      leaf_sync();  // every row's pieces are in the buffer
      if (lt == 0) {
        for (int p = 0; p < NPIECE; p++) tc::tma_store_2d(&opmap, As + p * A_PIECE, J * W, oprow0 + p * nb);
        tc::bulk_commit();
      }
    }
    if (lt == 0) tc::bulk_wait_all();
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy into shared memory outlives the loop
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace

emu_status launch_prep(emu_ctx *ctx, const double *t64, long tile, const long *d_tiles, int n, float *L32,
                       uint16_t *pieces, int nb) {
  if (n <= 0) return EMU_OK;
  if (nb % 32 != 0) return EMU_EINVAL;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 18.0 * n * (double)nb * nb);
  k_lkk_prep<<<dim3(nb / 32, nb / 32, n), 256, 0, ctx->stream>>>(t64, d_tiles, tile, L32, pieces, nb, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status make_map(emu_ctx *ctx, CUtensorMap *map, const uint16_t *pieces, int nb, int nslots) {
  return gemm_tc::make_map_bf16_sw128(ctx, map, pieces, (uint64_t)nb, (uint64_t)nslots * NPIECE * nb, (uint32_t)W);
}

emu_status make_op_map(emu_ctx *ctx, CUtensorMap *map, const uint16_t *op, int nb, long ntiles) {
  if ((uint64_t)ntiles * NPIECE * nb >= (1ull << 31)) {
    ctx->last_error = "piece arena too large for 32-bit TMA coordinates";
    return EMU_EINVAL;
  }
  return gemm_tc::make_map_bf16_sw128(ctx, map, op, (uint64_t)nb, (uint64_t)ntiles * NPIECE * nb, (uint32_t)RB);
}

emu_status launch(emu_ctx *ctx, const CUtensorMap &lmap, const CUtensorMap &opmap, const float *lkk0, float *t32,
                  int nb, int NT, int k, const int *d_rows, const int2 *d_jobs, int n) {
  if (n <= 0) return EMU_OK;
  if (!supports(nb)) return EMU_EINVAL;
  static std::atomic<uint64_t> attr_done{0};
  EMU_CUDA_TRY(ctx, smem_limit_once(attr_done, ctx->device, (const void *)k_trsm32_tc, SMEM_BYTES));
  const double nb3 = (double)nb * nb * nb;
  ProfScope ps(ctx, PROF_TRSM32, n * nb3, 14.0 * n * (double)nb * nb, 6.0 * n * (nb3 - (double)nb * nb * W));
  k_trsm32_tc<<<dim3(nb / RB, n), NTHREADS, SMEM_BYTES, ctx->stream>>>(lmap, opmap, lkk0, t32, nb, NT, k, d_rows,
                                                                       d_jobs, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

}  // namespace trsm_tc
