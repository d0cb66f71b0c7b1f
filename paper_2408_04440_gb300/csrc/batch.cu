// batch.cu -- many independent covariances of uneven bandlimit, built,
// factored by the adaptive per-tile precision Cholesky and sampled in one
// call (emu_batch_potrf_sample in include/emucov.h).
//
// The paper factors one large covariance; the batched workload factors many
// small ones (n = 64 .. 4096).  Launching the single-matrix path per matrix
// would leave the GPU idle between tiny launches, so here every step k of the
// tile algorithm runs ONCE for all matrices that still have a step k:
//   POTRF(k, k) of every such matrix in one dataflow launch, the panel TRSMs
//   of all of them in one launch per kind, their FP64 updates in one launch
//   and their tensor-core updates as one item list of one persistent GEMM.
// All matrices share one tile arena (each at its tile_base), one stack of
// samples (each at its row_base) and the same kernels as the single-matrix
// path, addressed through explicit tile indices.  The launches after the
// precision map are captured in one CUDA graph, which the context keeps and
// replays when the same batch comes again.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "emu_internal.h"
#include "gemm_f64.h"
#include "gemm_tc.h"
#include "trsm_tc.h"

namespace {

__device__ inline bool failed_b(const int *st) { return *((volatile const int *)st) != DEV_OK; }

// Zero the strict upper triangle of the listed diagonal tiles.
__global__ void k_tril_list(double *__restrict__ t64, const long *__restrict__ tiles, int nb, const int *st) {
  if (failed_b(st)) return;
  double *D = t64 + (size_t)tiles[blockIdx.y] * nb * nb;
  int c = blockIdx.x;
  for (int r = threadIdx.x; r < c; r += blockDim.x) D[r + (size_t)c * nb] = 0.0;
}

// Y_b (n_b x s, leading dimension n_b) from matrix b's rows of the stacked Y.
__global__ void k_gather_rows(const double *__restrict__ Y, long ldy, const BatchInst *__restrict__ inst, int s,
                              double *const *__restrict__ out) {
  BatchInst I = inst[blockIdx.y];
  double *o = out[blockIdx.y];
  long total = (long)I.n * s;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    long r = q % I.n, c = q / I.n;
    o[r + c * I.n] = Y[I.row_base + r + c * ldy];
  }
}

// Work of step k for all matrices: offsets and counts into the plan's lists.
struct Step {
  int d_off = 0, d_n = 0;      // diagonal tiles (k, k): POTRF (slot = position in this list)
  int dl_off = 0, dl_n = 0;    // those of a low class: FP32 master -> FP64 first
  int t64_off = 0, t64_n = 0;  // FP64 TRSM jobs {tile (i,k), tile (k,k)}
  int s64_off = 0, s64_n = 0;  // their tiles, split into BF16 pieces afterwards
  int t32_off = 0, t32_n = 0;  // FP32 TRSM jobs {tile (i,k), slot of L_kk}
  int q_off = 0, q_n = 0;      // panel tiles quantized to E4M3
  int u_off = 0, u_n = 0;      // FP64-class updates: tensor-core digit-product items
  int z_off = 0, z_n = 0;      // panel tiles digit-sliced for them {tile, slot}
  double u_flops = 0.0;
  int it_off = 0, it_n = 0;    // tensor-core items
  double tc_flops = 0.0, tc_mma = 0.0;
};

template <typename T>
T *dalloc(size_t n, emu_status *s) {
  if (n == 0) n = 1;
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *s = (e == cudaErrorMemoryAllocation) ? EMU_ENOMEM : EMU_ECUDA;
    return nullptr;
  }
  return static_cast<T *>(p);
}

// Everything one batch needs, kept in the context between calls.
struct BatchState {
  // what the state was built for
  std::vector<emu_cov_params> params;
  int nb = 0, s = 0;
  bool want_L = false;
  double eps = 0.0, u[EMU_NCLASS] = {};
  unsigned mask = 0;
  int diag_fp64 = 0;
  int band = EMU_MAP_NORM;
  double sp_frac = 0.0;
  // layout
  int count = 0, maxNT = 0, maxL = 0, s_pad = 0;
  long ntiles = 0, nrows = 0, ntab = 0;
  std::vector<BatchInst> inst;
  std::vector<unsigned char> cls;
  std::vector<Step> steps;
  std::vector<long> diag_lists;  // per step (see Step::d_off)
  bool any_low = false, any_e4m3 = false;
  int ntasks = 0, max_active = 0;
  int graph_launches = 0;
  long n_items_sample = 0;
  double sample_flops = 0.0, sample_mma = 0.0;
  std::vector<std::vector<double>> upd_flops;  // per matrix, per class
  // device arenas
  double *t64 = nullptr, *partial = nullptr, *tnorm = nullptr, *frob = nullptr, *tables = nullptr;
  float *t32 = nullptr, *slots = nullptr, *scale8 = nullptr;
  uint16_t *op = nullptr, *zp = nullptr;
  uint16_t *lpieces = nullptr;  // BF16 pieces of the step's L_kk, per slot (tensor-core TRSM)
  CUtensorMap lmap, opmap;
  bool tc_trsm = false;
  uint8_t *op8 = nullptr;
  unsigned char *d_cls = nullptr;
  BatchInst *d_inst = nullptr;
  int *d_tile_inst = nullptr;
  double *Z = nullptr, *Y = nullptr;
  int *ws = nullptr;
  double *rinv = nullptr;
  void *tasks = nullptr;
  double **d_Yptr = nullptr, **d_Lptr = nullptr;
  uint64_t *d_seed = nullptr;
  // device lists
  long *d_diag = nullptr, *d_all_diag = nullptr;
  int *d_bad = nullptr;  // per (step, diagonal slot): first non-positive pivot column, 0 = none
  int *d_all_diag_int = nullptr;
  int2 *d_t64 = nullptr, *d_t32 = nullptr;
  int *d_t64slot = nullptr;  // per FP64 TRSM job: the step slot of its L_kk (pre-scaled blocks)
  double *ls64 = nullptr, *rinv64 = nullptr;  // pre-scaled diagonal blocks of the step's L_kk, per slot
  int *d_s64 = nullptr, *d_q = nullptr;
  int4 *d_pairs = nullptr;
  gemm64::Item *d_items64 = nullptr, *d_items64s = nullptr;
  gemm64::Seg *d_segs64 = nullptr, *d_segs64s = nullptr;
  int4 *d_z = nullptr, *d_zs = nullptr;  // slice jobs: factor panel tiles / the sampler's FP64 tiles
  int2 *d_zblk = nullptr;                 // per matrix: {first row, rows} of Z
  int nslots = 0, nslots_s = 0, nzs = 0;
  long n_items64s = 0;
  double samp64_flops = 0.0;
  uint16_t *digits = nullptr;  // factor digits, then (after the factor) the sampler's L and Z digits
  int *exp64 = nullptr, *exp_s = nullptr, *exp_z = nullptr;
  size_t dig_s_off = 0;        // where the sampler's Z digits start in `digits` (elements)
  CUtensorMap map64a, map64b, map_sa, map_sz;
  gemm_tc::Item *d_items = nullptr, *d_items_s = nullptr;
  gemm_tc::Seg *d_segs = nullptr, *d_segs_s = nullptr;
  long n_all_diag = 0, n_pairs = 0;
  gemm_tc::Operands ops_f, ops_s;
  cudaGraphExec_t graph = nullptr;

  void release() {
    void *ps[] = {t64, partial, tnorm, frob, tables, t32, slots, scale8, op, zp, op8, d_cls, d_inst, d_tile_inst,
                  Z, Y, ws, rinv, tasks, d_Yptr, d_Lptr, d_seed, d_diag, d_bad, d_all_diag, d_all_diag_int, d_t64,
                  d_t64slot, ls64, rinv64,
                  d_t32, d_s64, d_q, d_pairs, d_items, d_items_s, d_segs, d_segs_s, d_items64,
                  d_items64s, d_segs64, d_segs64s, d_z, d_zs, d_zblk, digits, exp64, exp_s, exp_z, lpieces};
    for (void *p : ps)
      if (p) cudaFree(p);
    if (graph) cudaGraphExecDestroy(graph);
  }
};

bool same_params(const emu_cov_params &a, const emu_cov_params &b) {
  return a.L == b.L && a.beta == b.beta && a.sigma_exp == b.sigma_exp && a.nugget_rel == b.nugget_rel;
}

}  // namespace

namespace {

// Instances, tile/row/table offsets and the arenas of the build and the map.
emu_status batch_layout(emu_ctx *ctx, BatchState *B, int count, const emu_cov_params *p, int nb) {
  B->count = count;
  B->nb = nb;
  B->params.assign(p, p + count);
  B->inst.resize(count);
  long tiles = 0, rows = 0, tab = 0;
  int maxNT = 0, maxL = 0;
  for (int b = 0; b < count; b++) {
    BatchInst &I = B->inst[b];
    I.L = p[b].L;
    I.n = p[b].L * p[b].L;
    I.NT = (I.n + nb - 1) / nb;
    I.stream_id = b;
    I.beta = p[b].beta;
    I.sigma_exp = p[b].sigma_exp;
    I.nugget_rel = p[b].nugget_rel;
    I.tile_base = tiles;
    I.row_base = rows;
    I.tab_base = tab;
    tiles += (long)I.NT * (I.NT + 1) / 2;
    rows += (long)I.NT * nb;
    tab += (long)(2 * I.L - 1) * (4 * I.L - 3) + I.L + 1;
    maxNT = std::max(maxNT, I.NT);
    maxL = std::max(maxL, I.L);
  }
  B->ntiles = tiles;
  B->nrows = rows;
  B->ntab = tab;
  B->maxNT = maxNT;
  B->maxL = maxL;
  if (tiles * 3L * nb >= (1L << 31) || rows >= (1L << 31)) {
    ctx->last_error = "batch too large for 32-bit TMA coordinates";
    return EMU_EINVAL;
  }
  size_t te = (size_t)nb * nb;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  // FP64 + FP32 + three BF16 pieces per element, with some headroom
  if ((double)tiles * te * 18.0 > 0.9 * (double)free_b) {
    ctx->last_error = "batch arenas do not fit in free device memory";
    return EMU_ENOMEM;
  }
  std::vector<int> tile_inst(tiles);
  for (int b = 0; b < count; b++) {
    const BatchInst &I = B->inst[b];
    for (long t = 0; t < (long)I.NT * (I.NT + 1) / 2; t++) tile_inst[I.tile_base + t] = b;
  }
  emu_status s = EMU_OK;
  B->t64 = dalloc<double>(tiles * te, &s);
  B->partial = dalloc<double>(tiles * (nb / 32), &s);
  B->tnorm = dalloc<double>(tiles, &s);
  B->frob = dalloc<double>(count, &s);
  B->tables = dalloc<double>(tab, &s);
  B->d_cls = dalloc<unsigned char>(tiles, &s);
  B->d_inst = dalloc<BatchInst>(count, &s);
  B->d_tile_inst = dalloc<int>(tiles, &s);
  if (s != EMU_OK) {
    ctx->last_error = "batch arena allocation failed";
    return s;
  }
  EMU_CUDA_TRY(ctx, cudaMemcpy(B->d_inst, B->inst.data(), count * sizeof(BatchInst), cudaMemcpyHostToDevice));
  EMU_CUDA_TRY(ctx, cudaMemcpy(B->d_tile_inst, tile_inst.data(), tiles * sizeof(int), cudaMemcpyHostToDevice));
  return EMU_OK;
}

template <typename T>
emu_status upload(emu_ctx *ctx, T **dst, const std::vector<T> &v) {
  emu_status s = EMU_OK;
  *dst = dalloc<T>(v.size(), &s);
  if (s != EMU_OK) return s;
  if (!v.empty()) EMU_CUDA_TRY(ctx, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return EMU_OK;
}

// Step lists, item lists and the remaining arenas, from the class map.
emu_status batch_plan(emu_ctx *ctx, BatchState *B) {
  const int nb = B->nb, count = B->count;
  const size_t te = (size_t)nb * nb;
  const double nb3 = (double)nb * nb * nb;
  auto C = [&](long g) { return (int)B->cls[g]; };
  std::vector<long> longs;
  std::vector<int2> j64, j32;
  std::vector<int> j64slot;
  std::vector<int> s64, q;
  std::vector<gemm64::Item> items64;
  std::vector<gemm64::Seg> segs64;
  std::vector<int4> zjobs;
  std::vector<int> slot_of_tile(B->ntiles, -1);
  std::vector<gemm_tc::Item> items;
  std::vector<gemm_tc::Seg> segs;
  B->steps.assign(B->maxNT, Step());
  B->any_low = B->any_e4m3 = false;
  B->max_active = 0;
  B->upd_flops.assign(count, std::vector<double>(EMU_NCLASS, 0.0));
  for (int b = 0; b < count; b++) {
    const BatchInst &I = B->inst[b];
    for (int j = 0; j < I.NT; j++)
      for (int i = j; i < I.NT; i++) {
        int c = C(I.tile_base + tile_index(i, j, I.NT));
        if (c != EMU_CLASS_FP64) B->any_low = true;
        B->upd_flops[b][c] += (i == j ? 1.0 : 2.0) * j * nb3 + (i > j ? nb3 : 0.0);
      }
  }
  for (int k = 0; k < B->maxNT; k++) {
    Step &st = B->steps[k];
    std::vector<int> slot(count, -1);
    st.d_off = (int)longs.size();
    for (int b = 0; b < count; b++)
      if (B->inst[b].NT > k) {
        slot[b] = st.d_n++;
        longs.push_back(B->inst[b].tile_base + tile_index(k, k, B->inst[b].NT));
      }
    B->max_active = std::max(B->max_active, st.d_n);
    st.dl_off = (int)longs.size();
    for (int b = 0; b < count; b++)
      if (B->inst[b].NT > k) {
        long g = B->inst[b].tile_base + tile_index(k, k, B->inst[b].NT);
        if (C(g) != EMU_CLASS_FP64) {
          longs.push_back(g);
          st.dl_n++;
        }
      }
    st.t64_off = (int)j64.size();
    st.s64_off = (int)s64.size();
    st.t32_off = (int)j32.size();
    st.q_off = (int)q.size();
    st.u_off = (int)items64.size();
    st.z_off = (int)zjobs.size();
    st.it_off = (int)items.size();
    for (int b = 0; b < count; b++) {
      const BatchInst &I = B->inst[b];
      if (I.NT <= k + 1) continue;
      long gkk = I.tile_base + tile_index(k, k, I.NT);
      for (int i = k + 1; i < I.NT; i++) {
        long gik = I.tile_base + tile_index(i, k, I.NT);
        if (C(gik) == EMU_CLASS_FP64) {
          j64.push_back(make_int2((int)gik, (int)gkk));
          j64slot.push_back(slot[b]);
          if (B->any_low) s64.push_back((int)gik);  // BF16 pieces only feed tensor-core updates
        } else {
          j32.push_back(make_int2((int)gik, slot[b]));
        }
      }
      bool inst_f8 = false;
      for (int j = k + 1; j < I.NT; j++)
        for (int i = j; i < I.NT; i++) {
          long gij = I.tile_base + tile_index(i, j, I.NT);
          long gik = I.tile_base + tile_index(i, k, I.NT), gjk = I.tile_base + tile_index(j, k, I.NT);
          int c = C(gij);
          if (c == EMU_CLASS_FP64) {
            // digit products on the tensor cores; panel tiles sliced after this step's TRSMs
            for (long t : {gik, gjk})
              if (slot_of_tile[t] < 0) {
                slot_of_tile[t] = B->nslots++;
                zjobs.push_back(make_int4((int)t, slot_of_tile[t], slot_of_tile[t] * nb, 0));
              }
            int si = slot_of_tile[gik], sj = slot_of_tile[gjk];
            for (int nbk = 0; nbk < nb / gemm64::BN; nbk++)
              for (int mb = 0; mb < nb / gemm64::BM; mb++) {
                if (i == j && mb * gemm64::BM + gemm64::BM - 1 < nbk * gemm64::BN) continue;
                gemm64::Seg sg;
                sg.a_row = si * gemm64::NS * nb + mb * gemm64::BM;
                sg.b_row = sj * gemm64::NS * nb + nbk * gemm64::BN;
                sg.a_x = sg.b_x = 0;
                gemm64::Item it;
                it.out_off = gij * (long)te + mb * gemm64::BM + (long)nbk * gemm64::BN * nb;
                it.a_sc = si * nb + mb * gemm64::BM;
                it.b_sc = sj * nb + nbk * gemm64::BN;
                it.seg_begin = (int)segs64.size();
                segs64.push_back(sg);
                it.seg_end = (int)segs64.size();
                it.rows_valid = gemm64::BM;
                it.cols_valid = gemm64::BN;
                items64.push_back(it);
              }
            st.u_flops += 2.0 * nb3;
            continue;
          }
          int cc = (c == EMU_CLASS_FP32) ? EMU_CLASS_FP32 : (c == EMU_CLASS_E4M3) ? EMU_CLASS_E4M3 : EMU_CLASS_BF16;
          bool f8 = cc == EMU_CLASS_E4M3;
          inst_f8 |= f8;
          for (int nbk = 0; nbk < nb / gemm_tc::BN; nbk++)
            for (int mb = 0; mb < nb / gemm_tc::BM; mb++) {
              if (i == j && mb * gemm_tc::BM + gemm_tc::BM - 1 < nbk * gemm_tc::BN) continue;
              gemm_tc::Seg sg;
              sg.ax = 0;
              sg.ay = (int)(gik * (f8 ? 1 : 3) * nb + mb * gemm_tc::BM);
              sg.ay_step = nb;
              sg.bx = 0;
              sg.by = (int)(gjk * (f8 ? 1 : 3) * nb + nbk * gemm_tc::BN);
              sg.by_step = nb;
              sg.cls = cc;
              sg.pad = 0;
              gemm_tc::Item it;
              it.seg_begin = (int)segs.size();
              segs.push_back(sg);
              it.seg_end = (int)segs.size();
              it.out_off = gij * (long)te + mb * gemm_tc::BM + (long)nbk * gemm_tc::BN * nb;
              it.rows_valid = gemm_tc::BM;
              it.cols_valid = gemm_tc::BN;
              it.sa = f8 ? (int)gik : -1;
              it.sb = f8 ? (int)gjk : -1;
              items.push_back(it);
              double f = 2.0 * gemm_tc::BM * gemm_tc::BN * nb;
              st.tc_flops += f;
              st.tc_mma += f * (cc == EMU_CLASS_FP32 ? 6.0 : f8 ? 0.5 : 1.0);
            }
        }
      if (inst_f8) {
        B->any_e4m3 = true;
        for (int i = k + 1; i < I.NT; i++) q.push_back((int)(I.tile_base + tile_index(i, k, I.NT)));
      }
    }
    st.t64_n = (int)j64.size() - st.t64_off;
    st.s64_n = (int)s64.size() - st.s64_off;
    st.t32_n = (int)j32.size() - st.t32_off;
    st.q_n = (int)q.size() - st.q_off;
    st.u_n = (int)items64.size() - st.u_off;
    st.z_n = (int)zjobs.size() - st.z_off;
    st.it_n = (int)items.size() - st.it_off;
  }
  std::vector<long> all_diag;
  std::vector<int> all_diag_int;
  std::vector<int4> pairs;
  std::vector<gemm64::Item> items64s;
  std::vector<gemm64::Seg> segs64s;
  std::vector<int4> zs;
  std::vector<int2> zblk;
  std::vector<int> slot_s(B->ntiles, -1);
  B->nslots_s = 0;
  B->samp64_flops = 0.0;
  std::vector<gemm_tc::Item> items_s;
  std::vector<gemm_tc::Seg> segs_s;
  B->s_pad = ((B->s + gemm_tc::BN - 1) / gemm_tc::BN) * gemm_tc::BN;
  B->sample_flops = B->sample_mma = 0.0;
  for (int b = 0; b < count; b++) {
    const BatchInst &I = B->inst[b];
    for (int k = 0; k < I.NT; k++) {
      all_diag.push_back(I.tile_base + tile_index(k, k, I.NT));
      all_diag_int.push_back((int)(I.tile_base + tile_index(k, k, I.NT)));
    }
    if (B->want_L)
      for (int tj = 0; tj < I.NT; tj++)
        for (int ti = 0; ti < I.NT; ti++) pairs.push_back(make_int4(b, ti, tj, 0));
    if (B->s <= 0) continue;
    // the sampler's FP64-class tiles: digit slots, one exponent per row of the stacked rows
    zblk.push_back(make_int2((int)I.row_base, I.NT * nb));
    for (int j = 0; j < I.NT; j++)
      for (int i = j; i < I.NT; i++) {
        long t = I.tile_base + tile_index(i, j, I.NT);
        if (C(t) != EMU_CLASS_FP64) continue;
        slot_s[t] = B->nslots_s++;
        zs.push_back(make_int4((int)t, slot_s[t], (int)(I.row_base + (long)i * nb), 0));
      }
    for (int i = 0; i < I.NT; i++) {
      for (int nbk = 0; nbk < B->s_pad / gemm64::BN; nbk++)
        for (int mb = 0; mb < nb / gemm64::BM; mb++) {
          long row0 = (long)i * nb + mb * gemm64::BM;
          int cols = std::min(gemm64::BN, B->s - nbk * gemm64::BN);
          if (row0 >= I.n || cols <= 0) continue;
          gemm64::Item it;
          it.seg_begin = (int)segs64s.size();
          for (int k = 0; k <= i; k++) {
            int sl = slot_s[I.tile_base + tile_index(i, k, I.NT)];
            if (sl < 0) continue;
            gemm64::Seg sg;
            sg.a_row = sl * gemm64::NS * nb + mb * gemm64::BM;
            sg.b_row = nbk * gemm64::BN;
            sg.a_x = 0;
            sg.b_x = (int)(I.row_base + (long)k * nb);
            segs64s.push_back(sg);
            B->samp64_flops += 2.0 * gemm64::BM * gemm64::BN * nb;
          }
          it.seg_end = (int)segs64s.size();
          if (it.seg_end == it.seg_begin) continue;
          it.out_off = I.row_base + row0 + (long)nbk * gemm64::BN * B->nrows;
          it.a_sc = (int)(I.row_base + row0);
          it.b_sc = (int)zblk.size() - 1;  // block index; times s_pad below
          it.b_sc = it.b_sc * B->s_pad + nbk * gemm64::BN;
          it.rows_valid = (int)std::min<long>(gemm64::BM, I.n - row0);
          it.cols_valid = cols;
          items64s.push_back(it);
        }
      for (int nbk = 0; nbk < B->s_pad / gemm_tc::BN; nbk++)
        for (int mb = 0; mb < nb / gemm_tc::BM; mb++) {
          long row0 = (long)i * nb + mb * gemm_tc::BM;
          if (row0 >= I.n) continue;
          gemm_tc::Item it;
          it.seg_begin = (int)segs_s.size();
          for (int k = 0; k <= i; k++) {
            long gik = I.tile_base + tile_index(i, k, I.NT);
            int c = C(gik);
            if (c == EMU_CLASS_FP64) continue;
            gemm_tc::Seg sg;
            sg.ax = 0;
            sg.ay = (int)(gik * 3 * nb + mb * gemm_tc::BM);
            sg.ay_step = nb;
            sg.bx = (int)(I.row_base + (long)k * nb);
            sg.by = nbk * gemm_tc::BN;
            sg.by_step = B->s_pad;
            // E4M3-class tiles are sampled through their leading BF16 piece
            sg.cls = (c == EMU_CLASS_FP32) ? EMU_CLASS_FP32 : EMU_CLASS_BF16;
            sg.pad = 0;
            segs_s.push_back(sg);
            double f = 2.0 * gemm_tc::BM * gemm_tc::BN * nb;
            B->sample_flops += f;
            B->sample_mma += f * (sg.cls == EMU_CLASS_FP32 ? 6.0 : 1.0);
          }
          it.seg_end = (int)segs_s.size();
          if (it.seg_end == it.seg_begin) continue;
          it.out_off = I.row_base + row0 + (long)nbk * gemm_tc::BN * B->nrows;
          it.rows_valid = (int)std::min<long>(gemm_tc::BM, I.n - row0);
          it.cols_valid = B->s - nbk * gemm_tc::BN;
          it.sa = it.sb = -1;
          items_s.push_back(it);
        }
    }
  }
  B->n_all_diag = (long)all_diag.size();
  B->n_pairs = (long)pairs.size();
  B->n_items64s = (long)items64s.size();
  B->nzs = (int)zs.size();
  B->n_items_sample = (long)items_s.size();
  B->diag_lists = longs;
  // device lists
  emu_status s;
  B->d_bad = dalloc<int>(longs.size(), &s);
  if (!B->d_bad) return s;
  if ((s = upload(ctx, &B->d_diag, longs)) != EMU_OK || (s = upload(ctx, &B->d_all_diag, all_diag)) != EMU_OK ||
      (s = upload(ctx, &B->d_all_diag_int, all_diag_int)) != EMU_OK || (s = upload(ctx, &B->d_t64, j64)) != EMU_OK ||
      (s = upload(ctx, &B->d_t64slot, j64slot)) != EMU_OK ||
      (s = upload(ctx, &B->d_t32, j32)) != EMU_OK || (s = upload(ctx, &B->d_s64, s64)) != EMU_OK ||
      (s = upload(ctx, &B->d_q, q)) != EMU_OK || (s = upload(ctx, &B->d_items64, items64)) != EMU_OK ||
      (s = upload(ctx, &B->d_z, zjobs)) != EMU_OK || (s = upload(ctx, &B->d_segs64, segs64)) != EMU_OK ||
      (s = upload(ctx, &B->d_items64s, items64s)) != EMU_OK || (s = upload(ctx, &B->d_segs64s, segs64s)) != EMU_OK ||
      (s = upload(ctx, &B->d_zs, zs)) != EMU_OK || (s = upload(ctx, &B->d_zblk, zblk)) != EMU_OK ||
      (s = upload(ctx, &B->d_pairs, pairs)) != EMU_OK || (s = upload(ctx, &B->d_items, items)) != EMU_OK ||
      (s = upload(ctx, &B->d_segs, segs)) != EMU_OK || (s = upload(ctx, &B->d_items_s, items_s)) != EMU_OK ||
      (s = upload(ctx, &B->d_segs_s, segs_s)) != EMU_OK)
    return s;
  // remaining arenas
  s = EMU_OK;
  B->tc_trsm = trsm_tc::supports(nb);
  if (B->any_low) {
    B->t32 = dalloc<float>(B->ntiles * te, &s);
    B->slots = dalloc<float>((size_t)B->max_active * te, &s);
    if (B->tc_trsm) B->lpieces = dalloc<uint16_t>((size_t)B->max_active * 3 * te, &s);
  }
  B->op = dalloc<uint16_t>(B->ntiles * 3 * te, &s);
  if (B->any_e4m3) {
    B->op8 = dalloc<uint8_t>(B->ntiles * te, &s);
    B->scale8 = dalloc<float>(B->ntiles, &s);
  }
  // one digit arena: the factor's panel digits, reused after the factor for
  // the sampler's FP64 tiles (first) and Z (from dig_s_off)
  size_t need_f = (size_t)B->nslots * gemm64::NS * te;
  size_t need_s = (size_t)B->nslots_s * gemm64::NS * te;
  B->dig_s_off = need_s;
  if (B->nslots_s > 0) need_s += (size_t)gemm64::NS * B->s_pad * B->nrows;
  if (need_f + need_s > 0) B->digits = dalloc<uint16_t>(std::max(need_f, need_s), &s);
  if (B->nslots > 0) B->exp64 = dalloc<int>((size_t)B->nslots * nb, &s);
  if (B->nslots_s > 0) {
    B->exp_s = dalloc<int>(B->nrows, &s);
    B->exp_z = dalloc<int>((size_t)count * B->s_pad, &s);
  }
  if (!j64.empty()) {
    B->ls64 = dalloc<double>((size_t)B->max_active * nb * 32, &s);
    B->rinv64 = dalloc<double>((size_t)B->max_active * nb, &s);
  }
  B->ntasks = (int)potrf_dag_task_count(nb);
  B->tasks = dalloc<short4>(B->ntasks, &s);
  B->ws = dalloc<int>(potrf_batch_ws_ints(nb, B->max_active), &s);
  B->rinv = dalloc<double>((size_t)B->max_active * nb, &s);
  B->d_Yptr = dalloc<double *>(count, &s);
  B->d_Lptr = dalloc<double *>(count, &s);
  B->d_seed = dalloc<uint64_t>(1, &s);
  if (B->s > 0) {
    B->Z = dalloc<double>((size_t)B->nrows * B->s, &s);
    B->Y = dalloc<double>((size_t)B->nrows * B->s, &s);
    B->zp = dalloc<uint16_t>((size_t)3 * B->s_pad * B->nrows, &s);
  }
  if (s != EMU_OK) {
    ctx->last_error = "batch arena allocation failed";
    return s;
  }
  if ((s = potrf_dag_tasks_upload(ctx, nb, B->tasks, ctx->stream)) != EMU_OK) return s;
  // tensor maps: factor operands (BF16 pieces, FP8 copies) and sampler operands
  uint64_t rows16 = (uint64_t)B->ntiles * 3 * nb;
  if ((s = gemm_tc::make_map_bf16(ctx, &B->ops_f.a16, B->op, nb, rows16, gemm_tc::BM)) != EMU_OK) return s;
  if ((s = gemm_tc::make_map_bf16(ctx, &B->ops_f.b16, B->op, nb, rows16, gemm_tc::BN)) != EMU_OK) return s;
  B->ops_f.a8 = B->ops_f.a16;
  B->ops_f.b8 = B->ops_f.b16;
  B->ops_f.scale8 = B->scale8;
  if (B->any_e4m3) {
    uint64_t rows8 = (uint64_t)B->ntiles * nb;
    if ((s = gemm_tc::make_map_e4m3(ctx, &B->ops_f.a8, B->op8, nb, rows8, gemm_tc::BM)) != EMU_OK) return s;
    if ((s = gemm_tc::make_map_e4m3(ctx, &B->ops_f.b8, B->op8, nb, rows8, gemm_tc::BN)) != EMU_OK) return s;
  }
  if (B->nslots > 0) {
    uint64_t drows = (uint64_t)B->nslots * gemm64::NS * nb;
    if (drows >= (1ull << 31)) {
      ctx->last_error = "batch digit arena too large for 32-bit TMA coordinates";
      return EMU_EINVAL;
    }
    if ((s = gemm64::make_map(ctx, &B->map64a, B->digits, nb, drows, gemm64::BM)) != EMU_OK) return s;
    if ((s = gemm64::make_map(ctx, &B->map64b, B->digits, nb, drows, gemm64::BN)) != EMU_OK) return s;
  }
  if (B->nslots_s > 0) {
    uint64_t arows = (uint64_t)B->nslots_s * gemm64::NS * nb;
    if (arows >= (1ull << 31)) {
      ctx->last_error = "batch digit arena too large for 32-bit TMA coordinates";
      return EMU_EINVAL;
    }
    if ((s = gemm64::make_map(ctx, &B->map_sa, B->digits, nb, arows, gemm64::BM)) != EMU_OK) return s;
    if ((s = gemm64::make_map(ctx, &B->map_sz, B->digits + B->dig_s_off, B->nrows, (uint64_t)gemm64::NS * B->s_pad,
                              gemm64::BN)) != EMU_OK)
      return s;
  }
  if (B->any_low && B->tc_trsm &&
      ((s = trsm_tc::make_map(ctx, &B->lmap, B->lpieces, nb, B->max_active)) != EMU_OK ||
       (s = trsm_tc::make_op_map(ctx, &B->opmap, B->op, nb, B->ntiles)) != EMU_OK))
    return s;
  B->ops_s = B->ops_f;
  if (B->s > 0 &&
      (s = gemm_tc::make_map_bf16(ctx, &B->ops_s.b16, B->zp, B->nrows, (uint64_t)3 * B->s_pad, gemm_tc::BN)) !=
          EMU_OK)
    return s;
  return EMU_OK;
}

}  // namespace

namespace {

// A tile size chosen by timing, for one batch signature.
struct TuneRec {
  std::vector<emu_cov_params> params;
  double eps;
  unsigned mask;
  int diag_fp64, s;
  int band;
  double sp_frac;
  bool want_L;
  int nb;
};

// Per-context batch data: the last batch's state, the tuning records and the
// stream the graph is captured on (the legacy default stream cannot be).
struct BatchCtx {
  BatchState *state = nullptr;
  std::vector<TuneRec> tuned;
  cudaStream_t cap = nullptr;
};

// Every launch of the factor, the diagonal fix-up, the samples and the
// export, in order, on ctx->stream (which is being captured).
emu_status batch_record(emu_ctx *ctx, BatchState *B) {
  const int nb = B->nb;
  const size_t te = (size_t)nb * nb;
  emu_status s;
  if (B->any_low && (s = launch_to_f32_tiles(ctx, B->t64, B->t32, B->d_cls, B->ntiles, te)) != EMU_OK) return s;
  // exponent arrays start at the floor on every run (atomic max)
  if (B->exp64) EMU_CUDA_TRY(ctx, cudaMemsetAsync(B->exp64, 0, (size_t)B->nslots * nb * sizeof(int), ctx->stream));
  if (B->exp_s) EMU_CUDA_TRY(ctx, cudaMemsetAsync(B->exp_s, 0, (size_t)B->nrows * sizeof(int), ctx->stream));
  for (int k = 0; k < B->maxNT; k++) {
    const Step &st = B->steps[k];
    if ((s = launch_tiles_to_f64(ctx, B->t32, B->t64, B->d_diag + st.dl_off, st.dl_n, te)) != EMU_OK) return s;
    if ((s = launch_potrf64_batch(ctx, B->t64, nb, k, B->d_diag + st.d_off, st.d_n, B->tasks, B->ntasks, B->ws,
                                  B->rinv, B->d_bad + st.d_off)) != EMU_OK)
      return s;
    if (st.t32_n > 0) {
      // FP32 copies (and, for the tensor-core TRSM, BF16 pieces) of the step's L_kk, one slot per matrix
      s = B->tc_trsm ? trsm_tc::launch_prep(ctx, B->t64, 0, B->d_diag + st.d_off, st.d_n, B->slots, B->lpieces, nb)
                     : launch_diag_to_f32_slots(ctx, B->t64, B->slots, B->d_diag + st.d_off, st.d_n, te);
      if (s != EMU_OK) return s;
    }
    if (st.t64_n > 0) {
      // the step's L_kk with their diagonal blocks pre-scaled, one slot per matrix, then the FP64 TRSMs
      if ((s = launch_trsm64_prep(ctx, B->t64, nb, B->ls64, B->rinv64, B->d_diag + st.d_off, st.d_n)) != EMU_OK ||
          (s = launch_trsm64_jobs(ctx, B->t64, nb, B->d_t64 + st.t64_off, st.t64_n, B->ls64, B->rinv64,
                                  B->d_t64slot + st.t64_off)) != EMU_OK)
        return s;
    }
    if ((s = launch_split_tiles64(ctx, B->t64, B->op, B->d_s64 + st.s64_off, st.s64_n, nb, 0)) != EMU_OK) return s;
    s = B->tc_trsm ? trsm_tc::launch(ctx, B->lmap, B->opmap, B->slots, B->t32, nb, 0, 0, nullptr,
                                     B->d_t32 + st.t32_off, st.t32_n)
                   : launch_trsm32_jobs(ctx, B->slots, B->t32, B->op, nb, B->d_t32 + st.t32_off, st.t32_n);
    if (s != EMU_OK) return s;
    if ((s = launch_quant_e4m3(ctx, B->op, B->op8, B->scale8, B->d_q + st.q_off, st.q_n, nb)) != EMU_OK) return s;
    if ((s = gemm64::launch_row_exponents(ctx, B->t64, B->t32, B->d_cls, B->d_z + st.z_off, st.z_n, nb,
                                          B->exp64)) != EMU_OK ||
        (s = gemm64::launch_slice(ctx, B->t64, B->t32, B->d_cls, B->d_z + st.z_off, st.z_n, nb, B->exp64,
                                  B->digits)) != EMU_OK)
      return s;
    if (st.u_n > 0) {
      ProfScope ps(ctx, PROF_UPDATE64, st.u_flops, 0.0, 36.0 * st.u_flops);
      if ((s = gemm64::launch(ctx, B->map64a, B->map64b, B->d_items64 + st.u_off, st.u_n, B->d_segs64, nb, nb, nb,
                              B->exp64, B->exp64, gemm64::TC64_SUB, B->t64, nb, ctx->sm_count)) != EMU_OK)
        return s;
    }
    if (st.it_n > 0) {
      ProfScope ps(ctx, PROF_TC_FACTOR, st.tc_flops, 0.0, st.tc_mma);
      if ((s = gemm_tc::launch(ctx, B->ops_f, B->d_items + st.it_off, st.it_n, B->d_segs, nb / gemm_tc::BK,
                               gemm_tc::TC_SUB_F32, B->t32, nullptr, nb, ctx->sm_count)) != EMU_OK)
        return s;
    }
  }
  // diagonal factor tiles: zeros above the diagonal; BF16 pieces for the sampler
  k_tril_list<<<dim3(nb, (unsigned)B->n_all_diag), 128, 0, ctx->stream>>>(B->t64, B->d_all_diag, nb, ctx->d_status);
  EMU_LAUNCHED(ctx);
  if (B->s > 0 && B->any_low &&
      (s = launch_split_tiles64(ctx, B->t64, B->op, B->d_all_diag_int, (int)B->n_all_diag, nb, 1)) != EMU_OK)
    return s;
  if (B->s > 0) {
    if ((s = launch_normals_batch(ctx, B->d_seed, B->d_inst, B->count, B->maxNT, nb, B->s, B->Z, B->nrows)) !=
        EMU_OK)
      return s;
    // Y = 0; FP64-class tiles as digit products (FP64 accurate) on the tensor cores
    EMU_CUDA_TRY(ctx, cudaMemsetAsync(B->Y, 0, (size_t)B->nrows * B->s * sizeof(double), ctx->stream));
    if (B->n_items64s > 0) {
      uint16_t *dz = B->digits + B->dig_s_off;
      if ((s = gemm64::launch_row_exponents(ctx, B->t64, B->t32, B->d_cls, B->d_zs, B->nzs, nb, B->exp_s)) !=
              EMU_OK ||
          (s = gemm64::launch_slice(ctx, B->t64, B->t32, B->d_cls, B->d_zs, B->nzs, nb, B->exp_s, B->digits)) !=
              EMU_OK ||
          (s = gemm64::launch_slice_z(ctx, B->Z, B->nrows, B->s, B->s_pad, B->d_zblk, B->count, B->nrows, B->exp_z,
                                      dz)) != EMU_OK)
        return s;
      ProfScope ps(ctx, PROF_TRMM64, B->samp64_flops, 0.0, 36.0 * B->samp64_flops);
      if ((s = gemm64::launch(ctx, B->map_sa, B->map_sz, B->d_items64s, (int)B->n_items64s, B->d_segs64s, nb, nb,
                              B->s_pad, B->exp_s, B->exp_z, gemm64::TC64_ADD, B->Y, (int)B->nrows, ctx->sm_count)) !=
          EMU_OK)
        return s;
    }
    if (B->n_items_sample > 0) {
      if ((s = launch_split_z(ctx, B->Z, B->nrows, B->nrows, B->s, B->s_pad, B->zp)) != EMU_OK) return s;
      ProfScope ps(ctx, PROF_TC_SAMPLE, B->sample_flops, 0.0, B->sample_mma);
      if ((s = gemm_tc::launch(ctx, B->ops_s, B->d_items_s, (int)B->n_items_sample, B->d_segs_s, nb / gemm_tc::BK,
                               gemm_tc::TC_ADD_F64, nullptr, B->Y, (int)B->nrows, ctx->sm_count)) != EMU_OK)
        return s;
    }
    k_gather_rows<<<dim3(64, B->count), 256, 0, ctx->stream>>>(B->Y, B->nrows, B->d_inst, B->s, B->d_Yptr);
    EMU_LAUNCHED(ctx);
  }
  if (B->want_L &&
      (s = launch_export_batch(ctx, B->d_inst, B->d_pairs, B->n_pairs, nb, B->t64, B->any_low ? B->t32 : nullptr,
                               B->any_low ? B->d_cls : nullptr, B->d_Lptr)) != EMU_OK)
    return s;
  return EMU_OK;
}

emu_status batch_capture(emu_ctx *ctx, BatchCtx *BC, BatchState *B) {
  if (!BC->cap) EMU_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&BC->cap, cudaStreamNonBlocking));
  cudaStream_t user = ctx->stream;
  bool prof = ctx->prof;
  uint64_t l0 = ctx->launches, h0 = ctx->host_launches;
  ctx->prof = false;  // no profiler events inside the graph
  ctx->stream = BC->cap;
  // relaxed: the launchers set kernel attributes while the stream is captured
  cudaError_t e = cudaStreamBeginCapture(BC->cap, cudaStreamCaptureModeRelaxed);
  emu_status s = (e == cudaSuccess) ? batch_record(ctx, B) : emu_cuda_fail(ctx, e, "begin capture");
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) e = cudaStreamEndCapture(BC->cap, &g);
  ctx->stream = user;
  ctx->prof = prof;
  B->graph_launches = (int)(ctx->launches - l0);
  ctx->launches = l0;  // counted when the graph runs
  ctx->host_launches = h0;
  if (s != EMU_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return emu_cuda_fail(ctx, e, "end capture");
  e = cudaGraphInstantiate(&B->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return emu_cuda_fail(ctx, e, "graph instantiate");
  return EMU_OK;
}

bool state_matches(const BatchState *B, int count, const emu_cov_params *p, int nb, const double *u, double eps,
                   unsigned mask, int diag_fp64, int band, double sp_frac, int s, bool want_L) {
  if (!B || B->count != count || B->nb != nb || B->s != s || B->want_L != want_L || B->eps != eps ||
      B->mask != mask || B->diag_fp64 != diag_fp64 || B->band != band || B->sp_frac != sp_frac)
    return false;
  for (int c = 0; c < EMU_NCLASS; c++)
    if (B->u[c] != u[c]) return false;
  for (int b = 0; b < count; b++)
    if (!same_params(B->params[b], p[b])) return false;
  return true;
}

emu_status batch_run(emu_ctx *ctx, int count, const emu_cov_params *p, int nb, const emu_mp_opts *o, int nsamples,
                     uint64_t seed, double *const *dY, double *const *dL, emu_factor_info *infos, float *ms_out) {
  BatchCtx *BC = static_cast<BatchCtx *>(ctx->batch);
  // options: the single-matrix path's defaults (FP32 class with its sqrt(nb) growth)
  double eps = o ? o->eps : 0.0;
  double u[EMU_NCLASS] = {0x1p-53, 0x1p-24 * std::sqrt((double)nb), 0x1p-11, 0x1p-8, 0x1p-4};
  unsigned mask = 1u;
  int diag_fp64 = o ? o->diag_fp64 : 0;
  const int band = o ? o->band : EMU_MAP_NORM;
  const double sp_frac = o ? band_sp_frac(o) : 0.05;
  if (eps > 0.0) {
    for (int c = 0; c < EMU_NCLASS; c++)
      if (o->u[c] > 0.0) u[c] = o->u[c];
    // the batched plan makes no TF32 copies: the TF32 class is left out here
    mask = (o->prec_mask | 1u) & ((1u << EMU_CLASS_FP32) | (1u << EMU_CLASS_BF16) | (1u << EMU_CLASS_E4M3) | 1u);
  }
  bool want_L = dL != nullptr;
  BatchState *B = BC->state;
  bool reuse = state_matches(B, count, p, nb, u, eps, mask, diag_fp64, band, sp_frac, nsamples, want_L);
  emu_status s;
  if (!reuse) {
    if (B) {
      B->release();
      delete B;
    }
    B = BC->state = new BatchState();
    B->s = nsamples;
    B->want_L = want_L;
    B->eps = eps;
    B->mask = mask;
    B->diag_fp64 = diag_fp64;
    B->band = band;
    B->sp_frac = sp_frac;
    std::memcpy(B->u, u, sizeof(u));
    if ((s = batch_layout(ctx, B, count, p, nb)) != EMU_OK) return s;
  }
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, ST_WORDS * sizeof(int), ctx->stream));
  // covariances, tile norms and the precision map of every matrix
  if ((s = launch_cov_build_batch(ctx, B->d_inst, count, B->maxL, B->ntab, B->d_tile_inst, B->ntiles, nb, B->tables,
                                  B->t64, B->partial)) != EMU_OK)
    return s;
  if ((s = launch_precision_map_batch(ctx, B->d_inst, count, nb, B->partial, B->tnorm, B->frob, B->d_cls, eps, u,
                                      mask, diag_fp64, band, sp_frac)) != EMU_OK)
    return s;
  std::vector<unsigned char> cls(B->ntiles);
  std::vector<double> frob(count);
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(cls.data(), B->d_cls, B->ntiles, cudaMemcpyDeviceToHost, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(frob.data(), B->frob, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (reuse && cls != B->cls) {
    // the same batch mapped differently (not expected): plan again
    BatchState *nbs = new BatchState();
    nbs->s = nsamples;
    nbs->want_L = want_L;
    nbs->eps = eps;
    nbs->mask = mask;
    nbs->diag_fp64 = diag_fp64;
    nbs->band = band;
    nbs->sp_frac = sp_frac;
    std::memcpy(nbs->u, u, sizeof(u));
    B->release();
    delete B;
    B = BC->state = nbs;
    return batch_run(ctx, count, p, nb, o, nsamples, seed, dY, dL, infos, ms_out);
  }
  if (!reuse) {
    B->cls = cls;
    if ((s = batch_plan(ctx, B)) != EMU_OK) return s;
    if ((s = batch_capture(ctx, BC, B)) != EMU_OK) return s;
  }
  // caller pointers and the seed, read by the graph's kernels
  if (nsamples > 0)
    EMU_CUDA_TRY(ctx, cudaMemcpyAsync(B->d_Yptr, dY, count * sizeof(double *), cudaMemcpyHostToDevice, ctx->stream));
  if (want_L)
    EMU_CUDA_TRY(ctx, cudaMemcpyAsync(B->d_Lptr, dL, count * sizeof(double *), cudaMemcpyHostToDevice, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(B->d_seed, &seed, sizeof(seed), cudaMemcpyHostToDevice, ctx->stream));
  // the per-matrix pivot records (allocated with the step plan, after the map)
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(B->d_bad, 0, B->diag_lists.size() * sizeof(int), ctx->stream));
  EMU_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  if (ctx->prof) {
    // profiling: the same launches issued one by one, so that each kernel
    // group gets its own events
    if ((s = batch_record(ctx, B)) != EMU_OK) return s;
  } else {
    EMU_CUDA_TRY(ctx, cudaGraphLaunch(B->graph, ctx->stream));
    ctx->launches += B->graph_launches;
    ctx->host_launches++;
  }
  EMU_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, ST_WORDS * sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream));
  std::vector<int> hbad(B->diag_lists.size());
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(hbad.data(), B->d_bad, hbad.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream));
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  if (ms_out) *ms_out = ms;
  int code = ctx->h_status[ST_CODE];
  // matrices that met a non-positive pivot: the first such column of each
  // (the other matrices of the batch went on and are complete)
  std::vector<int> pivots(count, 0);
  int nbad = 0;
  for (int k = 0; k < B->maxNT; k++) {
    const Step &st = B->steps[k];
    for (int slot = 0; slot < st.d_n; slot++) {
      const int col = hbad[st.d_off + slot];
      if (col <= 0) continue;
      const long g = B->diag_lists[st.d_off + slot];
      for (int b = 0; b < count; b++)
        if (g >= B->inst[b].tile_base && g < B->inst[b].tile_base + (long)B->inst[b].NT * (B->inst[b].NT + 1) / 2) {
          if (pivots[b] == 0) nbad++;
          if (pivots[b] == 0 || col < pivots[b]) pivots[b] = col;
        }
    }
  }
  if (infos) {
    for (int b = 0; b < count; b++) {
      const BatchInst &I = B->inst[b];
      emu_factor_info &f = infos[b];
      std::memset(&f, 0, sizeof(f));
      f.n = I.n;
      f.nb = nb;
      f.nt = I.NT;
      f.pivot = pivots[b];
      for (long t = 0; t < (long)I.NT * (I.NT + 1) / 2; t++) f.tiles[B->cls[I.tile_base + t]]++;
      for (int c = 0; c < EMU_NCLASS; c++) f.update_flops[c] = B->upd_flops[b][c];
      f.frob = frob[b];
      f.ms = ms;
    }
  }
  if (code == DEV_TIMEOUT) {
    ctx->last_error = "device wait timed out";
    return EMU_ETIMEOUT;
  }
  if (nbad > 0 || code == DEV_NOTPD) {
    ctx->last_error = "covariances of the batch are not positive definite (see their info.pivot; the others are complete)";
    return EMU_ENOTPD;
  }
  return EMU_OK;
}

}  // namespace

void batch_ctx_release(emu_ctx *ctx) {
  BatchCtx *BC = static_cast<BatchCtx *>(ctx->batch);
  if (!BC) return;
  cudaStreamSynchronize(ctx->stream);
  if (BC->state) {
    BC->state->release();
    delete BC->state;
  }
  if (BC->cap) cudaStreamDestroy(BC->cap);
  delete BC;
  ctx->batch = nullptr;
}

extern "C" {

emu_status emu_batch_potrf_sample(emu_ctx *ctx, int count, const emu_cov_params *p, int nb, const emu_mp_opts *o,
                                  int nsamples, uint64_t seed, double *const *dY, double *const *dL,
                                  emu_factor_info *infos) {
  if (!ctx || count < 1 || !p || nsamples < 0 || (nsamples > 0 && !dY)) return EMU_EINVAL;
  if (o && (o->band < EMU_MAP_NORM || o->band > EMU_MAP_DP_HP)) {
    ctx->last_error = "unknown precision map";
    return EMU_EINVAL;
  }
  if (!(nb == 0 || (nb >= 256 && nb <= 1024 && nb % 256 == 0))) {
    ctx->last_error = "batch tile size must be 0 (tuned) or a multiple of 256 in [256, 1024]";
    return EMU_EINVAL;
  }
  for (int b = 0; b < count; b++) {
    if (p[b].L < 1 || p[b].L > 256 || !(p[b].beta > 0.0) || !(p[b].nugget_rel > -1.0 && p[b].nugget_rel < 1e300)) {
      ctx->last_error = "batch needs 1 <= L <= 256, beta > 0, finite nugget_rel > -1 for every matrix";
      return EMU_EINVAL;
    }
    if ((nsamples > 0 && !dY[b]) || (dL && !dL[b])) return EMU_EINVAL;
  }
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (!ctx->batch) ctx->batch = new BatchCtx();
  BatchCtx *BC = static_cast<BatchCtx *>(ctx->batch);
  if (nb != 0) return batch_run(ctx, count, p, nb, o, nsamples, seed, dY, dL, infos, nullptr);
  // nb == 0: the tile size this batch signature was tuned to, else tune it now
  // by timing the whole call with each candidate (the last candidate's results
  // are kept when it is the best, else the best runs once more)
  double eps = o ? o->eps : 0.0;
  unsigned mask = o ? o->prec_mask : 1u;
  int diag = o ? o->diag_fp64 : 0;
  const int band = o ? o->band : EMU_MAP_NORM;
  const double sp_frac = o ? band_sp_frac(o) : 0.05;
  for (const TuneRec &t : BC->tuned) {
    if (t.params.size() != (size_t)count || t.eps != eps || t.mask != mask || t.diag_fp64 != diag ||
        t.band != band || t.sp_frac != sp_frac ||
        t.s != nsamples || t.want_L != (dL != nullptr))
      continue;
    bool same = true;
    for (int b = 0; b < count && same; b++) same = same_params(t.params[b], p[b]);
    if (same) return batch_run(ctx, count, p, t.nb, o, nsamples, seed, dY, dL, infos, nullptr);
  }
  const int cand[2] = {512, 256};
  float best_ms = 0.f;
  int best = 0;
  for (int c : cand) {
    float ms = 0.f;
    emu_status s = batch_run(ctx, count, p, c, o, nsamples, seed, dY, dL, infos, &ms);
    if (s == EMU_ENOMEM) continue;
    if (s != EMU_OK) return s;
    if (best == 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  if (best == 0) return EMU_ENOMEM;
  TuneRec t;
  t.params.assign(p, p + count);
  t.eps = eps;
  t.mask = mask;
  t.diag_fp64 = diag;
  t.band = band;
  t.sp_frac = sp_frac;
  t.s = nsamples;
  t.want_L = dL != nullptr;
  t.nb = best;
  BC->tuned.push_back(t);
  if (best != cand[1]) return batch_run(ctx, count, p, best, o, nsamples, seed, dY, dL, infos, nullptr);
  return EMU_OK;
}

emu_status emu_batch_release(emu_ctx *ctx) {
  if (!ctx) return EMU_EINVAL;
  batch_ctx_release(ctx);
  return EMU_OK;
}

}  // extern "C"
