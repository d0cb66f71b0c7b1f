// api.cu -- the C ABI of libemucov: context and matrix lifetime, argument
// checks, and the host-side order of kernel launches (the tile-DAG schedule
// of the factor, sampling, solves).  See include/emucov.h for the contract.
#include <stdio.h>
#include <string.h>

#include <new>

#include <vector>

#include "emu_internal.h"
#include "gemm_f64.h"
#include "mixed.h"

emu_status emu_cuda_fail(emu_ctx *ctx, cudaError_t e, const char *what) {
  if (ctx) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    ctx->last_error = buf;
  }
  return EMU_ECUDA;
}

static emu_status collect_status(emu_ctx *ctx, int *pivot);

static emu_status fail_msg(emu_ctx *ctx, emu_status s, const char *msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

// ------------------------------------------------------------- profiling
ProfScope::ProfScope(emu_ctx *c, int group, double flops, double bytes, double mma_flops)
    : ctx(c), on(c && c->prof) {
  if (!on) return;
  for (int q = 0; q < 2; q++) {
    cudaEvent_t e;
    if (ctx->ev_pool.empty()) {
      if (cudaEventCreate(&e) != cudaSuccess) {
        on = false;
        return;
      }
    } else {
      e = ctx->ev_pool.back();
      ctx->ev_pool.pop_back();
    }
    (q == 0 ? rec.a : rec.b) = e;
  }
  rec.group = group;
  rec.flops = flops;
  rec.bytes = bytes;
  rec.mma_flops = mma_flops;
  rec.launches0 = ctx->launches;
  rec.stream = ctx->stream;
  cudaEventRecord(rec.a, ctx->stream);
}

ProfScope::~ProfScope() {
  if (!on) return;
  cudaEventRecord(rec.b, ctx->stream);
  rec.launches0 = ctx->launches - rec.launches0;  // launches inside the scope
  ctx->prof_open.push_back(rec);
}

static void prof_collect(emu_ctx *ctx) {
  if (ctx->prof_open.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (const ProfRec &r : ctx->prof_open) {
    float ms = 0.f, t0 = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    if (ctx->prof_base && cudaEventElapsedTime(&t0, ctx->prof_base, r.a) == cudaSuccess)
      ctx->timeline.push_back({r.group, r.stream, (double)t0, (double)t0 + ms});
    ctx->prof_ms[r.group] += ms;
    ctx->prof_launches[r.group] += (int)r.launches0;
    ctx->prof_flops[r.group] += r.flops;
    ctx->prof_bytes[r.group] += r.bytes;
    ctx->prof_mma[r.group] += r.mma_flops;
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->prof_open.clear();
}

extern "C" {

const char *emu_status_str(emu_status s) {
  switch (s) {
    case EMU_OK: return "ok";
    case EMU_EINVAL: return "invalid argument";
    case EMU_ENOMEM: return "out of device memory or size limit exceeded";
    case EMU_ENOTPD: return "matrix not positive definite";
    case EMU_ENOCONV: return "refinement did not converge";
    case EMU_ETIMEOUT: return "device wait timed out";
    case EMU_ECUDA: return "CUDA error";
    case EMU_ESTATE: return "matrix in wrong state";
  }
  return "unknown status";
}

const char *emu_last_error(const emu_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

uint64_t emu_launch_count(const emu_ctx *ctx) { return ctx ? ctx->launches : 0; }

uint64_t emu_host_launch_count(const emu_ctx *ctx) { return ctx ? ctx->host_launches : 0; }

emu_status emu_create(emu_ctx **out, int device, void *stream) {
  if (!out) return EMU_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return EMU_EINVAL;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return EMU_ECUDA;
  if (p.major != 10 || p.minor != 3) return EMU_EINVAL;  // sm_103 only
  emu_ctx *ctx = new (std::nothrow) emu_ctx();
  if (!ctx) return EMU_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  ctx->sm_count = p.multiProcessorCount;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, ST_WORDS * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_status, ST_WORDS * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, ST_WORDS * sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
  if (e == cudaSuccess) {
    // matrices are allocated stream-ordered from the device's default pool;
    // keep released blocks cached so that rebuilding a matrix is cheap
    cudaMemPool_t pool;
    e = cudaDeviceGetDefaultMemPool(&pool, device);
    uint64_t keep = UINT64_MAX;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e != cudaSuccess) {
    emu_destroy(ctx);
    return EMU_ECUDA;
  }
  *out = ctx;
  return EMU_OK;
}

emu_status emu_destroy(emu_ctx *ctx) {
  if (!ctx) return EMU_EINVAL;
  cudaSetDevice(ctx->device);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  prof_collect(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->prof_base) cudaEventDestroy(ctx->prof_base);
  cudaFree(ctx->dag_tasks);
  cudaFree(ctx->dag_ws);
  cudaFree(ctx->trace_buf);
  mixed_ctx_release(ctx);
  batch_ctx_release(ctx);
  for (cudaEvent_t e : ctx->xev)
    if (e) cudaEventDestroy(e);
  if (ctx->xfer) cudaStreamDestroy(ctx->xfer);
  delete ctx;
  return EMU_OK;
}

emu_status emu_set_stream(emu_ctx *ctx, void *stream) {
  if (!ctx) return EMU_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return EMU_OK;
}

emu_status emu_prof_enable(emu_ctx *ctx, int on) {
  if (!ctx) return EMU_EINVAL;
  prof_collect(ctx);
  for (int g = 0; g < PROF_NGROUPS; g++) {
    ctx->prof_launches[g] = 0;
    ctx->prof_ms[g] = ctx->prof_flops[g] = ctx->prof_bytes[g] = ctx->prof_mma[g] = 0.0;
  }
  ctx->prof = on != 0;
  ctx->timeline.clear();
  if (ctx->prof) {
    if (!ctx->prof_base) EMU_CUDA_TRY(ctx, cudaEventCreate(&ctx->prof_base));
    EMU_CUDA_TRY(ctx, cudaEventRecord(ctx->prof_base, ctx->stream));
  }
  return EMU_OK;
}

emu_status emu_prof_timeline(emu_ctx *ctx, double *h_out, size_t max_records, size_t *n_records) {
  if (!ctx || !n_records) return EMU_EINVAL;
  prof_collect(ctx);
  *n_records = ctx->timeline.size();
  if (!h_out) return EMU_OK;
  size_t n = ctx->timeline.size() < max_records ? ctx->timeline.size() : max_records;
  for (size_t i = 0; i < n; i++) {
    const auto &r = ctx->timeline[i];
    int sid = r.stream == ctx->crit ? 1 : r.stream == ctx->mid ? 2 : r.stream == ctx->bulk ? 3 : 0;
    h_out[4 * i] = r.group;
    h_out[4 * i + 1] = sid;
    h_out[4 * i + 2] = r.t0;
    h_out[4 * i + 3] = r.t1;
  }
  return EMU_OK;
}

emu_status emu_trace_enable(emu_ctx *ctx, int on) {
  if (!ctx) return EMU_EINVAL;
  ctx->trace_on = on != 0;
  ctx->trace_records = 0;
  return EMU_OK;
}

emu_status emu_schedule(emu_ctx *ctx, int use_graphs, int tuning) {
  if (!ctx) return EMU_EINVAL;
  mixed_set_schedule(ctx, use_graphs, tuning);
  return EMU_OK;
}

emu_status emu_schedule_info(emu_ctx *ctx, int *tried, int *reserved, int *reserved_fp64) {
  if (!ctx) return EMU_EINVAL;
  int t = 0, r = 0, r64 = 0;
  if (mixed_tuned_choice(ctx, &t, &r, &r64) < 0) t = r = r64 = 0;
  if (tried) *tried = t;
  if (reserved) *reserved = r;
  if (reserved_fp64) *reserved_fp64 = r64;
  return EMU_OK;
}

emu_status emu_test_wait_hook(emu_ctx *ctx, long long wait_cycles, int withhold_index) {
  if (!ctx) return EMU_EINVAL;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return set_dag_wait_hook(ctx, wait_cycles, withhold_index);
}

emu_status emu_trace_read(emu_ctx *ctx, uint64_t *h_records, size_t max_records, size_t *n_records) {
  if (!ctx || !n_records) return EMU_EINVAL;
  *n_records = ctx->trace_records;
  if (!h_records || ctx->trace_records == 0) return EMU_OK;
  size_t n = ctx->trace_records < max_records ? ctx->trace_records : max_records;
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(h_records, ctx->trace_buf, n * 5 * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                    ctx->stream));
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return EMU_OK;
}

emu_status emu_prof_read(emu_ctx *ctx, int group, int *launches, double *total_ms, double *flops,
                         double *bytes, double *mma_flops) {
  if (!ctx || group < 0 || group >= PROF_NGROUPS) return EMU_EINVAL;
  prof_collect(ctx);
  if (launches) *launches = ctx->prof_launches[group];
  if (total_ms) *total_ms = ctx->prof_ms[group];
  if (flops) *flops = ctx->prof_flops[group];
  if (bytes) *bytes = ctx->prof_bytes[group];
  if (mma_flops) *mma_flops = ctx->prof_mma[group];
  return EMU_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- matrices
static emu_status mat_alloc(emu_ctx *ctx, int n, int nb, emu_mat **out, bool arena64 = true) {
  if (!ctx || !out || n <= 0 || nb < 64 || nb > 2048 || (nb % 64) != 0)
    return fail_msg(ctx, EMU_EINVAL, "need n > 0 and nb a multiple of 64 in [64, 2048]");
  *out = nullptr;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  emu_mat *A = new (std::nothrow) emu_mat();
  if (!A) return EMU_ENOMEM;
  A->ctx = ctx;
  A->n = n;
  A->nb = nb;
  A->nt = (n + nb - 1) / nb;
  A->ntiles = tile_count(A->nt);
  A->tile_elems = (size_t)nb * nb;
  A->nchunk = nb / 32;
  size_t bytes64 = arena64 ? (size_t)A->ntiles * A->tile_elems * sizeof(double) : 0;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if (bytes64 + (64u << 20) > free_b) {
    delete A;
    return fail_msg(ctx, EMU_ENOMEM, "FP64 tile arena does not fit in free device memory");
  }
  cudaStream_t s = ctx->stream;
  cudaError_t e = arena64 ? cudaMallocAsync(&A->t64, bytes64, s) : cudaSuccess;
  if (e == cudaSuccess) e = cudaMallocAsync(&A->d_partial, (size_t)A->ntiles * A->nchunk * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&A->d_tnorm, (size_t)A->ntiles * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&A->d_frob, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&A->d_cls, (size_t)A->ntiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->d_cls, 0, (size_t)A->ntiles, ctx->stream);
  if (e != cudaSuccess) {
    emu_mat_free(A);
    return e == cudaErrorMemoryAllocation ? EMU_ENOMEM : emu_cuda_fail(ctx, e, "mat_alloc");
  }
  A->h_cls = new (std::nothrow) unsigned char[A->ntiles];
  if (!A->h_cls) {
    emu_mat_free(A);
    return EMU_ENOMEM;
  }
  memset(A->h_cls, 0, A->ntiles);
  *out = A;
  return EMU_OK;
}

extern "C" {

emu_status emu_mat_free(emu_mat *A) {
  if (!A) return EMU_EINVAL;
  cudaStream_t s = A->ctx ? A->ctx->stream : nullptr;
  if (A->ctx) cudaSetDevice(A->ctx->device);
  void *bufs[] = {A->t64, A->t32, A->d_partial, A->d_tnorm, A->d_frob, A->d_cls, A->op_bf16, A->op_e4m3,
                  A->scale_e4m3, A->op_tf32};
  for (void *b : bufs)
    if (b) cudaFreeAsync(b, s);
  mixed_mat_release(A);
  classfmt_release(A);
  delete[] A->h_cls;
  delete A;
  return EMU_OK;
}

emu_status emu_cov_build_classfmt(emu_ctx *ctx, const emu_cov_params *p, int nb, const emu_mp_opts *o,
                                  emu_mat **out) {
  if (!ctx || !p || !o || !out) return EMU_EINVAL;
  if (p->L < 1 || p->L > 4096 || !(p->beta > 0.0) || !(p->nugget_rel > -1.0 && p->nugget_rel < 1e300))
    return fail_msg(ctx, EMU_EINVAL, "need 1 <= L <= 4096, beta > 0, finite nugget_rel > -1");
  if (o->band < EMU_MAP_NORM || o->band > EMU_MAP_DP_HP) return fail_msg(ctx, EMU_EINVAL, "unknown precision map");
  if (nb % 256 != 0) return fail_msg(ctx, EMU_EINVAL, "class-format storage needs nb a multiple of 256");
  emu_mat *A = nullptr;
  emu_status s = mat_alloc(ctx, p->L * p->L, nb, &A, false);
  if (s != EMU_OK) return s;
  s = classfmt_build(ctx, A, p, o);
  if (s != EMU_OK) {
    emu_mat_free(A);
    return s;
  }
  *out = A;
  return EMU_OK;
}

emu_status emu_backward_error_est(emu_ctx *ctx, const emu_mat *L, const emu_cov_params *p, int nprobes,
                                  uint64_t seed, double *est) {
  if (!ctx || !L || !p || !est || nprobes < 1) return EMU_EINVAL;
  if (L->state != MAT_FACTOR64 && L->state != MAT_FACTOR_MIXED)
    return fail_msg(ctx, EMU_ESTATE, "the estimate needs a factored matrix");
  if (p->L * p->L != L->n) return fail_msg(ctx, EMU_EINVAL, "the parameters' n = L^2 differs from the factor's");
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return factor_backward_error_est(ctx, L, p, nprobes, seed, est);
}

emu_status emu_cov_build(emu_ctx *ctx, const emu_cov_params *p, int nb, emu_mat **out) {
  if (!ctx || !p || !out) return EMU_EINVAL;
  if (p->L < 1 || p->L > 4096 || !(p->beta > 0.0) || !(p->nugget_rel > -1.0 && p->nugget_rel < 1e300))
    return fail_msg(ctx, EMU_EINVAL, "need 1 <= L <= 4096, beta > 0, finite nugget_rel > -1");
  emu_mat *A = nullptr;
  emu_status s = mat_alloc(ctx, p->L * p->L, nb, &A);
  if (s != EMU_OK) return s;
  s = launch_cov_build(ctx, A, p);
  if (s != EMU_OK) {
    emu_mat_free(A);
    return s;
  }
  *out = A;
  return EMU_OK;
}

emu_status emu_mat_import(emu_ctx *ctx, const double *dA, int n, long lda, int nb,
                          emu_mat **out) {
  if (!ctx || !dA || !out || lda < n) return EMU_EINVAL;
  emu_mat *A = nullptr;
  emu_status s = mat_alloc(ctx, n, nb, &A);
  if (s != EMU_OK) return s;
  s = launch_import(ctx, A, dA, lda);
  if (s != EMU_OK) {
    emu_mat_free(A);
    return s;
  }
  *out = A;
  return EMU_OK;
}

emu_status emu_cov_from_residuals(emu_ctx *ctx, const double *dXi, int n, long m, long ldxi, double nugget_rel,
                                  int nb, emu_mat **out) {
  if (!ctx || !dXi || !out || n < 1 || m < 1 || ldxi < n || !(nugget_rel >= 0.0)) return EMU_EINVAL;
  if (nb % 256 != 0) return fail_msg(ctx, EMU_EINVAL, "the empirical covariance needs nb a multiple of 256");
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  emu_mat *A = nullptr;
  emu_status s = mat_alloc(ctx, n, nb, &A);
  if (s != EMU_OK) return s;
  const int NT = A->nt, npad = NT * nb;
  // K per segment (a multiple of the 256-column exact accumulation chunk) and
  // per launch (the digit arena stays within 2 GB)
  const long Kc = 512;
  const long mpad = (m + Kc - 1) / Kc * Kc;
  long kb = ((1L << 31) / (16L * npad)) / Kc * Kc;
  kb = std::max(Kc, std::min(kb, mpad));
  // every 128 x 64 block of every lower tile (diagonal tiles in full, so that
  // their norms cover both triangles as the covariance build's do), one
  // segment per Kc columns of a launch
  std::vector<gemm64::Item> items;
  std::vector<gemm64::Seg> segs;
  for (int I = 0; I < NT; I++)
    for (int J = 0; J <= I; J++)
      for (int nbk = 0; nbk < nb / gemm64::BN; nbk++)
        for (int mb = 0; mb < nb / gemm64::BM; mb++) {
          gemm64::Item it;
          it.out_off = tile_index(I, J, NT) * (long)nb * nb + mb * gemm64::BM + (long)nbk * gemm64::BN * nb;
          it.a_sc = I * nb + mb * gemm64::BM;
          it.b_sc = J * nb + nbk * gemm64::BN;
          it.seg_begin = (int)segs.size();
          for (long kc = 0; kc < kb / Kc; kc++) {
            gemm64::Seg sg;
            sg.a_row = it.a_sc;
            sg.b_row = it.b_sc;
            sg.a_x = sg.b_x = (int)(kc * Kc);
            segs.push_back(sg);
          }
          it.seg_end = (int)segs.size();
          it.rows_valid = gemm64::BM;
          it.cols_valid = gemm64::BN;
          items.push_back(it);
        }
  gemm64::Item *d_items = nullptr;
  gemm64::Seg *d_segs = nullptr;
  int *d_exps = nullptr;
  uint16_t *d_digits = nullptr;
  unsigned long long *d_maxbits = nullptr;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemsetAsync(ctx->d_status, 0, ST_WORDS * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_items, items.size() * sizeof(gemm64::Item), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_segs, segs.size() * sizeof(gemm64::Seg), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_exps, (size_t)npad * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_digits, (size_t)gemm64::NS * npad * kb * sizeof(uint16_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_maxbits, sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(gemm64::Item), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(gemm64::Seg), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->t64, 0, (size_t)A->ntiles * A->tile_elems * sizeof(double), st);
  CUtensorMap ma, mbm;
  if (e == cudaSuccess) s = gemm64::make_map(ctx, &ma, d_digits, kb, (uint64_t)gemm64::NS * npad, gemm64::BM);
  if (e == cudaSuccess && s == EMU_OK)
    s = gemm64::make_map(ctx, &mbm, d_digits, kb, (uint64_t)gemm64::NS * npad, gemm64::BN);
  for (long k0 = 0; k0 < m && e == cudaSuccess && s == EMU_OK; k0 += kb) {
    const long ncols = std::min(kb, m - k0);
    s = gemm64::launch_dense_digits(ctx, dXi, ldxi, n, k0, ncols, npad, kb, d_exps, d_digits);
    if (s == EMU_OK) {
      ProfScope ps(ctx, PROF_UPDATE64, (double)npad * (npad + nb) * (double)kb, 0.0, 36.0 * npad * (double)npad * kb);
      s = gemm64::launch(ctx, ma, mbm, d_items, (int)items.size(), d_segs, (int)Kc, npad, npad, d_exps, d_exps,
                         gemm64::TC64_ADD, A->t64, nb, ctx->sm_count);
    }
  }
  if (e == cudaSuccess && s == EMU_OK) s = launch_emp_finish(ctx, A, m, nugget_rel, d_maxbits);
  for (void *p : {(void *)d_items, (void *)d_segs, (void *)d_exps, (void *)d_digits, (void *)d_maxbits})
    if (p) cudaFreeAsync(p, st);
  if (e == cudaSuccess && s == EMU_OK) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) s = emu_cuda_fail(ctx, e, "cov_from_residuals");
  if (s == EMU_OK) {
    int pivot = 0;
    s = collect_status(ctx, &pivot);
  }
  if (s != EMU_OK) {
    emu_mat_free(A);
    return s;
  }
  *out = A;
  return EMU_OK;
}

emu_status emu_mat_import_host(emu_ctx *ctx, const double *hA, int n, long lda, int nb,
                               emu_mat **out) {
  if (!ctx || !hA || !out || lda < n) return EMU_EINVAL;
  emu_mat *A = nullptr;
  emu_status s = mat_alloc(ctx, n, nb, &A);
  if (s != EMU_OK) return s;
  // Tile column j: its lower part (rows r0 .. n-1) is copied on the copy
  // stream into staging buffer j % 2 while the import kernel of column j - 1
  // reads the other one; events order copy -> import and import -> reuse.
  cudaError_t e = cudaSuccess;
  if (!ctx->xfer) e = cudaStreamCreateWithFlags(&ctx->xfer, cudaStreamNonBlocking);
  for (int i = 0; i < 5 && e == cudaSuccess; i++)
    if (!ctx->xev[i]) e = cudaEventCreateWithFlags(&ctx->xev[i], cudaEventDisableTiming);
  cudaEvent_t ev_alloc = ctx->xev[0], ev_copied[2] = {ctx->xev[1], ctx->xev[2]}, ev_free[2] = {ctx->xev[3], ctx->xev[4]};
  double *stage[2] = {nullptr, nullptr};
  for (int b = 0; b < 2 && e == cudaSuccess; b++)
    e = cudaMallocAsync(&stage[b], (size_t)n * nb * sizeof(double), ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev_alloc, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->xfer, ev_alloc, 0);
  for (int j = 0; j < A->nt && e == cudaSuccess && s == EMU_OK; j++) {
    const int b = j & 1;
    long r0 = (long)j * nb;
    long cols = (r0 + nb <= n) ? nb : n - r0;
    if (j >= 2) e = cudaStreamWaitEvent(ctx->xfer, ev_free[b], 0);  // column j - 2 is imported
    // rows r0 .. n-1 of columns r0 .. r0+cols-1: the lower part of tile column j
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(stage[b], (size_t)(n - r0) * sizeof(double), hA + r0 + r0 * lda, lda * sizeof(double),
                            (size_t)(n - r0) * sizeof(double), cols, cudaMemcpyHostToDevice, ctx->xfer);
    if (e == cudaSuccess) e = cudaEventRecord(ev_copied[b], ctx->xfer);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ev_copied[b], 0);
    if (e == cudaSuccess) s = launch_import_col(ctx, A, j, stage[b], n - r0);
    if (e == cudaSuccess && s == EMU_OK) e = cudaEventRecord(ev_free[b], ctx->stream);
  }
  // every copy issued (also on an error path) is ordered before the frees
  if (cudaEventRecord(ev_alloc, ctx->xfer) == cudaSuccess) cudaStreamWaitEvent(ctx->stream, ev_alloc, 0);
  for (int b = 0; b < 2; b++)
    if (stage[b]) cudaFreeAsync(stage[b], ctx->stream);
  if (e == cudaSuccess && s == EMU_OK) s = launch_precision_map(ctx, A, 0.0, nullptr, 0u, 0, EMU_MAP_NORM, 0.0);
  if (e == cudaSuccess && s == EMU_OK) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) s = emu_cuda_fail(ctx, e, "import_host");
  if (s != EMU_OK) {
    emu_mat_free(A);
    return s;
  }
  *out = A;
  return EMU_OK;
}

emu_status emu_mat_clone(emu_ctx *ctx, const emu_mat *A, emu_mat **out) {
  if (!ctx || !A || !out) return EMU_EINVAL;
  if (A->state != MAT_COV) return fail_msg(ctx, EMU_ESTATE, "clone supports covariance matrices");
  if (A->cs) return fail_msg(ctx, EMU_ESTATE, "clone supports FP64-tiled matrices");
  emu_mat *B = nullptr;
  emu_status s = mat_alloc(ctx, A->n, A->nb, &B);
  if (s != EMU_OK) return s;
  cudaError_t e = cudaMemcpyAsync(B->t64, A->t64, (size_t)A->ntiles * A->tile_elems * sizeof(double),
                                  cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_partial, A->d_partial, (size_t)A->ntiles * A->nchunk * sizeof(double),
                        cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_tnorm, A->d_tnorm, (size_t)A->ntiles * sizeof(double),
                        cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_frob, A->d_frob, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
  if (e != cudaSuccess) {
    emu_mat_free(B);
    return emu_cuda_fail(ctx, e, "clone");
  }
  *out = B;
  return EMU_OK;
}

emu_status emu_mat_export(emu_ctx *ctx, const emu_mat *A, double *dOut, long ld) {
  if (!ctx || !A || !dOut || ld < A->n) return EMU_EINVAL;
  if (A->cs) return classfmt_export(ctx, A, dOut, ld);
  return launch_export(ctx, A, dOut, ld);
}

emu_status emu_mat_tile_info(emu_ctx *ctx, const emu_mat *A, unsigned char *h_cls,
                             double *h_norms) {
  if (!ctx || !A) return EMU_EINVAL;
  int NT = A->nt;
  unsigned char *cls = new (std::nothrow) unsigned char[A->ntiles];
  double *tn = new (std::nothrow) double[A->ntiles];
  if (!cls || !tn) {
    delete[] cls;
    delete[] tn;
    return EMU_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(cls, A->d_cls, A->ntiles, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tn, A->d_tnorm, A->ntiles * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    delete[] cls;
    delete[] tn;
    return emu_cuda_fail(ctx, e, "tile_info");
  }
  for (int j = 0; j < NT; j++)
    for (int i = 0; i < NT; i++) {
      size_t o = (size_t)i + (size_t)j * NT;
      if (i < j) {
        if (h_cls) h_cls[o] = 255;
        if (h_norms) h_norms[o] = 0.0;
      } else {
        long t = tile_index(i, j, NT);
        if (h_cls) h_cls[o] = cls[t];
        if (h_norms) h_norms[o] = tn[t];
      }
    }
  delete[] cls;
  delete[] tn;
  return EMU_OK;
}

emu_status emu_mat_shape(const emu_mat *A, int *n, int *nb, int *nt, int *state) {
  if (!A) return EMU_EINVAL;
  if (n) *n = A->n;
  if (nb) *nb = A->nb;
  if (nt) *nt = A->nt;
  if (state) *state = A->state;
  return EMU_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ factor
// Reads the device status word after the stream drains.
static emu_status collect_status(emu_ctx *ctx, int *pivot) {
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, ST_WORDS * sizeof(int),
                                    cudaMemcpyDeviceToHost, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (pivot) *pivot = ctx->h_status[ST_PIVOT];
  if (ctx->h_status[ST_CODE] == DEV_NOTPD) return EMU_ENOTPD;
  if (ctx->h_status[ST_CODE] == DEV_TIMEOUT) return fail_msg(ctx, EMU_ETIMEOUT, "device wait timed out");
  return EMU_OK;
}

// Plain FP64 right-looking tile Cholesky: POTRF(k), TRSM(:,k), SYRK/GEMM of
// the trailing tiles, k = 0 .. NT-1.
static emu_status factor64(emu_ctx *ctx, emu_mat *A) {
  for (int k = 0; k < A->nt; k++) {
    emu_status s = launch_potrf64_tile(ctx, A, k);
    if (s == EMU_OK) s = launch_trsm64_panel(ctx, A, k);
    if (s == EMU_OK) s = launch_update64(ctx, A, k);
    if (s != EMU_OK) return s;
  }
  return launch_tril_diag(ctx, A);
}

extern "C" emu_status emu_potrf_mp(emu_ctx *ctx, emu_mat *A, const emu_mp_opts *o,
                                   emu_factor_info *info) {
  if (!ctx || !A) return EMU_EINVAL;
  if (A->state != MAT_COV) return fail_msg(ctx, EMU_ESTATE, "matrix is already factored");
  if (o && (o->band < EMU_MAP_NORM || o->band > EMU_MAP_DP_HP))
    return fail_msg(ctx, EMU_EINVAL, "unknown precision map");
  bool mixed = o && (o->eps > 0.0 || o->band != EMU_MAP_NORM);
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, ST_WORDS * sizeof(int), ctx->stream));
  EMU_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  emu_status s;
  if (A->cs) {
    mixed = true;  // the precision map was fixed when the matrix was built
    s = classfmt_factor(ctx, A);
  } else if (mixed) {
    s = factor_mixed(ctx, A, o);
  } else {
    s = factor64(ctx, A);
  }
  if (s != EMU_OK) return s;
  EMU_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  int pivot = 0;
  s = collect_status(ctx, &pivot);
  mixed_tune_record(ctx, s == EMU_OK);  // the device time of the schedule choice, for the tuner
  A->state = mixed ? MAT_FACTOR_MIXED : MAT_FACTOR64;
  if (info) {
    memset(info, 0, sizeof *info);
    info->n = A->n;
    info->nb = A->nb;
    info->nt = A->nt;
    info->pivot = (s == EMU_ENOTPD) ? pivot : 0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    info->ms = ms;
    double nb3 = (double)A->nb * A->nb * A->nb;
    if (A->cs) {
      classfmt_fill_info(A, info);
    } else if (mixed) {
      mixed_fill_info(A, info);
    } else {
      info->tiles[EMU_CLASS_FP64] = (int)A->ntiles;
      int NT = A->nt;
      double f = 0.0;
      for (int j = 0; j < NT; j++) f += (double)(NT - j - 1) * nb3 + (double)(NT - j - 1) * (NT - j) * nb3;
      info->update_flops[EMU_CLASS_FP64] = f;
    }
  }
  return s;
}

// ---------------------------------------------------------------- sampling
extern "C" emu_status emu_sample(emu_ctx *ctx, const emu_mat *L, int nsamples, uint64_t seed,
                                 uint32_t stream_id, double *dY, long ldy, double *dZ) {
  if (!ctx || !L || !dY || nsamples < 0 || ldy < L->n) return EMU_EINVAL;
  if (L->state != MAT_FACTOR64 && L->state != MAT_FACTOR_MIXED)
    return fail_msg(ctx, EMU_ESTATE, "sampling needs a factored matrix");
  if (nsamples == 0) return EMU_OK;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  long npad = (long)L->nt * L->nb;
  double *Z = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&Z, (size_t)npad * nsamples * sizeof(double), ctx->stream));
  emu_status s = launch_normals(ctx, seed, stream_id, (int)npad, nsamples, Z, npad);
  if (s == EMU_OK) {
    if (L->cs)
      s = classfmt_sample(ctx, L, Z, npad, nsamples, dY, ldy);
    else if (L->state == MAT_FACTOR64)
      s = launch_trmm64(ctx, L, Z, npad, nsamples, dY, ldy);
    else
      s = mixed_sample(ctx, L, Z, npad, nsamples, dY, ldy);
  }
  if (s == EMU_OK && dZ) {
    cudaError_t e = cudaMemcpy2DAsync(dZ, ldy * sizeof(double), Z, npad * sizeof(double),
                                      (size_t)L->n * sizeof(double), nsamples,
                                      cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) s = emu_cuda_fail(ctx, e, "copy Z");
  }
  cudaFreeAsync(Z, ctx->stream);
  return s;
}

extern "C" emu_status emu_sample_host(emu_ctx *ctx, const emu_mat *L, int nsamples, uint64_t seed,
                                      uint32_t stream_id, double *hY, long ldy) {
  if (!ctx || !L || !hY || nsamples < 0 || ldy < L->n) return EMU_EINVAL;
  if (nsamples == 0) return EMU_OK;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  double *Y = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&Y, (size_t)L->n * nsamples * sizeof(double), ctx->stream));
  emu_status s = emu_sample(ctx, L, nsamples, seed, stream_id, Y, L->n, nullptr);
  if (s == EMU_OK) {
    cudaError_t e = cudaMemcpy2DAsync(hY, ldy * sizeof(double), Y, (size_t)L->n * sizeof(double),
                                      (size_t)L->n * sizeof(double), nsamples,
                                      cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) s = emu_cuda_fail(ctx, e, "copy Y to host");
  }
  cudaFreeAsync(Y, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  return s;
}

// ------------------------------------------------------------------ solves
// Copies B (n rows) into a zero-padded npad-row buffer, solves there.
static emu_status potrs_padded(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs) {
  if (L->state == MAT_FACTOR64) return launch_potrs64(ctx, L, X, ldx, nrhs);
  return mixed_potrs(ctx, L, X, ldx, nrhs);
}

extern "C" emu_status emu_potrs(emu_ctx *ctx, const emu_mat *L, const double *dB, long ldb,
                                double *dX, long ldx, int nrhs) {
  if (!ctx || !L || !dB || !dX || nrhs < 0 || ldb < L->n || ldx < L->n) return EMU_EINVAL;
  if (L->state != MAT_FACTOR64 && L->state != MAT_FACTOR_MIXED)
    return fail_msg(ctx, EMU_ESTATE, "solve needs a factored matrix");
  if (L->cs) return fail_msg(ctx, EMU_ESTATE, "solves need the FP32-master storage (emu_cov_build)");
  if (nrhs == 0) return EMU_OK;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  long npad = (long)L->nt * L->nb;
  double *W = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&W, (size_t)npad * nrhs * sizeof(double), ctx->stream));
  cudaError_t e = cudaMemsetAsync(W, 0, (size_t)npad * nrhs * sizeof(double), ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(W, npad * sizeof(double), dB, ldb * sizeof(double),
                          (size_t)L->n * sizeof(double), nrhs, cudaMemcpyDeviceToDevice, ctx->stream);
  emu_status s = (e == cudaSuccess) ? potrs_padded(ctx, L, W, npad, nrhs) : emu_cuda_fail(ctx, e, "potrs copy-in");
  if (s == EMU_OK) {
    e = cudaMemcpy2DAsync(dX, ldx * sizeof(double), W, npad * sizeof(double),
                          (size_t)L->n * sizeof(double), nrhs, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) s = emu_cuda_fail(ctx, e, "potrs copy-out");
  }
  cudaFreeAsync(W, ctx->stream);
  return s;
}

extern "C" emu_status emu_solve_refine(emu_ctx *ctx, const emu_mat *L, const emu_mat *S,
                                       const double *dB, long ldb, double *dX, long ldx, int nrhs,
                                       double tol, int maxit, emu_refine_info *info) {
  if (!ctx || !L || !S || !dB || !dX || nrhs < 0 || ldb < L->n || ldx < L->n || maxit < 0 ||
      !(tol > 0.0))
    return EMU_EINVAL;
  if (S->state != MAT_COV || S->n != L->n || S->nb != L->nb)
    return fail_msg(ctx, EMU_ESTATE, "S must be the unfactored covariance with the factor's tiling");
  if (L->state != MAT_FACTOR64 && L->state != MAT_FACTOR_MIXED)
    return fail_msg(ctx, EMU_ESTATE, "refinement needs a factored matrix");
  if (L->cs || S->cs) return fail_msg(ctx, EMU_ESTATE, "refinement needs the FP32-master storage (emu_cov_build)");
  return refine_solve(ctx, L, S, dB, ldb, dX, ldx, nrhs, tol, maxit, info);
}
