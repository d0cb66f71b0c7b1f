// emu_internal.h -- internal types shared by the CUDA translation units of
// libemucov (context, tiled matrix, tile indexing, launch bookkeeping).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/emucov.h"

// ----------------------------------------------------------------- tiling
// Lower tiles (i >= j) of an NT x NT tiling are packed column by column:
// tile (i, j) has index j*NT - j*(j-1)/2 + (i - j).  Each tile is nb x nb,
// column-major (element (r, c) at r + c*nb).
__host__ __device__ inline long tile_index(int i, int j, int NT) {
  return (long)j * NT - (long)j * (j - 1) / 2 + (i - j);
}
__host__ __device__ inline void tile_coords(long t, int NT, int *i, int *j) {
  int jj = 0;
  long base = 0;
  while (base + (NT - jj) <= t) {
    base += NT - jj;
    jj++;
  }
  *j = jj;
  *i = jj + (int)(t - base);
}
inline long tile_count(int NT) { return (long)NT * (NT + 1) / 2; }

// Device status word written by kernels and read back at sync points.
enum { ST_CODE = 0, ST_PIVOT = 1, ST_AUX = 2, ST_WORDS = 4 };
enum { DEV_OK = 0, DEV_NOTPD = 1, DEV_TIMEOUT = 2 };

// Matrix states.
enum { MAT_COV = 0, MAT_FACTOR64 = 1, MAT_FACTOR_MIXED = 2 };

// Kernel groups timed by the optional per-launch profiler (emu_prof_*).
enum {
  PROF_COV = 0, PROF_MAP, PROF_POTRF, PROF_TRSM64, PROF_TRSM32, PROF_UPDATE64,
  PROF_TC_FACTOR, PROF_TC_SAMPLE, PROF_TRMM64, PROF_RNG, PROF_SPLIT, PROF_SOLVE,
  PROF_NGROUPS
};

struct ProfRec {
  cudaEvent_t a, b;
  cudaStream_t stream;
  int group;
  uint64_t launches0;
  double flops, bytes, mma_flops;
};

struct emu_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int *d_status = nullptr;    // ST_WORDS ints
  int *h_status = nullptr;    // pinned mirror
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  uint64_t launches = 0;       // kernels of this library, graph nodes included
  uint64_t host_launches = 0;  // launch calls the host made (a graph replay counts once)
  std::string last_error;
  bool prof = false;
  std::vector<ProfRec> prof_open;   // recorded, not yet collected
  std::vector<cudaEvent_t> ev_pool;  // reusable events
  int prof_launches[PROF_NGROUPS] = {};
  double prof_ms[PROF_NGROUPS] = {}, prof_flops[PROF_NGROUPS] = {}, prof_bytes[PROF_NGROUPS] = {};
  double prof_mma[PROF_NGROUPS] = {};
  cudaEvent_t prof_base = nullptr;  // recorded when profiling is enabled
  struct TimelineRec {
    int group;
    cudaStream_t stream;
    double t0, t1;  // ms after prof_base
  };
  std::vector<TimelineRec> timeline;
  // mixed factor schedule: high-priority stream for the critical path
  // (POTRF, TRSM, next-column update), low-priority stream for the bulk
  // trailing update, and events ordering them
  cudaStream_t crit = nullptr, mid = nullptr, bulk = nullptr;
  std::vector<cudaEvent_t> sched_ev;
  // host imports: copy stream and its ordering events (allocation, copied[2],
  // staging buffer free[2]), created on first use
  cudaStream_t xfer = nullptr;
  cudaEvent_t xev[5] = {};
  // dataflow POTRF of a diagonal tile: task list and workspace (per nb)
  void *dag_tasks = nullptr;
  int *dag_ws = nullptr;
  size_t dag_ws_bytes = 0;
  int dag_ntasks = 0, dag_nbb = 0;
  // 1: the single-tile POTRF runs its chain on a cluster of three CTAs; 0: on
  // one CTA (clusters of this kernel cannot be resident); -1: not yet probed
  int dag_clus = -1;
  // batched factor (batch.cu): arenas, plan and captured graph of the last batch
  void *batch = nullptr;
  // single-matrix mixed factor (mixed.cu): captured graph, tuning table
  void *mixed = nullptr;
  // optional device-side task trace of the dataflow POTRF
  bool trace_on = false;
  unsigned long long *trace_buf = nullptr;
  size_t trace_cap = 0, trace_records = 0;
};

// Brackets the launches issued during its lifetime with CUDA events on the
// context stream when profiling is on; `flops` / `bytes` are the algorithmic
// work of those launches, `mma_flops` the tensor-core multiply-adds they
// execute (x2), split products included.
struct ProfScope {
  emu_ctx *ctx;
  ProfRec rec;
  bool on;
  ProfScope(emu_ctx *c, int group, double flops = 0.0, double bytes = 0.0, double mma_flops = 0.0);
  ~ProfScope();
};

// Class-format storage (classfmt.cu): every tile in the format of its
// precision class, column-major nb x nb, in the arena of its class at index
// slot[tile]; diagonal tiles are FP64.  E4M3 entries are codes q of the value
// q / sc8[slot].
struct ClassStore {
  std::vector<unsigned char> cls;  // per tile (TF32 is stored as FP32)
  std::vector<int> slot;           // per tile
  int nslot[EMU_NCLASS] = {};
  int *d_slot = nullptr;
  double *t64 = nullptr;
  float *t32 = nullptr;
  uint16_t *t16 = nullptr;
  uint8_t *t8 = nullptr;
  float *sc8 = nullptr;
  void *work = nullptr;            // factor plan (classfmt.cu)
  bool samp_ready = false;         // sampler digit slices of the FP64 tiles made
  uint16_t *samp_dig = nullptr;
  int *samp_exp = nullptr;
};
// Device pointers of the class arenas, for the class-format covariance store.
struct ClassArenas {
  const int *slot;
  const unsigned char *cls;
  double *t64;
  float *t32;
  uint16_t *t16;
  uint8_t *t8;
  const float *sc8;
};

struct emu_mat {
  emu_ctx *ctx = nullptr;
  int n = 0, nb = 0, nt = 0;
  int state = MAT_COV;
  long ntiles = 0;
  size_t tile_elems = 0;       // nb*nb
  double *t64 = nullptr;       // FP64 arena: ntiles tiles
  float *t32 = nullptr;        // FP32 master arena (mixed factor), ntiles tiles
  // norm pass: per-tile partial sums of squares, tile norms, classes
  int nchunk = 0;              // column chunks per tile (nb / 32)
  double *d_partial = nullptr; // ntiles * nchunk
  double *d_tnorm = nullptr;   // ntiles
  double *d_frob = nullptr;    // 1
  unsigned char *d_cls = nullptr; // ntiles
  unsigned char *h_cls = nullptr; // ntiles (host copy, valid for mixed)
  double frob = 0.0;
  // mixed factor operand copies (three BF16 pieces per tile, row-major)
  uint16_t *op_bf16 = nullptr; // ntiles * 3 * nb*nb
  uint8_t *op_e4m3 = nullptr;  // ntiles * nb*nb FP8-E4M3 copies (row-major), when E4M3 tiles exist
  float *scale_e4m3 = nullptr; // ntiles power-of-two scales of those copies
  float *op_tf32 = nullptr;     // ntiles * nb*nb TF32 copies (row-major), when TF32 tiles exist
  void *plan = nullptr;        // mixed-factor schedule (mixed.cu)
  ClassStore *cs = nullptr;    // class-format storage (t64 / t32 / op unused)
};

// ------------------------------------------------------------- bookkeeping
emu_status emu_cuda_fail(emu_ctx *ctx, cudaError_t e, const char *what);
#define EMU_CUDA_TRY(ctx, expr)                                   \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return emu_cuda_fail((ctx), _e, #expr); \
  } while (0)
// After a launch: count it and surface launch-configuration errors.
#define EMU_LAUNCHED(ctx)                                                   \
  do {                                                                      \
    (ctx)->launches++;                                                      \
    (ctx)->host_launches++;                                                 \
    cudaError_t _e = cudaGetLastError();                                    \
    if (_e != cudaSuccess) return emu_cuda_fail((ctx), _e, "kernel launch"); \
  } while (0)

// Kernel attributes belong to the device's context: raise a kernel's dynamic
// shared-memory limit once per device (bit `device` of `done`), from any
// thread.  Devices beyond 63 set it on every call.
inline cudaError_t smem_limit_once(std::atomic<uint64_t> &done, int device, const void *func, int bytes) {
  uint64_t bit = (device >= 0 && device < 64) ? (1ull << device) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// ------------------------------------------------------------- batches
// One covariance of a batch (batch.cu): its tiles, rows and covariance tables
// sit at these offsets of the batch's shared arenas.
struct BatchInst {
  long tile_base;  // first tile (packed lower tiles, column by column)
  long row_base;   // first row of its padded block of the stacked Z and Y
  long tab_base;   // first entry of its correlation table (sigma and nugget follow)
  int L, n, NT, stream_id;
  double beta, sigma_exp, nugget_rel;
};

// Kernel launch wrappers (defined in the .cu files that own the kernels).
// cov.cu
emu_status launch_cov_build(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p);
// Class-format build (cov.cu): the norm partials without storing any tile;
// then every tile stored in its class's arena.  Tables: rho, sigma, nugget.
emu_status launch_cov_norms(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p);
emu_status launch_cov_store_class(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p, const ClassArenas &ar);
emu_status launch_cov_tables(emu_ctx *ctx, const emu_cov_params *p, double *tables);
emu_status launch_import(emu_ctx *ctx, emu_mat *A, const double *dA, long lda);
// Empirical covariance: scale the raw sums by 1/m, nugget, padding, norms (cov.cu).
emu_status launch_emp_finish(emu_ctx *ctx, emu_mat *A, long m, double nugget_rel, unsigned long long *d_maxbits);
emu_status launch_import_col(emu_ctx *ctx, emu_mat *A, int tj, const double *dS, long ld);
emu_status launch_precision_map(emu_ctx *ctx, emu_mat *A, double eps,
                                const double *u, unsigned mask, int diag_fp64, int band, double sp_frac);
// sp_frac of a band map: 0 means the paper's 5 %
inline double band_sp_frac(const emu_mp_opts *o) { return o->sp_frac == 0.0 ? 0.05 : o->sp_frac; }
emu_status launch_export(emu_ctx *ctx, const emu_mat *A, double *dOut, long ld);
// fp64.cu
emu_status launch_potrf64_tile(emu_ctx *ctx, emu_mat *A, int k);
// Task list and workspace of the dataflow POTRF for tile size nb (allocated on
// first use; called before any stream capture).
emu_status potrf_dag_prepare(emu_ctx *ctx, int nb);
// The same on the tile at D (nb x nb, column-major), step k (pivot columns k nb + ..).
emu_status launch_potrf64_ptr(emu_ctx *ctx, double *D, int nb, int k);
// Test hook of the timeout path (emu_test_wait_hook).
emu_status set_dag_wait_hook(emu_ctx *ctx, long long wait_cycles, int withhold_index);
// d_rows: device list of the tile rows i > k to solve (nullptr: all of them)
emu_status launch_trsm64_panel(emu_ctx *ctx, emu_mat *A, int k, const int *d_rows = nullptr, int nrows = 0,
                               const double *Ls = nullptr, const double *rinvs = nullptr);
// Pre-scaled 32x32 diagonal blocks of FP64 factor tiles (nb x nb,
// column-major) for the FP64 panel TRSM: slot z of Ls[n][nb * 32] and
// rinvs[n][nb] from tile d_tiles[z] of the arena L (or L itself, n = 1, when
// d_tiles is null).
emu_status launch_trsm64_prep(emu_ctx *ctx, const double *L, int nb, double *Ls, double *rinvs,
                              const long *d_tiles = nullptr, int n = 1);
emu_status launch_update64(emu_ctx *ctx, emu_mat *A, int k);
emu_status launch_tril_diag(emu_ctx *ctx, emu_mat *A);
// cls != nullptr: only the FP64-class tiles contribute (mixed factors)
emu_status launch_trmm64(emu_ctx *ctx, const emu_mat *L, const double *Z,
                         long ldz, int s, double *Y, long ldy,
                         const unsigned char *cls = nullptr);
emu_status launch_potrs64(emu_ctx *ctx, const emu_mat *L, double *X, long ldx,
                          int nrhs);
// rng.cu
emu_status launch_normals(emu_ctx *ctx, uint64_t seed, uint32_t stream_id,
                          int nrows, int s, double *Z, long ldz);
// batched kernels over explicit tile indices (batch.cu drives them)
emu_status launch_cov_build_batch(emu_ctx *ctx, const BatchInst *d_inst, int count, int maxL, long ntab,
                                  const int *d_tile_inst, long ntiles, int nb, double *tables, double *t64,
                                  double *partial);
emu_status launch_precision_map_batch(emu_ctx *ctx, const BatchInst *d_inst, int count, int nb, double *partial,
                                      double *tnorm, double *frob, unsigned char *cls, double eps,
                                      const double *u, unsigned mask, int diag_fp64, int band, double sp_frac);
emu_status launch_export_batch(emu_ctx *ctx, const BatchInst *d_inst, const int4 *d_pairs, long npairs, int nb,
                               const double *t64, const float *t32, const unsigned char *cls,
                               double *const *d_out);
emu_status launch_normals_batch(emu_ctx *ctx, const uint64_t *d_seed, const BatchInst *d_inst, int count,
                                int maxNT, int nb, int s, double *Z, long ldz);
// jobs {tile (i,k), tile (k,k)}; with Ls / rinvs, job j's L_kk is pre-scaled in slot d_jslots[j]
emu_status launch_trsm64_jobs(emu_ctx *ctx, double *t64, int nb, const int2 *d_jobs, int njobs,
                              const double *Ls = nullptr, const double *rinvs = nullptr,
                              const int *d_jslots = nullptr);
emu_status launch_to_f32_tiles(emu_ctx *ctx, const double *t64, float *t32, const unsigned char *cls, long ntiles,
                               size_t te);
emu_status launch_tiles_to_f64(emu_ctx *ctx, const float *t32, double *t64, const long *d_tiles, int n, size_t te);
emu_status launch_diag_to_f32_slots(emu_ctx *ctx, const double *t64, float *slots, const long *d_tiles, int n,
                                    size_t te);
emu_status launch_trsm32_jobs(emu_ctx *ctx, const float *slots, float *t32, uint16_t *op, int nb, const int2 *d_jobs,
                              int njobs);
emu_status launch_split_tiles64(emu_ctx *ctx, const double *t64, uint16_t *op, const int *d_tiles, int n, int nb,
                                int lower_only);
emu_status launch_quant_e4m3(emu_ctx *ctx, const uint16_t *op, uint8_t *op8, float *scales, const int *d_tiles, int n,
                             int nb);
emu_status launch_split_z(emu_ctx *ctx, const double *Z, long ldz, long npad, int s, int s_pad, uint16_t *zp);
size_t potrf_dag_task_count(int nb);
emu_status potrf_dag_tasks_upload(emu_ctx *ctx, int nb, void *d_tasks, cudaStream_t s);
size_t potrf_batch_ws_ints(int nb, int nbat);
// bad: nbat ints, zero before the launch; a tile whose factor meets a
// non-positive pivot gets its 1-based global column there and the launch
// goes on (only that matrix is flagged)
emu_status launch_potrf64_batch(emu_ctx *ctx, double *t64, int nb, int k, const long *d_tiles, int nbat,
                                const void *d_tasks, int ntasks, int *ws, double *rinv, int *bad);
