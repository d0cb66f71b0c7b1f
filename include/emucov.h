/*
 * emucov.h -- C ABI of the GB300 (sm_103a) covariance-factorisation library
 * for spherical-harmonic climate emulators (arXiv 2408.04440).
 *
 * What the library computes (paper sections):
 *   - "Modeling the Temporal Dependence and Constructing a Covariance Matrix":
 *     the L^2 x L^2 covariance U-hat of the spherical-harmonic coefficients,
 *     made positive definite by a small diagonal perturbation, and its
 *     Cholesky factor U-hat = V V^T (the O(L^6) step).
 *   - "Advancements in Dense Linear Algebra" and "Mixed-Precision Computation
 *     Innovations": the factor is a tile algorithm (POTRF on diagonal tiles,
 *     TRSM on the panel, SYRK/GEMM on the trailing tiles) in which each tile
 *     runs in its own precision.
 *   - "Performance of Mixed-Precision Cholesky on Summit": a panel tile is
 *     converted once, by its producer, into the precision of its consumers.
 *   - "Generating Emulations": draws xi = V z with z ~ N(0, I).
 *
 * Conventions shared by every entry point:
 *   - Matrices are indexed from 0.  Dense arrays passed in or out are FP64,
 *     column-major, with a leading dimension `ld` >= number of rows, and live
 *     in DEVICE memory unless a parameter says "host".
 *   - The library owns `emu_ctx` and `emu_mat` objects; they are released only
 *     by emu_destroy / emu_mat_free.  A matrix keeps a pointer to the context
 *     it was made in: free every matrix before destroying that context.
 *     Caller pointers are borrowed for the duration of the call and of the
 *     stream work it enqueues.
 *   - All device work is enqueued on the context's stream (the one given to
 *     emu_create; NULL = the legacy default stream).  Calls that fill an
 *     `info` struct, or that return a status decided on the device
 *     (EMU_ENOTPD, EMU_ETIMEOUT, EMU_ENOCONV), synchronise that stream.
 *   - Every call returns an emu_status.  No exception or signal crosses the
 *     ABI.  On EMU_ECUDA the CUDA error string is kept in the context
 *     (emu_last_error).  Arguments are validated on the host before any launch.
 *   - The library runs on one GPU, the device given to emu_create, which must
 *     be an sm_103 (GB300) device.
 */
#ifndef EMUCOV_H
#define EMUCOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EMU_OK = 0,
  EMU_EINVAL = 1,   /* bad argument (checked on the host)                    */
  EMU_ENOMEM = 2,   /* device allocation failed or a size limit was exceeded */
  EMU_ENOTPD = 3,   /* factor met a non-positive pivot; see info->pivot      */
  EMU_ENOCONV = 4,  /* refinement did not reach tol within maxit             */
  EMU_ETIMEOUT = 5, /* a bounded device wait expired                         */
  EMU_ECUDA = 6,    /* CUDA runtime/driver error; see emu_last_error         */
  EMU_ESTATE = 7    /* matrix in the wrong state for this call               */
} emu_status;

/* Precision classes of a tile, most precise first.  The unit roundoff u that
 * the precision rule uses for each class is in emu_mp_opts.u (defaults:
 * 2^-53, 2^-24 * sqrt(nb), 2^-11, 2^-8, 2^-4).  "fp32" is computed on the
 * tensor cores as a three-way BF16 split of each operand (six partial
 * products, FP32 accumulation); its default u carries the sqrt(nb) growth of
 * the error of an nb-term FP32 accumulation relative to the tile norm.
 * "e4m3" carries a power-of-two scale per tile. */
enum {
  EMU_CLASS_FP64 = 0,
  EMU_CLASS_FP32 = 1,
  EMU_CLASS_TF32 = 2,
  EMU_CLASS_BF16 = 3,
  EMU_CLASS_E4M3 = 4,
  EMU_NCLASS = 5
};

typedef struct emu_ctx emu_ctx;
typedef struct emu_mat emu_mat;

/* Synthetic covariance of the spherical-harmonic coefficients, a stand-in for
 * the empirical U-hat ("Modeling the Temporal Dependence ...", equation for
 * U-hat, and the diagonal perturbation that follows it).  Row k holds the
 * coefficient (l, m), k = l^2 + l + m, 0 <= l < L, |m| <= l, n = L^2:
 *   S[i,j] = s(l_i) s(l_j) exp(-sqrt((l_i-l_j)^2 + (m_i-m_j)^2) / beta),
 *   s(l) = (1 + l)^(-sigma_exp),   S[k,k] += nugget_rel * max_k S[k,k].
 * nugget_rel is finite and > -1; a negative value shifts the diagonal down,
 * and S may then not be positive definite (the factor reports EMU_ENOTPD with
 * the first non-positive pivot). */
typedef struct {
  int L;
  double beta;
  double sigma_exp;
  double nugget_rel;
} emu_cov_params;

/* Band-based precision maps of the paper's experiments ("Performance
 * Results": DP, DP/SP, DP/SP/HP with 5 % SP, DP/HP), with SP the "fp32" class
 * and HP the "bf16" class.  In every map the diagonal band (tiles i == j) is
 * FP64.  DP/SP: all other tiles fp32.  DP/HP: all other tiles bf16.
 * DP/SP/HP: the sub-diagonal bands i - j = 1 .. b are fp32 and the rest bf16,
 * b the fewest whole bands that hold at least sp_frac of the NT(NT+1)/2
 * tiles (sp_frac == 0 means 0.05; sp_frac < 0 gives b = 0). */
enum {
  EMU_MAP_NORM = 0,     /* the per-tile norm rule (eps, prec_mask, u) */
  EMU_MAP_DP_SP = 1,
  EMU_MAP_DP_SP_HP = 2,
  EMU_MAP_DP_HP = 3
};

/* Options of the factorisation ("Mixed-Precision Computation Innovations").
 * With band = EMU_MAP_NORM: eps <= 0 selects the plain FP64 tile Cholesky;
 * eps > 0 selects the adaptive per-tile precision: tile (i,j) runs in the
 * least precise class c allowed by prec_mask for which
 * ||S_ij||_F * u[c] <= eps * ||S||_F / NT (NT = number of tile rows, ||S||_F
 * over the full symmetric matrix); FP64 when none passes.  diag_fp64 != 0
 * also pins the diagonal tiles' storage and updates to FP64.  u[c] <= 0 takes
 * the default.  band = EMU_MAP_DP_SP .. EMU_MAP_DP_HP selects a band map
 * instead (eps, prec_mask, diag_fp64 and u are then not used; sp_frac == 0
 * means 0.05).  The diagonal POTRF is always FP64. */
typedef struct {
  double eps;
  unsigned prec_mask; /* bit c enables class c; bit 0 (FP64) is implied */
  int diag_fp64;
  double u[EMU_NCLASS];
  int band;           /* EMU_MAP_* */
  double sp_frac;     /* DP/SP/HP: least fraction of the tiles in fp32 bands */
} emu_mp_opts;

typedef struct {
  int n, nb, nt;
  int pivot;                  /* EMU_ENOTPD: 1-based global column, else 0  */
  int tiles[EMU_NCLASS];      /* lower tiles per class                      */
  double update_flops[EMU_NCLASS]; /* SYRK/GEMM/TRSM flops per class        */
  double frob;                /* ||S||_F of the input (0 for plain FP64)    */
  double ms;                  /* device time of the factor, CUDA events     */
} emu_factor_info;

typedef struct {
  int iters;        /* refinement corrections applied                       */
  double rel_resid; /* at exit, max over columns of the normwise backward
                       error ||b - S x||_2 / (||S||_F ||x||_2 + ||b||_2)     */
  double ms;
} emu_refine_info;

/* ---------------------------------------------------------------- context */
/* Create a context on `device` that enqueues on `stream` (a cudaStream_t;
 * NULL = legacy default stream).  Fails with EMU_EINVAL when the device is
 * not sm_103. */
emu_status emu_create(emu_ctx **ctx, int device, void *stream);
emu_status emu_destroy(emu_ctx *ctx);
emu_status emu_set_stream(emu_ctx *ctx, void *stream);
const char *emu_status_str(emu_status s);
const char *emu_last_error(const emu_ctx *ctx);
/* Number of this library's kernels launched through `ctx` so far (the kernels
 * of a replayed CUDA graph included). */
uint64_t emu_launch_count(const emu_ctx *ctx);
/* Number of launch calls the host made through `ctx` so far: kernel launches
 * issued one by one, plus one per CUDA graph replay. */
uint64_t emu_host_launch_count(const emu_ctx *ctx);

/* Optional per-kernel-group timing, for roofline accounting.  When enabled,
 * every group of launches is bracketed by CUDA events on the context stream
 * (which adds a small gap between launches).  emu_prof_enable resets the
 * counters; emu_prof_read synchronises the stream and returns, for `group`
 * (EMU_PROF_*), the launches, their total device time, their algorithmic
 * flops and bytes, and the tensor-core flops they executed (split products
 * included). */
enum {
  EMU_PROF_COV = 0, EMU_PROF_MAP, EMU_PROF_POTRF, EMU_PROF_TRSM64, EMU_PROF_TRSM32,
  EMU_PROF_UPDATE64, EMU_PROF_TC_FACTOR, EMU_PROF_TC_SAMPLE, EMU_PROF_TRMM64,
  EMU_PROF_RNG, EMU_PROF_SPLIT, EMU_PROF_SOLVE, EMU_PROF_NGROUPS
};
emu_status emu_prof_enable(emu_ctx *ctx, int on);
/* Timeline of the profiled kernel groups since emu_prof_enable: four doubles
 * per record (group, stream: 0 = context stream, 1 = critical, 2 = panel,
 * 3 = bulk stream of the mixed factor, start ms, end ms, both relative to the
 * enable call).  Reports the number of records in *n_records. */
emu_status emu_prof_timeline(emu_ctx *ctx, double *h_out, size_t max_records,
                             size_t *n_records);
/* Device-side task trace of the dataflow FP64 POTRF of the diagonal tiles
 * (off by default).  While enabled, each factor records, for every task of
 * every diagonal tile (tile k's records follow tile k-1's), five 64-bit words:
 * kind | r << 8 | c << 24 | s << 40 (kind 0 = leaf with its sub-diagonal
 * solve, 1 = TRSM, 2 = update of
 * 16x16 block (r,c) by panel s), the SM id, and %globaltimer nanoseconds when
 * the task was fetched, when its inputs were ready, and when it completed.
 * The master CTA's records (one per 16-column step, after the tile's task
 * records) hold the step's start, the end of its leaf and its end; their
 * second word packs the SM id (bits 0-7) with three saturated durations in SM
 * clock cycles: the leaf (bits 8-25), the wait for the next sub-diagonal
 * block after it (bits 26-44) and the whole step (bits 45-63).  (When the
 * chain runs on one CTA because clusters of three cannot be resident, the
 * second word holds the solve of block (s, s-1) and the compute warps' second
 * phase instead, and the middle timestamp ends the solve.)  In the cluster
 * form the first helper's records follow (kind 5, one per step s < nb/16 - 1):
 * r = s+1, c = s, the start of its step, the arrival of its inputs
 * (X_{s+1,s-1} and block (s+1, s)) and the time its part of
 * X_{s+1,s} X_{s+1,s}^T was sent and X_{s+1,s} published; the second word
 * packs the SM id with the nanoseconds from the inputs to the end of the
 * solve (bits 8-25).  Then the
 * second helper's (kind 6, one per step s < nb/16 - 2): r = s+2, c = s, the
 * start of its step, the arrival of X_{s+2,s-1} and X_{s,s-1} (its update by
 * panel s-1), the publication of X_{s+2,s}, and in the second word the
 * nanoseconds from that arrival to the end of its solves.
 * emu_trace_read copies up to max_records records to host memory and reports
 * how many the last factor wrote. */
emu_status emu_trace_enable(emu_ctx *ctx, int on);
emu_status emu_trace_read(emu_ctx *ctx, uint64_t *h_records, size_t max_records,
                          size_t *n_records);
/* The task list of the dataflow POTRF of one nb x nb FP64 diagonal tile (the
 * "POTRF on the diagonal tile" step of the tile Cholesky), in the order the
 * kernel's CTAs fetch it.  Host only: no device work, no context.  Four
 * int16 per task: kind (0 = step s of the chain: solve block (s, s-1) against
 * L_{s-1,s-1}, update and factor block (s, s); 1 = TRSM of block (r, c)
 * against L_cc after applying panel c-1; 2 = update of block (r, c) by panel
 * s; 3 = the single-tile master that runs every step of the chain), r, c, s
 * (16x16 blocks).  No task applies panel s to blocks (s+1, s+1) and
 * (s+2, s+1): the chain does.  single_tile = 1 gives the list of the
 * single-matrix factor whose chain runs on one CTA (one master task at the
 * head), 2 the list when the chain runs on a cluster of three CTAs (the head
 * task is not fetched, and the chain also solves blocks (c+2, c) and applies
 * panel s to block (s+2, s+2)), 0 the batch form (one kind-0 task per step).  Writes min(n, max_tasks) tasks to h_tasks (may be
 * NULL with max_tasks 0) and n to *n_tasks.  EMU_EINVAL unless nb is a
 * positive multiple of 16 no larger than 2048. */
emu_status emu_potrf_task_list(int nb, int single_tile, int16_t *h_tasks, size_t max_tasks, size_t *n_tasks);
/* Schedule of the single-matrix mixed factor (FP32-master storage).  With
 * use_graphs != 0 (the default) the launches after the precision map are
 * recorded once into a CUDA graph over the factor's four streams and replayed
 * while the map, the tiling and the arenas' addresses stay the same (one host
 * launch per factor; profiling or tracing turns replay off).  With
 * tuning != 0 (the default) the first factors of each (NT, nb, class map)
 * each try one of four counts of SMs left free of the bulk trailing update
 * (16/32, 8/16, 24/48, 32/64, without/with FP64-class panel work near), timed
 * on the device; later factors use the fastest.  Every choice gives the same
 * factor bit for bit. */
emu_status emu_schedule(emu_ctx *ctx, int use_graphs, int tuning);
/* The tuner's state for the last signature factored: choices timed so far
 * (0..4), and the SMs left free without / with FP64-class panel work in the
 * choice the next factor of that signature uses.  All 0 before any mixed
 * factor. */
emu_status emu_schedule_info(emu_ctx *ctx, int *tried, int *reserved, int *reserved_fp64);

/* Measured FMA rates of the context's device, in TFLOP/s (2 flops per FMA):
 * eight independent FP64 (FP32) FMA chains per thread, eight CTAs of 256
 * threads per SM, timed with CUDA events; the denominators of the rooflines of
 * the kernels bound by plain FP64 or FP32 arithmetic.  Synchronises. */
emu_status emu_measure_alu_peaks(emu_ctx *ctx, double *fp64_tflops, double *fp32_tflops);

/* Test hook of the timeout path (failure detection; the paper has no
 * counterpart).  Every wait of the dataflow FP64 diagonal POTRF on another
 * task's flag is bounded; this sets that bound, in SM clock cycles, for every
 * context on ctx's device (wait_cycles <= 0 restores the default, about 2 s)
 * and names one flag that every such wait treats as never set:
 * withhold_index = r * (nb / 16) + c for the 16 x 16 block (r, c) of a
 * diagonal tile, -1 for none.  A factor that meets a withheld flag returns
 * EMU_ETIMEOUT once the bound runs out: the waiting kernel records the
 * timeout in the status word and returns, the others see the status and
 * leave, and the context stays usable.  Synchronises the device.  For tests
 * of failure detection only. */
emu_status emu_test_wait_hook(emu_ctx *ctx, long long wait_cycles, int withhold_index);
emu_status emu_prof_read(emu_ctx *ctx, int group, int *launches, double *total_ms,
                         double *flops, double *bytes, double *mma_flops);

/* ---------------------------------------------------------------- matrices */
/* Build the synthetic covariance on the device as an n x n tiled matrix with
 * tile size nb (n = L^2).  The lower tiles are stored packed, each tile
 * nb x nb column-major in FP64; a ragged last tile row is padded with zeros
 * and a unit diagonal, which the factor carries through as an identity block.
 * The per-tile Frobenius norms are computed in the same pass. */
emu_status emu_cov_build(emu_ctx *ctx, const emu_cov_params *p, int nb,
                         emu_mat **out);
/* Import a user covariance: dA is n x n FP64 column-major on the device, only
 * its lower triangle is read. */
emu_status emu_mat_import(emu_ctx *ctx, const double *dA, int n, long lda,
                          int nb, emu_mat **out);
/* Same from HOST memory hA (pinned memory gives full copy bandwidth): only
 * the lower triangle is copied, one tile column at a time, through a device
 * staging buffer of n x nb doubles.  The call synchronises the stream before
 * returning, so hA may be reused at once. */
emu_status emu_mat_import_host(emu_ctx *ctx, const double *hA, int n, long lda,
                               int nb, emu_mat **out);
/* Empirical covariance of residual vectors ("Modeling the Temporal
 * Dependence", the estimate U-hat and the diagonal perturbation after it):
 *   U[i,j] = (1/m) sum_t Xi[i,t] Xi[j,t],   U[k,k] += nugget_rel * max_k U[k,k],
 * Xi: device, column-major n x m (leading dimension ldxi >= n), one residual
 * vector per column (m = R (T - P) in the paper); read only during the call.
 * The paper adds the perturbation when m < n; pass nugget_rel = 0 for none.
 * The lower tiles are formed on the tensor cores with FP64 accuracy (exact
 * digit products of the rows, accumulated exactly in fixed point and rounded
 * once to FP64), then scaled; the result is
 * a matrix in the state emu_cov_build leaves (tiles, tile norms, ||U||_F).
 * nb must be a multiple of 256.  EMU_EINVAL on bad arguments, EMU_ENOMEM if
 * the tile arena does not fit, EMU_ETIMEOUT if a bounded device wait expired. */
emu_status emu_cov_from_residuals(emu_ctx *ctx, const double *dXi, int n, long m, long ldxi,
                                  double nugget_rel, int nb, emu_mat **out);
/* The steps after sampling that turn draws into emulations ("Generating
 * Emulations").  Coefficients are real-form, row k = l^2 + l + m as in
 * emu_cov_params, one time step per column (column-major, device memory).
 *
 * emu_var_recursion: the VAR(P) recursion with diagonal Phi_p ("Modeling the
 * Temporal Dependence"), f_t = sum_{p=1..P} Phi_p f_{t-p} + xi_t for
 * t = 0 .. T-1 with f before t = 0 taken as zero.  Xi: n x T (ld ldxi);
 * Phi: n x P (the diagonal of Phi_p in column p-1); F: n x T (ld ldf), may
 * not overlap Xi.  0 <= P <= 8.
 *
 * emu_isht: the inverse spherical-harmonic transform of each column of F
 * (n = L^2, ld ldf) to a grid of ntheta colatitudes t_i = pi i/(ntheta-1)
 * (poles included) by nphi longitudes p_j = 2 pi j/nphi:
 *   Z[i + j ntheta, t] = sum_{l<L, |m|<=l} F[l^2+l+m, t] Y_lm(t_i, p_j)
 * with the real orthonormal basis Y_l0 = N_l0 P_l(cos t),
 * Y_lm = sqrt(2) N_lm P_l^m(cos t) cos(m p), Y_l,-m = sqrt(2) N_lm P_l^m(cos t) sin(m p)
 * (m > 0), N_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!, P_l^m with the
 * Condon-Shortley phase.  Z: ld ldz >= ntheta nphi.  1 <= L <= 2048.
 * Both return EMU_EINVAL on bad arguments and synchronise the stream. */
emu_status emu_var_recursion(emu_ctx *ctx, const double *dXi, int n, int T, long ldxi, const double *dPhi, int P,
                             double *dF, long ldf);
emu_status emu_isht(emu_ctx *ctx, const double *dF, int L, int T, long ldf, int ntheta, int nphi, double *dZ,
                    long ldz);
/* emu_sht: the forward transform of grid data Z (layout of emu_isht) to the
 * real-form coefficients F (L^2 x T, ld ldf), by the paper's method
 * ("Spherical Harmonic Transform"): the integral in longitude by a DFT
 * (C_m, S_m), the extension of each to the full circle in colatitude
 * (g(2 pi - t) = (-1)^m g(t)), its Fourier coefficients K_q, and their
 * contraction with S_{l,m,q} = sum_q' c_{l,m,q'} I(q + q'), c the Fourier
 * coefficients of the extended Legendre factor of Y_lm and
 * I(k) = int_0^pi e^{ikt} sin t dt.  Exact for data band-limited at L when
 * ntheta > L and nphi >= 2L - 1 (the synthesis of emu_isht is then inverted).
 * Shared-memory bound: (4 (2L-1) + ntheta) doubles <= 48 KB; EMU_EINVAL
 * beyond it. */
emu_status emu_sht(emu_ctx *ctx, const double *dZ, int ntheta, int nphi, int T, long ldz, int L, double *dF,
                   long ldf);

/* emu_emulate_grid: the last step of "Generating Emulations" and Eq.
 * decouple ("Climate Emulator Design -- Formulation"): from the synthesis Zs
 * of emu_isht (G grid points x T time steps, ld ldz, device) it forms, for
 * t = 1..T (column t-1),
 *   Z_t(g) = Zs_t(g) + v(g) e_t(g)        (the nugget eps_t ~ N(0, v^2)),
 *   y_t(g) = m_t(g) + sigma(g) Z_t(g),
 * into Y (G x T, ld ldy, device; Y == Zs with ldy == ldz is allowed, other
 * overlaps are not).  e_t(g) is the library's standard normal of row g and
 * column t-1 for (seed, stream_id) (the generator of emu_sample).  The mean
 * trend is the paper's distributed-lag model of the forcing x plus K
 * harmonics:
 *   m_t = beta0 + beta1 x_y + beta2 (1 - rho) sum_{s>=1} rho^(s-1) x_(y-s)
 *         + sum_{k=1..K} a_k cos(2 pi t k / tau) + b_k sin(2 pi t k / tau),
 * y = ceil(t / tau), with every year before the trajectory taken at x[0].
 * Per-point parameters beta0, beta1, beta2, rho (rho in [0, 1]), sigma and v
 * are device arrays of length G; a and b are K x G (amplitude k of point g at
 * [k-1 + g K]).  The paper fits these parameters to data; the library takes
 * them as given.  Returns EMU_EINVAL for bad arguments (K > 8, tau <= 0,
 * nyears < ceil(T / tau), G > 2^31 - 1) and synchronises the stream. */
typedef struct emu_trend {
  int K;                 /* harmonic pairs, 0..8 */
  double tau;            /* period of the harmonics in time steps (12, 365, 8760 ...) */
  const double *beta0;   /* intercept, G */
  const double *beta1;   /* slope on the current forcing, G */
  const double *beta2;   /* slope on the lagged forcing, G */
  const double *rho;     /* lag decay in [0, 1], G */
  const double *a, *b;   /* K x G cosine / sine amplitudes; NULL when K = 0 */
  const double *x;       /* forcing x[0..nyears] (device); x[0] also stands for earlier years */
  int nyears;
} emu_trend;
emu_status emu_emulate_grid(emu_ctx *ctx, const double *dZs, long G, int T, long ldz, const emu_trend *m,
                            const double *dsigma, const double *dv, uint64_t seed, uint32_t stream_id, double *dY,
                            long ldy);

/* -------------------------------------------- class-format tile storage */
/* emu_cov_build_classfmt: the synthetic covariance of emu_cov_build stored
 * tile by tile in the format of its precision class ("Mixed-Precision
 * Computation Innovations": tiles allocated at the size of their precision),
 * for covariances whose FP64 lower triangle does not fit the device.  The
 * precision map is computed first from a norm pass that stores nothing (the
 * rule of emu_mp_opts o; every diagonal tile FP64; TF32 is stored as FP32),
 * then every tile is computed again and stored: FP64 8 bytes, FP32 4, BF16 2
 * (nearest); E4M3-class tiles take 2 bytes per entry and hold BF16 values
 * while they are trailing tiles of the factor.  nb must be a multiple of 256.
 * emu_potrf_mp factors such a matrix in place with this map (o is not read):
 * each trailing update is accumulated in FP32 on the tensor cores and the tile
 * is re-rounded to its working format (FP32 or BF16); each panel is decoded,
 * solved as in the FP32-master factor and rounded to its class (E4M3 tiles to
 * codes of x s, s = 2^floor(log2(448 / amax)) per tile, stored in the first
 * byte of each entry's slot), and the operands of later updates are made from
 * the rounded values.  emu_sample, emu_mat_export,
 * emu_mat_tile_info and emu_backward_error_est accept it; emu_potrs,
 * emu_solve_refine and emu_mat_clone return EMU_ESTATE.  Device memory:
 * about the stored bytes plus, while factoring, a ring of three panels
 * (FP64 + FP32 + three BF16 pieces + FP8 + eight digit planes per tile of a
 * tile column, about 35 bytes per element of nb x NT rows). */
emu_status emu_cov_build_classfmt(emu_ctx *ctx, const emu_cov_params *p, int nb, const emu_mp_opts *o,
                                  emu_mat **out);
/* emu_backward_error_est: an estimate of ||L L^T - S||_F / ||S||_F for a
 * factor L of the covariance with parameters p, without S in memory (the
 * randomised trace estimate of Hutchinson): with nprobes Gaussian probe
 * columns G (the library's normals for `seed`, stream id 7),
 * ||(L L^T - S) G||_F^2 / nprobes estimates ||L L^T - S||_F^2; L^T G and
 * L (L^T G) are computed from the stored tiles and S G from p (the entries
 * regenerated as the builder computes them), all in FP64.  Any storage.
 * Relative spread of the estimate about sqrt(2 / nprobes). */
emu_status emu_backward_error_est(emu_ctx *ctx, const emu_mat *L, const emu_cov_params *p, int nprobes,
                                  uint64_t seed, double *est);

/* Deep copy (device to device), e.g. to keep S for emu_solve_refine. */
emu_status emu_mat_clone(emu_ctx *ctx, const emu_mat *A, emu_mat **out);
/* Write the matrix as a dense FP64 lower triangle (upper set to 0) into dOut
 * (n x n, column-major, device).  For a mixed factor each tile is widened
 * from its stored precision. */
emu_status emu_mat_export(emu_ctx *ctx, const emu_mat *A, double *dOut,
                          long ld);
/* Copy the per-tile precision classes (NT x NT column-major bytes, upper =
 * 255) and tile norms (NT x NT doubles, upper = 0) to HOST arrays; either
 * pointer may be NULL. */
emu_status emu_mat_tile_info(emu_ctx *ctx, const emu_mat *A,
                             unsigned char *h_cls, double *h_norms);
/* n, nb, NT and state (0 = covariance, 1 = FP64 factor, 2 = mixed factor). */
emu_status emu_mat_shape(const emu_mat *A, int *n, int *nb, int *nt,
                         int *state);
emu_status emu_mat_free(emu_mat *A);

/* ------------------------------------------------------------------ factor */
/* Factor A = L L^T in place (A must hold a covariance, state 0).  Plain FP64
 * when o == NULL or o->eps <= 0, otherwise the adaptive mixed-precision tile
 * factor described at emu_mp_opts.  On a non-positive pivot returns
 * EMU_ENOTPD with info->pivot set and leaves A in an unspecified state. */
emu_status emu_potrf_mp(emu_ctx *ctx, emu_mat *A, const emu_mp_opts *o,
                        emu_factor_info *info);

/* ---------------------------------------------------------------- sampling */
/* Draw `nsamples` emulations Y = L Z ("Generating Emulations", xi = V z) with
 * Z ~ N(0, I) generated on the device: entry (r, c) of Z comes from
 * Philox4x32-10 (Salmon et al., SC'11) at counter {r/2 mod 2^32, r/2 >> 32,
 * c, stream_id} and key {seed mod 2^32, seed >> 32}, turned into two 53-bit
 * uniforms and a Box-Muller pair for rows (2p, 2p+1), so Y is bit-identical
 * for the same (seed, factor) whatever the launch shape.  dY: n x nsamples
 * FP64, column-major, ldy >= n.  If dZ != NULL the normals are also written
 * there (n x nsamples, ld ldy). */
emu_status emu_sample(emu_ctx *ctx, const emu_mat *L, int nsamples,
                      uint64_t seed, uint32_t stream_id, double *dY, long ldy,
                      double *dZ);

/* Same, with Y and (optionally) Z in HOST memory: the device work and both
 * copies are enqueued on the context stream and the call returns after the
 * copies complete. */
emu_status emu_sample_host(emu_ctx *ctx, const emu_mat *L, int nsamples,
                           uint64_t seed, uint32_t stream_id, double *hY,
                           long ldy);

/* ------------------------------------------------------------------ solves */
/* X = (L L^T)^{-1} B with the factor L: a forward and a backward triangular
 * sweep over the tile rows.  A plain FP64 factor solves in FP64.  A mixed
 * factor solves in FP32 arithmetic: the diagonal blocks against FP32 values
 * of their FP64 factor tiles, the off-diagonal tiles as stored (FP64 tiles
 * rounded to FP32, FP32 masters as they are), each tile's product accumulated
 * in FP32 and added to the FP64 right-hand sides (it is the preconditioner of
 * emu_solve_refine, whose residual and update are FP64).  dB, dX: n x nrhs,
 * column-major; dX may equal dB. */
emu_status emu_potrs(emu_ctx *ctx, const emu_mat *L, const double *dB,
                     long ldb, double *dX, long ldx, int nrhs);

/* Solve S X = B by iterative refinement: X0 = (L L^T)^{-1} B, then FP64
 * residual R = B - S X against the FP64 covariance S (state 0, same n and
 * nb as L), correction D = (L L^T)^{-1} R in the factor's precisions, FP64
 * update X += D, until every column's normwise backward error
 * ||r||_2 / (||S||_F ||x||_2 + ||b||_2) is <= tol.  Returns EMU_ENOCONV when
 * maxit corrections do not reach tol (X then holds the last iterate). */
emu_status emu_solve_refine(emu_ctx *ctx, const emu_mat *L, const emu_mat *S,
                            const double *dB, long ldb, double *dX, long ldx,
                            int nrhs, double tol, int maxit,
                            emu_refine_info *info);

/* ------------------------------------------------------------------ batches */
/* Many independent covariances of uneven bandlimit (the batched workload:
 * n = L_b^2 from 64 to 4096), each built, factored by the adaptive per-tile
 * precision Cholesky and sampled, in one call.  Every step k of the tile
 * algorithm ("Advancements in Dense Linear Algebra") runs once for all
 * matrices that still have a step k, and the launches after the precision map
 * are captured in one CUDA graph that the context keeps and replays when the
 * same batch (parameters, nb, options, nsamples, dL given or not) comes
 * again.  The paper factors one matrix at a time; batching is this library's.
 *   count     number of matrices (>= 1)
 *   p         count parameter sets; 1 <= p[b].L <= 256
 *   nb        tile size: a multiple of 256 in [256, 1024], or 0 to let the
 *             library time 512 and 256 on the first call of this batch and
 *             keep the faster (later calls reuse the choice)
 *   o         factor options for every matrix (NULL or eps <= 0: plain FP64)
 *   nsamples  samples per matrix (0: factor only)
 *   seed      Philox key; matrix b draws its normals with stream id b, the
 *             draws emu_sample(L_b, nsamples, seed, b, ...) makes
 *   dY        count device pointers: Y_b = L_b Z_b, n_b x nsamples,
 *             column-major, leading dimension n_b (may be NULL if nsamples == 0)
 *   dL        NULL, or count device pointers: the factor L_b, n_b x n_b,
 *             column-major, leading dimension n_b, zeros above the diagonal
 *   infos     NULL, or count records; ms is the device time of the graph
 * Returns EMU_EINVAL for bad arguments, EMU_ENOMEM when the batch arenas do
 * not fit, EMU_ENOTPD when some matrices are not positive definite (each of
 * them has infos[b].pivot, its first non-positive pivot column; every other
 * matrix's factor and samples are complete and valid), EMU_ETIMEOUT,
 * EMU_ECUDA.  The arenas (about 18 bytes per element of every
 * padded lower tile) stay allocated in the context until emu_batch_release or
 * emu_destroy. */
emu_status emu_batch_potrf_sample(emu_ctx *ctx, int count, const emu_cov_params *p, int nb,
                                  const emu_mp_opts *o, int nsamples, uint64_t seed,
                                  double *const *dY, double *const *dL, emu_factor_info *infos);
/* Frees the context's batch arenas, plan and graph. */
emu_status emu_batch_release(emu_ctx *ctx);

/* ------------------------------------------------------- no-allocation build */
/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory while they call the library: code inside
 * a framework that owns the device heap, a process that reserved all memory up
 * front, or work issued while a CUDA graph is being built around it.  It needs
 * no context (creating one allocates).
 *
 * Writes the lower triangle (rows >= columns) of the synthetic covariance of
 * emu_cov_build, n = L^2, into dS (device, n x n FP64, column-major, ld >= n);
 * the strict upper triangle is not touched.  The values are those emu_cov_build
 * stores.  Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default)
 * and the call returns without synchronising.
 *
 * Scratch: the correlation and scale tables live in a fixed 1 MiB file-scope
 * device array instead of allocated memory, which bounds L to 128 (n <= 16384);
 * a larger L returns EMU_ENOMEM.  Every device that loads the library holds
 * the array until the process exits.  Each call on a stream that is not being
 * captured looks up the array's device address on the current device
 * (cudaGetSymbolAddress), so a device reset between calls is harmless; a call
 * on a capturing stream reuses the address of the last uncaptured call on that
 * device, so make at least one uncaptured call first, and none after a device
 * reset until an uncaptured one has run.  All calls share the one array: calls
 * whose work overlaps on the GPU (different streams, no ordering between them)
 * race and may produce wrong values.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  Returns EMU_EINVAL for bad arguments, EMU_ECUDA
 * for a launch failure or for a CUDA error already pending on the calling
 * thread (checked before any launch and left in place for the caller). */
emu_status emu_cov_build_dense_noalloc(int L, double beta, double sigma_exp,
                                       double nugget_rel, double *dS, long ld,
                                       void *stream);

#ifdef __cplusplus
}
#endif
#endif /* EMUCOV_H */
