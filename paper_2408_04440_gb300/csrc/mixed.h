// mixed.h -- entry points of the adaptive-precision factor, its sampler and
// solves, and the iterative-refinement driver (mixed.cu, refine.cu).
#pragma once
#include "emu_internal.h"

emu_status factor_mixed(emu_ctx *ctx, emu_mat *A, const emu_mp_opts *o);
void mixed_fill_info(const emu_mat *A, emu_factor_info *info);
emu_status mixed_sample(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz, int s,
                        double *Y, long ldy);
emu_status mixed_potrs(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs);
// blocked right-looking sweeps (solve.cu), for nb a multiple of 64 up to 1024
bool mixed_potrs_blocked_supports(int nb);
emu_status mixed_potrs_blocked(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs);
void mixed_ctx_release(emu_ctx *ctx);
// graph replay and reserved-SM tuning of the single-matrix factor
void mixed_set_schedule(emu_ctx *ctx, int use_graphs, int tuning);
void mixed_tune_record(emu_ctx *ctx, bool ok);
int mixed_tuned_choice(emu_ctx *ctx, int *tried, int *R, int *R64);
// the internal streams of the lookahead schedule and at least nev events
emu_status mixed_sched_streams(emu_ctx *ctx, int nev);
// SMs left free of the bulk GEMM beside FP64-class panel work or not
int mixed_reserved_sms(bool fp64_near);
// class-format storage (classfmt.cu)
emu_status classfmt_build(emu_ctx *ctx, emu_mat *A, const emu_cov_params *p, const emu_mp_opts *o);
emu_status classfmt_factor(emu_ctx *ctx, emu_mat *A);
void classfmt_fill_info(const emu_mat *A, emu_factor_info *info);
emu_status classfmt_sample(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz, int s, double *Y, long ldy);
emu_status classfmt_export(emu_ctx *ctx, const emu_mat *A, double *dOut, long ld);
void classfmt_release(emu_mat *A);
emu_status factor_backward_error_est(emu_ctx *ctx, const emu_mat *A, const emu_cov_params *cp, int nprobes,
                                     uint64_t seed, double *est);
// batch.cu: arenas, plan and graph of the context's last batch
void batch_ctx_release(emu_ctx *ctx);
void mixed_mat_release(emu_mat *A);
emu_status refine_solve(emu_ctx *ctx, const emu_mat *L, const emu_mat *S, const double *dB,
                        long ldb, double *dX, long ldx, int nrhs, double tol, int maxit,
                        emu_refine_info *info);
