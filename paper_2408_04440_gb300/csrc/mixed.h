// mixed.h -- entry points of the adaptive-precision factor, its sampler and
// solves, and the iterative-refinement driver (mixed.cu, refine.cu).
#pragma once
#include "emu_internal.h"

emu_status factor_mixed(emu_ctx *ctx, emu_mat *A, const emu_mp_opts *o);
void mixed_fill_info(const emu_mat *A, emu_factor_info *info);
emu_status mixed_sample(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz, int s,
                        double *Y, long ldy);
emu_status mixed_potrs(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs);
void mixed_ctx_release(emu_ctx *ctx);
// batch.cu: arenas, plan and graph of the context's last batch
void batch_ctx_release(emu_ctx *ctx);
void mixed_mat_release(emu_mat *A);
emu_status refine_solve(emu_ctx *ctx, const emu_mat *L, const emu_mat *S, const double *dB,
                        long ldb, double *dX, long ldx, int nrhs, double tol, int maxit,
                        emu_refine_info *info);
