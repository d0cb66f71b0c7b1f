// mixed.cu -- adaptive per-tile precision factor (placeholder until the
// tensor-core path lands).
#include "mixed.h"

emu_status factor_mixed(emu_ctx *ctx, emu_mat *, const emu_mp_opts *) {
  ctx->last_error = "mixed-precision factor not available in this build";
  return EMU_EINVAL;
}
void mixed_fill_info(const emu_mat *, emu_factor_info *) {}
emu_status mixed_sample(emu_ctx *ctx, const emu_mat *, const double *, long, int, double *, long) {
  ctx->last_error = "mixed-precision sampler not available in this build";
  return EMU_EINVAL;
}
emu_status mixed_potrs(emu_ctx *ctx, const emu_mat *, double *, long, int) {
  ctx->last_error = "mixed-precision solve not available in this build";
  return EMU_EINVAL;
}
void mixed_ctx_release(emu_ctx *) {}
