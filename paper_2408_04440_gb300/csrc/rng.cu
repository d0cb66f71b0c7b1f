// rng.cu -- standard normals z ~ N(0, I) for drawing emulations
// ("Generating Emulations": xi = V z).  Counter-based, so every entry depends
// only on (seed, stream id, row, column) and never on the launch shape:
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) at counter
// {p mod 2^32, p >> 32, column, stream id}, key {seed mod 2^32, seed >> 32},
// p = row / 2; two 53-bit uniforms u1 in (0,1], u2 in [0,1); Box-Muller gives
// rows 2p (cosine) and 2p+1 (sine).
#include <algorithm>

#include "emu_internal.h"
#include "rng.cuh"

namespace {

__global__ void k_normals(uint64_t seed, uint32_t stream_id, int nrows, int s,
                          double *__restrict__ Z, long ldz) {
  long npairs = (nrows + 1) / 2;
  long total = npairs * s;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
       q += (long)gridDim.x * blockDim.x) {
    long p = q % npairs;
    int col = (int)(q / npairs);
    normal_pair(seed, stream_id, p, col, nrows, Z + (size_t)col * ldz + 2 * p);
  }
}

// Batch: blockIdx.y = matrix b, all NT_b * nb padded rows of its block of the
// stacked Z (rows row_base ..), with its own stream id.
// The seed is read from device memory so that a captured graph can be
// replayed with another seed.
__global__ void k_normals_batch(const uint64_t *__restrict__ seed_p, const BatchInst *__restrict__ inst, int nb,
                                int s, double *__restrict__ Z, long ldz) {
  const uint64_t seed = *seed_p;
  BatchInst I = inst[blockIdx.y];
  int nrows = I.NT * nb;
  long npairs = (nrows + 1) / 2;
  long total = npairs * s;
  double *Zb = Z + I.row_base;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    long p = q % npairs;
    int col = (int)(q / npairs);
    normal_pair(seed, (uint32_t)I.stream_id, p, col, nrows, Zb + (size_t)col * ldz + 2 * p);
  }
}
}  // namespace

emu_status launch_normals(emu_ctx *ctx, uint64_t seed, uint32_t stream_id, int nrows,
                          int s, double *Z, long ldz) {
  long total = (long)((nrows + 1) / 2) * s;
  long blocks = (total + 255) / 256;
  if (blocks > 8L * ctx->sm_count) blocks = 8L * ctx->sm_count;
  if (blocks < 1) blocks = 1;
  ProfScope ps(ctx, PROF_RNG, 0.0, 8.0 * nrows * (double)s);
  k_normals<<<(unsigned)blocks, 256, 0, ctx->stream>>>(seed, stream_id, nrows, s, Z, ldz);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_normals_batch(emu_ctx *ctx, const uint64_t *d_seed, const BatchInst *d_inst, int count,
                                int maxNT, int nb, int s, double *Z, long ldz) {
  long per = (long)((maxNT * nb + 1) / 2) * s;
  int bx = (int)std::min<long>(std::max<long>((per + 255) / 256, 1), 64);
  ProfScope ps(ctx, PROF_RNG, 0.0, 0.0);
  k_normals_batch<<<dim3(bx, count), 256, 0, ctx->stream>>>(d_seed, d_inst, nb, s, Z, ldz);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}
