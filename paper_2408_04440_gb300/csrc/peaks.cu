// peaks.cu -- measured FP64 and FP32 FMA rates of the device, the roofline
// denominators of the kernels bound by plain ALU arithmetic (the diagonal
// POTRF, the FP64 panel TRSM, the triangular solves).  Each thread runs eight
// independent FMA chains (enough to cover the pipe latency), every SM holds
// several CTAs, and the device time of the launch is taken with CUDA events.
#include "emu_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, T seed, T *out) {
  T a0 = seed + (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  const T m = (T)0.999999, c = (T)1e-7;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
      a0 = fma(a0, m, c);
      a1 = fma(a1, m, c);
      a2 = fma(a2, m, c);
      a3 = fma(a3, m, c);
      a4 = fma(a4, m, c);
      a5 = fma(a5, m, c);
      a6 = fma(a6, m, c);
      a7 = fma(a7, m, c);
    }
  }
  const T r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (r == (T)-1) *out = r;  // never true: keeps the chains alive
}

template <typename T>
emu_status time_fma(emu_ctx *ctx, int iters, double *tflops) {
  const int blocks = ctx->sm_count * 8, threads = 256;
  T *out = nullptr;
  EMU_CUDA_TRY(ctx, cudaMallocAsync(&out, sizeof(T), ctx->stream));
  k_fma_loop<T><<<blocks, threads, 0, ctx->stream>>>(8, (T)1, out);  // warm-up
  EMU_LAUNCHED(ctx);
  EMU_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  k_fma_loop<T><<<blocks, threads, 0, ctx->stream>>>(iters, (T)1, out);
  EMU_LAUNCHED(ctx);
  EMU_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  EMU_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev1));
  float ms = 0.f;
  EMU_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  cudaFreeAsync(out, ctx->stream);
  const double flop = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads;
  *tflops = ms > 0.f ? flop / (ms * 1e-3) / 1e12 : 0.0;
  return EMU_OK;
}

}  // namespace

extern "C" emu_status emu_measure_alu_peaks(emu_ctx *ctx, double *fp64_tflops, double *fp32_tflops) {
  if (!ctx || !fp64_tflops || !fp32_tflops) return EMU_EINVAL;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  emu_status s = time_fma<double>(ctx, 2000, fp64_tflops);
  if (s == EMU_OK) s = time_fma<float>(ctx, 40000, fp32_tflops);
  return s;
}
