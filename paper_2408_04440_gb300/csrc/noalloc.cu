// noalloc.cu -- covariance build into a caller-provided dense buffer without
// any device allocation (emu_cov_build_dense_noalloc in include/emucov.h).
//
// Some callers cannot allocate device memory while they call this library:
// code running inside a framework that owns the device heap, a process that
// has reserved all memory up front, or work issued while a CUDA graph is
// being built around it.  For them the correlation and scale tables that
// emu_cov_build keeps in stream-ordered scratch live here in a file-scope
// __device__ array instead.  The array is part of the loaded module, so every
// device that loads the library holds it until the process exits.
#include <mutex>

#include "emu_internal.h"

namespace {

// Tables of one call: rho[(2L-1)(4L-3)], sigma[L], nugget[1].  1 MiB of
// doubles, enough for every L <= 128 (n = L^2 <= 16384).
constexpr int kNoAllocMaxL = 128;
constexpr size_t kNoAllocScratchDoubles = 131072;
static_assert((size_t)(2 * kNoAllocMaxL - 1) * (4 * kNoAllocMaxL - 3) + kNoAllocMaxL + 1 <= kNoAllocScratchDoubles,
              "scratch too small for kNoAllocMaxL");

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Host-side record of the array's device address, per device.  In host code
// the symbol name is only a stand-in, so the address comes from
// cudaGetSymbolAddress with that device current.  It is looked up again on
// every call whose stream is not being captured (the module may sit at a new
// address after a device reset); a captured call uses the last address seen.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {};

__device__ inline int degree_na(long k) {
  int l = (int)sqrtf((float)k);
  while ((long)l * l > k) l--;
  while ((long)(l + 1) * (l + 1) <= k) l++;
  return l;
}

// Same tables, same operations and order as the tiled builder's.
__global__ void k_noalloc_tables(int L, double beta, double sexp, double nugget_rel, double *sigma, double *rho,
                                 double *nugget) {
  int W = 4 * L - 3;
  long total = (long)(2 * L - 1) * W;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    int a = (int)(t / W), b = (int)(t % W);
    double dl = (double)(a - (L - 1)), dm = (double)(b - (2 * L - 2));
    double d = sqrt(dl * dl + dm * dm);
    rho[t] = exp(-d / beta);
  }
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x)
    sigma[l] = pow(1.0 + l, -sexp);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double dmax = 0.0;
    for (int l = 0; l < L; l++) {
      double s = pow(1.0 + l, -sexp);
      double v = s * s * 1.0;
      if (v > dmax) dmax = v;
    }
    *nugget = nugget_rel * dmax;
  }
}

// Lower triangle of S (column-major, leading dimension ld): column gj =
// blockIdx.y, rows gj .. n-1 strided over the grid's x dimension.
__global__ void k_noalloc_dense(int L, long n, const double *__restrict__ sigma, const double *__restrict__ rho,
                                const double *__restrict__ nugget, double *__restrict__ S, long ld) {
  long gj = blockIdx.y;
  int W = 4 * L - 3;
  int lj = degree_na(gj), mj = (int)(gj - (long)lj * lj - lj);
  double nug = *nugget;
  for (long gi = gj + blockIdx.x * (long)blockDim.x + threadIdx.x; gi < n; gi += (long)gridDim.x * blockDim.x) {
    int li = degree_na(gi);
    int mi = (int)(gi - (long)li * li - li);
    double e = rho[(long)(li - lj + L - 1) * W + (mi - mj + 2 * L - 2)];
    double v = __dmul_rn(__dmul_rn(sigma[li], sigma[lj]), e);
    if (gi == gj) v = __dadd_rn(v, nug);
    S[gi + gj * ld] = v;
  }
}

// Device address of the scratch array on the current device.
emu_status noalloc_scratch(cudaStream_t st, double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EMU_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return EMU_EINVAL;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return EMU_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return EMU_ECUDA;
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return EMU_OK;
}

}  // namespace

extern "C" emu_status emu_cov_build_dense_noalloc(int L, double beta, double sigma_exp, double nugget_rel,
                                                  double *dS, long ld, void *stream) {
  if (!dS || L < 1 || !(beta > 0.0) || !(nugget_rel > -1.0 && nugget_rel < 1e300) || ld < (long)L * L) return EMU_EINVAL;
  if (L > kNoAllocMaxL) return EMU_ENOMEM;  // tables would not fit the fixed scratch array
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // an error already pending on this thread is not this call's: report it
  // before launching anything, and leave it for the caller to read
  if (cudaPeekAtLastError() != cudaSuccess) return EMU_ECUDA;
  double *scratch = nullptr;
  emu_status s = noalloc_scratch(st, &scratch);
  if (s != EMU_OK) return s;
  size_t ntab = (size_t)(2 * L - 1) * (4 * L - 3);
  double *rho = scratch, *sigma = scratch + ntab, *nug = scratch + ntab + L;
  // every table entry used below is rewritten by this call before it is read
  int blocks = (int)((ntab + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  k_noalloc_tables<<<blocks, 256, 0, st>>>(L, beta, sigma_exp, nugget_rel, sigma, rho, nug);
  if (cudaGetLastError() != cudaSuccess) return EMU_ECUDA;
  long n = (long)L * L;
  unsigned gx = (unsigned)((n + 255) / 256);
  if (gx > 64) gx = 64;
  k_noalloc_dense<<<dim3(gx, (unsigned)n), 256, 0, st>>>(L, n, sigma, rho, nug, dS, ld);
  if (cudaGetLastError() != cudaSuccess) return EMU_ECUDA;
  return EMU_OK;
}
