// emulate.cu -- the steps after sampling that turn draws of the coefficient
// covariance into emulations ("Generating Emulations"): the VAR(P) recursion
// of the spherical-harmonic coefficients with diagonal Phi_p, and the inverse
// spherical-harmonic transform of the coefficients to a latitude-longitude
// grid ("Spherical Harmonic Transform", the synthesis sum over (l, m)).
//
// Coefficients are real-form and ordered by degree then order,
// k = l^2 + l + m, |m| <= l < L, as the covariance's rows.  The real basis:
//   Y_l0 = N_l0 P_l(cos t),  Y_lm = sqrt(2) N_lm P_l^m(cos t) cos(m p) (m > 0),
//   Y_l,-m = sqrt(2) N_lm P_l^m(cos t) sin(m p),  N_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!,
// P_l^m with the Condon-Shortley phase (-1)^m.  Grid: colatitudes
// t_i = pi i / (ntheta - 1) (poles included), longitudes p_j = 2 pi j / nphi.
//
// The last step builds the emulations of Eq. decouple from the synthesis Zs:
// y_t = m_t + sigma (Zs_t + v e_t), with the nugget e drawn by the library's
// Philox generator and the distributed-lag mean trend m_t.
#include <cmath>

#include "emu_internal.h"
#include "rng.cuh"

namespace {

__device__ inline bool failed(const int *st) { return *((volatile const int *)st) != DEV_OK; }

// f_t = sum_p phi_p f_{t-p} + xi_t per coefficient (f before t = 0 is zero):
// one thread per coefficient, the P previous values in registers.
constexpr int kMaxP = 8;
__global__ void k_var(const double *__restrict__ xi, long ldxi, int n, int T, const double *__restrict__ phi, int P,
                      double *__restrict__ f, long ldf, const int *st) {
  if (failed(st)) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double c[kMaxP], h[kMaxP];
#pragma unroll
  for (int p = 0; p < kMaxP; p++) {
    c[p] = p < P ? phi[k + (long)p * n] : 0.0;
    h[p] = 0.0;  // h[p] = f_{t-1-p}
  }
  for (int t = 0; t < T; t++) {
    double v = 0.0;
#pragma unroll
    for (int p = 0; p < kMaxP; p++) v = fma(c[p], h[p], v);
    v += xi[k + (long)t * ldxi];
#pragma unroll
    for (int p = kMaxP - 1; p > 0; p--) h[p] = h[p - 1];
    h[0] = v;
    f[k + (long)t * ldf] = v;
  }
}

// Normalised associated Legendre table: lam[off(m) + (l - m) * ntheta + i] =
// c_m N_lm P_l^m(cos t_i), c_0 = 1, c_m = sqrt(2), off(m) = ntheta * (m L - m(m-1)/2).
// One thread per (m, i): the standard stable recursion in l,
//   Pb_mm = -sqrt((2m+1)/(2m)) sin t Pb_{m-1,m-1},  Pb_00 = 1/sqrt(4 pi),
//   Pb_{m+1,m} = sqrt(2m+3) cos t Pb_mm,
//   Pb_lm = a_lm (cos t Pb_{l-1,m} - Pb_{l-2,m} / a_{l-1,m}),  a_lm = sqrt((4l^2-1)/(l^2-m^2)).
__global__ void k_legendre(int L, int ntheta, double *__restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
  if (i >= ntheta || m >= L) return;
  const double th = M_PI * (double)i / (double)(ntheta - 1);
  double s, c;
  sincos(th, &s, &c);
  double pmm = 0.28209479177387814;  // 1 / sqrt(4 pi)
  for (int q = 1; q <= m; q++) pmm *= -sqrt((2.0 * q + 1.0) / (2.0 * q)) * s;
  const double cm = m > 0 ? 1.4142135623730951 : 1.0;
  double *out = lam + (size_t)ntheta * ((size_t)m * L - (size_t)m * (m - 1) / 2);
  out[i] = cm * pmm;
  if (m + 1 >= L) return;
  double p1 = sqrt(2.0 * m + 3.0) * c * pmm;  // l = m + 1
  out[(size_t)ntheta + i] = cm * p1;
  double p0 = pmm, a_prev = sqrt(2.0 * m + 3.0);
  for (int l = m + 2; l < L; l++) {
    const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
    const double p = a * (c * p1 - p0 / a_prev);
    out[(size_t)(l - m) * ntheta + i] = cm * p;
    p0 = p1;
    p1 = p;
    a_prev = a;
  }
}

// Per order m and time t: A_m(t_i) = sum_l f_{l,m} lam_lm(t_i) and
// B_m(t_i) = sum_l f_{l,-m} lam_lm(t_i) (m > 0).  ab[(m * 2 + {0,1}) * ntheta + i, t].
__global__ void k_isht_legendre(int L, int T, const double *__restrict__ f, long ldf, int ntheta,
                                const double *__restrict__ lam, double *__restrict__ ab, long ldab, const int *st) {
  if (failed(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y, t = blockIdx.z;
  if (i >= ntheta) return;
  const double *lm = lam + (size_t)ntheta * ((size_t)m * L - (size_t)m * (m - 1) / 2);
  const double *ft = f + (long)t * ldf;
  double a = 0.0, b = 0.0;
  for (int l = m; l < L; l++) {
    const double y = lm[(size_t)(l - m) * ntheta + i];
    a = fma(ft[(long)l * l + l + m], y, a);
    if (m > 0) b = fma(ft[(long)l * l + l - m], y, b);
  }
  ab[(size_t)(2 * m) * ntheta + i + (long)t * ldab] = a;
  ab[(size_t)(2 * m + 1) * ntheta + i + (long)t * ldab] = b;
}

// Z(t_i, p_j) = sum_m A_m(t_i) cos(m p_j) + B_m(t_i) sin(m p_j): one CTA per
// (latitude ring, time), the ring's 2L sums in shared memory; cos / sin of
// (m j mod nphi) 2 pi / nphi from a table.
__global__ void k_isht_fourier(int L, int ntheta, int nphi, const double *__restrict__ ab, long ldab,
                               const double *__restrict__ cs, double *__restrict__ z, long ldz, const int *st) {
  if (failed(st)) return;
  extern __shared__ double sab[];  // [2L]
  const int i = blockIdx.x, t = blockIdx.y;
  for (int q = threadIdx.x; q < 2 * L; q += blockDim.x) sab[q] = ab[(size_t)q * ntheta + i + (long)t * ldab];
  __syncthreads();
  for (int j = threadIdx.x; j < nphi; j += blockDim.x) {
    double v = 0.0;
    for (int m = 0; m < L; m++) {
      const long r = ((long)m * j) % nphi;
      v = fma(sab[2 * m], cs[2 * r], v);
      v = fma(sab[2 * m + 1], cs[2 * r + 1], v);
    }
    z[i + (long)j * ntheta + (long)t * ldz] = v;
  }
}

__global__ void k_cossin(int nphi, double *__restrict__ cs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nphi) return;
  double s, c;
  sincospi(2.0 * (double)r / (double)nphi, &s, &c);
  cs[2 * r] = c;
  cs[2 * r + 1] = s;
}

// ---------------------------------------------------------------- forward SHT
// The forward transform of the grid data (the coefficient as the integral of
// Z Y_lm over the sphere): C_m / S_m by a DFT in longitude, the circle
// extension g(t_{M-i}) = (-1)^m g(t_i) over M = 2 ntheta - 2 colatitudes,
// Fourier coefficients K_q of g, and the contraction with
// S_{l,m,q} = sum_q' c_{l,m,q'} I(q + q'), c the Fourier coefficients of the
// extended Legendre factor and I(k) = int_0^pi e^{ikt} sin t dt: 2/(1-k^2)
// for even k, +-i pi/2 at k = +-1, and 0 for the other odd k.

// C_m(t_i), S_m(t_i) = (2 pi / nphi) sum_j Z_ij {cos, sin}(m p_j): one CTA per
// (ring, time), the ring in shared memory.  cs[(2m + {0,1}) * ntheta + i, t].
__global__ void k_sht_fourier(const double *__restrict__ z, long ldz, int ntheta, int nphi, int L,
                              const double *__restrict__ csp, double *__restrict__ cs, long ldcs, const int *st) {
  if (failed(st)) return;
  extern __shared__ double ring[];  // [nphi]
  const int i = blockIdx.x, t = blockIdx.y;
  for (int j = threadIdx.x; j < nphi; j += blockDim.x) ring[j] = z[i + (long)j * ntheta + (long)t * ldz];
  __syncthreads();
  const double w = 6.283185307179586 / (double)nphi;
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    double c = 0.0, sn = 0.0;
    // r = m j mod nphi, stepped without a division
    const int step = m % nphi;
    int r = 0;
    for (int j = 0; j < nphi; j++) {
      c = fma(ring[j], csp[2 * r], c);
      sn = fma(ring[j], csp[2 * r + 1], sn);
      r += step;
      if (r >= nphi) r -= nphi;
    }
    cs[(size_t)(2 * m) * ntheta + i + (long)t * ldcs] = c * w;
    cs[(size_t)(2 * m + 1) * ntheta + i + (long)t * ldcs] = sn * w;
  }
}

// Fourier coefficients over the M-point circle (M = 2N, N = ntheta - 1) of
// the extended function g: g_i = v[i] for i <= N (v[i] at t_i = 2 pi i / M)
// and g_i = sgn v[M - i] above: out[q + L - 1] for |q| < L, complex, of
// (1/M) sum_i g_i exp(-2 pi i q i / M).  The samples i and M - i (0 < i < N)
// pair up: for sgn = +1 their sum is 2 v[i] cos(2 pi q i / M) and the sines
// cancel, for sgn = -1 the cosines cancel and -2 v[i] sin(2 pi q i / M) is
// left; i = 0 and i = N add v[0] + (-1)^q v[N].  g is real, so the
// coefficient at -q is the conjugate of the one at q.  cm: table of
// cos / sin (2 pi r / M); r = q i mod M is stepped without a division.
__device__ inline void circle_coeffs(const double *v, double sgn, int ntheta, int M, int L, const double *cm,
                                     double *outr, double *outi) {
  const int N = ntheta - 1;
  const double invM = 1.0 / (double)M;
  const int odd = sgn < 0.0 ? 1 : 0;  // sine sums
  for (int q = threadIdx.x; q <= L - 1; q += blockDim.x) {
    const int step = q % M;
    int r = step;
    double acc = 0.0;
    for (int i = 1; i < N; i++) {
      acc = fma(v[i], cm[2 * r + odd], acc);
      r += step;
      if (r >= M) r -= M;
    }
    const double ends = v[0] + ((q & 1) ? -v[N] : v[N]);
    const double re = odd ? ends * invM : (ends + 2.0 * acc) * invM;
    const double im = odd ? -2.0 * acc * invM : 0.0;
    outr[q + L - 1] = re;
    outi[q + L - 1] = im;
    if (q > 0) {
      outr[L - 1 - q] = re;
      outi[L - 1 - q] = -im;
    }
  }
}

// S_{l,m,q} for one (l, m) per CTA: the Legendre factor's circle coefficients
// in shared memory, then their convolution with I.  sq[(pair) * 2Q + {re, im} * Q + q].
__global__ void k_sht_S(int L, int ntheta, const double *__restrict__ lam, const double *__restrict__ cm,
                        double *__restrict__ sq) {
  extern __shared__ double sh[];  // cr[Q], ci[Q], v[ntheta]
  const int Q = 2 * L - 1, M = 2 * ntheta - 2;
  double *cr = sh, *ci = sh + Q, *v = sh + 2 * Q;
  const int pair = blockIdx.x;  // m * L - m (m - 1) / 2 + (l - m)
  int m = 0;
  while (pair >= (m + 1) * L - (m + 1) * m / 2) m++;
  const int l = m + pair - (m * L - m * (m - 1) / 2);
  const double *h = lam + (size_t)ntheta * pair;
  for (int i = threadIdx.x; i < ntheta; i += blockDim.x) v[i] = h[i];
  __syncthreads();
  circle_coeffs(v, (m & 1) ? -1.0 : 1.0, ntheta, M, L, cm, cr, ci);
  __syncthreads();
  double *o = sq + (size_t)pair * 2 * Q;
  for (int q = threadIdx.x - (L - 1); q <= L - 1; q += blockDim.x) {
    double sr = 0.0, si = 0.0;
    // I(k) is real for even k, +-i pi/2 at k = +-1 and zero at the other odd
    // k: the even k first (q2 of q's parity), then the two imaginary terms
    for (int q2 = -(L - 1) + ((q - (L - 1)) & 1); q2 <= L - 1; q2 += 2) {
      const int k = q + q2;
      const double ir = 2.0 / (1.0 - (double)k * k);
      sr = fma(cr[q2 + L - 1], ir, sr);
      si = fma(ci[q2 + L - 1], ir, si);
    }
    for (int sgn1 = -1; sgn1 <= 1; sgn1 += 2) {
      const int q2 = sgn1 - q;
      if (q2 >= -(L - 1) && q2 <= L - 1) {
        const double ii = sgn1 * 1.5707963267948966;
        sr = fma(-ci[q2 + L - 1], ii, sr);
        si = fma(cr[q2 + L - 1], ii, si);
      }
    }
    o[q + L - 1] = sr;
    o[Q + q + L - 1] = si;
  }
  (void)l;
}

// K_q of C_m and S_m for one (m, time) per CTA, then the contraction
// f_{l,+-m} = Re sum_q K_q S_{l,m,q} for l = m .. L-1.
__global__ void k_sht_contract(int L, int T, int ntheta, const double *__restrict__ cs, long ldcs,
                               const double *__restrict__ cm, const double *__restrict__ sq, double *__restrict__ f,
                               long ldf, const int *st) {
  if (failed(st)) return;
  extern __shared__ double sh[];  // kc_r, kc_i, ks_r, ks_i [Q each], v [ntheta]
  const int Q = 2 * L - 1, M = 2 * ntheta - 2;
  const int m = blockIdx.x, t = blockIdx.y;
  double *kcr = sh, *kci = sh + Q, *ksr = sh + 2 * Q, *ksi = sh + 3 * Q, *v = sh + 4 * Q;
  const double sgn = (m & 1) ? -1.0 : 1.0;
  for (int c = 0; c < 2; c++) {
    for (int i = threadIdx.x; i < ntheta; i += blockDim.x) v[i] = cs[(size_t)(2 * m + c) * ntheta + i + (long)t * ldcs];
    __syncthreads();
    circle_coeffs(v, sgn, ntheta, M, L, cm, c ? ksr : kcr, c ? ksi : kci);
    __syncthreads();
  }
  const size_t pair0 = (size_t)m * L - (size_t)m * (m - 1) / 2;
  for (int l = m + threadIdx.x; l < L; l += blockDim.x) {
    const double *o = sq + (pair0 + (l - m)) * 2 * Q;
    double fc = 0.0, fs = 0.0;
    for (int q = 0; q < Q; q++) {
      fc += kcr[q] * o[q] - kci[q] * o[Q + q];
      fs += ksr[q] * o[q] - ksi[q] * o[Q + q];
    }
    f[(long)l * l + l + m + (long)t * ldf] = fc;
    if (m > 0) f[(long)l * l + l - m + (long)t * ldf] = fs;
  }
}

// Emulations of Eq. decouple on the grid, for time steps t = 1..T (column
// t-1): y_t(g) = m_t(g) + sigma(g) (Zs_t(g) + v(g) e_t(g)), e_t(g) the
// library's normal of row g, column t-1 (Philox stream `sid`), and
//   m_t = b0 + b1 x_y + b2 D_y + sum_k a_k cos(2 pi t k / tau) + b_k sin(2 pi t k / tau),
// y = ceil(t / tau), D_y = (1 - rho) sum_{s>=1} rho^(s-1) x_(y-s) with the
// years before the trajectory at x[0]: D_1 = x[0], D_(y+1) = (1 - rho) x_y + rho D_y.
// One thread per grid-point pair (the two rows of one Box-Muller pair) and
// chunk of kEmTC time steps (blockIdx.y); the harmonic values of the chunk
// are shared by the block.  HBM-bound: 16 bytes in, 8 out per entry.
constexpr int kMaxK = 8, kEmTC = 32;
struct TrendDev {
  int K, nyears;
  double tau;
  const double *b0, *b1, *b2, *rho, *a, *b, *x;
};
__global__ void __launch_bounds__(128) k_emulate_grid(const double *__restrict__ Zs, long G, int T, long ldz,
                                                      TrendDev m, const double *__restrict__ sigma,
                                                      const double *__restrict__ v, uint64_t seed, uint32_t sid,
                                                      double *Y, long ldy) {
  __shared__ double cs[kMaxK][kEmTC], sn[kMaxK][kEmTC];
  const int t0 = blockIdx.y * kEmTC + 1;
  const int nt = min(kEmTC, T - t0 + 1);
  const double two_pi = 6.283185307179586476925286766559;
  for (int q = threadIdx.x; q < m.K * kEmTC; q += blockDim.x) {
    int k = q / kEmTC + 1, tt = q % kEmTC;
    sincos(two_pi * (double)(t0 + tt) * (double)k / m.tau, &sn[k - 1][tt], &cs[k - 1][tt]);
  }
  __syncthreads();
  const long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (2 * p >= G) return;
  const int npt = (2 * p + 1 < G) ? 2 : 1;
  double b0[2], b1[2], b2[2], rho[2], sg[2], vv[2], D[2], a[2][kMaxK], b[2][kMaxK];
  long yc = (long)ceil((double)t0 / m.tau);  // forcing year of the chunk's first step
  for (int u = 0; u < 2; u++) {
    long g = 2 * p + (u < npt ? u : 0);
    b0[u] = m.b0[g];
    b1[u] = m.b1[g];
    b2[u] = m.b2[g];
    rho[u] = m.rho[g];
    sg[u] = sigma[g];
    vv[u] = v[g];
#pragma unroll
    for (int k = 0; k < kMaxK; k++) {
      a[u][k] = k < m.K ? m.a[k + g * m.K] : 0.0;
      b[u][k] = k < m.K ? m.b[k + g * m.K] : 0.0;
    }
    D[u] = m.x[0];
    for (long yy = 1; yy < yc; yy++) D[u] = (1.0 - rho[u]) * m.x[yy] + rho[u] * D[u];
  }
  for (int tt = 0; tt < nt; tt++) {
    const int t = t0 + tt;
    const long y = (long)ceil((double)t / m.tau);
    while (yc < y) {
      for (int u = 0; u < 2; u++) D[u] = (1.0 - rho[u]) * m.x[yc] + rho[u] * D[u];
      yc++;
    }
    double e[2] = {0.0, 0.0};
    normal_pair(seed, sid, p, t - 1, (int)(G < 0x7fffffff ? G : 0x7fffffff), e);
    const double xy = m.x[y];
    for (int u = 0; u < npt; u++) {
      double mt = b0[u] + b1[u] * xy + b2[u] * D[u];
      for (int k = 0; k < m.K; k++) mt += a[u][k] * cs[k][tt] + b[u][k] * sn[k][tt];
      const long g = 2 * p + u;
      const double z = Zs[g + (long)(t - 1) * ldz] + vv[u] * e[u];
      Y[g + (long)(t - 1) * ldy] = mt + sg[u] * z;
    }
  }
}

}  // namespace


extern "C" {

emu_status emu_var_recursion(emu_ctx *ctx, const double *dXi, int n, int T, long ldxi, const double *dPhi, int P,
                             double *dF, long ldf) {
  if (!ctx || !dXi || !dF || n < 1 || T < 1 || ldxi < n || ldf < n || P < 0 || P > kMaxP || (P > 0 && !dPhi))
    return EMU_EINVAL;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, ST_WORDS * sizeof(int), ctx->stream));
  k_var<<<(n + 127) / 128, 128, 0, ctx->stream>>>(dXi, ldxi, n, T, dPhi, P, dF, ldf, ctx->d_status);
  EMU_LAUNCHED(ctx);
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return EMU_OK;
}

emu_status emu_isht(emu_ctx *ctx, const double *dF, int L, int T, long ldf, int ntheta, int nphi, double *dZ,
                    long ldz) {
  if (!ctx || !dF || !dZ || L < 1 || L > 2048 || T < 1 || ldf < (long)L * L || ntheta < 2 || nphi < 1 ||
      ldz < (long)ntheta * nphi)
    return EMU_EINVAL;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, ST_WORDS * sizeof(int), s));
  const size_t nlam = (size_t)ntheta * ((size_t)L * (L + 1) / 2);
  const long ldab = 2L * L * ntheta;
  double *lam = nullptr, *ab = nullptr, *cs = nullptr;
  cudaError_t e = cudaMallocAsync(&lam, nlam * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&ab, (size_t)ldab * T * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&cs, 2 * (size_t)nphi * sizeof(double), s);
  emu_status st = EMU_OK;
  if (e == cudaSuccess) {
    ProfScope ps(ctx, PROF_SOLVE, 2.0 * (double)L * L * ntheta * T + 4.0 * (double)L * ntheta * nphi * T, 0.0);
    k_legendre<<<dim3((ntheta + 127) / 128, L), 128, 0, s>>>(L, ntheta, lam);
    k_cossin<<<(nphi + 255) / 256, 256, 0, s>>>(nphi, cs);
    k_isht_legendre<<<dim3((ntheta + 127) / 128, L, T), 128, 0, s>>>(L, T, dF, ldf, ntheta, lam, ab, ldab,
                                                                     ctx->d_status);
    k_isht_fourier<<<dim3(ntheta, T), 256, 2 * L * sizeof(double), s>>>(L, ntheta, nphi, ab, ldab, cs, dZ, ldz,
                                                                        ctx->d_status);
    e = cudaGetLastError();
    ctx->launches += 4;
  }
  for (void *p : {(void *)lam, (void *)ab, (void *)cs})
    if (p) cudaFreeAsync(p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) st = emu_cuda_fail(ctx, e, "isht");
  return st;
}


emu_status emu_sht(emu_ctx *ctx, const double *dZ, int ntheta, int nphi, int T, long ldz, int L, double *dF,
                   long ldf) {
  if (!ctx || !dZ || !dF || L < 1 || L > 1024 || T < 1 || ntheta < 2 || nphi < 1 || ldz < (long)ntheta * nphi ||
      ldf < (long)L * L)
    return EMU_EINVAL;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, ST_WORDS * sizeof(int), s));
  const int Q = 2 * L - 1, M = 2 * ntheta - 2;
  const size_t npair = (size_t)L * (L + 1) / 2;
  const long ldcs = 2L * L * ntheta;
  double *lam = nullptr, *csp = nullptr, *cm = nullptr, *sq = nullptr, *cs = nullptr;
  cudaError_t e = cudaMallocAsync(&lam, npair * ntheta * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&csp, 2 * (size_t)nphi * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&cm, 2 * (size_t)M * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&sq, npair * 2 * Q * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&cs, (size_t)ldcs * T * sizeof(double), s);
  const size_t sm_S = (2 * (size_t)Q + ntheta) * sizeof(double), sm_K = (4 * (size_t)Q + ntheta) * sizeof(double);
  if (e == cudaSuccess && (sm_S > 48 * 1024 || sm_K > 48 * 1024 || nphi * sizeof(double) > 48 * 1024)) {
    e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) {
    ProfScope ps(ctx, PROF_SOLVE, 2.0 * (double)L * ntheta * nphi * T + 8.0 * (double)L * Q * M * T, 0.0);
    k_legendre<<<dim3((ntheta + 127) / 128, L), 128, 0, s>>>(L, ntheta, lam);
    k_cossin<<<(nphi + 255) / 256, 256, 0, s>>>(nphi, csp);
    k_cossin<<<(M + 255) / 256, 256, 0, s>>>(M, cm);
    k_sht_S<<<(unsigned)npair, 128, sm_S, s>>>(L, ntheta, lam, cm, sq);
    k_sht_fourier<<<dim3(ntheta, T), 128, nphi * sizeof(double), s>>>(dZ, ldz, ntheta, nphi, L, csp, cs, ldcs,
                                                                      ctx->d_status);
    k_sht_contract<<<dim3(L, T), 128, sm_K, s>>>(L, T, ntheta, cs, ldcs, cm, sq, dF, ldf, ctx->d_status);
    e = cudaGetLastError();
    ctx->launches += 6;
  }
  for (void *p : {(void *)lam, (void *)csp, (void *)cm, (void *)sq, (void *)cs})
    if (p) cudaFreeAsync(p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaErrorInvalidValue) return EMU_EINVAL;
  if (e != cudaSuccess) return emu_cuda_fail(ctx, e, "sht");
  return EMU_OK;
}


emu_status emu_emulate_grid(emu_ctx *ctx, const double *dZs, long G, int T, long ldz, const emu_trend *m,
                            const double *dsigma, const double *dv, uint64_t seed, uint32_t stream_id, double *dY,
                            long ldy) {
  if (!ctx || !dZs || !dY || !m || !dsigma || !dv || G < 1 || T < 1 || ldz < G || ldy < G) return EMU_EINVAL;
  if (!(m->tau > 0.0) || m->K < 0 || m->K > kMaxK || (m->K > 0 && (!m->a || !m->b)) || !m->beta0 || !m->beta1 ||
      !m->beta2 || !m->rho || !m->x || m->nyears < 0)
    return EMU_EINVAL;
  if ((long)std::ceil((double)T / m->tau) > (long)m->nyears) return EMU_EINVAL;  // forcing too short
  if (G > 0x7fffffffL) return EMU_EINVAL;  // Philox row counter of one column
  if (dY == dZs && ldy != ldz) return EMU_EINVAL;
  if (dY != dZs && (dY < dZs + G + (long)(T - 1) * ldz && dZs < dY + G + (long)(T - 1) * ldy)) return EMU_EINVAL;
  EMU_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  TrendDev td{m->K, m->nyears, m->tau, m->beta0, m->beta1, m->beta2, m->rho, m->a, m->b, m->x};
  long pairs = (G + 1) / 2;
  dim3 grid((unsigned)((pairs + 127) / 128), (unsigned)((T + kEmTC - 1) / kEmTC));
  {
    ProfScope ps(ctx, PROF_RNG, 0.0, 24.0 * (double)G * T);
    k_emulate_grid<<<grid, 128, 0, ctx->stream>>>(dZs, G, T, ldz, td, dsigma, dv, seed, stream_id, dY, ldy);
    EMU_LAUNCHED(ctx);
  }
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return EMU_OK;
}

}  // extern "C"
