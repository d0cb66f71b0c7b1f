/*
 * emu_oracle.c -- plain CPU FP64 oracle (TEST INFRASTRUCTURE ONLY; see
 * emu_oracle.h).  Slow on purpose: straight loops in the order the
 * definitions are written, no blocking beyond the tile algorithm itself,
 * OpenMP only across independent columns.  Shares nothing with the CUDA
 * library.
 */
#include "emu_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ---------------------------------------------------------------- indexing */
void orc_lm_of_index(long k, int *l, int *m) {
  /* k = l^2 + l + m with |m| <= l, so l = floor(sqrt(k)). */
  long ll = 0;
  while ((ll + 1) * (ll + 1) <= k) ll++;
  *l = (int)ll;
  *m = (int)(k - ll * ll - ll);
}

/* -------------------------------------------------------------- covariance */
void orc_cov_build(int L, double beta, double sigma_exp, double nugget_rel,
                   double *S, long ld) {
  long n = (long)L * L;
#pragma omp parallel for schedule(static)
  for (long j = 0; j < n; j++) {
    int lj, mj;
    orc_lm_of_index(j, &lj, &mj);
    double sj = pow(1.0 + lj, -sigma_exp);
    for (long i = 0; i < n; i++) {
      int li, mi;
      orc_lm_of_index(i, &li, &mi);
      double si = pow(1.0 + li, -sigma_exp);
      double dl = (double)(li - lj), dm = (double)(mi - mj);
      double d = sqrt(dl * dl + dm * dm);
      S[IDX(i, j, ld)] = si * sj * exp(-d / beta);
    }
  }
  double dmax = 0.0;
  for (long k = 0; k < n; k++)
    if (S[IDX(k, k, ld)] > dmax) dmax = S[IDX(k, k, ld)];
  for (long k = 0; k < n; k++) S[IDX(k, k, ld)] += nugget_rel * dmax;
}

void orc_cov_rows(int L, double beta, double sigma_exp, double nugget_rel,
                  const long *rows, int nrows, double *out) {
  long n = (long)L * L;
  /* max diagonal entry: the diagonal of the correlation part is exp(0) = 1 */
  double dmax = 0.0;
  for (int l = 0; l < L; l++) {
    double s = pow(1.0 + l, -sigma_exp);
    if (s * s > dmax) dmax = s * s;
  }
#pragma omp parallel for schedule(static)
  for (int q = 0; q < nrows; q++) {
    long i = rows[q];
    int li, mi;
    orc_lm_of_index(i, &li, &mi);
    double si = pow(1.0 + li, -sigma_exp);
    for (long j = 0; j < n; j++) {
      int lj, mj;
      orc_lm_of_index(j, &lj, &mj);
      double sj = pow(1.0 + lj, -sigma_exp);
      double dl = (double)(li - lj), dm = (double)(mi - mj);
      double v = si * sj * exp(-sqrt(dl * dl + dm * dm) / beta);
      if (j == i) v += nugget_rel * dmax;
      out[q + j * (long)nrows] = v;
    }
  }
}

/* ------------------------------------------------------ norms and the map */
void orc_tile_norms(int n, const double *S, long ld, int nb, double *t) {
  int NT = (n + nb - 1) / nb;
  for (int j = 0; j < NT; j++) {
    for (int i = 0; i < NT; i++) {
      if (i < j) {
        t[i + (size_t)j * NT] = 0.0;
        continue;
      }
      double ss = 0.0;
      int r1 = (i + 1) * nb < n ? (i + 1) * nb : n;
      int c1 = (j + 1) * nb < n ? (j + 1) * nb : n;
      for (int c = j * nb; c < c1; c++) {
        for (int r = i * nb; r < r1; r++) {
          if (i == j && r < c) continue; /* lower triangle only */
          double v = S[IDX(r, c, ld)];
          double w = (i == j && r != c) ? 2.0 : 1.0; /* mirrored entry */
          ss += w * v * v;
        }
      }
      t[i + (size_t)j * NT] = sqrt(ss);
    }
  }
}

double orc_frob_from_tiles(int NT, const double *t) {
  double ss = 0.0;
  for (int j = 0; j < NT; j++)
    for (int i = j; i < NT; i++) {
      double v = t[i + (size_t)j * NT];
      ss += (i == j ? 1.0 : 2.0) * v * v;
    }
  return sqrt(ss);
}

void orc_precision_map(int NT, const double *t, double eps, const double *u,
                       int nclass, unsigned mask, int diag_fp64,
                       unsigned char *cls) {
  double thr = eps * orc_frob_from_tiles(NT, t) / (double)NT;
  for (int j = 0; j < NT; j++)
    for (int i = 0; i < NT; i++) {
      if (i < j) {
        cls[i + (size_t)j * NT] = 255;
        continue;
      }
      int c = 0;
      if (!(diag_fp64 && i == j)) {
        for (int cc = nclass - 1; cc >= 1; cc--) {
          if (((mask >> cc) & 1u) && t[i + (size_t)j * NT] * u[cc] <= thr) {
            c = cc;
            break;
          }
        }
      }
      cls[i + (size_t)j * NT] = (unsigned char)c;
    }
}

/* Band-based precision maps of the paper's experiments ("Performance Results"
 * section: DP, DP/SP, DP/SP/HP with 5 % SP, DP/HP).  band: 1 DP/SP, 2
 * DP/SP/HP, 3 DP/HP.  Classes: 0 FP64 (DP), 1 FP32 (SP), 3 BF16 (HP).  The
 * diagonal band is DP.  For DP/SP/HP the SP tiles are whole sub-diagonal
 * bands nearest the diagonal, as few as hold at least sp_frac of the
 * NT (NT + 1) / 2 lower tiles; the bands beyond are HP.  Returns that number
 * of SP bands (0 for the other maps).  Upper tiles get 255. */
int orc_precision_map_band(int NT, int band, double sp_frac, unsigned char *cls) {
  int nsp = 0;
  if (band == 2 && sp_frac > 0.0) {
    /* count tiles band by band until the SP share is reached */
    double total = 0.5 * (double)NT * (double)(NT + 1);
    long in_sp = 0;
    while (nsp < NT - 1 && (double)in_sp < sp_frac * total) {
      nsp++;
      in_sp += NT - nsp; /* band d holds the NT - d tiles (j + d, j) */
    }
  }
  for (int j = 0; j < NT; j++)
    for (int i = 0; i < NT; i++) {
      unsigned char c;
      if (i < j)
        c = 255;
      else if (i == j)
        c = 0;
      else if (band == 1)
        c = 1;
      else if (band == 3)
        c = 3;
      else
        c = (i - j <= nsp) ? 1 : 3;
      cls[i + (size_t)j * NT] = c;
    }
  return nsp;
}

/* Empirical covariance of residual vectors ("Modeling the Temporal
 * Dependence": U-hat is the sum of xi xi^T over the R (T - P) residual vectors
 * divided by their number, then a perturbation of the diagonal).  Xi is n x m
 * column-major (leading dimension ld), one vector per column.  Writes the full
 * symmetric U (n x n, column-major): U[i,j] = (1/m) sum_t Xi[i,t] Xi[j,t], then
 * U[k,k] += nugget_rel * max_k U[k,k]. */
void orc_cov_from_residuals(int n, long m, const double *Xi, long ld, double nugget_rel, double *U) {
  const double inv_m = 1.0 / (double)m;
  for (int j = 0; j < n; j++)
    for (int i = j; i < n; i++) {
      double s = 0.0;
      for (long t = 0; t < m; t++) s += Xi[i + t * ld] * Xi[j + t * ld];
      U[i + (size_t)j * n] = s * inv_m;
      U[j + (size_t)i * n] = s * inv_m;
    }
  if (nugget_rel > 0.0) {
    double mx = 0.0;
    for (int k = 0; k < n; k++)
      if (U[k + (size_t)k * n] > mx) mx = U[k + (size_t)k * n];
    for (int k = 0; k < n; k++) U[k + (size_t)k * n] += nugget_rel * mx;
  }
}

static const double ORC_PI = 3.14159265358979323846;

/* VAR(P) recursion of the coefficients with diagonal Phi_p ("Modeling the
 * Temporal Dependence"): f_t = sum_{p=1..P} Phi_p f_{t-p} + xi_t, f before
 * t = 0 zero.  Column-major n x T arrays, phi n x P (column p-1 = diag Phi_p). */
void orc_var_recursion(int n, int T, const double *xi, long ldxi, const double *phi, int P, double *f, long ldf) {
  for (int k = 0; k < n; k++)
    for (int t = 0; t < T; t++) {
      double v = 0.0;
      for (int p = 1; p <= P; p++)
        if (t - p >= 0) v += phi[k + (long)(p - 1) * n] * f[k + (long)(t - p) * ldf];
      f[k + (long)t * ldf] = v + xi[k + (long)t * ldxi];
    }
}

/* Mean trend of the decoupled model (Eq. decouple and the distributed-lag
 * trend of "Climate Emulator Design -- Formulation") at one grid point and
 * time step t >= 1:
 *   m_t = b0 + b1 x_y + b2 (1 - rho) sum_{s>=1} rho^(s-1) x_(y-s)
 *         + sum_{k=1..K} { a_k cos(2 pi t k / tau) + b_k sin(2 pi t k / tau) },
 * y = ceil(t / tau).  The forcing trajectory is x[0..nyears]; every year
 * before the first (index <= 0) carries x[0], so the lag terms with y - s <= 0
 * sum in closed form to rho^(y-1) x[0] / (1 - rho) and the infinite sum is
 *   (1 - rho) sum_{s=1..y-1} rho^(s-1) x[y-s] + rho^(y-1) x[0].
 * a and b hold the K harmonic amplitudes of this grid point. */
double orc_mean_trend(long t, double tau, double b0, double b1, double b2, double rho, int K, const double *a,
                      const double *b, const double *x) {
  const double pi = 3.14159265358979323846;
  long y = (long)ceil((double)t / tau);
  double lag = 0.0;
  for (long s = 1; s <= y - 1; s++) lag += pow(rho, (double)(s - 1)) * x[y - s];
  lag = (1.0 - rho) * lag + pow(rho, (double)(y - 1)) * x[0];
  double m = b0 + b1 * x[y] + b2 * lag;
  for (int k = 1; k <= K; k++) {
    double w = 2.0 * pi * (double)t * (double)k / tau;
    m += a[k - 1] * cos(w) + b[k - 1] * sin(w);
  }
  return m;
}

/* Emulations on the grid ("Generating Emulations" and Eq. decouple): for grid
 * point g and time step t = 1..T (column t-1),
 *   Z_t(g) = Zs_t(g) + v(g) e_t(g)          (the nugget eps_t ~ N(0, v^2))
 *   y_t(g) = m_t(g) + sigma(g) Z_t(g),
 * Zs the inverse SHT of the coefficients (G x T, ld ldz), e the standard
 * normals of the nugget (G x T, ld lde; an input, drawn by the caller),
 * per-point trend parameters b0, b1, b2, rho (length G) and amplitudes
 * a, bh (K x G, amplitude k-1 of point g at [k-1 + g K]). */
void orc_emulate_grid(long G, int T, const double *Zs, long ldz, const double *e, long lde, int K, double tau,
                      const double *b0, const double *b1, const double *b2, const double *rho, const double *a,
                      const double *bh, const double *x, const double *sigma, const double *v, double *Y,
                      long ldy) {
  for (long g = 0; g < G; g++)
    for (int t = 1; t <= T; t++) {
      double m = orc_mean_trend(t, tau, b0[g], b1[g], b2[g], rho[g], K, a + g * K, bh + g * K, x);
      double Z = Zs[g + (long)(t - 1) * ldz] + v[g] * e[g + (long)(t - 1) * lde];
      Y[g + (long)(t - 1) * ldy] = m + sigma[g] * Z;
    }
}

/* Real orthonormal spherical harmonic of degree l, order m (|m| <= l) at
 * colatitude theta, longitude phi ("Spherical Harmonic Transform": the
 * orthonormal Y_lm, real form): N_l|m| P_l^|m|(cos theta) times 1 (m = 0),
 * sqrt(2) cos(m phi) (m > 0) or sqrt(2) sin(|m| phi) (m < 0), with
 * N_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)! and P_l^m carrying the
 * Condon-Shortley phase.  P_l^m from the unnormalised three-term recurrence
 * in l, the normalisation through log-factorials (valid while (2m-1)!! stays
 * in range, l < 150). */
double orc_real_sh(int l, int m, double theta, double phi) {
  const int am = m < 0 ? -m : m;
  const double x = cos(theta), sx = sin(theta);
  double pmm = 1.0; /* P_am^am = (-1)^am (2am-1)!! sin^am */
  for (int q = 1; q <= am; q++) pmm *= -(2.0 * q - 1.0) * sx;
  double p = pmm;
  if (l > am) {
    double p0 = pmm, p1 = x * (2.0 * am + 1.0) * pmm; /* l = am + 1 */
    for (int ll = am + 2; ll <= l; ll++) {
      double p2 = ((2.0 * ll - 1.0) * x * p1 - (ll + am - 1.0) * p0) / (double)(ll - am);
      p0 = p1;
      p1 = p2;
    }
    p = p1;
  }
  const double lognorm = 0.5 * (log((2.0 * l + 1.0) / (4.0 * ORC_PI)) + lgamma(l - am + 1.0) - lgamma(l + am + 1.0));
  double y = exp(lognorm) * p;
  if (m > 0) y *= sqrt(2.0) * cos(m * phi);
  if (m < 0) y *= sqrt(2.0) * sin(am * phi);
  return y;
}

/* Inverse spherical-harmonic transform by the synthesis sum: for each column
 * t of F (row k = l^2 + l + m), Z[i + j ntheta, t] = sum_{l,m} F[k, t]
 * Y_lm(theta_i, phi_j), theta_i = pi i / (ntheta - 1), phi_j = 2 pi j / nphi. */
void orc_isht(int L, int T, const double *F, long ldf, int ntheta, int nphi, double *Z, long ldz) {
  for (int i = 0; i < ntheta; i++) {
    const double th = ORC_PI * (double)i / (double)(ntheta - 1);
    for (int j = 0; j < nphi; j++) {
      const double ph = 2.0 * ORC_PI * (double)j / (double)nphi;
      for (int t = 0; t < T; t++) Z[i + (long)j * ntheta + (long)t * ldz] = 0.0;
      for (int l = 0; l < L; l++)
        for (int m = -l; m <= l; m++) {
          const double y = orc_real_sh(l, m, th, ph);
          const long k = (long)l * l + l + m;
          for (int t = 0; t < T; t++) Z[i + (long)j * ntheta + (long)t * ldz] += F[k + (long)t * ldf] * y;
        }
    }
  }
}

/* Forward spherical-harmonic transform on the equiangular grid of orc_isht
 * ("Spherical Harmonic Transform": the coefficient as the integral of Z times
 * Y_lm over the sphere, computed through G_m(theta), its extension to the
 * full circle in theta, its Fourier coefficients K, and the integrals
 * I(q) = int_0^pi e^{i q t} sin t dt).  Real-form coefficients of the basis of
 * orc_real_sh.  Steps, per column t of Z:
 *   C_m(t_i) = (2 pi / nphi) sum_j Z_ij cos(m p_j),  S_m(t_i) = (same) sin(m p_j);
 *   g(t_{M-i}) = (-1)^m g(t_i) extends g in {C_m, S_m} to M = 2 ntheta - 2 points
 *     t_i = 2 pi i / M of the circle (Z(2pi - t, p) = Z(t, p + pi));
 *   K_q = (1/M) sum_i g(t_i) e^{-i q t_i},  |q| < L;
 *   h_lm(t) = c_m N_lm P_l^m(cos t) extends the same way; its coefficients
 *     c_q' likewise; S_{l,m,q} = sum_q' c_q' I(q + q');
 *   f_{l,m} = Re sum_q K_q(C_m) S_{l,m,q},  f_{l,-m} = Re sum_q K_q(S_m) S_{l,m,q}.
 * Exact for data band-limited at L when ntheta > L and nphi >= 2L - 1. */
static void orc_I(int k, double *re, double *im) {
  if (k == 1 || k == -1) {
    *re = 0.0;
    *im = k * ORC_PI / 2.0;
  } else {
    *re = (k % 2 == 0) ? 2.0 / (1.0 - (double)k * k) : 0.0;
    *im = 0.0;
  }
}
void orc_I_pub(int k, double *re, double *im) { orc_I(k, re, im); }

void orc_sht(int L, int T, const double *Z, long ldz, int ntheta, int nphi, double *F, long ldf) {
  const int M = 2 * ntheta - 2, Q = 2 * L - 1;
  double *g = (double *)malloc(sizeof(double) * M);
  double *Kr = (double *)malloc(sizeof(double) * Q), *Ki = (double *)malloc(sizeof(double) * Q);
  double *cr = (double *)malloc(sizeof(double) * Q), *ci = (double *)malloc(sizeof(double) * Q);
  double *Sr = (double *)malloc(sizeof(double) * Q), *Si = (double *)malloc(sizeof(double) * Q);
  double *CS = (double *)malloc(sizeof(double) * 2 * (size_t)L * ntheta);
  for (int t = 0; t < T; t++) {
    const double *z = Z + (long)t * ldz;
    /* C_m, S_m on the ntheta rings */
    for (int m = 0; m < L; m++)
      for (int i = 0; i < ntheta; i++) {
        double c = 0.0, sn = 0.0;
        for (int j = 0; j < nphi; j++) {
          const double ph = 2.0 * ORC_PI * (double)(((long)m * j) % nphi) / (double)nphi;
          c += z[i + (long)j * ntheta] * cos(ph);
          sn += z[i + (long)j * ntheta] * sin(ph);
        }
        CS[(2 * m) * ntheta + i] = c * 2.0 * ORC_PI / nphi;
        CS[(2 * m + 1) * ntheta + i] = sn * 2.0 * ORC_PI / nphi;
      }
    for (int m = 0; m < L; m++) {
      const double sgn = (m % 2 == 0) ? 1.0 : -1.0;
      for (int cs = 0; cs < 2; cs++) {
        if (m == 0 && cs == 1) continue;
        /* extension and Fourier coefficients of g */
        for (int i = 0; i < ntheta; i++) g[i] = CS[(2 * m + cs) * ntheta + i];
        for (int i = ntheta; i < M; i++) g[i] = sgn * g[M - i];
        for (int q = -(L - 1); q <= L - 1; q++) {
          double re = 0.0, im = 0.0;
          for (int i = 0; i < M; i++) {
            const double a = 2.0 * ORC_PI * (double)((((long)q * i) % M + M) % M) / (double)M;
            re += g[i] * cos(a);
            im -= g[i] * sin(a);
          }
          Kr[q + L - 1] = re / M;
          Ki[q + L - 1] = im / M;
        }
        for (int l = m; l < L; l++) {
          /* coefficients of h_lm on the same circle, then S and the contraction */
          for (int i = 0; i < ntheta; i++) g[i] = orc_real_sh(l, m, 2.0 * ORC_PI * i / M, 0.0);
          for (int i = ntheta; i < M; i++) g[i] = sgn * g[M - i];
          for (int q = -(L - 1); q <= L - 1; q++) {
            double re = 0.0, im = 0.0;
            for (int i = 0; i < M; i++) {
              const double a = 2.0 * ORC_PI * (double)((((long)q * i) % M + M) % M) / (double)M;
              re += g[i] * cos(a);
              im -= g[i] * sin(a);
            }
            cr[q + L - 1] = re / M;
            ci[q + L - 1] = im / M;
          }
          double fr = 0.0;
          for (int q = -(L - 1); q <= L - 1; q++) {
            double sr = 0.0, si = 0.0;
            for (int q2 = -(L - 1); q2 <= L - 1; q2++) {
              double ir, ii;
              orc_I(q + q2, &ir, &ii);
              sr += cr[q2 + L - 1] * ir - ci[q2 + L - 1] * ii;
              si += cr[q2 + L - 1] * ii + ci[q2 + L - 1] * ir;
            }
            fr += Kr[q + L - 1] * sr - Ki[q + L - 1] * si;
          }
          const long k = (long)l * l + l + (cs == 0 ? m : -m);
          F[k + (long)t * ldf] = fr;
        }
      }
    }
  }
  free(g);
  free(Kr);
  free(Ki);
  free(cr);
  free(ci);
  free(Sr);
  free(Si);
  free(CS);
}

/* -------------------------------------------------------------- Cholesky */
int orc_potrf_unblocked(int n, double *A, long ld) {
  /* Cholesky-Banachiewicz: row i of L from rows 0..i-1. */
  for (int i = 0; i < n; i++) {
    for (int j = 0; j <= i; j++) {
      double s = A[IDX(i, j, ld)];
      for (int p = 0; p < j; p++) s -= A[IDX(i, p, ld)] * A[IDX(j, p, ld)];
      if (i == j) {
        if (!(s > 0.0)) return i + 1;
        A[IDX(i, i, ld)] = sqrt(s);
      } else {
        A[IDX(i, j, ld)] = s / A[IDX(j, j, ld)];
      }
    }
  }
  return 0;
}

/* Diagonal-block factor used inside the blocked algorithm: column-by-column
 * (Cholesky-Crout), a different loop order from the unblocked routine above
 * so that the two cross-check each other. */
static int potrf_block(int kb, double *A, long ld) {
  for (int j = 0; j < kb; j++) {
    double d = A[IDX(j, j, ld)];
    for (int p = 0; p < j; p++) d -= A[IDX(j, p, ld)] * A[IDX(j, p, ld)];
    if (!(d > 0.0)) return j + 1;
    d = sqrt(d);
    A[IDX(j, j, ld)] = d;
    for (int i = j + 1; i < kb; i++) {
      double s = A[IDX(i, j, ld)];
      for (int p = 0; p < j; p++) s -= A[IDX(i, p, ld)] * A[IDX(j, p, ld)];
      A[IDX(i, j, ld)] = s / d;
    }
  }
  return 0;
}

int orc_potrf_blocked_steps(int n, int nb, double *A, long ld, int k0, int k1) {
  int NT = (n + nb - 1) / nb;
  if (k1 > NT) k1 = NT;
  for (int k = k0; k < k1; k++) {
    int c0 = k * nb;
    int kb = (c0 + nb <= n) ? nb : n - c0;
    /* POTRF(k,k) */
    int info = potrf_block(kb, &A[IDX(c0, c0, ld)], ld);
    if (info) return c0 + info;
    int r0 = c0 + kb;
    if (r0 >= n) break;
    /* TRSM: A(r0:n, c0:c0+kb) <- A(r0:n, c0:c0+kb) * L_kk^{-T}, i.e. each row
     * x solves L_kk x^T = a^T by forward substitution over the columns. */
    for (int c = 0; c < kb; c++) {
      double *xc = &A[IDX(r0, c0 + c, ld)];
      for (int p = 0; p < c; p++) {
        double l = A[IDX(c0 + c, c0 + p, ld)];
        const double *xp = &A[IDX(r0, c0 + p, ld)];
        for (int i = 0; i < n - r0; i++) xc[i] -= xp[i] * l;
      }
      double d = A[IDX(c0 + c, c0 + c, ld)];
      for (int i = 0; i < n - r0; i++) xc[i] /= d;
    }
    /* SYRK/GEMM: A(j:n, j) -= A(j:n, panel) * A(j, panel)^T for j >= r0. */
#pragma omp parallel for schedule(dynamic, 8)
    for (int j = r0; j < n; j++) {
      double *cj = &A[IDX(j, j, ld)];
      for (int p = 0; p < kb; p++) {
        double ajp = A[IDX(j, c0 + p, ld)];
        const double *ap = &A[IDX(j, c0 + p, ld)];
        for (int i = 0; i < n - j; i++) cj[i] -= ap[i] * ajp;
      }
    }
  }
  return 0;
}

int orc_potrf_blocked(int n, int nb, double *A, long ld, int kmax) {
  int NT = (n + nb - 1) / nb;
  if (kmax < 0 || kmax > NT) kmax = NT;
  return orc_potrf_blocked_steps(n, nb, A, ld, 0, kmax);
}

/* ----------------------------------------------------- sampling and solve */
void orc_trmm_lower(int n, int s, const double *Lf, long ldl, const double *Z,
                    long ldz, double *Y, long ldy) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < s; c++) {
    double *y = &Y[IDX(0, c, ldy)];
    for (int i = 0; i < n; i++) y[i] = 0.0;
    for (int p = 0; p < n; p++) {
      double z = Z[IDX(p, c, ldz)];
      const double *lp = &Lf[IDX(0, p, ldl)];
      for (int i = p; i < n; i++) y[i] += lp[i] * z;
    }
  }
}

void orc_potrs(int n, int nrhs, const double *Lf, long ldl, const double *B,
               long ldb, double *X, long ldx) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < nrhs; c++) {
    double *x = &X[IDX(0, c, ldx)];
    for (int i = 0; i < n; i++) x[i] = B[IDX(i, c, ldb)];
    /* L y = b */
    for (int p = 0; p < n; p++) {
      x[p] /= Lf[IDX(p, p, ldl)];
      const double *lp = &Lf[IDX(0, p, ldl)];
      for (int i = p + 1; i < n; i++) x[i] -= lp[i] * x[p];
    }
    /* L^T x = y */
    for (int p = n - 1; p >= 0; p--) {
      const double *lp = &Lf[IDX(0, p, ldl)];
      double s = x[p];
      for (int i = p + 1; i < n; i++) s -= lp[i] * x[i];
      x[p] = s / Lf[IDX(p, p, ldl)];
    }
  }
}

double orc_logdet_chol(int n, const double *Lf, long ldl) {
  double s = 0.0;
  for (int k = 0; k < n; k++) s += log(Lf[IDX(k, k, ldl)]);
  return 2.0 * s;
}

double orc_backward_error(int n, const double *A, long lda, const double *Lf,
                          long ldl) {
  double num = 0.0, den = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : num, den)
  for (int j = 0; j < n; j++) {
    for (int i = j; i < n; i++) {
      double m = 0.0;
      for (int p = 0; p <= j; p++) m += Lf[IDX(i, p, ldl)] * Lf[IDX(j, p, ldl)];
      double a = A[IDX(i, j, lda)];
      double w = (i == j) ? 1.0 : 2.0;
      num += w * (m - a) * (m - a);
      den += w * a * a;
    }
  }
  return sqrt(num) / sqrt(den);
}

/* ------------------------------------------------------------------- RNG */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u; /* Weyl sequence key schedule */
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_uniform_pair(uint64_t seed, uint32_t stream, long p, int c,
                      double *u1, double *u2) {
  uint32_t ctr[4] = {(uint32_t)((uint64_t)p & 0xffffffffu),
                     (uint32_t)((uint64_t)p >> 32), (uint32_t)c, stream};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  uint64_t a = ((uint64_t)w[0] << 21) | (uint64_t)(w[1] >> 11); /* 53 bits */
  uint64_t b = ((uint64_t)w[2] << 21) | (uint64_t)(w[3] >> 11);
  *u1 = ((double)a + 1.0) * 0x1.0p-53; /* (0, 1] */
  *u2 = (double)b * 0x1.0p-53;         /* [0, 1) */
}

void orc_normal_matrix(uint64_t seed, uint32_t stream, int n, int s, double *Z,
                       long ldz) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int c = 0; c < s; c++) {
    for (int r = 0; r < n; r += 2) {
      double u1, u2;
      orc_uniform_pair(seed, stream, r / 2, c, &u1, &u2);
      double rad = sqrt(-2.0 * log(u1));
      double th = two_pi * u2;
      Z[IDX(r, c, ldz)] = rad * cos(th);
      if (r + 1 < n) Z[IDX(r + 1, c, ldz)] = rad * sin(th);
    }
  }
}
