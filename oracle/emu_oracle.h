/*
 * emu_oracle.h -- plain CPU FP64 oracle for the spherical-harmonic emulator's
 * covariance factorisation and sampling path (arXiv 2408.04440).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that tests, the smoke
 * check and the benchmark's CPU-baseline leg can compare the CUDA library
 * against an obviously correct, slow reference.  The product path never links,
 * loads or calls it, and it shares no code, header, table or constant with the
 * CUDA library.
 *
 * Storage convention: every matrix is a full, dense, column-major FP64 array
 * with leading dimension `ld`; only the lower triangle of symmetric inputs is
 * read and only the lower triangle of a Cholesky factor is written.
 *
 * Pins (tests/test_oracle.py): exact recovery of an integer factor, blocked vs
 * unblocked agreement, log-det vs eigenvalue sum, backward error, closed-form
 * covariance entries, Philox known-answer vectors, Box-Muller moments.
 */
#ifndef EMU_ORACLE_H
#define EMU_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Row k of the coefficient vector holds the spherical-harmonic coefficient
 * (l, m) with k = l*l + l + m, 0 <= l < L, -l <= m <= l: ordered by degree l,
 * then order m.  The coefficient vector (z_00, ..., z_{L-1,L-1}) has L^2 rows
 * (Section "Modeling the Temporal Dependence"). */
void orc_lm_of_index(long k, int *l, int *m);

/* Synthetic stand-in for the empirical covariance U-hat of the VAR residuals
 * (Section "Modeling the Temporal Dependence", equation for U-hat):
 *   S[i,j] = s(l_i) s(l_j) exp(-|| (l_i,m_i) - (l_j,m_j) ||_2 / beta),
 *   s(l) = (1 + l)^(-sigma_exp),
 * then the diagonal perturbation ("nugget") that keeps the matrix positive
 * definite: S[k,k] += nugget_rel * max_k S[k,k].  Writes the full n x n
 * matrix (n = L^2), both triangles. */
void orc_cov_build(int L, double beta, double sigma_exp, double nugget_rel,
                   double *S, long ld);

/* Selected rows of the same covariance: out[q + c*nrows] = S[rows[q], c]
 * for c < n (nrows x n, column-major), without forming the full matrix. */
void orc_cov_rows(int L, double beta, double sigma_exp, double nugget_rel,
                  const long *rows, int nrows, double *out);

/* Frobenius norm of every lower tile (i >= j) of the tiling with tile size nb
 * (the last tile row/column is ragged when nb does not divide n).
 * t[i + j*NT] = ||S_ij||_F, NT = ceil(n/nb); upper entries set to 0. */
void orc_tile_norms(int n, const double *S, long ld, int nb, double *t);

/* ||S||_F of the full symmetric matrix from its lower tile norms:
 * sqrt( sum_i t_ii^2 + 2 sum_{i>j} t_ij^2 ). */
double orc_frob_from_tiles(int NT, const double *t);

/* Per-tile precision rule: tile (i,j) may use precision class c (unit
 * roundoff u[c]) only if t_ij * u[c] <= eps * ||S||_F / NT.  Classes are
 * numbered from the most precise (0 = FP64) to the least; the tile takes the
 * least precise class in `mask` (bit c = class c enabled) that satisfies the
 * rule, and class 0 when none does.  diag_fp64 != 0 pins diagonal tiles to
 * class 0.  cls[i + j*NT] for i >= j; upper entries set to 255. */
void orc_precision_map(int NT, const double *t, double eps, const double *u,
                       int nclass, unsigned mask, int diag_fp64,
                       unsigned char *cls);
int orc_precision_map_band(int NT, int band, double sp_frac, unsigned char *cls);
void orc_cov_from_residuals(int n, long m, const double *Xi, long ld, double nugget_rel, double *U);
void orc_var_recursion(int n, int T, const double *xi, long ldxi, const double *phi, int P, double *f, long ldf);
double orc_real_sh(int l, int m, double theta, double phi);
double orc_mean_trend(long t, double tau, double b0, double b1, double b2, double rho, int K, const double *a,
                      const double *b, const double *x);
void orc_emulate_grid(long G, int T, const double *Zs, long ldz, const double *e, long lde, int K, double tau,
                      const double *b0, const double *b1, const double *b2, const double *rho, const double *a,
                      const double *bh, const double *x, const double *sigma, const double *v, double *Y,
                      long ldy);
void orc_isht(int L, int T, const double *F, long ldf, int ntheta, int nphi, double *Z, long ldz);
void orc_sht(int L, int T, const double *Z, long ldz, int ntheta, int nphi, double *F, long ldf);
void orc_I_pub(int k, double *re, double *im);

/* Unblocked Cholesky (row-by-row, the textbook Cholesky-Banachiewicz form):
 * A = L L^T, L lower with positive diagonal, overwritten in place.
 * Returns 0, or the 1-based column of the first non-positive pivot. */
int orc_potrf_unblocked(int n, double *A, long ld);

/* Right-looking blocked Cholesky with block size nb, the tile algorithm of
 * the paper's DAG (POTRF on the diagonal tile, TRSM on the panel, SYRK/GEMM
 * on the trailing tiles).  Runs panel steps k = 0 .. kmax-1 (kmax < 0: all).
 * Returns 0, or the 1-based global column of the first non-positive pivot. */
int orc_potrf_blocked(int n, int nb, double *A, long ld, int kmax);
/* Panel steps k0 .. k1-1 of the same algorithm on a matrix whose steps
 * 0 .. k0-1 are already done. */
int orc_potrf_blocked_steps(int n, int nb, double *A, long ld, int k0, int k1);

/* Y = L Z for lower-triangular L (n x n) and Z (n x s): drawing emulations
 * xi = V z (Section "Generating Emulations"). */
void orc_trmm_lower(int n, int s, const double *Lf, long ldl, const double *Z,
                    long ldz, double *Y, long ldy);

/* Solve (L L^T) X = B by forward then backward substitution. */
void orc_potrs(int n, int nrhs, const double *Lf, long ldl, const double *B,
               long ldb, double *X, long ldx);

/* log det(L L^T) = 2 sum_k log L[k,k]. */
double orc_logdet_chol(int n, const double *Lf, long ldl);

/* ||A - L L^T||_F / ||A||_F over the full symmetric matrix (A read from
 * its lower triangle). */
double orc_backward_error(int n, const double *A, long lda, const double *Lf,
                          long ldl);

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* Standard normals for an n x s matrix Z, independent of any launch shape:
 * entry (r, c) is drawn from counter {r/2, 0, c, stream} under key
 * {seed_lo, seed_hi}; the four output words give two 53-bit uniforms
 * u1 in (0,1], u2 in [0,1) and Box-Muller gives the pair
 * (sqrt(-2 ln u1) cos(2 pi u2), sqrt(-2 ln u1) sin(2 pi u2)) for rows
 * (2p, 2p+1). */
void orc_normal_matrix(uint64_t seed, uint32_t stream, int n, int s, double *Z,
                       long ldz);
/* The two uniforms of counter (p, c, stream) under `seed`, for tests. */
void orc_uniform_pair(uint64_t seed, uint32_t stream, long p, int c,
                      double *u1, double *u2);

#ifdef __cplusplus
}
#endif
#endif
