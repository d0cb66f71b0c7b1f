"""Pins for the CPU oracle against facts that do not come from the oracle itself:
exact recovery of a known integer factor, two different Cholesky loop orders,
eigenvalue log-determinants, backward error, closed-form covariance values,
published Philox known-answer vectors, hand-derived precision maps and the
distribution of the Box-Muller normals.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = np.array([2.0**-53, 2.0**-24, 2.0**-11, 2.0**-8, 2.0**-4])


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.logspace(0, -math.log10(cond), n)
    return np.asfortranarray((Q * ev) @ Q.T)


def _int_factor(n, seed):
    """Lower-triangular integer L0, entries in [-3, 3], diagonal 2^k, k in {1,2,3}."""
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.integers(-3, 4, size=(n, n)).astype(np.float64), -1)
    L0[np.diag_indices(n)] = 2.0 ** rng.integers(1, 4, size=n)
    return L0


# ------------------------------------------------------------------ factor
@pytest.mark.parametrize("n,nb", [(1, 1), (7, 3), (32, 8), (64, 16), (64, 64), (50, 16)])
def test_exact_recovery_of_integer_factor(n, nb):
    # Sigma = L0 L0^T is exact in FP64 (small integers); every division is by a
    # power of two and every square root is of a perfect square, so both
    # algorithms must return L0 bit for bit.
    L0 = _int_factor(n, seed=n * 131 + nb)
    S = np.asfortranarray(L0 @ L0.T)
    Lu, iu = O.potrf_unblocked(S)
    Lb, ib = O.potrf_blocked(S, nb)
    assert iu == 0 and ib == 0
    assert np.array_equal(Lu, L0)
    assert np.array_equal(Lb, L0)


@pytest.mark.parametrize("n,nb", [(256, 64), (200, 64), (130, 17), (96, 128)])
def test_blocked_matches_unblocked(n, nb):
    S = _spd(n, seed=n + nb)
    Lu, _ = O.potrf_unblocked(S)
    Lb, _ = O.potrf_blocked(S, nb)
    assert np.linalg.norm(Lb - Lu) / np.linalg.norm(Lu) < 1e-14
    assert np.all(np.diag(Lb) > 0)
    assert np.all(np.triu(Lb, 1) == 0)


@pytest.mark.parametrize("n", [16, 100, 512])
def test_logdet_equals_eigenvalue_sum(n):
    S = _spd(n, seed=7 * n, cond=1e4)
    Lb, _ = O.potrf_blocked(S, 32)
    ld = O.logdet_chol(Lb)
    ref = float(np.sum(np.log(np.linalg.eigvalsh(S))))
    assert abs(ld - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("L,nb,beta", [(8, 16, 4.0), (16, 64, 4.0), (32, 128, 4.0)])
def test_backward_error_on_covariance(L, nb, beta):
    S = O.cov_build(L, beta)
    Lb, info = O.potrf_blocked(S, nb)
    assert info == 0
    assert np.all(np.diag(Lb) > 0)
    rel = np.linalg.norm(Lb @ Lb.T - S) / np.linalg.norm(S)
    assert rel <= 1e-13
    # the oracle's own backward-error routine agrees with numpy's product
    assert abs(O.backward_error(S, Lb) - rel) <= 1e-15 + 1e-3 * rel


def test_partial_factor_steps():
    # kmax panel steps leave the first kmax*nb columns final and the trailing
    # block equal to its Schur complement.
    S = _spd(96, seed=3)
    A, info = O.potrf_blocked(S, 32, kmax=1, inplace=False)
    assert info == 0
    Lfull, _ = O.potrf_blocked(S, 32)
    assert np.allclose(A[:, :32], Lfull[:, :32], rtol=0, atol=1e-13)
    L11 = Lfull[:32, :32]
    L21 = Lfull[32:, :32]
    schur = S[32:, 32:] - L21 @ L21.T
    assert np.allclose(np.tril(A[32:, 32:]), np.tril(schur), atol=1e-13)
    assert np.allclose(L11 @ L11.T, S[:32, :32], atol=1e-13)


@pytest.mark.parametrize("blocked", [False, True])
def test_not_positive_definite_reports_pivot(blocked):
    n = 40
    S = np.asfortranarray(np.eye(n))
    S[22, 22] = -1.0  # first failing pivot: column 23 (1-based)
    if blocked:
        _, info = O.potrf_blocked(S, 16)
    else:
        _, info = O.potrf_unblocked(S)
    assert info == 23


# -------------------------------------------------------------- covariance
def test_index_order_by_degree_then_order():
    k = 0
    for l in range(12):
        for m in range(-l, l + 1):
            assert O.lm_of_index(k) == (l, m)
            k += 1


def test_covariance_closed_form_values():
    L, beta = 8, 4.0
    S = O.cov_build(L, beta)
    n = L * L
    assert S.shape == (n, n)
    assert np.array_equal(S, S.T)
    # sigma_0 = 1 is the largest diagonal entry, so the nugget is 1e-8 exactly
    assert S[0, 0] == 1.0 + 1e-8
    # diagonal: (1+l)^-3 + 1e-8; for l = 1, 3, 7 this is 1/8, 1/64, 1/512
    for l, v in [(1, 1 / 8), (3, 1 / 64), (7, 1 / 512)]:
        k = l * l + l
        assert abs(S[k, k] - (v + 1e-8)) <= 4e-16 * v
    # correlation depends on the distance between (l,m) pairs only and is
    # exp(-d/beta): collinear steps multiply, rho(d1 + d2) = rho(d1) rho(d2)
    D = np.sqrt(np.diag(S) - 1e-8)
    R = S / np.outer(D, D)

    def rho(a, b):
        return R[a[0] ** 2 + a[0] + a[1], b[0] ** 2 + b[0] + b[1]]

    assert abs(rho((2, 0), (4, 0)) - rho((2, 0), (3, 0)) * rho((3, 0), (4, 0))) < 1e-15
    assert abs(rho((3, -2), (3, 2)) - rho((3, -2), (3, 0)) ** 2) < 1e-15
    # translation invariance in (l, m)
    assert abs(rho((2, 1), (5, 3)) - rho((3, 1), (6, 3))) < 1e-15
    # unit distance: rho = e^{-1/beta}; distance 5 via the 3-4-5 triangle
    assert abs(rho((4, 0), (5, 0)) - math.exp(-0.25)) < 1e-15
    assert abs(rho((1, 0), (4, 4)) - math.exp(-5 / 4)) < 1e-15


def test_covariance_limits_and_definiteness():
    # beta -> 0 removes all correlation: S = diag((1+l)^-3) + nugget
    S0 = O.cov_build(5, 1e-4)
    off = S0 - np.diag(np.diag(S0))
    assert np.max(np.abs(off)) == 0.0
    # the exponential kernel is positive definite, so lambda_min >= nugget
    S = O.cov_build(8, 4.0)
    lam = np.linalg.eigvalsh(S)
    assert lam.min() >= 1e-8 * (1 - 1e-6)


@pytest.mark.parametrize("L,beta,sigma_exp,nugget", [
    (5, 2.0, 1.5, 1e-8),
    (16, 8.0, 1.5, 1e-8),
    (33, 12.0, 1.5, 1e-8),
    # growing sigma_l: the largest diagonal entry is the last degree's, not
    # sigma_0's, so the nugget's max-diagonal rule is exercised off l = 0
    (9, 3.0, -0.75, 1e-3),
    # a negative nugget (the indefinite inputs of the not-positive-definite tests)
    (12, 3.0, 1.5, -1e-3),
])
def test_cov_rows_equals_rows_of_full_build(L, beta, sigma_exp, nugget):
    """The row generator (used as the expected value at sizes where the full
    matrix does not fit) is the full build's rows bit for bit: same entries,
    same nugget, same index decode (Modeling the Temporal Dependence...: the
    covariance and its diagonal perturbation)."""
    n = L * L
    S = O.cov_build(L, beta, sigma_exp=sigma_exp, nugget_rel=nugget)
    rows = {0, n - 1, n // 2, n // 3 + 1}
    rows |= {l * l + l for l in range(L)}          # m = 0 of every degree
    rows |= {l * l for l in range(L)}              # m = -l
    rows |= {l * l + 2 * l for l in range(L)}      # m = +l
    rows = np.array(sorted(rows), dtype=np.int64)
    R = O.cov_rows(L, beta, rows, sigma_exp=sigma_exp, nugget_rel=nugget)
    assert R.shape == (len(rows), n)
    assert np.array_equal(R, S[rows, :])
    # every row carries the nugget on its diagonal entry and nowhere else
    dmax = max((1.0 + l) ** (-2 * sigma_exp) for l in range(L))
    for q, i in enumerate(rows):
        l = int(math.isqrt(int(i)))
        s2 = (1.0 + l) ** (-2 * sigma_exp)
        # relative to the terms, not to their sum (a negative nugget cancels)
        assert abs(R[q, i] - (s2 + nugget * dmax)) <= 4e-16 * (s2 + abs(nugget) * dmax)


def test_tile_norms_against_numpy():
    S = O.cov_build(10, 3.0)  # n = 100, ragged with nb = 32
    nb = 32
    t = O.tile_norms(S, nb)
    NT = 4
    for i in range(NT):
        for j in range(NT):
            blk = S[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]
            ref = np.linalg.norm(blk) if i >= j else 0.0
            assert abs(t[i, j] - ref) <= 1e-14 * max(ref, 1e-300)
    assert abs(O.frob_from_tiles(t) - np.linalg.norm(S)) <= 1e-14 * np.linalg.norm(S)


# ------------------------------------------------------------ precision map
def _hand_cases():
    rows = []
    with open(os.path.join(GOLDEN, "precision_map_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split(":")
            eps, mask, dg = lhs.split()
            rows.append((float(eps), int(mask), int(dg), [int(x) for x in rhs.split()]))
    return rows


@pytest.mark.parametrize("eps,mask,dg,expect", _hand_cases())
def test_precision_map_hand_derived(eps, mask, dg, expect):
    t = np.array([[2.0, 0.0], [1e-6, 1.0]], order="F")
    c = O.precision_map(t, eps, U, mask, bool(dg))
    assert [c[0, 0], c[1, 0], c[1, 1]] == expect
    assert c[0, 1] == 255


def test_precision_map_properties():
    S = O.cov_build(16, 6.0)
    t = O.tile_norms(S, 32)
    NT = t.shape[0]
    for eps in [1e-12, 1e-8, 1e-6, 1e-3]:
        c = O.precision_map(t, eps, U, 0b11111, False)
        thr = eps * np.linalg.norm(S) / NT
        err2 = 0.0
        for i in range(NT):
            for j in range(i + 1):
                cc = c[i, j]
                assert cc == 0 or t[i, j] * U[cc] <= thr
                for lower in range(cc + 1, 5):  # every less precise class fails
                    assert t[i, j] * U[lower] > thr
                err2 += (1 if i == j else 2) * (t[i, j] * U[cc]) ** 2
        # the rule's purpose: summed tile-level rounding stays below eps*||S||
        assert math.sqrt(err2) <= eps * np.linalg.norm(S) * (1 + 1e-12) or np.all(
            c[np.tril_indices(NT)] == 0)
    # eps tiny -> all fp64; eps huge -> everything in the least precise class
    assert np.all(O.precision_map(t, 1e-300, U, 31)[np.tril_indices(NT)] == 0)
    assert np.all(O.precision_map(t, 1e6, U, 31)[np.tril_indices(NT)] == 4)
    assert np.all(O.precision_map(t, 1e6, U, 0b01011)[np.tril_indices(NT)] == 3)


# The paper's band variants ("Performance Results": DP, DP/SP, DP/SP/HP with
# 5 % SP, DP/HP).  Counts below are worked by hand from the definition: NT(NT+1)/2
# lower tiles, NT on the diagonal (DP), band d holding NT - d tiles.
@pytest.mark.parametrize("NT,band,frac,expect", [
    (7, 1, 0.05, (7, 21, 0)),          # DP/SP: the 21 off-diagonal tiles are SP
    (7, 3, 0.05, (7, 0, 21)),          # DP/HP
    (32, 2, 0.05, (32, 31, 465)),      # 5 % of 528 = 26.4 <= band 1 (31 tiles)
    (100, 2, 0.05, (100, 294, 4656)),  # 5 % of 5050 = 252.5: bands 1..3 = 99+98+97 = 294
    (100, 2, -1.0, (100, 0, 4950)),    # no SP bands
    (4, 2, 0.99, (4, 6, 0)),           # the share cannot be reached: every off-diagonal band SP
])
def test_band_maps_hand_derived(NT, band, frac, expect):
    c, nsp = O.precision_map_band(NT, band, frac)
    low = c[np.tril_indices(NT)]
    assert (int((low == 0).sum()), int((low == 1).sum()), int((low == 3).sum())) == expect
    assert np.all(np.diag(c) == 0) and np.all(c[np.triu_indices(NT, 1)] == 255)
    # classes depend only on the band i - j, and SP bands come before HP bands
    for d in range(1, NT):
        band_cls = {int(c[j + d, j]) for j in range(NT - d)}
        assert len(band_cls) == 1
        if band == 2:
            assert band_cls == ({1} if d <= nsp else {3})


def test_band_map_sp_share_is_minimal():
    rng = np.random.default_rng(4)
    for _ in range(50):
        NT = int(rng.integers(2, 300))
        frac = float(rng.uniform(0.001, 0.5))
        c, nsp = O.precision_map_band(NT, 2, frac)
        total = NT * (NT + 1) // 2
        sp = int((c[np.tril_indices(NT)] == 1).sum())
        assert sp == sum(NT - d for d in range(1, nsp + 1))
        if nsp < NT - 1:
            assert sp >= frac * total
        assert sp - (NT - nsp) < frac * total  # one band fewer falls short


# Empirical covariance U = Xi Xi^T / m (+ nugget_rel * max diag on the diagonal):
# pins that do not restate the sum.
def _hadamard(m):
    H = np.array([[1.0]])
    while H.shape[0] < m:
        H = np.block([[H, H], [H, -H]])
    return H


def test_empirical_cov_recovers_integer_factor_exactly():
    # rows of a Hadamard matrix are orthogonal with H H^T = m I, so for an
    # integer lower-triangular L0 and Xi = L0 H[:n] the estimate is L0 L0^T exactly
    rng = np.random.default_rng(3)
    for n, m in [(5, 8), (12, 16), (16, 64)]:
        L0 = np.tril(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
        np.fill_diagonal(L0, rng.integers(1, 4, size=n))
        Xi = L0 @ _hadamard(m)[:n]
        assert np.array_equal(O.cov_from_residuals(Xi), L0 @ L0.T)


def test_empirical_cov_closed_forms_and_invariants():
    rng = np.random.default_rng(5)
    # scaled identity columns: U = c^2 / n I
    assert np.array_equal(O.cov_from_residuals(2.0 * np.eye(4)), np.eye(4))
    # one nonzero entry among m columns: U = a^2 / m at (i, i) only
    Xi = np.zeros((6, 8))
    Xi[2, 5] = 3.0
    U = O.cov_from_residuals(Xi)
    E = np.zeros((6, 6))
    E[2, 2] = 9.0 / 8.0
    assert np.array_equal(U, E)
    # trace = squared Frobenius norm / m; symmetric; positive semidefinite
    Xi = rng.standard_normal((30, 17))
    U = O.cov_from_residuals(Xi)
    assert abs(np.trace(U) - np.linalg.norm(Xi) ** 2 / 17) <= 1e-14 * np.trace(U)
    assert np.array_equal(U, U.T)
    assert np.linalg.eigvalsh(U).min() >= -1e-13 * np.trace(U)
    assert np.linalg.matrix_rank(U) == 17  # m < n: singular without the perturbation
    # the order of the residual vectors does not matter
    perm = rng.permutation(17)
    assert np.allclose(O.cov_from_residuals(Xi[:, perm]), U, rtol=0, atol=1e-14 * np.abs(U).max())
    # the perturbation touches the diagonal only, by nugget_rel * max diag
    Un = O.cov_from_residuals(Xi, 1e-3)
    off = ~np.eye(30, dtype=bool)
    assert np.array_equal(Un[off], U[off])
    assert np.allclose(np.diag(Un) - np.diag(U), 1e-3 * np.diag(U).max(), rtol=1e-12, atol=0)
    assert np.linalg.eigvalsh(Un).min() > 0


# VAR recursion and inverse SHT of the emulation steps ("Generating Emulations").
def test_var_recursion_closed_forms():
    rng = np.random.default_rng(1)
    Xi = rng.standard_normal((5, 9))
    assert np.array_equal(O.var_recursion(Xi, None), Xi)            # no lags: f = xi
    assert np.array_equal(O.var_recursion(Xi, np.zeros((5, 2))), Xi)
    imp = np.zeros((3, 12))
    imp[:, 0] = 1.0
    F = O.var_recursion(imp, np.full((3, 1), 0.5))                   # AR(1) impulse: phi^t
    assert np.array_equal(F[0], 0.5 ** np.arange(12))
    F = O.var_recursion(imp, np.tile([1.0, -1.0], (3, 1)))           # f_t = f_{t-1} - f_{t-2}: period 6
    assert np.array_equal(F[1], np.resize([1.0, 1.0, 0.0, -1.0, -1.0, 0.0], 12))
    # linearity in the innovations
    X2 = rng.standard_normal((5, 9))
    Ph = rng.uniform(-0.3, 0.3, (5, 3))
    assert np.allclose(O.var_recursion(Xi + X2, Ph), O.var_recursion(Xi, Ph) + O.var_recursion(X2, Ph), atol=1e-14)


def test_real_spherical_harmonics_pins():
    rng = np.random.default_rng(2)
    for _ in range(5):
        th, ph = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
        # closed forms (Condon-Shortley phase, real form)
        c = math.sqrt(3 / (4 * math.pi))
        assert abs(O.real_sh(0, 0, th, ph) - 1 / math.sqrt(4 * math.pi)) < 1e-15
        assert abs(O.real_sh(1, 0, th, ph) - c * math.cos(th)) < 1e-15
        assert abs(O.real_sh(1, 1, th, ph) + c * math.sin(th) * math.cos(ph)) < 1e-15
        assert abs(O.real_sh(1, -1, th, ph) + c * math.sin(th) * math.sin(ph)) < 1e-15
        assert abs(O.real_sh(2, 0, th, ph) - math.sqrt(5 / (16 * math.pi)) * (3 * math.cos(th) ** 2 - 1)) < 1e-14
        # addition theorem: sum_m Y_lm^2 = (2l+1)/(4 pi) at every point
        for l in (3, 17, 60):
            s2 = sum(O.real_sh(l, m, th, ph) ** 2 for m in range(-l, l + 1))
            assert abs(s2 - (2 * l + 1) / (4 * math.pi)) <= 1e-12 * (2 * l + 1)


def test_isht_single_coefficients_and_orthonormality():
    L, nt, nph = 5, 181, 64
    n = L * L
    Z = O.isht(np.eye(n), L, nt, nph)  # column k: Y_k on the grid
    th = np.pi * np.arange(nt) / (nt - 1)
    # column of Y_10 is sqrt(3/4pi) cos(theta) on every longitude
    y10 = Z[:, 2].reshape(nph, nt)
    assert np.allclose(y10, np.sqrt(3 / (4 * np.pi)) * np.cos(th)[None, :], atol=1e-15)
    # orthonormality by quadrature (trapezoid in theta with sin weights, exact in phi)
    w = np.sin(th) * (np.pi / (nt - 1))
    w[[0, -1]] *= 0.5
    W = np.tile(w, nph) * (2 * np.pi / nph)
    G = Z.T @ (Z * W[:, None])
    assert np.abs(G - np.eye(n)).max() < 1e-3  # the trapezoid rule in theta is second order: h^2 ~ 3e-4


def test_forward_sht_pins():
    # I(q) = int_0^pi e^{iqt} sin t dt, worked by hand
    assert O.I_of(0) == 2.0 and abs(O.I_of(2) + 2.0 / 3.0) < 1e-16 and O.I_of(3) == 0.0
    assert abs(O.I_of(1) - 1j * math.pi / 2) < 1e-16 and abs(O.I_of(-1) + 1j * math.pi / 2) < 1e-16
    # the constant field 1 has f_00 = int Y_00 = sqrt(4 pi) and nothing else
    L, nt, nph = 5, 6, 10
    F = O.sht(np.ones((nt * nph, 1)), L, nt, nph)
    assert abs(F[0, 0] - math.sqrt(4 * math.pi)) < 1e-13 and np.abs(F[1:, 0]).max() < 1e-13
    # exact recovery of band-limited data on the paper's minimal grid (ntheta = L + 1,
    # nphi = 2L) and on a larger one: the synthesis sum is inverted
    rng = np.random.default_rng(7)
    for L, nt, nph in [(6, 7, 12), (9, 10, 17), (8, 20, 31)]:
        f0 = rng.standard_normal((L * L, 3))
        assert np.abs(O.sht(O.isht(f0, L, nt, nph), L, nt, nph) - f0).max() < 1e-12
    # one coarser grid (ntheta = L) is no longer exact
    L = 8
    f0 = rng.standard_normal((L * L, 1))
    assert np.abs(O.sht(O.isht(f0, L, L, 2 * L), L, L, 2 * L) - f0).max() > 1e-6


# -------------------------------------------------------------------- RNG
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split(":")
            w = [int(x, 16) for x in lhs.split()]
            rows.append((w[:4], w[4:], [int(x, 16) for x in rhs.split()]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert O.philox4x32_10(ctr, key) == out


def test_uniform_ranges_and_counter_independence():
    u1, u2 = O.uniform_pair(0, 0, 0, 0)
    assert 0.0 < u1 <= 1.0 and 0.0 <= u2 < 1.0
    assert O.uniform_pair(0, 0, 0, 0) != O.uniform_pair(1, 0, 0, 0)  # seed
    assert O.uniform_pair(0, 0, 0, 0) != O.uniform_pair(0, 1, 0, 0)  # stream
    assert O.uniform_pair(0, 0, 1, 0) != O.uniform_pair(0, 0, 0, 1)  # row pair vs column


def test_box_muller_distribution():
    from scipy import stats

    Z = O.normal_matrix(seed=12345, stream=0, n=1000, s=400)
    z = Z.ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the two members of a Box-Muller pair are uncorrelated, and their squared
    # radius is -2 ln u1
    a, b = Z[0::2, :].ravel(), Z[1::2, :].ravel()
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(a.size)
    u1, _ = O.uniform_pair(12345, 0, 3, 7)
    assert abs(Z[6, 7] ** 2 + Z[7, 7] ** 2 + 2 * math.log(u1)) < 1e-12
    # odd n: the last row takes the cosine member
    Zo = O.normal_matrix(seed=12345, stream=0, n=7, s=3)
    assert np.array_equal(Zo, Z[:7, :3])


# ----------------------------------------------------------- sample, solve
def test_trmm_matches_numpy_and_reproduces_covariance():
    S = O.cov_build(4, 2.0)  # n = 16
    Lb, _ = O.potrf_blocked(S, 8)
    Z = O.normal_matrix(seed=5, stream=0, n=16, s=64)
    Y = O.trmm_lower(Lb, Z)
    assert np.allclose(Y, Lb @ Z, rtol=0, atol=1e-14)
    # second moment: E[Y Y^T] = L L^T = S
    Zb = O.normal_matrix(seed=6, stream=0, n=16, s=200000)
    Yb = O.trmm_lower(Lb, Zb)
    C = Yb @ Yb.T / Yb.shape[1]
    d = np.sqrt(np.diag(S))
    assert np.max(np.abs(C - S) / np.outer(d, d)) < 6 / math.sqrt(Yb.shape[1])


def test_potrs_solves():
    S = O.cov_build(6, 3.0)
    Lb, _ = O.potrf_blocked(S, 16)
    rng = np.random.default_rng(0)
    B = np.asfortranarray(rng.standard_normal((36, 5)))
    X = O.potrs(Lb, B)
    ref = np.linalg.solve(S, B)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-11


def test_blocked_steps_compose():
    S = _spd(200, seed=9)
    A1, _ = O.potrf_blocked(S, 64)
    A2 = np.array(S, order="F", copy=True)
    for k in range(4):
        assert O.lib().orc_potrf_blocked_steps(200, 64, O._dp(A2), 200, k, k + 1) == 0
    assert np.array_equal(np.tril(A2), A1)


# ------------------------------------------- mean trend and grid emulations
def test_mean_trend_closed_forms():
    """Eq. decouple's trend m_t: lag weights (1 - rho) rho^(s-1) and the
    harmonic terms, checked on cases whose value is known without the sum."""
    x = np.array([0.5, 1.0, 2.0, 4.0, 8.0, 16.0])
    # rho = 0: only the previous year's forcing carries the lag slope
    for t, tau in [(1, 12.0), (13, 12.0), (30, 12.0), (5, 1.0)]:
        y = math.ceil(t / tau)
        want = 0.3 + 2.0 * x[y] + 5.0 * x[y - 1]
        assert O.mean_trend(t, tau, 0.3, 2.0, 5.0, 0.0, [], [], x) == pytest.approx(want, rel=1e-15)
    # the lag weights sum to one: a constant forcing c gives b0 + (b1 + b2) c for any rho
    c = np.full(9, 3.25)
    for rho in (0.0, 0.3, 0.9, 1.0):
        for t in (1, 7, 40):
            got = O.mean_trend(t, 5.0, 1.0, 0.5, 2.0, rho, [], [], c)
            assert got == pytest.approx(1.0 + 2.5 * 3.25, rel=1e-14)
    # an impulse in year j reaches year y with weight (1 - rho) rho^(y - j - 1)
    imp = np.zeros(12)
    imp[4] = 1.0
    rho = 0.6
    for y in range(1, 12):
        want = 0.0 if y <= 4 else (1 - rho) * rho ** (y - 5)
        if y == 4:
            want = 0.0  # the current year's forcing has slope b1 = 0 here
        assert O.mean_trend(y, 1.0, 0.0, 0.0, 1.0, rho, [], [], imp) == pytest.approx(want, abs=1e-16)
    # years before the trajectory carry x[0]: at y = 1 the lag term is x[0], whatever rho
    assert O.mean_trend(1, 12.0, 0.0, 0.0, 1.0, 0.7, [], [], x) == pytest.approx(x[0], rel=1e-15)
    # rho = 1 keeps the pre-trajectory level for ever
    assert O.mean_trend(50, 12.0, 0.0, 0.0, 1.0, 1.0, [], [], x) == pytest.approx(x[0], rel=1e-15)
    # harmonics with tau = 12: a_1 cos(2 pi t / 12) + b_2 sin(4 pi t / 12)
    z = np.zeros(3)
    for t, want in [(3, 0.0 + math.sin(math.pi)), (6, -1.0 + 0.0), (12, 1.0), (1, math.cos(math.pi / 6) + math.sin(math.pi / 3))]:
        got = O.mean_trend(t, 12.0, 0.0, 0.0, 0.0, 0.0, [1.0, 0.0], [0.0, 1.0], z)
        assert abs(got - want) < 1e-14
    # a full period of any harmonic sums to zero
    tot = sum(O.mean_trend(t, 12.0, 0.0, 0.0, 0.0, 0.0, [0.7, -0.2, 1.3], [0.4, 0.9, -0.6], z) for t in range(1, 13))
    assert abs(tot) < 1e-13


def test_emulate_grid_pins():
    """Eq. decouple with the nugget of "Generating Emulations":
    y = m + sigma (Zs + v e)."""
    rng = np.random.default_rng(5)
    G, T, K = 7, 30, 2
    Zs = rng.standard_normal((G, T))
    E = rng.standard_normal((G, T))
    zero, one = np.zeros(G), np.ones(G)
    x = rng.standard_normal(4)
    AB0 = np.zeros((K, G))
    # no trend, unit scale, no nugget: the synthesis itself, bit for bit
    Y = O.emulate_grid(Zs, E, 12.0, zero, zero, zero, zero, AB0, AB0, x, one, zero)
    assert np.array_equal(Y, Zs)
    # no trend, Zs = 0: the nugget scaled by sigma v, exactly
    sig, v = np.full(G, 2.0), np.full(G, 3.0)
    Y = O.emulate_grid(np.zeros((G, T)), E, 12.0, zero, zero, zero, zero, AB0, AB0, x, sig, v)
    assert np.array_equal(Y, 6.0 * E)
    # full model: each entry equals the single-point trend plus the scaled stochastic part
    b0, b1, b2 = rng.standard_normal(G), rng.standard_normal(G), rng.standard_normal(G)
    rho = rng.uniform(0, 1, G)
    A, B = rng.standard_normal((K, G)), rng.standard_normal((K, G))
    sig, v = rng.uniform(0.5, 2, G), rng.uniform(0, 0.3, G)
    Y = O.emulate_grid(Zs, E, 12.0, b0, b1, b2, rho, A, B, x, sig, v)
    for g in (0, 3, 6):
        for t in (1, 12, 13, 30):
            m = O.mean_trend(t, 12.0, b0[g], b1[g], b2[g], rho[g], A[:, g], B[:, g], x)
            assert Y[g, t - 1] == m + sig[g] * (Zs[g, t - 1] + v[g] * E[g, t - 1])
    # the trend is shared by all ensembles: two draws differ only by sigma (Zs + v e)
    Y2 = O.emulate_grid(Zs + 1.0, E, 12.0, b0, b1, b2, rho, A, B, x, sig, v)
    assert np.allclose(Y2 - Y, np.outer(sig, np.ones(T)), rtol=0, atol=1e-13)


@pytest.mark.parametrize("L,beta,nugget,nb", [(12, 3.0, -1e-3, 16), (20, 3.0, -1e-3, 64), (12, 2.0, -0.05, 32)])
def test_potrf_failure_column_is_the_first_indefinite_leading_block(L, beta, nugget, nb):
    """The oracle's blocked Cholesky reports the 1-based column p of its first
    non-positive pivot.  Sylvester's criterion fixes p independently: the
    leading (p-1) x (p-1) block of S is positive definite and the leading
    p x p block is not (numpy's symmetric eigensolver, not the oracle)."""
    S = O.cov_build(L, beta, 1.5, nugget)
    _, p = O.potrf_blocked(S, nb)
    assert p > 1
    lam_prev = np.linalg.eigvalsh(S[:p - 1, :p - 1])[0]
    lam = np.linalg.eigvalsh(S[:p, :p])[0]
    assert lam_prev > 1e-12 * np.abs(S).max()
    assert lam < 0.0
