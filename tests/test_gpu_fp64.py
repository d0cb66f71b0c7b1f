"""Parity of the plain FP64 GPU path with the CPU oracle, through the C ABI:
covariance build, tile norms, FP64 tile Cholesky (<= 1e-12 relative), the
sampler (Y = L Z) and the solves.  Sizes span several tiles and a ragged tail.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import paper_2408_04440_gb300 as E
    from paper_2408_04440_gb300 import build

    build.build()
    return E


@pytest.fixture(scope="module")
def ctx(E):
    c = E.Context(0)
    yield c
    c.close()


def _np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("L,nb,beta", [(8, 64, 4.0), (12, 64, 3.0), (20, 128, 4.0), (32, 128, 4.0)])
def test_cov_build_and_norms(E, ctx, L, nb, beta):
    A = E.emu_cov_build(ctx, L, beta, nb)
    S = O.cov_build(L, beta)
    G = _np(E.emu_mat_export(ctx, A))
    ref = np.tril(S)
    assert np.max(np.abs(G - ref)) <= 4e-16 * np.max(np.abs(ref))
    cls, tn = E.emu_mat_tile_info(ctx, A)
    t_ref = O.tile_norms(S, nb)
    assert np.allclose(tn, t_ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("L,nb,beta", [(8, 64, 4.0), (12, 64, 3.0), (20, 128, 4.0), (32, 128, 4.0)])
def test_fp64_factor_matches_oracle(E, ctx, L, nb, beta):
    A = E.emu_cov_build(ctx, L, beta, nb)
    info = E.emu_potrf_mp(ctx, A)
    assert info.status == E.EMU_OK and info.pivot == 0
    G = _np(E.emu_mat_export(ctx, A))
    Lo, oinfo = O.potrf_blocked(O.cov_build(L, beta), nb)
    assert oinfo == 0
    rel = np.linalg.norm(G - Lo) / np.linalg.norm(Lo)
    assert rel <= 1e-12, rel
    assert np.all(np.triu(G, 1) == 0)


def test_fp64_factor_of_imported_matrix(E, ctx):
    import torch

    rng = np.random.default_rng(11)
    n = 200  # ragged with nb = 64
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    S = (Q * np.logspace(0, -6, n)) @ Q.T
    S = 0.5 * (S + S.T)
    A = E.emu_mat_import(ctx, torch.from_numpy(S).cuda(), 64)
    E.emu_potrf_mp(ctx, A)
    G = _np(E.emu_mat_export(ctx, A))
    Lo, _ = O.potrf_blocked(S, 64)
    assert np.linalg.norm(G - Lo) / np.linalg.norm(Lo) <= 1e-12


@pytest.mark.parametrize("scale", [2.0**-1010, 2.0**1005])
def test_fp64_factor_with_extreme_pivots(E, ctx, scale):
    # pivots below 2^-1000 or above 2^1000 leave the hardware reciprocal's
    # range and take IEEE division in the diagonal-block leaf
    import torch

    rng = np.random.default_rng(5)
    n = 150
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    S = (Q * np.linspace(1.0, 8.0, n)) @ Q.T
    S = 0.5 * (S + S.T) * scale
    A = E.emu_mat_import(ctx, torch.from_numpy(S).cuda(), 64)
    E.emu_potrf_mp(ctx, A)
    G = _np(E.emu_mat_export(ctx, A))
    Lo, info = O.potrf_blocked(S, 64)
    assert info == 0
    assert np.all(np.isfinite(G))
    assert np.linalg.norm(G - Lo) / np.linalg.norm(Lo) <= 1e-12


def _hadamard(m):
    H = np.array([[1.0]])
    while H.shape[0] < m:
        H = np.block([[H, H], [H, -H]])
    return H


@pytest.mark.parametrize("n,m", [(700, 500), (700, 1300), (256, 64)])
def test_empirical_covariance_matches_oracle(E, ctx, n, m):
    import torch

    rng = np.random.default_rng(n + m)
    Xi = rng.standard_normal((n, m)) * np.logspace(0, -3, n)[:, None]
    U, st = E.emu_cov_from_residuals(ctx, torch.from_numpy(np.asfortranarray(Xi)).cuda(), nb=256)
    assert st == E.EMU_OK
    G = _np(E.emu_mat_export(ctx, U))
    nug = 1e-8 if m < n else 0.0
    Uo = O.cov_from_residuals(Xi, nug)
    assert np.abs(G - np.tril(Uo)).max() <= 1e-13 * np.abs(Uo).max()
    # the matrix is in the covariance state: its norms feed the precision map
    cls, tn = E.emu_mat_tile_info(ctx, U)
    to = O.tile_norms(Uo, 256)
    NT = to.shape[0]
    assert np.allclose(tn[np.tril_indices(NT)], to[np.tril_indices(NT)], rtol=1e-12, atol=0)
    U.free()


def test_empirical_covariance_exact_for_integer_factor(E, ctx):
    # Xi = L0 H[:n] with Hadamard rows: the estimate is L0 L0^T, exactly (integer digit products)
    import torch

    rng = np.random.default_rng(9)
    n, m = 300, 512
    L0 = np.tril(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
    np.fill_diagonal(L0, rng.integers(1, 4, size=n))
    Xi = L0 @ _hadamard(m)[:n]
    U, _ = E.emu_cov_from_residuals(ctx, torch.from_numpy(np.asfortranarray(Xi)).cuda(), nb=256, nugget_rel=0.0)
    G = _np(E.emu_mat_export(ctx, U))
    assert np.array_equal(G, np.tril(L0 @ L0.T))
    U.free()


def test_empirical_covariance_in_several_launches_then_factor(E, ctx):
    # n = 2048 rows: the digit arena holds 65536 columns, so 70000 residuals take two
    # launches; sampled entries against the oracle on the same rows; then the
    # mixed factor of the estimate meets eps
    import torch

    n, m, nb = 2048, 70000, 256
    S = O.cov_build(46, 6.0)[:n, :n]  # n = 2116, leading 2048 x 2048 block
    Lo, _ = O.potrf_blocked(S, nb)
    rng = np.random.default_rng(2)
    Xg = torch.from_numpy(np.asfortranarray(Lo)).cuda() @ torch.randn(n, m, dtype=torch.float64, device="cuda",
                                                                       generator=torch.Generator("cuda").manual_seed(4))
    U, st = E.emu_cov_from_residuals(ctx, Xg, nb=nb)
    assert st == E.EMU_OK
    G = _np(E.emu_mat_export(ctx, U))
    rows = np.sort(rng.choice(n, 24, replace=False))
    Xr = Xg[torch.from_numpy(rows).cuda()].cpu().numpy()
    Uo = O.cov_from_residuals(Xr)  # entries (rows x rows) of the estimate
    Gr = G[np.ix_(rows, rows)]
    low = np.tril(np.ones_like(Gr, dtype=bool))
    assert np.abs(Gr[low] - Uo[low]).max() <= 1e-13 * np.abs(Uo).max()
    info = E.emu_potrf_mp(ctx, U, eps=1e-8)
    assert info.status == E.EMU_OK
    L = _np(E.emu_mat_export(ctx, U))
    Uf = G + np.tril(G, -1).T
    assert np.linalg.norm(L @ L.T - Uf) / np.linalg.norm(Uf) <= 1e-8
    U.free()


def test_var_recursion_matches_oracle(E, ctx):
    import torch

    rng = np.random.default_rng(6)
    n, T, P = 500, 300, 3
    Xi = rng.standard_normal((n, T))
    Ph = rng.uniform(-0.3, 0.3, (n, P))
    F = _np(E.emu_var_recursion(ctx, torch.from_numpy(np.asfortranarray(Xi)).cuda(),
                                torch.from_numpy(np.asfortranarray(Ph)).cuda()))
    Fo = O.var_recursion(Xi, Ph)
    assert np.abs(F - Fo).max() <= 1e-13 * np.abs(Fo).max()


@pytest.mark.parametrize("L,nt,nph", [(24, 25, 48), (9, 10, 17)])
def test_isht_matches_oracle(E, ctx, L, nt, nph):
    import torch

    rng = np.random.default_rng(L)
    T = 4
    F = rng.standard_normal((L * L, T)) / (1.0 + np.repeat(np.arange(L), 2 * np.arange(L) + 1))[:, None]
    Z = _np(E.emu_isht(ctx, torch.from_numpy(np.asfortranarray(F)).cuda(), L, nt, nph))
    Zo = O.isht(F, L, nt, nph)
    assert np.abs(Z - Zo).max() <= 1e-12 * np.abs(Zo).max()


@pytest.mark.parametrize("L,nt,nph", [(24, 25, 48), (9, 20, 31)])
def test_sht_matches_oracle_and_inverts_isht(E, ctx, L, nt, nph):
    import torch

    rng = np.random.default_rng(L + nt)
    T = 3
    Z = rng.standard_normal((nt * nph, T))  # not band-limited: the method's estimate
    F = _np(E.emu_sht(ctx, torch.from_numpy(np.asfortranarray(Z)).cuda(), L, nt, nph))
    Fo = O.sht(Z, L, nt, nph)
    assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()
    f0 = rng.standard_normal((L * L, T))
    Zb = E.emu_isht(ctx, torch.from_numpy(np.asfortranarray(f0)).cuda(), L, nt, nph)
    assert np.abs(_np(E.emu_sht(ctx, Zb, L, nt, nph)) - f0).max() <= 1e-12  # exact recovery


def test_emulation_chain_from_the_mixed_factor(E, ctx):
    # draws xi = L z of the mixed factor, VAR(3) in time, synthesis on the grid:
    # the chain runs in our kernels and equals the oracle's VAR and synthesis of
    # the same draws
    import torch

    Lb, nb, beta, T = 16, 256, 4.0, 40
    A = E.emu_cov_build(ctx, Lb, beta, nb)
    E.emu_potrf_mp(ctx, A, eps=1e-8)
    Xi = E.emu_sample(ctx, A, T, seed=8)
    A.free()
    n = Lb * Lb
    Ph = torch.from_numpy(np.asfortranarray(np.tile([0.5, 0.2, 0.1], (n, 1)))).cuda()
    F = E.emu_var_recursion(ctx, Xi, Ph)
    Z = _np(E.emu_isht(ctx, F, Lb, Lb + 1, 2 * Lb))
    Fo = O.var_recursion(_np(Xi), _np(Ph))
    Zo = O.isht(Fo, Lb, Lb + 1, 2 * Lb)
    assert np.abs(Z - Zo).max() <= 1e-12 * np.abs(Zo).max()


def _trend_inputs(G, T, K, tau, seed):
    rng = np.random.default_rng(seed)
    ny = -(-T // int(tau)) if float(tau).is_integer() else int(np.ceil(T / tau))
    return dict(beta0=rng.standard_normal(G), beta1=rng.standard_normal(G), beta2=rng.standard_normal(G),
                rho=np.concatenate([[0.0, 1.0], rng.uniform(0, 1, G - 2)]), A=rng.standard_normal((K, G)),
                B=rng.standard_normal((K, G)), x=rng.standard_normal(ny + 1), sigma=rng.uniform(0.5, 2.0, G),
                v=rng.uniform(0.0, 0.5, G))


@pytest.mark.parametrize("G,T,K,tau", [(1175, 70, 3, 12.0), (33, 5, 0, 1.0), (64, 40, 8, 7.5)])
def test_emulate_grid_matches_oracle(E, ctx, G, T, K, tau):
    # y = m + sigma (Zs + v e), Eq. decouple: trend, nugget and scale against
    # the oracle, given the oracle's own Philox normals for the nugget
    import torch

    p = _trend_inputs(G, T, K, tau, seed=G + T)
    Zs = np.random.default_rng(1).standard_normal((G, T))
    seed, sid = 77, 5
    cu = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in p.items()}
    Y = _np(E.emu_emulate_grid(ctx, torch.from_numpy(np.asfortranarray(Zs)).cuda(), tau, cu["beta0"],
                               cu["beta1"], cu["beta2"], cu["rho"], cu["A"] if K else None,
                               cu["B"] if K else None, cu["x"], cu["sigma"], cu["v"], seed, sid))
    e = O.normal_matrix(seed, sid, G, T)
    Yo = O.emulate_grid(Zs, e, tau, p["beta0"], p["beta1"], p["beta2"], p["rho"], p["A"], p["B"], p["x"],
                        p["sigma"], p["v"])
    assert np.abs(Y - Yo).max() <= 1e-12 * np.abs(Yo).max()
    # zero nugget and trend, unit scale: the synthesis itself, bit for bit
    z = torch.zeros(G, dtype=torch.float64, device="cuda")
    Y1 = _np(E.emu_emulate_grid(ctx, torch.from_numpy(np.asfortranarray(Zs)).cuda(), tau, z, z, z, z, None, None,
                                cu["x"], torch.ones_like(z), z, seed, sid))
    assert np.array_equal(Y1, Zs)


def test_emulation_chain_to_the_grid_fields(E, ctx):
    # the whole of "Generating Emulations": draws of the mixed factor, VAR(2),
    # synthesis, nugget, trend and scale, against the oracle's chain on the
    # same draws and nugget normals
    import torch

    Lb, nb, beta, T, tau, K = 12, 256, 4.0, 36, 12.0, 2
    A = E.emu_cov_build(ctx, Lb, beta, nb)
    E.emu_potrf_mp(ctx, A, eps=1e-8)
    Xi = E.emu_sample(ctx, A, T, seed=9)
    A.free()
    n = Lb * Lb
    Ph = torch.from_numpy(np.asfortranarray(np.tile([0.6, 0.2], (n, 1)))).cuda()
    nt, nph = Lb + 1, 2 * Lb
    G = nt * nph
    Zs = E.emu_isht(ctx, E.emu_var_recursion(ctx, Xi, Ph), Lb, nt, nph)
    p = _trend_inputs(G, T, K, tau, seed=3)
    cu = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in p.items()}
    Y = _np(E.emu_emulate_grid(ctx, Zs, tau, cu["beta0"], cu["beta1"], cu["beta2"], cu["rho"], cu["A"], cu["B"],
                               cu["x"], cu["sigma"], cu["v"], 11, 2))
    Zo = O.isht(O.var_recursion(_np(Xi), _np(Ph)), Lb, nt, nph)
    Yo = O.emulate_grid(Zo, O.normal_matrix(11, 2, G, T), tau, p["beta0"], p["beta1"], p["beta2"], p["rho"],
                        p["A"], p["B"], p["x"], p["sigma"], p["v"])
    assert np.abs(Y - Yo).max() <= 1e-12 * np.abs(Yo).max()


def test_emulate_grid_rejects_a_short_forcing(E, ctx):
    import torch

    G, T = 10, 25
    z = torch.zeros(G, dtype=torch.float64, device="cuda")
    x = torch.zeros(2, dtype=torch.float64, device="cuda")  # one year; 25 monthly steps need three
    Zs = torch.zeros((T, G), dtype=torch.float64, device="cuda").t()
    with pytest.raises(E.EmuError):
        E.emu_emulate_grid(ctx, Zs, 12.0, z, z, z, z, None, None, x, z, z, 1)


@pytest.mark.parametrize("eps", [0.0, 1e-8])
def test_withheld_flag_times_out_and_the_context_recovers(E, ctx, eps):
    # failure detection without a GPU fault: a flag that nothing sets (the
    # test hook withholds block (1, 0)'s flag of the diagonal POTRF) and a wait
    # bound of 2e5 cycles; the factor reports EMU_ETIMEOUT, every kernel
    # returns, and the same context then factors correctly
    L, nb, beta = 32, 256, 4.0
    A = E.emu_cov_build(ctx, L, beta, nb)
    ctx.test_wait_hook(wait_cycles=200000, withhold_index=1 * (nb // 16) + 0)
    try:
        with pytest.raises(E.EmuError) as err:
            E.emu_potrf_mp(ctx, A, eps=eps)
        assert err.value.status == E.EMU_ETIMEOUT
    finally:
        ctx.test_wait_hook(0, -1)
    A.free()
    A = E.emu_cov_build(ctx, L, beta, nb)
    E.emu_potrf_mp(ctx, A, eps=eps)
    Lg = _np(E.emu_mat_export(ctx, A))
    A.free()
    S = O.cov_build(L, beta)
    if eps == 0.0:
        Lo, _ = O.potrf_blocked(S, nb)
        assert np.linalg.norm(Lg - Lo) / np.linalg.norm(Lo) <= 1e-12
    else:
        assert np.linalg.norm(Lg @ Lg.T - S) / np.linalg.norm(S) <= eps


@pytest.mark.parametrize("bad", [1, 70, 199])
def test_not_positive_definite_reports_pivot(E, ctx, bad):
    import torch

    n = 200
    S = np.eye(n)
    S[bad - 1, bad - 1] = -1.0
    A = E.emu_mat_import(ctx, torch.from_numpy(S).cuda(), 64)
    info = E.emu_potrf_mp(ctx, A, raise_on_error=False)
    assert info.status == E.EMU_ENOTPD
    assert info.pivot == bad
    # the context stays usable after the failure
    B = E.emu_cov_build(ctx, 6, 2.0, 64)
    assert E.emu_potrf_mp(ctx, B).status == E.EMU_OK


@pytest.mark.parametrize("nugget", [-1e-3, -0.05])
def test_negative_nugget_reports_the_oracles_pivot(E, ctx, nugget):
    """A negative nugget makes the covariance indefinite; the FP64 factor
    reports EMU_ENOTPD at the oracle's first non-positive pivot column."""
    L, beta, nb = 20, 3.0, 64
    _, piv = O.potrf_blocked(O.cov_build(L, beta, 1.5, nugget), nb)
    assert piv > 0
    A = E.emu_cov_build(ctx, L, beta, nb, nugget_rel=nugget)
    info = E.emu_potrf_mp(ctx, A, raise_on_error=False)
    assert info.status == E.EMU_ENOTPD
    assert info.pivot == piv


@pytest.mark.parametrize("L,nb,s", [(12, 64, 5), (32, 128, 64)])
def test_fp64_sampling(E, ctx, L, nb, s):
    A = E.emu_cov_build(ctx, L, 4.0, nb)
    E.emu_potrf_mp(ctx, A)
    Y, Z = E.emu_sample(ctx, A, s, seed=0, return_z=True)
    Zo = O.normal_matrix(0, 0, L * L, s)
    Zg = _np(Z)
    assert np.max(np.abs(Zg - Zo)) <= 1e-14 * np.max(np.abs(Zo))
    Lo, _ = O.potrf_blocked(O.cov_build(L, 4.0), nb)
    Yo = O.trmm_lower(Lo, Zo)
    Yg = _np(Y)
    assert np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo) <= 1e-12
    # bit-identical on rerun
    Y2 = _np(E.emu_sample(ctx, A, s, seed=0))
    assert np.array_equal(Y2, Yg)
    # a different seed or stream id gives different draws
    assert not np.array_equal(_np(E.emu_sample(ctx, A, s, seed=1)), Yg)
    assert not np.array_equal(_np(E.emu_sample(ctx, A, s, seed=0, stream_id=1)), Yg)


def test_fp64_sampling_host_buffers(E, ctx):
    A = E.emu_cov_build(ctx, 10, 3.0, 64)
    E.emu_potrf_mp(ctx, A)
    Yh = E.emu_sample_host(ctx, A, 7, seed=3)
    Yd = _np(E.emu_sample(ctx, A, 7, seed=3))
    assert np.array_equal(Yh, Yd)


def test_fp64_solves(E, ctx):
    import torch

    L, nb = 16, 64
    A = E.emu_cov_build(ctx, L, 4.0, nb)
    S = E.emu_mat_clone(ctx, A)
    E.emu_potrf_mp(ctx, A)
    rng = np.random.default_rng(2)
    B = rng.standard_normal((L * L, 3))
    X = _np(E.emu_potrs(ctx, A, torch.from_numpy(B).cuda()))
    So = O.cov_build(L, 4.0)
    Lo, _ = O.potrf_blocked(So, nb)
    Xo = O.potrs(Lo, B)
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-9
    Xr, ri = E.emu_solve_refine(ctx, A, S, torch.from_numpy(B).cuda(), tol=1e-15, maxit=10)
    assert ri.status == E.EMU_OK
    Xr = _np(Xr)
    eta = np.linalg.norm(B - So @ Xr, axis=0) / (np.linalg.norm(So) * np.linalg.norm(Xr, axis=0)
                                                 + np.linalg.norm(B, axis=0))
    assert eta.max() <= 1e-15


def test_bad_arguments(E, ctx):
    import ctypes

    h = ctypes.c_void_p()
    p = E.emu_cov_params(0, 1.0, 1.5, 1e-8)
    assert ctx.lib.emu_cov_build(ctx.h, ctypes.byref(p), 64, ctypes.byref(h)) == E.EMU_EINVAL
    p = E.emu_cov_params(8, 1.0, 1.5, 1e-8)
    assert ctx.lib.emu_cov_build(ctx.h, ctypes.byref(p), 100, ctypes.byref(h)) == E.EMU_EINVAL
    A = E.emu_cov_build(ctx, 8, 2.0, 64)
    with pytest.raises(E.EmuError):
        E.emu_sample(ctx, A, 4, seed=0)  # not factored yet: EMU_ESTATE
    E.emu_potrf_mp(ctx, A)
    with pytest.raises(E.EmuError):
        E.emu_potrf_mp(ctx, A)  # already factored


def test_launch_count_increases(E, ctx):
    before = ctx.launch_count
    A = E.emu_cov_build(ctx, 8, 2.0, 64)
    E.emu_potrf_mp(ctx, A)
    assert ctx.launch_count > before


def test_import_from_host_buffer(E, ctx):
    L, nb, beta = 14, 64, 3.0  # n = 196: ragged last tile column
    S = O.cov_build(L, beta)
    A = E.emu_mat_import_host(ctx, np.asfortranarray(S), nb)
    G = _np(E.emu_mat_export(ctx, A))
    assert np.array_equal(G, np.tril(S))
    _, tn = E.emu_mat_tile_info(ctx, A)
    assert np.allclose(tn, O.tile_norms(S, nb), rtol=1e-13, atol=0)
    E.emu_potrf_mp(ctx, A)
    Lo, _ = O.potrf_blocked(S, nb)
    G = _np(E.emu_mat_export(ctx, A))
    assert np.linalg.norm(G - Lo) / np.linalg.norm(Lo) <= 1e-12


def test_profiler_counts_launches(E, ctx):
    ctx.prof_enable(True)
    A = E.emu_cov_build(ctx, 12, 3.0, 64)
    E.emu_potrf_mp(ctx, A)
    prof = ctx.prof_read()
    ctx.prof_enable(False)
    assert prof["cov"]["launches"] >= 1 and prof["potrf"]["launches"] >= 3
    assert prof["update64"]["flops"] > 0 and prof["potrf"]["ms"] > 0


def test_matrix_outliving_its_context(E):
    # closing a context frees the matrices made in it; a Python handle that
    # outlives the context then frees nothing (no use of the freed context)
    c = E.Context(0)
    A = E.emu_cov_build(c, 6, 2.0, 64)
    c.close()
    assert A.h is None
    A.free()
    del A
