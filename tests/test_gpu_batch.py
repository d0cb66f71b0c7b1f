"""Batched path on the GPU (emu_batch_potrf_sample): many covariances of
uneven bandlimit factored and sampled in one call, against the oracle.

* plain FP64 batch: every L_b equals the oracle's blocked Cholesky to 1e-12,
  Z_b equals the oracle's Philox/Box-Muller draws with stream id b, and
  Y_b = L_b Z_b to 1e-12;
* adaptive batch: every matrix meets ||L L^T - S||_F / ||S||_F <= eps against
  the oracle's S, and its per-class tile counts are the rule's on the oracle's
  tile norms;
* the batch agrees with the single-matrix path run matrix by matrix;
* a second call replays the captured graph with the same results.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

MASK_FP64_FP32_BF16 = 0b01011
MASK_WITH_E4M3 = 0b11011


def U_of(nb):
    return np.array([2.0**-53, 2.0**-24 * np.sqrt(nb), 2.0**-11, 2.0**-8, 2.0**-4])


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


# uneven bandlimits: one tile (n = 25 .. 256), several tiles, a ragged last tile
PARAMS = [(5, 2.0), (16, 3.0), (17, 2.5), (23, 4.0), (30, 5.0), (12, 7.5), (33, 3.5), (40, 6.0), (8, 2.2)]


def _bf(E, ctx, *a, **k):
    Ys, Ls, infos, s = E.emu_batch_potrf_sample(ctx, *a, **k)
    return ([y.cpu().numpy() for y in Ys] if Ys else None, [x.cpu().numpy() for x in Ls] if Ls else None, infos, s)


def test_fp64_batch_matches_oracle(E, ctx):
    nb, s, seed = 256, 40, 9
    Ys, Ls, infos, st = _bf(E, ctx, PARAMS, nb=nb, eps=0.0, nsamples=s, seed=seed, want_L=True)
    assert st == E.EMU_OK
    for b, (L, beta) in enumerate(PARAMS):
        n = L * L
        S = O.cov_build(L, beta)
        Lo, info = O.potrf_blocked(S, nb)
        assert info == 0
        assert infos[b].n == n and infos[b].tiles[0] == infos[b].nt * (infos[b].nt + 1) // 2
        rel = np.linalg.norm(Ls[b] - Lo) / np.linalg.norm(Lo)
        assert rel <= 1e-12, (b, rel)
        Zo = O.normal_matrix(seed, b, n, s)
        ref = Lo @ Zo
        ry = np.linalg.norm(Ys[b] - ref) / np.linalg.norm(ref)
        assert ry <= 1e-12, (b, ry)


@pytest.mark.parametrize("eps,mask", [(1e-8, MASK_FP64_FP32_BF16), (1e-4, MASK_WITH_E4M3)])
def test_mixed_batch_meets_eps(E, ctx, eps, mask):
    nb = 256
    _, Ls, infos, st = _bf(E, ctx, PARAMS, nb=nb, eps=eps, prec_mask=mask, want_L=True)
    assert st == E.EMU_OK
    low = 0
    for b, (L, beta) in enumerate(PARAMS):
        S = O.cov_build(L, beta)
        be = np.linalg.norm(Ls[b] @ Ls[b].T - S) / np.linalg.norm(S)
        assert be <= eps, (b, be)
        co = O.precision_map(O.tile_norms(S, nb), eps, U_of(nb), mask)
        NT = co.shape[0]
        counts = [int(sum(co[i, j] == c for i in range(NT) for j in range(i + 1))) for c in range(5)]
        assert infos[b].tiles == counts, (b, infos[b].tiles, counts)
        low += sum(counts[1:])
    assert low > 0  # the batch exercises the tensor-core classes


def test_band_map_batch(E, ctx):
    # DP/SP/HP per matrix of the batch: each matrix's map is the oracle's band
    # map for its own NT, and each factor meets the tolerance of that map
    nb = 256
    _, Ls, infos, st = _bf(E, ctx, PARAMS, nb=nb, band=E.MAP_DP_SP_HP, want_L=True)
    assert st == E.EMU_OK
    for b, (L, beta) in enumerate(PARAMS):
        NT = infos[b].nt
        co, _ = O.precision_map_band(NT, 2, 0.05)
        counts = [int((co[np.tril_indices(NT)] == c).sum()) for c in range(5)]
        assert infos[b].tiles == counts, (b, infos[b].tiles, counts)
        S = O.cov_build(L, beta)
        t = O.tile_norms(S, nb)
        U = U_of(nb)
        eps_map = NT * max(t[i, j] * U[co[i, j]] for i in range(NT) for j in range(i + 1)) / np.linalg.norm(S)
        be = np.linalg.norm(Ls[b] @ Ls[b].T - S) / np.linalg.norm(S)
        assert be <= max(eps_map, 1e-14), (b, be, eps_map)


def test_batch_agrees_with_single_path(E, ctx):
    nb, s, seed, eps = 256, 64, 5, 1e-6
    Ys, Ls, infos, st = _bf(E, ctx, PARAMS, nb=nb, eps=eps, prec_mask=MASK_WITH_E4M3, nsamples=s, seed=seed,
                            want_L=True)
    assert st == E.EMU_OK
    same = 0
    for b, (L, beta) in enumerate(PARAMS):
        A = E.emu_cov_build(ctx, L, beta, nb)
        E.emu_potrf_mp(ctx, A, eps=eps, prec_mask=MASK_WITH_E4M3)
        G = E.emu_mat_export(ctx, A).cpu().numpy()
        Y = E.emu_sample(ctx, A, s, seed=seed, stream_id=b).cpu().numpy()
        A.free()
        assert np.linalg.norm(Ls[b] - G) <= 1e-12 * np.linalg.norm(G), b
        assert np.linalg.norm(Ys[b] - Y) <= 1e-12 * np.linalg.norm(Y), b
        same += int(np.array_equal(Ls[b], G) and np.array_equal(Ys[b], Y))
    print(f"batch vs single path: {same} of {len(PARAMS)} matrices bit-identical")


def test_graph_replay_and_seed(E, ctx):
    nb, s = 256, 32
    p = PARAMS[:5]
    n0 = ctx.launch_count
    Y1, L1, _, _ = _bf(E, ctx, p, nb=nb, eps=1e-8, nsamples=s, seed=1, want_L=True)
    n1 = ctx.launch_count
    Y2, L2, _, _ = _bf(E, ctx, p, nb=nb, eps=1e-8, nsamples=s, seed=1, want_L=True)
    n2 = ctx.launch_count
    assert n1 > n0 and n2 - n1 > 0
    for b in range(len(p)):
        assert np.array_equal(L1[b], L2[b]) and np.array_equal(Y1[b], Y2[b])
    Y3, L3, _, _ = _bf(E, ctx, p, nb=nb, eps=1e-8, nsamples=s, seed=2, want_L=True)
    for b in range(len(p)):
        assert np.array_equal(L1[b], L3[b]) and not np.array_equal(Y1[b], Y3[b])


def test_tuned_tile_size(E, ctx):
    p = PARAMS[:6]
    _, Ls, infos, st = _bf(E, ctx, p, nb=0, eps=1e-8, want_L=True)
    assert st == E.EMU_OK and infos[0].nb in (256, 512)
    _, Ls2, infos2, _ = _bf(E, ctx, p, nb=0, eps=1e-8, want_L=True)
    assert infos2[0].nb == infos[0].nb  # the choice is remembered
    for b, (L, beta) in enumerate(p):
        S = O.cov_build(L, beta)
        assert np.linalg.norm(Ls2[b] @ Ls2[b].T - S) / np.linalg.norm(S) <= 1e-8
    E.emu_batch_release(ctx)


def test_batch_bad_arguments(E, ctx):
    lib = ctx.lib
    assert lib.emu_batch_potrf_sample(ctx.h, 0, None, 256, None, 0, 0, None, None, None) == E.EMU_EINVAL
    for bad in ([(300, 2.0)], [(8, -1.0)]):
        _, _, _, st = E.emu_batch_potrf_sample(ctx, bad, nb=256, raise_on_error=False)
        assert st == E.EMU_EINVAL
    _, _, _, st = E.emu_batch_potrf_sample(ctx, [(8, 2.0)], nb=128, raise_on_error=False)
    assert st == E.EMU_EINVAL


# nugget below the smallest conditional variances of the row order: not
# positive definite, with the first non-positive pivot well inside the matrix
BAD = (20, 3.0, 1.5, -1e-3)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("eps", [0.0, 1e-8])
def test_non_spd_instance_flags_only_that_instance(E, ctx, eps):
    """One matrix of the batch is not positive definite: the call reports
    EMU_ENOTPD, only that matrix's info.pivot is set (for the FP64 factor, the
    oracle's first non-positive pivot column), and every other matrix of the
    batch is complete and correct; the context stays usable."""
    params = PARAMS[:4] + [BAD] + PARAMS[4:6]
    nb, s, seed = 256, 16, 4
    Ys, Ls, infos, st = _bf(E, ctx, params, nb=nb, eps=eps, nsamples=s, seed=seed, want_L=True,
                            raise_on_error=False)
    assert st == E.EMU_ENOTPD
    _, piv = O.potrf_blocked(O.cov_build(*BAD), nb)
    assert piv > 16
    for b, q in enumerate(params):
        if q is BAD:
            assert infos[b].pivot > 0
            if eps == 0.0:
                assert infos[b].pivot == piv
            continue
        assert infos[b].pivot == 0, b
        L, beta = q
        n = L * L
        S = O.cov_build(L, beta)
        if eps == 0.0:
            Lo, _ = O.potrf_blocked(S, nb)
            assert _rel(Ls[b], Lo) <= 1e-12, b
            assert _rel(Ys[b], Lo @ O.normal_matrix(seed, b, n, s)) <= 1e-12, b
        else:
            assert _rel(Ls[b] @ Ls[b].T, S) <= eps, b
    _, _, _, st2 = _bf(E, ctx, PARAMS[:3], nb=nb, eps=eps)
    assert st2 == E.EMU_OK
