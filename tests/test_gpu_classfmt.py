"""Class-format tile storage (every tile in the format of its precision
class, re-rounded after each update) on the GPU, through the C ABI, against
the oracle: the stored covariance, the precision map, the factor's backward
error, the sampler, and the matrix-free backward-error estimate.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

MASK_ALL = 0b11011        # FP64, FP32, BF16, E4M3 (no TF32 storage class)
MASK_FP64_FP32_BF16 = 0b01011
U_NOMINAL = np.array([2.0**-53, 2.0**-24, 2.0**-11, 2.0**-8, 2.0**-4])


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


def _np(t):
    return t.cpu().numpy()


def _bf16_rn(x):
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def _expected_map(S, nb, eps, mask):
    """The oracle's rule with every diagonal tile FP64 (class-format storage
    keeps the diagonal in FP64)."""
    t = O.tile_norms(S, nb)
    return O.precision_map(t, eps, U_of(nb), mask, True), t


def _map_matches(cls_gpu, t, eps, mask, nb):
    U = U_of(nb)
    cls_o = O.precision_map(t, eps, U, mask, True)
    NT = t.shape[0]
    thr = eps * O.frob_from_tiles(t) / NT
    for i in range(NT):
        for j in range(i + 1):
            if cls_gpu[i, j] == cls_o[i, j]:
                continue
            margins = [abs(t[i, j] * U[c] - thr) / thr for c in range(1, 5)]
            assert min(margins) < 1e-12, (i, j, cls_gpu[i, j], cls_o[i, j])


@pytest.mark.parametrize("L,nb,beta,eps", [(40, 256, 5.0, 1e-4), (48, 256, 6.0, 1e-6)])
def test_classfmt_build_stores_each_tile_in_its_class(E, ctx, L, nb, beta, eps):
    A = E.emu_cov_build_classfmt(ctx, L, beta, nb, eps=eps, prec_mask=MASK_ALL)
    S = O.cov_build(L, beta)
    cls, _ = E.emu_mat_tile_info(ctx, A)
    _, t = _expected_map(S, nb, eps, MASK_ALL)
    _map_matches(cls, t, eps, MASK_ALL, nb)
    assert np.all(np.diag(cls) == 0)
    G = _np(E.emu_mat_export(ctx, A))
    A.free()
    n, NT = L * L, cls.shape[0]
    for i in range(NT):
        for j in range(i + 1):
            ri, cj = np.s_[i * nb:min(n, (i + 1) * nb)], np.s_[j * nb:min(n, (j + 1) * nb)]
            ref = np.tril(S)[ri, cj] if i == j else S[ri, cj]
            got = G[ri, cj]
            c = cls[i, j]
            err = np.abs(got - ref)
            # the device's pow may differ from libm's in the last places of s(l)
            if c == 0:
                assert np.all(err <= 1e-15 * np.abs(ref))
            elif c == 1:
                assert np.all(err <= (2.0**-24 + 1e-15) * np.abs(ref))
            else:
                # BF16, and the E4M3 class's BF16 working values (its codes are
                # written when the factor solves the tile)
                assert np.all(err <= (2.0**-8 + 1e-15) * np.abs(ref))
    print(f"L={L} eps={eps:g}: tiles per class {np.bincount(cls[np.tril_indices(NT)], minlength=5)}")


@pytest.mark.parametrize("L,nb,beta,eps,mask", [
    (40, 256, 5.0, 1e-4, MASK_ALL),
    (48, 256, 6.0, 1e-6, MASK_ALL),
    (32, 256, 4.0, 1e-8, MASK_FP64_FP32_BF16),
    (64, 1024, 4.0, 1e-6, MASK_ALL),        # nb = 1024: the SIMT FP32 panel TRSM, as at L = 480
    (44, 512, 6.0, 1e-5, MASK_ALL),          # ragged last tile
])
def test_classfmt_factor_meets_eps(E, ctx, L, nb, beta, eps, mask):
    A = E.emu_cov_build_classfmt(ctx, L, beta, nb, eps=eps, prec_mask=mask)
    info = E.emu_potrf_mp(ctx, A, eps=eps, prec_mask=mask)
    S = O.cov_build(L, beta)
    cls, _ = E.emu_mat_tile_info(ctx, A)
    G = _np(E.emu_mat_export(ctx, A))
    A.free()
    be = np.linalg.norm(G @ G.T - S) / np.linalg.norm(S)
    assert be <= eps, be
    assert np.all(np.triu(G, 1) == 0)
    assert list(info.tiles) == list(np.bincount(cls[np.tril_indices(cls.shape[0])], minlength=5))
    print(f"L={L} nb={nb} eps={eps:g}: backward {be:.2e}, tiles {info.tiles}")


def test_classfmt_all_fp64_matches_the_oracle(E, ctx):
    # eps <= 0: every tile FP64, the updates as exact digit products; the
    # factor is the FP64 Cholesky factor
    L, nb, beta = 24, 256, 4.0
    A = E.emu_cov_build_classfmt(ctx, L, beta, nb, eps=0.0)
    E.emu_potrf_mp(ctx, A, eps=0.0)
    G = _np(E.emu_mat_export(ctx, A))
    A.free()
    Lo, _ = O.potrf_blocked(O.cov_build(L, beta), nb)
    assert np.linalg.norm(G - Lo) / np.linalg.norm(Lo) <= 1e-12


def test_classfmt_sampling(E, ctx):
    # Y = L Z with the stored tiles: FP64 and FP32 tiles at their precision,
    # BF16 and E4M3 tiles (exact in BF16) against bf16(Z), FP32 accumulation
    L, nb, beta, eps, s = 40, 256, 5.0, 1e-4, 200
    A = E.emu_cov_build_classfmt(ctx, L, beta, nb, eps=eps, prec_mask=MASK_ALL)
    E.emu_potrf_mp(ctx, A, eps=eps, prec_mask=MASK_ALL)
    cls, _ = E.emu_mat_tile_info(ctx, A)
    assert (cls == 4).any() and (cls == 3).any()
    G = _np(E.emu_mat_export(ctx, A))
    Y, Z = E.emu_sample(ctx, A, s, seed=3, return_z=True)
    Y2 = _np(E.emu_sample(ctx, A, s, seed=3))
    A.free()
    Y, Z = _np(Y), _np(Z)
    assert np.array_equal(Y, Y2)  # bit-reproducible
    assert np.abs(Z - O.normal_matrix(3, 0, L * L, s)).max() <= 1e-14
    n, NT = L * L, cls.shape[0]
    Zb = _bf16_rn(Z)
    ref = np.zeros_like(Y)
    for i in range(NT):
        ri = np.s_[i * nb:min(n, (i + 1) * nb)]
        for k in range(i + 1):
            ck = np.s_[k * nb:min(n, (k + 1) * nb)]
            ref[ri] += G[ri, ck] @ (Zb[ck] if cls[i, k] in (3, 4) else Z[ck])
    rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert rel <= 1e-6, rel


@pytest.mark.parametrize("classfmt", [True, False])
def test_backward_error_estimate(E, ctx, classfmt):
    # the Hutchinson estimate from 32 probes (S G regenerated from the
    # parameters) against the exact backward error of the exported factor
    L, nb, beta, eps = 48, 256, 6.0, 1e-6
    if classfmt:
        A = E.emu_cov_build_classfmt(ctx, L, beta, nb, eps=eps, prec_mask=MASK_ALL)
        E.emu_potrf_mp(ctx, A, eps=eps, prec_mask=MASK_ALL)
    else:
        A = E.emu_cov_build(ctx, L, beta, nb)
        E.emu_potrf_mp(ctx, A, eps=eps, prec_mask=MASK_ALL)
    est = E.emu_backward_error_est(ctx, A, L, beta, nprobes=32, seed=5)
    G = _np(E.emu_mat_export(ctx, A))
    A.free()
    S = O.cov_build(L, beta)
    be = np.linalg.norm(G @ G.T - S) / np.linalg.norm(S)
    assert 0.5 * be <= est <= 2.0 * be, (est, be)
    print(f"classfmt={classfmt}: estimate {est:.3e}, exact {be:.3e}")


def test_backward_error_estimate_of_the_fp64_factor_is_tiny(E, ctx):
    L, nb, beta = 24, 256, 4.0
    A = E.emu_cov_build(ctx, L, beta, nb)
    E.emu_potrf_mp(ctx, A)
    est = E.emu_backward_error_est(ctx, A, L, beta, nprobes=8, seed=1)
    A.free()
    assert est <= 1e-14, est


def test_classfmt_rejects_solves(E, ctx):
    import torch

    A = E.emu_cov_build_classfmt(ctx, 16, 4.0, 256, eps=1e-6, prec_mask=MASK_ALL)
    E.emu_potrf_mp(ctx, A, eps=1e-6, prec_mask=MASK_ALL)
    B = torch.zeros((256, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(E.EmuError):
        E.emu_potrs(ctx, A, B)
    A.free()
