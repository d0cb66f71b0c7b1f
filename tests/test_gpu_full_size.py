"""Full-size parity cases on the GPU, through the C ABI.

Two workloads at their full sizes:
  * n = 16384 (L=128, nb=512, beta=8): FP64 vs adaptive FP64/FP32/BF16 at
    eps=1e-8, 256 samples with seed 1;
  * n = 65536 (L=256, nb=1024, beta=12): adaptive FP64/FP32/BF16/FP8-E4M3 at
    eps=1e-6, then 16 N(0,1) right-hand sides (Philox seed 4, stream 1)
    solved by iterative refinement with FP64 residuals.
The oracle cannot factor these sizes in seconds, so every check uses outputs
it computes one by one (rows of the covariance, norms of sampled tile rows,
the precision rule on given norms, one panel step of the blocked factor) or a
property that holds at any size (the backward error and the solve residual on
sampled rows, against the oracle's covariance rows).
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu



def U_of(nb):
    """The library's default unit roundoffs: the FP32 class carries the
    sqrt(nb) growth of an nb-term FP32 accumulation."""
    return np.array([2.0**-53, 2.0**-24 * np.sqrt(nb), 2.0**-11, 2.0**-8, 2.0**-4])

MASK_FP64_FP32_BF16 = 0b01011
MASK_WITH_E4M3 = 0b11011


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


def _rows(n, m, seed):
    """m rows spread over [0, n): one per equal stratum, seeded position."""
    rng = np.random.default_rng(seed)
    edges = np.linspace(0, n, m + 1).astype(np.int64)
    return np.array([rng.integers(edges[q], edges[q + 1]) for q in range(m)], dtype=np.int64)


def _bf16_rn(x):
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def _map_agrees(cls, t, eps, mask, nb):
    """Classes equal the rule's on norms t, except where a tile sits within
    1e-12 of a class threshold (both sides sum the norms in their own order)."""
    U = U_of(nb)
    co = O.precision_map(t, eps, U, mask)
    NT = t.shape[0]
    thr = eps * O.frob_from_tiles(t) / NT
    for i in range(NT):
        for j in range(i + 1):
            if cls[i, j] != co[i, j]:
                assert min(abs(t[i, j] * U[c] - thr) / thr for c in range(1, 5)) < 1e-12, (i, j)


def _export_rows(E, ctx, A, idx):
    """Rows idx of the exported lower factor (host) and the device export."""
    import torch

    Ld = E.emu_mat_export(ctx, A)
    ti = torch.as_tensor(idx, device=Ld.device)
    return Ld, ti


def _row_backward_error(E, ctx, A, idx, S_rows, frob):
    """sqrt(n/m) ||(L L^T - S)[idx, :]||_F / ||S||_F: the normwise backward
    error estimated from the sampled rows (unbiased for the squared norm)."""
    import torch

    Ld, ti = _export_rows(E, ctx, A, idx)
    LLt = (Ld[ti, :] @ Ld.t()).cpu().numpy()
    del Ld
    torch.cuda.empty_cache()
    n = S_rows.shape[1]
    R = LLt - S_rows
    return float(np.sqrt(n / len(idx)) * np.linalg.norm(R) / frob)


# ------------------------------------------------------------ n = 16384
L2, NB2, BETA2, EPS2, S2 = 128, 512, 8.0, 1e-8, 256


@pytest.fixture(scope="module")
def S16k():
    return O.cov_build(L2, BETA2)


def test_n16384_norms_map_backward_error(E, ctx, S16k):
    n = L2 * L2
    A = E.emu_cov_build(ctx, L2, BETA2, NB2)
    _, tn = E.emu_mat_tile_info(ctx, A)
    to = O.tile_norms(S16k, NB2)
    low = np.tril(np.ones_like(to, dtype=bool))
    # the oracle sums a tile's nb^2 squares in one recursive chain, whose
    # relative error bound is (nb^2 - 1) u; the entries agree to a few ulp
    rtol = NB2 * NB2 * 2.0**-53
    assert np.allclose(tn[low], to[low], rtol=rtol, atol=0)
    info = E.emu_potrf_mp(ctx, A, eps=EPS2, prec_mask=MASK_FP64_FP32_BF16)
    assert info.status == E.EMU_OK
    assert abs(info.frob - O.frob_from_tiles(to)) <= rtol * info.frob
    cls, _ = E.emu_mat_tile_info(ctx, A)
    _map_agrees(cls, to, EPS2, MASK_FP64_FP32_BF16, NB2)
    # the full backward error against the oracle's covariance (one FP64
    # product L L^T of 8.8e12 flop, done by torch on the device for the test)
    import torch

    Ld = E.emu_mat_export(ctx, A)
    Sg = torch.from_numpy(S16k).to(Ld.device)
    be = float(torch.linalg.norm(Ld @ Ld.t() - Sg) / torch.linalg.norm(Sg))
    del Ld, Sg
    torch.cuda.empty_cache()
    assert be <= EPS2, be
    print(f"n=16384 eps=1e-8: tiles {info.tiles}, full backward error {be:.2e}, factor {info.ms:.1f} ms")


def test_n16384_sampling_rows(E, ctx, S16k):
    # Z equals the oracle's Philox/Box-Muller normals; sampled rows of Y equal
    # the per-class product: FP64/FP32 tiles exact, BF16 tiles with both
    # operands rounded to BF16, up to FP32 accumulation
    import torch

    n = L2 * L2
    A = E.emu_cov_build(ctx, L2, BETA2, NB2)
    E.emu_potrf_mp(ctx, A, eps=EPS2, prec_mask=MASK_FP64_FP32_BF16)
    cls, _ = E.emu_mat_tile_info(ctx, A)
    Y, Z = E.emu_sample(ctx, A, S2, seed=1, return_z=True)
    idx = _rows(n, 64, 12)
    Ld, ti = _export_rows(E, ctx, A, idx)
    Lr = Ld[ti, :].cpu().numpy()
    del Ld
    torch.cuda.empty_cache()
    Yr = Y[torch.as_tensor(idx, device=Y.device), :].cpu().numpy()
    Z = Z.cpu().numpy()
    Zo = O.normal_matrix(1, 0, n, S2)
    assert np.max(np.abs(Z - Zo)) <= 1e-14 * np.max(np.abs(Zo))
    Zb = _bf16_rn(Z)
    ref = np.zeros_like(Yr)
    for q, r in enumerate(idx):
        i = r // NB2
        for k in range(i + 1):
            ck = np.s_[k * NB2:(k + 1) * NB2]
            if cls[i, k] in (3, 4):
                ref[q] += _bf16_rn(Lr[q, ck]) @ Zb[ck]
            else:
                ref[q] += Lr[q, ck] @ Z[ck]
    # the tensor cores accumulate up to n products per output in FP32:
    # probabilistic bound sqrt(n) 2^-24 on the relative error
    rel = np.linalg.norm(Yr - ref) / np.linalg.norm(ref)
    assert rel <= np.sqrt(n) * 2.0**-24, rel
    Y2 = E.emu_sample(ctx, A, S2, seed=1)
    assert torch.equal(Y, Y2)  # bit-reproducible per seed


def test_n16384_fp64_first_panel_and_rows(E, ctx, S16k):
    # the plain FP64 path: its first block column against the oracle's first
    # panel step (POTRF of tile (0,0) and the column's TRSM) to 1e-12, and the
    # backward error on sampled rows at FP64 level
    import torch

    n = L2 * L2
    A = E.emu_cov_build(ctx, L2, BETA2, NB2)
    info = E.emu_potrf_mp(ctx, A)
    assert info.status == E.EMU_OK
    Ld = E.emu_mat_export(ctx, A)
    col0 = Ld[:, :NB2].cpu().numpy()
    del Ld
    torch.cuda.empty_cache()
    P = O.potrf_blocked(S16k, NB2, kmax=1)[0]  # one panel step
    ref = P[:, :NB2]
    assert np.linalg.norm(col0 - ref) <= 1e-12 * np.linalg.norm(ref)
    idx = _rows(n, 64, 13)
    be = _row_backward_error(E, ctx, A, idx, S16k[idx, :], np.linalg.norm(S16k))
    assert be <= 1e-14, be
    print(f"n=16384 FP64: first panel vs oracle ok, backward (64 sampled rows) {be:.2e}, factor {info.ms:.1f} ms")


# ------------------------------------------------------------ n = 65536
L3, NB3, BETA3, EPS3, NRHS3 = 256, 1024, 12.0, 1e-6, 16


def test_n65536_e4m3_factor_and_refined_solve(E, ctx):
    import torch

    n = L3 * L3
    S_mat = E.emu_cov_build(ctx, L3, BETA3, NB3)
    _, tn = E.emu_mat_tile_info(ctx, S_mat)
    NT = tn.shape[0]
    # covariance entries on sampled rows against the oracle's closed form
    idx = _rows(n, 128, 21)
    S_rows = O.cov_rows(L3, BETA3, idx)
    Sd = E.emu_mat_export(ctx, S_mat)  # lower triangle
    ti = torch.as_tensor(idx, device=Sd.device)
    G_rows = torch.where(torch.arange(n, device=Sd.device)[None, :] <= ti[:, None], Sd[ti, :],
                         Sd[:, ti].t()).cpu().numpy()
    del Sd
    torch.cuda.empty_cache()
    assert np.max(np.abs(G_rows - S_rows)) <= 1e-15 * np.max(np.abs(S_rows))
    # tile norms of sampled tile rows against the oracle's rows
    for bi in (0, 29, NT - 1):
        rows = np.arange(bi * NB3, min(n, (bi + 1) * NB3))
        R = O.cov_rows(L3, BETA3, rows)
        for j in range(bi + 1):
            # numpy's norm and the GPU's per-thread partial sums both add in
            # short chains: far below the recursive-chain bound nb^2 u
            t = np.linalg.norm(R[:, j * NB3:(j + 1) * NB3])
            assert abs(tn[bi, j] - t) <= 1e-12 * t, (bi, j)
        del R
    # the factor: the rule on the norms, E4M3 tiles present, eps met
    A = E.emu_mat_clone(ctx, S_mat)
    info = E.emu_potrf_mp(ctx, A, eps=EPS3, prec_mask=MASK_WITH_E4M3)
    assert info.status == E.EMU_OK
    assert abs(info.frob - O.frob_from_tiles(tn)) <= 1e-13 * info.frob
    cls, _ = E.emu_mat_tile_info(ctx, A)
    _map_agrees(cls, tn, EPS3, MASK_WITH_E4M3, NB3)
    assert info.tiles[4] > 0 and info.tiles[3] > 0
    frob = info.frob
    be = _row_backward_error(E, ctx, A, idx, S_rows, frob)
    assert be <= EPS3, be
    # refinement: FP64 residuals against the FP64 covariance, corrections from
    # the mixed factor; the residual on the sampled rows is then checked
    # against the oracle's covariance rows
    B = O.normal_matrix(4, 1, n, NRHS3)
    X, ri = E.emu_solve_refine(ctx, A, S_mat, torch.from_numpy(B).cuda(), tol=1e-13, maxit=60)
    assert ri.status == E.EMU_OK
    X = X.cpu().numpy()
    r = B[idx, :] - S_rows @ X
    est = np.sqrt(n / len(idx)) * np.linalg.norm(r, axis=0)
    eta = est / (frob * np.linalg.norm(X, axis=0) + np.linalg.norm(B, axis=0))
    assert eta.max() <= 1e-12, eta.max()
    print(f"n=65536 eps=1e-6: tiles {info.tiles}, factor {info.ms:.1f} ms, backward (128 sampled rows) {be:.2e}; "
          f"refine {ri.iters} iterations in {ri.ms:.1f} ms, sampled-row backward error {eta.max():.2e}")
