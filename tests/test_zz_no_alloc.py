"""The no-allocation covariance build (emu_cov_build_dense_noalloc), for
callers that cannot allocate device memory while they call the library, gives
the same lower triangle as emu_cov_build followed by emu_mat_export, on two
calls in a row.  Collected last on purpose, so that a failure here leaves every
other test already run."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(E, lib, L, beta, out, stream):
    n = L * L
    return lib.emu_cov_build_dense_noalloc(L, beta, 1.5, 1e-8, ctypes.c_void_p(out.data_ptr()), n,
                                           ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_build_matches_tiled_build_twice():
    import torch

    import paper_2408_04440_gb300 as E
    from paper_2408_04440_gb300 import build

    build.build()
    lib = E.load()
    stream = torch.cuda.current_stream()
    with E.Context(0) as ctx:
        # two calls in a row, different sizes, the second reusing the scratch
        for L, beta in [(32, 4.0), (20, 3.0)]:
            n = L * L
            out = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()  # column-major
            assert _noalloc(E, lib, L, beta, out, stream) == E.EMU_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            A = E.emu_cov_build(ctx, L, beta, 128)
            ref = E.emu_mat_export(ctx, A).cpu().numpy()
            A.free()
            # same operations in the same order: the tolerance of the build tests,
            # and in practice bit equality
            assert np.max(np.abs(got - ref)) <= 4e-16 * np.max(np.abs(ref))
            assert np.array_equal(np.triu(got, 1), np.zeros_like(got))  # upper untouched


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch

    import paper_2408_04440_gb300 as E

    lib = E.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    s = lib.emu_cov_build_dense_noalloc(129, 4.0, 1.5, 1e-8, ctypes.c_void_p(buf.data_ptr()), 129 * 129,
                                        ctypes.c_void_p(0))
    assert s == E.EMU_ENOMEM
