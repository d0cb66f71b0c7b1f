"""The half-length form of the circle coefficients used by the forward SHT.

The forward transform extends each colatitude function from [0, pi] to the
full circle, g_i = v_i for i <= N and g_i = sgn v_{M-i} above (M = 2N,
N = ntheta - 1; sgn = (-1)^m), and needs its Fourier coefficients
c_q = (1/M) sum_i g_i exp(-2 pi i q i / M) for |q| < L.  The kernel pairs the
samples i and M - i: for sgn = +1, c_q = (v_0 + (-1)^q v_N + 2 sum_{0<i<N}
v_i cos(2 pi q i / M)) / M, real; for sgn = -1, c_q = (v_0 + (-1)^q v_N) / M
- 2i/M sum_{0<i<N} v_i sin(2 pi q i / M); and c_{-q} = conj(c_q).  These
checks compare that form with the FFT of the explicitly extended sequence.
"""
import numpy as np
import pytest


def extended(v, sgn):
    N = len(v) - 1
    M = 2 * N
    g = np.empty(M)
    g[: N + 1] = v
    for i in range(N + 1, M):
        g[i] = sgn * v[M - i]
    return g


def half_length(v, sgn, L):
    N = len(v) - 1
    M = 2 * N
    out = np.zeros(2 * L - 1, dtype=complex)
    i = np.arange(1, N)
    for q in range(L):
        ends = v[0] + (-1) ** q * v[N]
        if sgn > 0:
            c = (ends + 2.0 * np.sum(v[1:N] * np.cos(2 * np.pi * q * i / M))) / M
        else:
            c = ends / M - 2j / M * np.sum(v[1:N] * np.sin(2 * np.pi * q * i / M))
        out[q + L - 1] = c
        out[L - 1 - q] = np.conj(c)
    return out


@pytest.mark.parametrize("ntheta,L", [(2, 1), (9, 8), (33, 32), (65, 40), (129, 128)])
@pytest.mark.parametrize("sgn", [1.0, -1.0])
def test_half_length_form_matches_the_fft(ntheta, L, sgn):
    rng = np.random.default_rng(ntheta * 7 + int(sgn > 0))
    v = rng.standard_normal(ntheta)  # nonzero pole values too: i = 0 and i = N are not reflected
    g = extended(v, sgn)
    M = len(g)
    full = np.fft.fft(g) / M  # c_q at index q mod M
    ref = np.array([full[q % M] for q in range(-(L - 1), L)])
    got = half_length(v, sgn, L)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
