"""The factorisation of the band-limited inverse transform that the unfold kernel evaluates.

The analytic inverse (Sec. 4) of a band of M = N/4 bins starting at k_lo is
    z[n] = sum_j Z[j] exp(2 pi i (k_lo + j) n / N),  j in [0, M).
The kernel evaluates it at n = 4m + r as four M-point transforms split M = P x Q (pass 1: a
Q-point DFT per (r, ja); pass 2: a P-point DFT per (r, mb) over rows rotated by k_lo mod P).
Two layouts share that skeleton and differ in where the output twiddle
T1[r][mb][ja] = exp(2 pi i (k_lo + ja)(r + 4 mb) / N) is applied:
  * 1024 and 4096 samples: in pass 1, after its DFT;
  * 2048 samples: in pass 2, as c u^i per row i, with the rows past k_lo mod P shifted by
    one input slot in pass 1 (slot 0 turned by i^r).
This test restates both factorisations in numpy, in FP64, and checks them against the direct
sum for band offsets with every kind of k_lo mod P: it pins the mathematics the kernels
follow, not the kernels themselves (it runs no CUDA code and shares nothing with the oracle
or the CUDA path). The kernels' own index arithmetic for each k_lo mod P is pinned on the GPU
by tests/test_gpu_parity.py::test_parity_band_offsets (sampling rates that put k_lo at every
kind of residue, at each length, against the oracle), and on the tensor-core path and the
allocation-free entry point by the band-offset cases in tests/test_gpu_tc.py and
tests/test_zz_no_alloc.py.
"""
import numpy as np
import pytest

SHAPES = {1024: (16, 16), 2048: (32, 16), 4096: (32, 32)}   # N -> (Q, P)


def direct(Z, k_lo, n):
    k = k_lo + np.arange(Z.size)
    return np.exp(2j * np.pi * np.outer(np.arange(n), k) / n) @ Z


def _pass2(A, n, Q, P):
    """A[r][row][mb] -> z[4 (mb + Q ma) + r] = sum_row A[r][row][mb] exp(2 pi i row ma / P)."""
    F = np.exp(2j * np.pi * np.outer(np.arange(P), np.arange(P)) / P)     # [row][ma]
    out = np.einsum("rim,ia->rma", A, F)                                   # [r][mb][ma]
    z = np.empty(n, complex)
    for r in range(4):
        m = np.arange(Q)[:, None] + Q * np.arange(P)[None, :]              # m = mb + Q ma
        z[4 * m + r] = out[r]
    return z


def _pre(Q):
    return np.exp(2j * np.pi * np.outer(np.arange(4), np.arange(Q)) / (4 * Q))   # [r][jb]


def _dft_q(x, Q):
    W = np.exp(2j * np.pi * np.outer(np.arange(Q), np.arange(Q)) / Q)     # [jb][mb]
    return x @ W


def layout_twiddle_in_pass1(Z, k_lo, n):
    Q, P = SHAPES[n]
    Zr = Z.reshape(Q, P)                                                    # [jb][ja], j = ja + P jb
    A = np.empty((4, P, Q), complex)
    for r in range(4):
        X = _dft_q((Zr * _pre(Q)[r][:, None]).T, Q)                        # [ja][mb]
        ja = np.arange(P)[:, None]
        mb = np.arange(Q)[None, :]
        X = X * np.exp(2j * np.pi * (k_lo + ja) * (r + 4 * mb) / n)
        A[r, (k_lo + np.arange(P)) % P, :] = X
    return _pass2(A, n, Q, P)


def layout_twiddle_in_pass2(Z, k_lo, n, turn=True, shift=True):
    """turn / shift off: the two slips this layout invites (for the test that the check bites)."""
    Q, P = SHAPES[n]
    kr, f0 = k_lo % P, k_lo // P
    A = np.empty((4, P, Q), complex)
    for r in range(4):
        for ja in range(P):
            sh = shift and ja + kr >= P
            x = np.empty(Q, complex)
            if sh:   # one-slot cyclic shift of the input, slot 0 turned by i^r
                x[0] = Z[ja + P * (Q - 1)] * (1j ** r if turn else 1)
                x[1:] = Z[ja + P * np.arange(Q - 1)] * _pre(Q)[r][1:]
            else:
                x[:] = Z[ja + P * np.arange(Q)] * _pre(Q)[r]
            A[r, (kr + ja) % P, :] = _dft_q(x, Q)
    w = 4 * np.arange(Q)[None, :] + np.arange(4)[:, None]                  # [r][mb]: 4 mb + r
    c = np.exp(2j * np.pi * f0 * P * w / n)
    u = np.exp(2j * np.pi * w / n)
    tau = c[:, None, :] * u[:, None, :] ** np.arange(P)[None, :, None]     # [r][row][mb]
    return _pass2(A * tau, n, Q, P)


@pytest.mark.parametrize("n", [1024, 2048, 4096])
def test_both_layouts_equal_the_direct_inverse(n):
    Q, P = SHAPES[n]
    rng = np.random.default_rng(n)
    # band offsets with k_lo mod P = 0, 1, P / 2, P - 1 and the 200 MHz windows of the workloads
    offsets = sorted({8 * P, 8 * P + 1, 8 * P + P // 2, 9 * P - 1, round(0.15 * n + 0.5)})
    for k_lo in offsets:
        Z = rng.standard_normal(n // 4) + 1j * rng.standard_normal(n // 4)
        ref = direct(Z, k_lo, n)
        scale = np.abs(ref).max()
        for f in (layout_twiddle_in_pass1, layout_twiddle_in_pass2):
            err = np.abs(f(Z, k_lo, n) - ref).max() / scale
            assert err < 1e-12, (f.__name__, k_lo, err)


def test_a_plausible_slip_is_caught():
    """The check bites: the 2048-sample layout without slot 0's quarter turn, or without the
    one-slot shift of the rows past k_lo mod P, misses the direct inverse by far more than
    rounding; with k_lo mod P = 0 no row is shifted and both slips are harmless."""
    n = 2048
    Q, P = SHAPES[n]
    rng = np.random.default_rng(1)
    Z = rng.standard_normal(n // 4) + 1j * rng.standard_normal(n // 4)
    for k_lo, bites in ((8 * P + 5, True), (8 * P, False)):
        ref = direct(Z, k_lo, n)
        scale = np.abs(ref).max()
        assert np.abs(layout_twiddle_in_pass2(Z, k_lo, n) - ref).max() / scale < 1e-12
        for kw in (dict(turn=False), dict(shift=False)):
            err = np.abs(layout_twiddle_in_pass2(Z, k_lo, n, **kw) - ref).max() / scale
            assert (err > 1e-3) == bites, (k_lo, kw, err)
