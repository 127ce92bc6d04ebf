"""Textbook matrix forms of the one-level periodic DWT, used to pin the oracle.

TEST INFRASTRUCTURE ONLY (imported by the test suite).

These are built from the standard definition of a periodic two-channel filter
bank (analysis row i of the low-pass half holds h_k at column (2i + k) mod N),
not from the paper's per-index equations, so comparing them with the oracle's
literal Eq. 1-6 / 11-16 code applied to unit vectors checks the oracle against
an independent statement of the same transform.
"""
from __future__ import annotations

import numpy as np


def d4_filters():
    """Daubechies-4 low-pass h (closed form, sum h = sqrt 2) and its quadrature
    mirror g_k = (-1)^k h_{3-k}."""
    s3 = np.sqrt(3.0)
    h = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * np.sqrt(2.0))
    g = np.array([h[3], -h[2], h[1], -h[0]])
    return h, g


def analysis_matrix(N: int, wavelet: int) -> np.ndarray:
    """N x N periodic analysis matrix A: y = A x gives [approximation | detail]."""
    if wavelet == 0:
        h = np.array([0.5, 0.5])
        g = np.array([0.5, -0.5])
    else:
        h, g = d4_filters()
    A = np.zeros((N, N))
    for i in range(N // 2):
        for k in range(len(h)):
            A[i, (2 * i + k) % N] += h[k]
            A[N // 2 + i, (2 * i + k) % N] += g[k]
    return A


def lowpass_rows(N: int, wavelet: int) -> np.ndarray:
    """The N/2 x N low-pass half L of the analysis matrix."""
    return analysis_matrix(N, wavelet)[: N // 2]


def synthesis_scale(wavelet: int) -> float:
    """sigma with S = sigma * A^T: 1 for orthonormal D4, 2 for the /2 Haar."""
    return 2.0 if wavelet == 0 else 1.0


def fuse_closed_form(pan: np.ndarray, ms: np.ndarray, wavelet: int, gain: float) -> np.ndarray:
    """One band of the fusion written as a matrix identity rather than as steps:
        F = P + sigma^2 L_H^T (gain M - L_H P L_W^T) L_W,
    which follows from F = S_H Z' S_W^T with Z' = A_H P A_W^T except on LL, and
    S = sigma A^T.  For Haar this is P + rep2x2(M - blockmean2x2(P))."""
    H, W = pan.shape
    LH = lowpass_rows(H, wavelet)
    LW = lowpass_rows(W, wavelet)
    s2 = synthesis_scale(wavelet) ** 2
    return pan + s2 * LH.T @ (gain * ms - LH @ pan @ LW.T) @ LW


def adjoint_closed_form(grad: np.ndarray, wavelet: int, gain: float):
    """Adjoint of fuse_closed_form for one band: (grad_pan, grad_ms)
        grad_ms  = gain sigma^2 L_H G L_W^T
        grad_pan = G - sigma^2 L_H^T L_H G L_W^T L_W."""
    H, W = grad.shape
    LH = lowpass_rows(H, wavelet)
    LW = lowpass_rows(W, wavelet)
    s2 = synthesis_scale(wavelet) ** 2
    gm = gain * s2 * LH @ grad @ LW.T
    gp = grad - s2 * LH.T @ (LH @ grad @ LW.T) @ LW
    return gp, gm
