"""Oracle: the plain (dense) ST-BIEM time march.  TEST INFRASTRUCTURE ONLY.

T_n = sum_{m=0}^{n} K_m D_{n-m}   (Eq. 4; D = 0 before step 0, initial rest of Sec. 2.1.1)

``march`` is the definition written out (one contraction per step).
``march_rows_fft`` evaluates the same sum for a few receivers using an FFT
convolution in time (a library primitive used as one step of the definition),
for workloads too large for the direct loop.

Parity: pinned by tests/test_oracle_dense.py against (i) a pure-Python
quadruple loop at tiny N, (ii) the closed form T = -mu/(2 cs) D at interior
points of a long straight fault under uniform slip rate, before the edge
waves arrive (Sec. 6: the radiation-damping term), (iii) causality.
"""
import numpy as np


def march(K, D):
    """K[m, i, j] (m < M), D[n, j] (n < M)  ->  T[n, i]."""
    M = D.shape[0]
    T = np.zeros((M, K.shape[1]))
    for n in range(M):
        mm = min(n + 1, K.shape[0])
        # sum over m <= n of K_m @ D_{n-m}
        T[n] = np.einsum("mij,mj->i", K[:mm], D[n::-1][:mm])
    return T


def march_rows_fft(K_rows, D):
    """K_rows[m, r, j] for a set of receivers r, D[n, j] -> T[n, r] (same sum, FFT in time)."""
    M = D.shape[0]
    Mk = K_rows.shape[0]
    L = 1
    while L < M + Mk:
        L *= 2
    FD = np.fft.rfft(D, n=L, axis=0)                  # [f, j]
    out = np.zeros((M, K_rows.shape[1]))
    for r in range(K_rows.shape[1]):
        FK = np.fft.rfft(K_rows[:, r, :], n=L, axis=0)  # [f, j]
        out[:, r] = np.fft.irfft((FK * FD).sum(axis=1), n=L)[:M]
    return out
