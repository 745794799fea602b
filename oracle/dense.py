"""Oracle: the plain (dense) ST-BIEM time march.  TEST INFRASTRUCTURE ONLY.

T_n = sum_{m=0}^{n} K_m D_{n-m}   (Eq. 4; D = 0 before step 0, initial rest of Sec. 2.1.1)

``march`` is the definition written out (one contraction per step).
``march_rows_fft`` evaluates the same sum for a few receivers using an FFT
convolution in time (a library primitive used as one step of the definition),
for workloads too large for the direct loop.

``rupture_march`` is the dynamic-rupture time march of Sec. 6.2 on any kernel operator (the
plain one or the FDP=H compressed one): each step predicts the traction from the history,
solves the friction law element by element against the instantaneous self term K_{i,i,0}
(radiation damping; the instantaneous term is local when cs dt <= dx/2) and appends D_n.

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


def rupture_march(K, tau0, sigma_n, mu_s, mu_d, Dc, dt, M, law="linear"):
    """Dynamic rupture, Sec. 6.2.  Unruptured elements keep zero slip rate until the traction
    reaches the strength; slipping elements carry traction = strength; no back slip (D >= 0);
    the strength uses the slip u of the previous step:
        law "linear":      strength(u) = sigma_n (mu_s - (mu_s - mu_d) min(u / Dc, 1))
        law "exponential": strength(u) = (T_th - T_dy) exp(-u / Dc) + T_dy   (Sec. 6.2),
                           T_th = sigma_n mu_s, T_dy = sigma_n mu_d.
    K[m, i, j] with m < M.  Returns D[n, i], T[n, i] (total traction)."""
    N = K.shape[1]
    D = np.zeros((M, N))
    T = np.zeros((M, N))
    slip = np.zeros(N)
    k0 = np.diag(K[0]).copy()               # K_{i,i,0} = -mu / (2 cs)
    t_th, t_dy = sigma_n * mu_s, sigma_n * mu_d
    for n in range(M):
        mm = min(n + 1, K.shape[0])
        pred = np.einsum("mij,mj->i", K[1:mm], D[n - 1::-1][:mm - 1]) if n > 0 else np.zeros(N)
        tau = tau0 + pred
        if law == "exponential":
            strength = (t_th - t_dy) * np.exp(-slip / Dc) + t_dy
        elif law == "linear":
            strength = sigma_n * (mu_s - (mu_s - mu_d) * np.minimum(slip / Dc, 1.0))
        else:
            raise ValueError("law is 'linear' or 'exponential'")
        v = np.where(tau > strength, (tau - strength) / (-k0), 0.0)
        D[n] = v
        T[n] = tau + k0 * v
        slip = slip + v * dt
    return D, T
