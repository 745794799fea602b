"""Oracle: the quantization method of App. A (staircase approximation of a temporal kernel).
TEST INFRASTRUCTURE ONLY: nothing of the product path imports this module.

A temporal convolution T_n = sum_{m = M_init}^{M_fin - 1} K_m D_{n-m} is approximated by a
staircase of Q constant values Khat_q over the ranges b_q <= m < b_{q+1} (App. A.1.1):

    T_n ~ sum_q Khat_q Dhat_{n,q},   Dhat_{n,q} = sum_{m = b_q}^{b_{q+1} - 1} D_{n-m},

with the running update Dhat_{n,q} = Dhat_{n-1,q} + D_{n-b_q} - D_{n-b_{q+1}}.

Partition rule (the one the paper uses for the antiplane problem): b_0 = M_init; from b_q the
range grows while |K_m - K_{b_q}| / 2 <= eps_Q |Khat| with Khat = (K_{b_q} + K_m) / 2 (with the
optional absolute bound, min(eps_Q |Khat|, eps_abs)); b_{q+1} is the first m that breaks it, and
Khat_q = (K_{b_q} + K_{b_{q+1} - 1}) / 2.  Readings (the passage is partly garbled): the "end"
kernel value in Khat is K_{b_{q+1} - 1}, and the comparison is made with the candidate end m.
"""
import numpy as np


def partitions(K, eps_q, eps_abs=None, m_init=0):
    """Partitions b (length Q + 1, b[0] = m_init, b[-1] = len(K)) and values Khat (length Q) of
    the staircase approximation of K[m_init:] (App. A.1.1)."""
    K = np.asarray(K, dtype=np.float64)
    M = K.shape[0]
    b, khat = [m_init], []
    q0 = m_init
    while q0 < M:
        m = q0 + 1
        while m < M:
            kh = 0.5 * (K[q0] + K[m])
            bound = eps_q * abs(kh)
            if eps_abs is not None:
                bound = min(bound, eps_abs)
            if 0.5 * abs(K[m] - K[q0]) > bound:
                break
            m += 1
        khat.append(0.5 * (K[q0] + K[m - 1]))
        b.append(m)
        q0 = m
    return np.array(b, dtype=np.int64), np.array(khat)


def staircase(b, khat, M):
    """The quantized kernel as a sequence: Khat_q on b_q <= m < b_{q+1}, zero before b_0."""
    out = np.zeros(M)
    for q in range(len(khat)):
        out[b[q]:b[q + 1]] = khat[q]
    return out


def convolve_running(b, khat, D):
    """T_n = sum_q Khat_q Dhat_{n,q} for every n, the window sums Dhat kept by the running update
    of Eq. A.4 (D_n = 0 for n < 0).  D: (steps,) or (steps, N)."""
    D = np.asarray(D, dtype=np.float64)
    steps = D.shape[0]
    tail = D.shape[1:]
    Q = len(khat)
    dhat = np.zeros((Q,) + tail)
    T = np.zeros_like(D)

    def at(t):
        return D[t] if 0 <= t < steps else 0.0

    for n in range(steps):
        for q in range(Q):
            dhat[q] = dhat[q] + at(n - b[q]) - at(n - b[q + 1])
        T[n] = np.tensordot(khat, dhat, axes=(0, 0))
    return T
