"""Pins of the oracle's plain (dense) time march (CPU only)."""
import math

import numpy as np
import pytest

from oracle import dense
from oracle import kernel as kn
from paper_1903_02118_gb300 import inputs


def test_march_equals_quadruple_loop():
    N, M = 5, 7
    el = kn.element_table(inputs.kinked_fault(N))
    K = kn.discrete_kernel(el, 0.5, M, 1.0, 1.0)
    D = np.random.default_rng(1).standard_normal((M, N))
    T = dense.march(K, D)
    for n in range(M):
        for i in range(N):
            s = 0.0
            for m in range(n + 1):
                for j in range(N):
                    s += K[m, i, j] * D[n - m, j]
            assert abs(T[n, i] - s) < 1e-14 * (1 + abs(s))


def test_uniform_slip_rate_gives_radiation_damping_until_edge_waves():
    # Sec. 6: -mu/(2 cs) is the radiation damping; on an (effectively) infinite planar fault
    # under uniform slip rate V the stress stays exactly -mu V /(2 cs) (1-D plane wave) until
    # the waves from the fault ends reach the receiver.
    N, M, mu, cs, dt = 200, 120, 1.0, 1.0, 0.5
    el = kn.element_table(inputs.straight_fault(N))
    K = kn.discrete_kernel(el, dt, M, mu, cs)
    D = np.full((M, N), 0.7)
    T = dense.march(K, D)
    i = 100
    edge = el["mx"][i] - 0.0       # distance to the nearer fault end
    for n in range(M):
        if cs * (n + 1) * dt < edge - 1e-9:
            assert abs(T[n, i] - (-mu * 0.7 / (2 * cs))) < 1e-13
    assert abs(T[M - 1, 199] - (-mu * 0.7 / (2 * cs))) > 1e-3   # the end element feels its edge


def test_causality_of_march():
    N, M = 60, 80
    el = kn.element_table(inputs.curved_fault(N, 9))
    K = kn.discrete_kernel(el, 0.5, M, 1.0, 1.0)
    D = np.zeros((M, N))
    D[10:, 0] = 1.0
    T = dense.march(K, D)
    d = np.hypot(el["mx"] - el["bx"][0], el["my"] - el["by"][0])   # distance to nearest end of element 0
    for i in range(1, N):
        first = int(np.ceil(d[i] / 0.5)) - 1 + 10   # first step whose window reaches the front
        assert np.all(T[:max(first - 1, 0), i] == 0.0)


def test_fft_rows_equal_march():
    N, M = 40, 90
    el = kn.element_table(inputs.curved_fault(N, 3))
    K = kn.discrete_kernel(el, 0.5, M, 1.0, 1.0)
    D = inputs.gaussian_filtered_history(N, M, 4)
    T = dense.march(K, D)
    rows = [0, 7, 39]
    Tr = dense.march_rows_fft(K[:, rows, :], D)
    assert np.abs(Tr - T[:, rows]).max() < 1e-12 * np.abs(T).max()


@pytest.mark.parametrize("law", ["linear", "exponential"])
def test_rupture_follows_the_plane_wave_recursion_inside_the_causal_cone(law):
    # Uniform overstress on a long planar fault: before edge waves arrive every interior element
    # is a 1-D plane-wave problem, T = tau0 - mu/(2 cs) v, so the slip rate obeys
    # eta v_n = tau0 - strength(u_n), u_{n+1} = u_n + v_n dt exactly (Sec. 6.2 law).  For the
    # exponential law this explicit recursion is the Euler scheme of
    # eta du/dt = a - b exp(-u / Dc) (a = tau0 - T_dy, b = T_th - T_dy), whose solution is
    # exp(u / Dc) = b / a + (1 - b / a) exp(a t / (eta Dc)).
    N, M, dt = 160, 60, 0.5
    el = kn.element_table(inputs.straight_fault(N))
    K = kn.discrete_kernel(el, dt, M, 1.0, 1.0)
    tau0 = np.full(N, 0.62)
    Dc = 4.0
    D, T = dense.rupture_march(K, tau0, 1.0, 0.6, 0.3, Dc, dt, M, law=law)
    u, eta = 0.0, 0.5
    i = N // 2
    for n in range(M):
        if (n + 1) * dt >= el["mx"][i] - 1.0:   # edge waves could have arrived
            break
        if law == "linear":
            s = 0.6 - 0.3 * min(u / Dc, 1.0)
        else:
            s = 0.3 + 0.3 * math.exp(-u / Dc)
        v = max(0.62 - s, 0.0) / eta
        assert abs(D[n, i] - v) < 1e-12 and abs(T[n, i] - (0.62 - eta * v)) < 1e-12
        u += v * dt
    assert n > 40
    if law == "exponential":
        a, b, t = 0.32, 0.3, n * dt
        u_ode = Dc * math.log(b / a + (1 - b / a) * math.exp(a * t / (eta * Dc)))
        u_march = D[:n, i].sum() * dt
        # Euler (lambda dt = a dt / (eta Dc) = 0.08) is 6 % behind the ODE here; the linear law
        # with the same T_th, T_dy, Dc would be 28 % ahead
        assert abs(u_march - u_ode) < 0.1 * u_ode


def test_exponential_weakening_limits():
    # Sec. 6.2: rupture starts when the traction reaches T_th; after slip >> Dc the traction
    # of slipping elements settles at T_dy.
    N, M, dt = 120, 160, 0.5
    el = kn.element_table(inputs.straight_fault(N))
    K = kn.discrete_kernel(el, dt, M, 1.0, 1.0)
    tau0 = np.full(N, 0.5)
    tau0[55:65] = 0.7
    D, T = dense.rupture_march(K, tau0, 1.0, 0.6, 0.3, 0.5, dt, M, law="exponential")
    assert np.all(D[0, :55] == 0.0) and np.all(D[0, 55:65] > 0.0)
    assert np.all(T[D == 0.0] <= 0.6 + 1e-12)
    slip = D.sum(0) * dt
    deep = slip > 20 * 0.5
    assert deep.sum() > 10
    assert np.abs(T[-1, deep] - 0.3).max() < 1e-6


def test_rupture_respects_locking_and_no_back_slip():
    N, M, dt = 120, 90, 0.5
    el = kn.element_table(inputs.kinked_fault(N))
    K = kn.discrete_kernel(el, dt, M, 1.0, 1.0)
    tau0 = np.full(N, 0.45)
    tau0[55:65] = 0.61                          # overstressed nucleation patch
    D, T = dense.rupture_march(K, tau0, 1.0, 0.6, 0.3, 2.0, dt, M)
    assert np.all(D >= 0.0)
    assert np.all(D[0, :55] == 0.0) and np.all(D[0, 55:65] > 0.0)
    slipping = D > 0.0
    strength_max = 0.6
    assert np.all(T[~slipping] <= strength_max + 1e-12)    # locked cells stay below strength
