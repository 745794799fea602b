"""Pins of the oracle's discrete kernel (CPU only)."""
import json
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import kernel as kn
from paper_1903_02118_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _el(xy):
    return kn.element_table(xy)


@pytest.mark.parametrize("mu,cs", [(1.0, 1.0), (1.3, 0.5), (30.0, 4.0)])
def test_self_term_is_radiation_damping(mu, cs):
    # Sec. 6 normalisation: K_{i,i,0} = -mu / (2 cs) at CFL 1/2, eps_t = 1.
    dx = 2.0  # exact binary sizes: the CFL-1/2 arrival of the end-point waves is a knife edge
    dt = GOLD["cfl"]["value"] * dx / cs
    el = _el(inputs.straight_fault(9, dx))
    K = kn.discrete_kernel(el, dt, 3, mu, cs)
    want = GOLD["self_term_over_mu_over_cs"]["value"] * mu / cs
    assert np.allclose(np.diag(K[0]), want, rtol=0, atol=1e-15 * abs(want))


@pytest.mark.parametrize("geom", ["straight", "kinked", "curved"])
def test_instantaneous_term_is_local(geom):
    # At CFL 1/2 the nearest end point of any other element is at cs*dt: K_{ij,0} = 0 (j != i).
    xy = {"straight": inputs.straight_fault(40), "kinked": inputs.kinked_fault(40),
          "curved": inputs.curved_fault(40, 11)}[geom]
    el = _el(xy)
    K0 = kn.discrete_kernel(el, 0.5, 1, 1.0, 1.0)[0]
    off = K0 - np.diag(np.diag(K0))
    # the shared end point sits exactly on the causal front at t = dt; rounding of the
    # coordinates moves it by ~1e-16, which the square-root onset S ~ sqrt(2 r dr) turns
    # into ~1e-8 (chord lengths of the curved trace differ from dx by ~1e-14)
    assert np.abs(off).max() < 1e-7


def _screw_pair(px, py, ax, ay, bx, by, mu):
    """Textbook static field of a uniform slip segment = two opposite screw dislocations at the
    end points; a screw dislocation of Burgers vector b at the origin has
    sigma_xz = -mu b y / (2 pi r^2), sigma_yz = mu b x / (2 pi r^2)."""
    def disl(x0, y0):
        x = px - x0
        y = py - y0
        r2 = x * x + y * y
        return -mu * y / (2 * np.pi * r2), mu * x / (2 * np.pi * r2)
    # the slipped segment runs a -> b; with the left-normal convention the field is
    # (dislocation at b) - (dislocation at a)
    sb = disl(bx, by)
    sa = disl(ax, ay)
    return sb[0] - sa[0], sb[1] - sa[1]


def test_static_limit_matches_screw_dislocations():
    rng = np.random.default_rng(3)
    for _ in range(50):
        ax, ay = rng.uniform(-3, 3, 2)
        ang = rng.uniform(0, 2 * np.pi)
        ln = rng.uniform(0.5, 2.0)
        bx, by = ax + ln * np.cos(ang), ay + ln * np.sin(ang)
        px, py = rng.uniform(-6, 6, 2)
        el = _el(np.array([[ax, ay, bx, by]]))
        src = {k: el[k][0] for k in ("ax", "ay", "tx", "ty", "len")}
        want = _screw_pair(px, py, ax, ay, bx, by, 1.7)
        got = kn.stress_static(px, py, src, 1.7)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14)
        # and the dynamic kernel tends to it: [R(t+1) - R(t)] -> K_static at late t
        late = kn.stress_jump(px, py, src, 1e6, 1e6 + 1.0, 1.7, 1.3)
        assert np.allclose(late, want, rtol=1e-8, atol=1e-12)


def test_static_self_value():
    el = _el(inputs.straight_fault(5, 2.0))
    Ks = kn.static_kernel(el, 1.0)
    assert np.isclose(Ks[2, 2], -2.0 / (np.pi * 2.0), rtol=1e-14)


def test_causality():
    # K_{ij,m} = 0 while cs (m+1) dt <= distance from receiver to element (Sec. 2.2 causal cone)
    el = _el(inputs.curved_fault(60, 4))
    dt, cs = 0.5, 1.0
    M = 80
    K = kn.discrete_kernel(el, dt, M, 1.0, cs)
    # distance from midpoint i to segment j
    px, py = el["mx"][:, None], el["my"][:, None]
    ax, ay, bx, by = el["ax"][None], el["ay"][None], el["bx"][None], el["by"][None]
    ex, ey = bx - ax, by - ay
    u = np.clip(((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey), 0, 1)
    d = np.hypot(px - ax - u * ex, py - ay - u * ey)
    t_end = (np.arange(M) + 1.0) * dt
    dead = cs * t_end[:, None, None] <= d[None] - 1e-12
    assert dead.sum() > 1000
    assert np.all(K[dead] == 0.0)


def _w_quad(X, Y, ln, t, cs):
    """Displacement of unit-rate ramp slip on [0, ln] x {0}: w = Y/(2 pi cs) int S(r)/r^2 dxi
    (representation w = -mu int dxi d_Y B with B the ramp-convolved Green's function)."""
    def f(xi):
        r2 = (X - xi) ** 2 + Y * Y
        return np.sqrt(max(cs * cs * t * t - r2, 0.0)) / r2
    # break the integral at the causal-cone edges for the adaptive rule
    pts = []
    if cs * t > abs(Y):
        R = np.sqrt(cs * cs * t * t - Y * Y)
        pts = [p for p in (X - R, X, X + R) if 0 < p < ln]
    val, _ = integrate.quad(f, 0.0, ln, points=pts or None, epsabs=1e-14, epsrel=1e-13, limit=400)
    return Y / (2 * np.pi * cs) * val


def test_kernel_against_quadrature_and_finite_difference():
    # Independent route: quadrature of the displacement integral, then sigma = mu grad w by
    # central differences, compared with the closed form in the element's local frame.
    rng = np.random.default_rng(7)
    mu, cs, ln = 1.0, 1.0, 1.0
    el = _el(np.array([[0.0, 0.0, ln, 0.0]]))
    src = {k: el[k][0] for k in ("ax", "ay", "tx", "ty", "len")}
    h = 1e-4
    n_ok = 0
    for _ in range(30):
        X = rng.uniform(-2.0, 3.0)
        Y = rng.choice([-1, 1]) * rng.uniform(0.2, 2.0)
        r_min = np.hypot(max(0.0, max(-X, X - ln)), Y)
        t = r_min / cs + rng.uniform(0.05, 3.0)
        sX_fd = mu * (_w_quad(X + h, Y, ln, t, cs) - _w_quad(X - h, Y, ln, t, cs)) / (2 * h)
        sY_fd = mu * (_w_quad(X, Y + h, ln, t, cs) - _w_quad(X, Y - h, ln, t, cs)) / (2 * h)
        sxz, syz = kn.stress_ramp(X, Y, src, t, mu, cs)   # local frame = global here
        assert abs(sxz - sX_fd) < 2e-6 * (1 + abs(sX_fd)), (X, Y, t, sxz, sX_fd)
        assert abs(syz - sY_fd) < 2e-6 * (1 + abs(sY_fd)), (X, Y, t, syz, sY_fd)
        n_ok += 1
    assert n_ok == 30


def test_representation_gives_unit_slip_jump():
    # The displacement jump across the element equals the slip (t for unit slip rate) well
    # inside the causal cone (Sec. 2.1.1 definition of Delta u).
    t, cs, ln = 5.0, 1.0, 40.0
    up = _w_quad(20.0, 1e-4, ln, t, cs)
    dn = _w_quad(20.0, -1e-4, ln, t, cs)
    assert abs((up - dn) - t) < 1e-3


def test_translation_invariance_and_reciprocity_on_straight_fault():
    el = _el(inputs.straight_fault(24))
    K = kn.discrete_kernel(el, 0.5, 60, 1.0, 1.0)
    for d in range(-5, 6):
        diag = np.array([K[:, i, i - d] for i in range(max(d, 0), min(24, 24 + d))])
        assert np.abs(diag - diag[0]).max() < 1e-14
    assert np.abs(K - K.transpose(0, 2, 1)).max() < 1e-14


def test_tail_form_equals_difference():
    el = _el(inputs.curved_fault(30, 2))
    K = kn.discrete_kernel(el, 0.5, 300, 1.0, 1.0)
    Ks = kn.static_kernel(el, 1.0)
    T = kn.tail_kernel(el, 0.5, 300, 1.0, 1.0)
    assert np.abs(T - (K - 0.5 * Ks[None])).max() < 1e-13
