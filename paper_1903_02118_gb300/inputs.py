"""Seeded synthetic inputs shaped like the paper's 2-D antiplane workloads.

This module holds no arithmetic of the method: it only draws fault geometries
and slip-rate histories.  It is shared by the tests, the benchmark and the
oracle (the only module both sides may use).

Seeds: a workload with index k uses ``1903021180 + k``; sub-streams add +0
(geometry), +1000 (slip history), +2000 (friction heterogeneity) and +3000
(request arrivals).
"""
import math

import numpy as np

SEED_BASE = 1903021180
GEOMETRY, SLIP, FRICTION, ARRIVALS = 0, 1000, 2000, 3000


def seed_for(k, stream):
    return SEED_BASE + k + stream


def straight_fault(n, dx=1.0):
    """n elements [j dx, (j+1) dx] on the x axis: rows (x0, y0, x1, y1)."""
    x = np.arange(n + 1, dtype=np.float64) * dx
    xy = np.zeros((n, 4))
    xy[:, 0] = x[:-1]
    xy[:, 2] = x[1:]
    return xy


def kinked_fault(n, frac=0.625, angle=np.pi / 4, dx=1.0):
    """Planar fault kinked by `angle` after a fraction `frac` of its elements."""
    nk = int(round(frac * n))
    pts = [np.array([0.0, 0.0])]
    for j in range(n):
        a = 0.0 if j < nk else angle
        pts.append(pts[-1] + dx * np.array([np.cos(a), np.sin(a)]))
    pts = np.array(pts)
    return np.concatenate([pts[:-1], pts[1:]], axis=1)


def curved_fault(n, seed, max_slope=0.2, kappa_max=0.1, modes=8, dx=1.0):
    """Random Fourier curve y(x) = s * sum_k a_k sin(2 pi k x / L + phi_k), a_k ~ N(0,1)/k^2,
    L = n dx, scaled so that max |y'| = max_slope (a gently curved, single-valued
    fault trace) and then, if needed, further so that max |curvature| <= kappa_max / dx;
    cut into n chords of length dx by arc-length marching."""
    rng = np.random.default_rng(seed)
    L = n * dx
    a = rng.standard_normal(modes) / np.arange(1, modes + 1) ** 2
    ph = rng.uniform(0.0, 2.0 * np.pi, modes)
    k = np.arange(1, modes + 1)
    w = 2.0 * np.pi * k / L

    xs = np.linspace(0.0, 1.2 * L, 20001)
    y1 = np.sum(a * w * np.cos(w * xs[:, None] + ph), axis=1)
    y2 = np.sum(-a * w * w * np.sin(w * xs[:, None] + ph), axis=1)
    s = max_slope / np.abs(y1).max()
    curv = np.abs(s * y2) / (1.0 + (s * y1) ** 2) ** 1.5
    if curv.max() > kappa_max / dx:
        s *= (kappa_max / dx) / curv.max()
    # chord marching: each chord end solves (x - x0)^2 + (y(x) - y0)^2 = dx^2, by Newton's method in
    # scalar arithmetic from the tangent estimate (the slope is at most max_slope: a simple root)
    a_l, w_l, ph_l = [float(v) for v in a], [float(v) for v in w], [float(v) for v in ph]

    def ys(x):
        v = d = 0.0
        for ak, wk, pk in zip(a_l, w_l, ph_l):
            v += ak * math.sin(wk * x + pk)
            d += ak * wk * math.cos(wk * x + pk)
        return s * v, s * d

    x0, y0 = 0.0, ys(0.0)[0]
    pts = [(x0, y0)]
    for _ in range(n):
        x = x0 + dx / math.sqrt(1.0 + ys(x0)[1] ** 2)
        for _ in range(50):
            yv, dv = ys(x)
            step = ((x - x0) ** 2 + (yv - y0) ** 2 - dx * dx) / (2.0 * (x - x0) + 2.0 * (yv - y0) * dv)
            x -= step
            if abs(step) <= 1e-15 * (1.0 + abs(x)):
                break
        x0, y0 = x, ys(x)[0]
        pts.append((x0, y0))
    pts = np.array(pts)
    return np.concatenate([pts[:-1], pts[1:]], axis=1)


def gaussian_filtered_history(n, m, seed, sigma_x=4.0, sigma_t=4.0):
    """Slip rate D[step, element]: N(0,1) smoothed by a Gaussian of sigma_x cells
    and sigma_t steps (zero before t = 0 by construction of the march)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((m, n))
    return gaussian_filter(raw, sigma=(sigma_t, sigma_x), mode="constant")


def gaussian_pulse(n, m, dt, seed, width=16.0, duration_steps=8.0, nrhs=1):
    """D[step, element] = exp(-(s - s0)^2 / (2 width^2) - (t - t0)^2 / (2 (duration dt)^2)),
    s = element index (arc length in dx), t = (step + 1/2) dt; s0 ~ U[n/4, 3n/4],
    t0 ~ U[64 dt, 512 dt].  With nrhs > 1 returns [nrhs, m, n]."""
    rng = np.random.default_rng(seed)
    out = []
    s = np.arange(n, dtype=np.float64)
    t = (np.arange(m, dtype=np.float64) + 0.5) * dt
    for _ in range(nrhs):
        s0 = rng.uniform(0.25 * n, 0.75 * n)
        t0 = rng.uniform(64.0 * dt, min(512.0, max(64.0, 0.5 * m)) * dt)
        out.append(np.exp(-((s[None, :] - s0) ** 2) / (2.0 * width * width)
                          - ((t[:, None] - t0) ** 2) / (2.0 * (duration_steps * dt) ** 2)))
    return out[0] if nrhs == 1 else np.stack(out)
