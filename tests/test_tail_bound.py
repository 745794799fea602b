"""The bound that shortens the plan's threshold scans (m_S of App. H for the near pairs, the
transient's taps of App. B.3): fdph_kernel_tail returns the Domain-S remainder of the discrete
kernel, K(t1, t1 + dt) - Kstat dt, and an upper bound on it that falls with t1.  A scan for the last
step whose remainder reaches a threshold may stop where the bound is below half the threshold only
if the bound really bounds the remainder and really falls; both are checked here against the
oracle's closed form (oracle/kernel.py), on CPU."""
import numpy as np
import pytest

from oracle import kernel as kn
from paper_1903_02118_gb300 import build, fdph


@pytest.fixture(scope="module")
def L():
    build.build()
    return fdph.lib()


def _pairs(count, seed):
    """Random source elements (length 0.5-1.5, any orientation) and receiver points at distances
    0.3-80 from the first end point; with each its S-front time for c = 1 (farther end point)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        length = rng.uniform(0.5, 1.5)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        seg = np.array([rng.uniform(-5, 5), rng.uniform(-5, 5), np.cos(ang), np.sin(ang), length])
        r = np.exp(rng.uniform(np.log(0.3), np.log(80.0)))
        th = rng.uniform(0.0, 2.0 * np.pi)
        p = seg[:2] + r * np.array([np.cos(th), np.sin(th)])
        bx, by = seg[0] + length * seg[2], seg[1] + length * seg[3]
        front = max(np.hypot(p[0] - seg[0], p[1] - seg[1]), np.hypot(p[0] - bx, p[1] - by))
        out.append((p, seg, front))
    return out


def test_remainder_equals_the_oracle(L):
    """The library's remainder is the oracle's closed form (relative to the remainder's size)."""
    for p, seg, front in _pairs(200, 1):
        src = {"ax": seg[0], "ay": seg[1], "tx": seg[2], "ty": seg[3], "len": seg[4]}
        for t1 in (0.25 * front, front + 0.3, front + 7.0, front + 2e3):
            x, y, _ = fdph.kernel_tail(p, seg, t1, 0.5)
            ox, oy = kn.stress_tail(p[0], p[1], src, t1, t1 + 0.5, 1.0, 1.0)
            scale = abs(ox) + abs(oy)
            assert abs(x - ox) <= 1e-9 * scale + 1e-300 and abs(y - oy) <= 1e-9 * scale + 1e-300


@pytest.mark.parametrize("dt,mu,cs", [(0.5, 1.0, 1.0), (0.25, 3.0, 2.0)])
def test_bound_bounds_and_falls(L, dt, mu, cs):
    """Once both fronts have passed, the bound is >= |x|, |y| and |n . (x, y)| for the oracle's
    remainder, and it does not rise from one step to the next; before the fronts it is +inf."""
    rng = np.random.default_rng(2)
    for p, seg, front in _pairs(150, 3):
        src = {"ax": seg[0], "ay": seg[1], "tx": seg[2], "ty": seg[3], "len": seg[4]}
        t_front = front / cs
        assert fdph.kernel_tail(p, seg, 0.999 * t_front, dt, mu, cs)[2] == np.inf
        ts = t_front + np.concatenate([[1e-4, 1e-2], np.arange(1, 400) * dt, [1e3, 1e4, 1e5]])
        prev = np.inf
        for t1 in ts:
            b = fdph.kernel_tail(p, seg, t1, dt, mu, cs)[2]
            ox, oy = kn.stress_tail(p[0], p[1], src, t1, t1 + dt, mu, cs)
            a = rng.uniform(0.0, 2.0 * np.pi)
            proj = abs(np.cos(a) * ox + np.sin(a) * oy)
            assert b >= max(abs(ox), abs(oy), proj), (p, seg, t1, b, ox, oy)
            assert b <= prev
            prev = b


def test_bounded_scan_finds_the_full_scans_step(L):
    """m_S = 1 + last k < M with |n . remainder_k| >= thr (App. H): the scan that starts below the
    first step whose bound is under thr / 2 gives the full scan's m_S, and at eps_st = 1e-4 it covers
    well under a quarter of M = 4000 steps."""
    M, dt = 4000, 0.5
    saved = []
    for p, seg, front in _pairs(40, 5):
        src = {"ax": seg[0], "ay": seg[1], "tx": seg[2], "ty": seg[3], "len": seg[4]}
        n = np.array([-seg[3], seg[2]])
        t = np.arange(M) * dt
        ox, oy = kn.stress_tail(p[0], p[1], src, t, t + dt, 1.0, 1.0)
        val = np.abs(n[0] * ox + n[1] * oy)
        for thr in (0.5e-4, 0.5e-6):
            above = np.nonzero(val >= thr)[0]
            full = int(above[-1]) + 1 if above.size else 0
            k_lo, k_hi = 0, M
            while k_lo < k_hi:
                mid = (k_lo + k_hi) // 2
                if fdph.kernel_tail(p, seg, mid * dt, dt)[2] < 0.5 * thr:
                    k_hi = mid
                else:
                    k_lo = mid + 1
            bounded = next((k + 1 for k in range(k_lo - 1, -1, -1) if val[k] >= thr), 0)
            assert bounded == full
            if thr > 1e-5:
                saved.append(k_lo / M)
    assert np.median(saved) < 0.25
