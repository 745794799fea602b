"""Oracle: discrete kernel of the 2-D antiplane (SH) ST-BIEM.  TEST INFRASTRUCTURE ONLY.

What it computes (Sec. 2.1.2 of the paper):

* slip rate piecewise constant in space over straight elements (the spatial
  basis of Sec. 2.1.2) and in time over steps of length dt (Eq. "D
  interpolation");
* traction collocated at element midpoints and at t_n = (n + eps_t) dt with
  eps_t = 1 (Sec. 4.3 supposes eps_t = 1);
* K_{i,j,m} = integral of the kernel over (t_{m-1}, t_m]  (Eq. 4), i.e. the
  jump of the ramp response R_ij between t = m dt and t = (m+1) dt.

The paper does not print the 2-D kernel (it cites Tada & Madariaga 2001).  The
closed form used here is derived from the 2-D SH Green's function
G = cs / (2 pi mu) * H(cs t - r) / sqrt(cs^2 t^2 - r^2) and the representation
w(x, t) = -mu * int_elem d(xi) int dtau  slip(xi, tau) d_Y G.  For unit slip rate
switched on at t = 0 on an element with local axes (X along the element from
its first end point P_a, Y along the left normal), receiver at local (X, Y):

    c_a = -X, c_b = len - X, r_e^2 = c_e^2 + Y^2, S_e = sqrt(max(cs^2 t^2 - r_e^2, 0))
    Phi = asin(clamp(c_b / R)) - asin(clamp(c_a / R)),  R = sqrt(cs^2 t^2 - Y^2)
          (Phi = 0 while cs t <= |Y|)
    sigma_Y = -mu / (2 pi cs) * (Phi + c_b S_b / r_b^2 - c_a S_a / r_a^2)
    sigma_X = -mu / (2 pi cs) * (Y S_b / r_b^2 - Y S_a / r_a^2)

(sigma_X, sigma_Y) are the shear-stress components (sigma_xz, sigma_yz) of the
local frame; they are rotated to the global frame, and the traction is the
projection on the receiver's left normal (App. C.2: the method works on the
stress components and projects afterwards).

Jumps R(t2) - R(t1) are evaluated in differenced form, using
S(t2) - S(t1) = cs^2 (t2^2 - t1^2) / (S(t2) + S(t1)), which is exact algebra but
avoids cancelling two O(t) numbers.  The static limit (t -> infinity, per unit
slip) is the textbook screw-dislocation pair at the element end points.

Parity: pinned by tests/test_oracle_kernel.py against (i) the radiation-damping
self term -mu/(2 cs) (Sec. 6 normalisation), (ii) the textbook static screw-
dislocation field, (iii) causality (zero outside the causal cone, Sec. 2.2),
(iv) an independent route: adaptive quadrature of the displacement integral
plus a finite difference, (v) translation invariance on a straight fault.
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def element_table(xy):
    """Element table from end points xy[:, (x0, y0, x1, y1)] (Sec. 2.1.2).

    Returns dict with midpoints (collocation points), lengths, unit tangents and
    left unit normals (normal = tangent rotated by +90 degrees).
    """
    xy = np.asarray(xy, dtype=np.float64)
    ax, ay, bx, by = xy[:, 0], xy[:, 1], xy[:, 2], xy[:, 3]
    ex = bx - ax
    ey = by - ay
    length = np.sqrt(ex * ex + ey * ey)
    tx = ex / length
    ty = ey / length
    return {
        "ax": ax, "ay": ay, "bx": bx, "by": by,
        "mx": 0.5 * (ax + bx), "my": 0.5 * (ay + by),
        "len": length, "tx": tx, "ty": ty, "nx": -ty, "ny": tx,
    }


def _local(px, py, ax, ay, tx, ty, length):
    """Receiver coordinates in the source element's local frame."""
    dx = px - ax
    dy = py - ay
    X = dx * tx + dy * ty
    Y = dx * (-ty) + dy * tx
    ca = -X
    cb = length - X
    ra2 = ca * ca + Y * Y
    rb2 = cb * cb + Y * Y
    return X, Y, ca, cb, ra2, rb2


def _S(ct, r2):
    return np.sqrt(np.maximum(ct * ct - r2, 0.0))


def _Phi(ct, Y, ca, cb):
    R2 = ct * ct - Y * Y
    live = ct > np.abs(Y)
    R = np.sqrt(np.where(live, R2, 1.0))
    phi = np.arcsin(np.clip(cb / R, -1.0, 1.0)) - np.arcsin(np.clip(ca / R, -1.0, 1.0))
    return np.where(live, phi, 0.0)


def _dS(t1, t2, cs, r2):
    """S(t2) - S(t1) for t2 >= t1 >= 0, in cancellation-free form."""
    S1 = _S(cs * t1, r2)
    S2 = _S(cs * t2, r2)
    both = S1 > 0.0
    den = np.where(both, S2 + S1, 1.0)
    return np.where(both, cs * cs * (t2 - t1) * (t2 + t1) / den, S2)


def _to_global(sX, sY, tx, ty):
    # stress vector (sigma_xz, sigma_yz) = sX * t + sY * n, n = (-ty, tx)
    return sX * tx - sY * ty, sX * ty + sY * tx


def stress_jump(px, py, src, t1, t2, mu, cs):
    """R(t2) - R(t1) of the two global stress components (sigma_xz, sigma_yz).

    px, py: receiver point(s); src: dict with keys ax, ay, tx, ty, len for the
    source element(s) (broadcastable); t1 <= t2, both >= 0.
    """
    X, Y, ca, cb, ra2, rb2 = _local(px, py, src["ax"], src["ay"], src["tx"], src["ty"], src["len"])
    dPhi = _Phi(cs * t2, Y, ca, cb) - _Phi(cs * t1, Y, ca, cb)
    dSa = _dS(t1, t2, cs, ra2)
    dSb = _dS(t1, t2, cs, rb2)
    pref = -mu / (TWO_PI * cs)
    sY = pref * (dPhi + cb * dSb / rb2 - ca * dSa / ra2)
    sX = pref * (Y * dSb / rb2 - Y * dSa / ra2)
    return _to_global(sX, sY, src["tx"], src["ty"])


def stress_ramp(px, py, src, t, mu, cs):
    """Ramp response R(t): stress (sigma_xz, sigma_yz) for unit slip rate from t = 0."""
    t = np.maximum(np.asarray(t, dtype=np.float64), 0.0)
    return stress_jump(px, py, src, np.zeros_like(t), t, mu, cs)


def stress_static(px, py, src, mu):
    """Static stress per unit slip (t -> infinity limit of R(t) / t)."""
    X, Y, ca, cb, ra2, rb2 = _local(px, py, src["ax"], src["ay"], src["tx"], src["ty"], src["len"])
    pref = -mu / TWO_PI
    sY = pref * (cb / rb2 - ca / ra2)
    sX = pref * (Y / rb2 - Y / ra2)
    return _to_global(sX, sY, src["tx"], src["ty"])


def stress_tail(px, py, src, t1, t2, mu, cs):
    """[R(t2) - R(t1)] - K_static * (t2 - t1), in cancellation-free form.

    Uses cs t - S = r^2 / (cs t + S) so that no O(t) terms are subtracted.
    """
    X, Y, ca, cb, ra2, rb2 = _local(px, py, src["ax"], src["ay"], src["tx"], src["ty"], src["len"])
    dPhi = _Phi(cs * t2, Y, ca, cb) - _Phi(cs * t1, Y, ca, cb)

    def dev(r2):
        # S(t2) - S(t1) - cs (t2 - t1)
        S1 = _S(cs * t1, r2)
        S2 = _S(cs * t2, r2)
        both = S1 > 0.0
        den = np.where(both, S2 + S1, 1.0)
        g = r2 / (cs * t2 + S2) + r2 / np.where(both, cs * t1 + S1, 1.0)
        late = cs * (t2 - t1) * g / den
        return np.where(both, late, S2 - cs * (t2 - t1))

    da = dev(ra2)
    db = dev(rb2)
    pref = -mu / (TWO_PI * cs)
    sY = pref * (dPhi + cb * db / rb2 - ca * da / ra2)
    sX = pref * (Y * db / rb2 - Y * da / ra2)
    return _to_global(sX, sY, src["tx"], src["ty"])


def _src(el, j):
    return {k: el[k][j] for k in ("ax", "ay", "tx", "ty", "len")}


def traction(el, i, sxz, syz):
    return el["nx"][i] * sxz + el["ny"][i] * syz


def discrete_kernel(el, dt, M, mu, cs, receivers=None, sources=None):
    """K[m, i, j] (traction) for m in [0, M), eps_t = 1 (Eq. 4).

    K_{i,j,m} = R_ij((m+1) dt) - R_ij(m dt).
    """
    n = el["len"].shape[0]
    ri = np.arange(n) if receivers is None else np.asarray(receivers)
    sj = np.arange(n) if sources is None else np.asarray(sources)
    I = ri[None, :, None]
    J = sj[None, None, :]
    m = np.arange(M, dtype=np.float64)[:, None, None]
    sxz, syz = stress_jump(el["mx"][I], el["my"][I], _src(el, J), m * dt, (m + 1.0) * dt, mu, cs)
    return traction(el, I, sxz, syz)


def static_kernel(el, mu, receivers=None, sources=None):
    """K^stat[i, j] traction per unit slip (the Domain-S kernel of Sec. 2.2)."""
    n = el["len"].shape[0]
    ri = np.arange(n) if receivers is None else np.asarray(receivers)
    sj = np.arange(n) if sources is None else np.asarray(sources)
    I = ri[:, None]
    J = sj[None, :]
    sxz, syz = stress_static(el["mx"][I], el["my"][I], _src(el, J), mu)
    return traction(el, I, sxz, syz)


def tail_kernel(el, dt, M, mu, cs, receivers=None, sources=None):
    """K[m, i, j] - K^stat[i, j] * dt, computed without cancellation."""
    n = el["len"].shape[0]
    ri = np.arange(n) if receivers is None else np.asarray(receivers)
    sj = np.arange(n) if sources is None else np.asarray(sources)
    I = ri[None, :, None]
    J = sj[None, None, :]
    m = np.arange(M, dtype=np.float64)[:, None, None]
    sxz, syz = stress_tail(el["mx"][I], el["my"][I], _src(el, J), m * dt, (m + 1.0) * dt, mu, cs)
    return traction(el, I, sxz, syz)
