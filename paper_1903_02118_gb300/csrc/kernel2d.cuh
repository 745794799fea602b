// kernel2d.cuh -- discrete 2-D antiplane (SH) kernel of the ST-BIEM, host + device.
//
// Piecewise-constant slip rate over a straight element (Sec. 2.1.2) switched on at t = 0
// produces, at a receiver point, the shear-stress vector (s_xz, s_yz).  In the element's
// frame (origin at its first end point, X along it, Y along its left normal), with
// e0 = -X, e1 = len - X, q_e = e_e^2 + Y^2 and W_e(t) = sqrt(max(c^2 t^2 - q_e, 0)):
//
//   s_Y(t) = -mu/(2 pi c) [ Theta(t) + e1 W_1 / q_1 - e0 W_0 / q_0 ]
//   s_X(t) = -mu/(2 pi c) [ Y W_1 / q_1 - Y W_0 / q_0 ]
//   Theta(t) = asin(clamp(e1 / rho)) - asin(clamp(e0 / rho)),  rho = sqrt(c^2 t^2 - Y^2),
//              Theta = 0 while c t <= |Y|
//
// (2-D SH Green's function c/(2 pi mu) H(ct - r)/sqrt(c^2 t^2 - r^2) integrated over the
// element and twice in time; the paper cites this kernel without printing it).  The
// discrete kernel of Eq. 4 with eps_t = 1 is the jump of this ramp response between
// m dt and (m + 1) dt.  Jumps are taken in differenced form
//   W(t2) - W(t1) = c^2 (t2 - t1)(t2 + t1) / (W(t2) + W(t1))
// so that late-time coefficients do not lose digits; the static kernel per unit slip is
// the t -> infinity limit of the ramp slope.
#pragma once
#include <math.h>

#ifdef __CUDACC__
#define FDPH_HD __host__ __device__ __forceinline__
#else
#define FDPH_HD inline
#endif

namespace fdph {

struct Seg {          // source element: first end point, unit tangent, length
    double ax, ay, tx, ty, len;
};

struct Stress2 {      // global shear-stress vector (s_xz, s_yz)
    double x, y;
};

struct LocalPt {
    double Y, e0, e1, q0, q1;
};

FDPH_HD LocalPt seg_local(double px, double py, const Seg& s) {
    const double dx = px - s.ax;
    const double dy = py - s.ay;
    const double X = dx * s.tx + dy * s.ty;
    LocalPt p;
    p.Y = dy * s.tx - dx * s.ty;
    p.e0 = -X;
    p.e1 = s.len - X;
    p.q0 = p.e0 * p.e0 + p.Y * p.Y;
    p.q1 = p.e1 * p.e1 + p.Y * p.Y;
    return p;
}

FDPH_HD double ramp_W(double ct, double q) {
    const double v = ct * ct - q;
    return v > 0.0 ? sqrt(v) : 0.0;
}

FDPH_HD double clamp1(double v) { return v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v); }

FDPH_HD double theta(double ct, const LocalPt& p) {
    if (!(ct > fabs(p.Y))) return 0.0;
    const double rho = sqrt(ct * ct - p.Y * p.Y);
    return asin(clamp1(p.e1 / rho)) - asin(clamp1(p.e0 / rho));
}

// W(t2) - W(t1), t2 >= t1 >= 0
FDPH_HD double dW(double t1, double t2, double c, double q) {
    const double w1 = ramp_W(c * t1, q);
    const double w2 = ramp_W(c * t2, q);
    if (w1 > 0.0) return c * c * (t2 - t1) * (t2 + t1) / (w2 + w1);
    return w2;
}

// W(t2) - W(t1) - c (t2 - t1), using c t - W = q / (c t + W)
FDPH_HD double dW_minus_static(double t1, double t2, double c, double q) {
    const double w1 = ramp_W(c * t1, q);
    const double w2 = ramp_W(c * t2, q);
    if (w1 > 0.0) {
        const double g = q / (c * t2 + w2) + q / (c * t1 + w1);
        return c * (t2 - t1) * g / (w2 + w1);
    }
    return w2 - c * (t2 - t1);
}

FDPH_HD Stress2 to_global(double sX, double sY, const Seg& s) {
    // stress vector = sX * tangent + sY * normal, normal = (-ty, tx)
    Stress2 r;
    r.x = sX * s.tx - sY * s.ty;
    r.y = sX * s.ty + sY * s.tx;
    return r;
}

// Ramp-response jump R(t2) - R(t1) of the stress vector at (px, py).
FDPH_HD Stress2 stress_jump(double px, double py, const Seg& s, double t1, double t2, double mu,
                            double c) {
    const LocalPt p = seg_local(px, py, s);
    const double dth = theta(c * t2, p) - theta(c * t1, p);
    const double d0 = dW(t1, t2, c, p.q0);
    const double d1 = dW(t1, t2, c, p.q1);
    const double k = -mu / (2.0 * M_PI * c);
    const double sY = k * (dth + p.e1 * d1 / p.q1 - p.e0 * d0 / p.q0);
    const double sX = k * (p.Y * d1 / p.q1 - p.Y * d0 / p.q0);
    return to_global(sX, sY, s);
}

// [R(t2) - R(t1)] - (t2 - t1) * static stress, without cancellation.
FDPH_HD Stress2 stress_tail(double px, double py, const Seg& s, double t1, double t2, double mu,
                            double c) {
    const LocalPt p = seg_local(px, py, s);
    const double dth = theta(c * t2, p) - theta(c * t1, p);
    const double d0 = dW_minus_static(t1, t2, c, p.q0);
    const double d1 = dW_minus_static(t1, t2, c, p.q1);
    const double k = -mu / (2.0 * M_PI * c);
    const double sY = k * (dth + p.e1 * d1 / p.q1 - p.e0 * d0 / p.q0);
    const double sX = k * (p.Y * d1 / p.q1 - p.Y * d0 / p.q0);
    return to_global(sX, sY, s);
}

// Upper bound on |s_X| + |s_Y| of stress_tail(t1, t1 + dt) -- hence on either global component and
// on any unit projection of it -- once both end points' fronts have passed (c t1 > sqrt(q_e)); +inf
// before.  From the closed form: |d Theta / dt| = c^2 t / (c^2 t^2 - Y^2) sum_e |e| / W_e(t), and
// 0 <= dW_minus_static(t1, t1 + dt) <= dt q / (t1 W(t1)); every factor falls with t, so the bound
// falls with t1 (a threshold scan can stop where it drops below the threshold).
FDPH_HD double stress_tail_bound(double px, double py, const Seg& s, double t1, double dt, double mu, double c) {
    const LocalPt p = seg_local(px, py, s);
    const double ct = c * t1;
    const double qm = p.q0 > p.q1 ? p.q0 : p.q1;
    if (!(t1 > 0.0) || !(ct * ct > qm)) return INFINITY;
    const double w0 = sqrt(ct * ct - p.q0), w1 = sqrt(ct * ct - p.q1);
    const double dth = dt * c * ct / (ct * ct - p.Y * p.Y) * (fabs(p.e0) / w0 + fabs(p.e1) / w1);
    const double a0 = dt / (t1 * w0), a1 = dt / (t1 * w1);
    const double k = mu / (2.0 * M_PI * c);
    return k * (dth + fabs(p.e1) * a1 + fabs(p.e0) * a0 + fabs(p.Y) * (a0 + a1));
}

// Static stress vector per unit slip (screw-dislocation pair at the end points).
FDPH_HD Stress2 stress_static(double px, double py, const Seg& s, double mu) {
    const LocalPt p = seg_local(px, py, s);
    const double k = -mu / (2.0 * M_PI);
    const double sY = k * (p.e1 / p.q1 - p.e0 / p.q0);
    const double sX = k * (p.Y / p.q1 - p.Y / p.q0);
    return to_global(sX, sY, s);
}

}  // namespace fdph
