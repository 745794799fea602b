"""Oracle: the FDP=H plan and its compressed operator, evaluated by brute force.
TEST INFRASTRUCTURE ONLY.

The plan follows the paper's steps in its order:

1. Clustering (Sec. 2.3, Sec. 4.2.2): the root box is the axis-aligned bounding
   box of the element midpoints; a box is bisected at the middle of its
   longest side (x on ties), boxes are never re-tightened, so every box of one
   level has the same shape; an element belongs to the child holding its
   midpoint (a midpoint on the cut goes to the upper child); empty children
   are dropped.
2. Block-cluster tree (Sec. 2.3, Sec. 4.2.2): diam = largest box diagonal +
   largest element length in the two clusters, rbar = distance between the
   box centres, dist = rbar - diam.  Admissible leaf if diam < eta * dist
   (Eq. 8, tested first); inadmissible leaf if both clusters hold at most
   `leaf` elements or diam < l_min (Eq. 9); otherwise both clusters are
   bisected (4 children).
3. ART integers per admissible leaf with i*, j* = box centres (Sec. 4.2.2):
   dm_i = floor((r_{i j*} - rbar) / (c dt))                       (Eq. 30)
   mbar_j = floor((r_{i* j} - len_j / 2) / (c dt))                (App. C.3)
   Dm_j = ceil((r_{i* j} + len_j / 2) / (c dt)) - mbar_j + n_c    (App. C.3, App. H)
   discretised causality min(dm_i + mbar_j) >= 1 is checked  (Sec. 5.2).
4. Domain F, per global stress component c in {xz, yz} (App. C.2): amplitude
   Khat^F_ij = integral of the kernel over the leaf's discrete Domain-F window
   [a_ij, a_ij + Dm_j) steps, a_ij = dm_i + mbar_j (Eq. 28), projected on the
   receiver normal; waveform h_{j,m} = K_{i* j, mbar_j + m} / Khat^F_{i* j}
   (Eq. 29, receiver at the virtual point i*); low-rank approximation of the
   amplitude block (Eq. 13).
5. Domain S from a_ij + Dm_j on: the static kernel Khat^S (App. B.1 with the
   App. C.3 choice that cancels its second term), low-rank approximated.
6. 2-D Domain-S transient (App. B.3, App. H): temporal rank-2 form
   K ~ Khat^S + Khat^tr h^tr with the temporal pivot at the start of Domain S.
7. Inadmissible leaves (App. E): exact kernel up to the Domain-S start m_S,
   then the static kernel.

LRA (Sec. 2.3 criterion |K - K_LRA|_F < eps |K|_F): truncated SVD with the
minimal rank meeting the criterion; the block is kept exact when
rank * (N_r + N_s) >= N_r * N_s (the "original rank" fallback of Sec. 6.2).

Readings where the paper is silent or garbled:
* eps_t = 1; leaf size bounds the inadmissible clusters; l_min = 0 by default.
* Khat^F_ij is integrated over the ART-shifted discrete window of the pair (amp_window 0), so
  that amplitude, waveform and the static part that follows add up to the kernel's impulse;
  amp_window 1 takes Eq. 28 as written, the pair's own continuous Domain F
  (t-_ij, t+_ij) = mbar_j dt + (r_ij - r_{i* j}) / c + (0, Dm_j dt): the App. C.3 window of i*
  moved by the pair's travel-time difference (smooth in i, j; the placed window is not), and the
  transient below then takes its temporal pivot at the end of that window, t+_ij, instead of kS dt.
* Near a nodal direction the waveform of one stress component is ill
  conditioned (its amplitude at i* is nearly zero).  A component whose
  amplitude at i* is below 0.2 of the stress-vector impulse |Khat^F_{i* j}|
  uses instead the waveform of the stress vector projected on its impulse
  direction, h = (Khat . K(t)) / |Khat|^2.
* Transient: spatial pivot (p, q) = argmax |K_{p q, a+Dm} - Khat^S_pq dt| of the
  leaf (cross-approximation pivot), h^tr_m = that fibre normalised at m = 0,
  Khat^tr_ij = K_{ij, a_ij + Dm_j} - Khat^S_ij dt;  Dm_tr = 1 + last m < M with
  |fibre(m)| >= eps_st * mu / (2 cs) (0 if none).
* eps_q > 0: the transient's Dm_tr exact taps are replaced by their App. A staircase
  (oracle/quantization.py partition rule, applied to the normalised fibre); the operator then holds
  the staircase values, which the product evaluates by running window sums.
* m_S(i, j) = 1 + last k < M with |K_{ij,k} - K^stat_ij dt| >= eps_st * mu/(2 cs)
  (0 if none);  eps_st = 0 keeps the whole kernel (the plain ST-BIEM).
* Geometry arithmetic is FP64 with distances sqrt(dx*dx + dy*dy), no fused
  multiply-add, so that every integer and every tree decision is reproducible
  bit for bit by an independent implementation.

Parity: pinned by tests/test_oracle_fdph.py (cover of the index square by the
leaves, admissibility inequalities, causality, Eq. 24 effective wave-speed
bound, exact ART on a straight line, sum rules of the waveform and amplitude,
LRA criterion and minimality, closeness of the compressed operator to the
plain kernel, and FDP=H vs plain march error at the level the paper reports).
"""
import math

import numpy as np

from . import kernel as kn
from . import quantization as qz


NODAL_TAU = 0.2   # nodal-direction threshold of the waveform choice (reading, see header)


class Params:
    def __init__(self, eta=0.5, leaf=32, eps=1e-4, eps_st=1e-6, extra_steps=-1, lmin=0.0,
                 mu=1.0, cs=1.0, dt=0.5, M=256, soe_terms=0, eps_tr=None, art_interp=False, eta_scheme=0,
                 amp_window=0, transient=True, eps_q=0.0):
        self.eta, self.leaf, self.eps, self.eps_st = eta, leaf, eps, eps_st
        self.extra_steps, self.lmin, self.mu, self.cs, self.dt, self.M = extra_steps, lmin, mu, cs, dt, M
        self.soe_terms = soe_terms
        self.eps_tr = eps_st if eps_tr is None else eps_tr
        self.art_interp = art_interp
        self.eta_scheme = eta_scheme   # 0: constant eta (Eq. 8); 1: constant eta^2 dist (Eq. 25), needs lmin > 0
        # Domain-F amplitude window: 0 the pair's placed discrete window [a, a + Dm); 1 the pair's
        # own continuous Domain F of Eq. 28 (see the header)
        self.amp_window = amp_window
        self.transient = transient     # False drops the 2-D Domain-S transient (App. A.3 study)
        # eps_Q > 0: the transient's exact taps are quantized (App. A; App. B.3 applies it there)
        self.eps_q = eps_q


def soe_min_len(W):
    """The exponential tail is fitted only over at least max(512, 2 W) steps: shorter ranges
    make the basis nearly singular, and there the exact kernel is cheap to keep anyway."""
    return max(512, 2 * W)


def soe_rates(M, Q):
    """Decay rates of the exponential tail basis: Q rates spaced geometrically in [0.5/M, 1]."""
    return np.exp(np.log(0.5 / M) + np.arange(Q) / (Q - 1.0) * (np.log(1.0) - np.log(0.5 / M)))


def default_extra_steps(el, p):
    """n_c for an additional Domain-F width of 10 max-element-lengths / c (Sec. 6.3, App. H)."""
    return int(math.ceil(10.0 * float(el["len"].max()) / (p.cs * p.dt) - 1e-9))


def _dist(ax, ay, bx, by):
    dx = ax - bx
    dy = ay - by
    return np.sqrt(dx * dx + dy * dy)


# ----------------------------------------------------------------------------- clustering

class Cluster:
    __slots__ = ("lo", "hi", "idx", "level", "_kids")

    def __init__(self, lo, hi, idx, level):
        self.lo, self.hi, self.idx, self.level, self._kids = lo, hi, idx, level, None

    def centre(self):
        return 0.5 * (self.lo[0] + self.hi[0]), 0.5 * (self.lo[1] + self.hi[1])

    def diag(self):
        w = self.hi[0] - self.lo[0]
        h = self.hi[1] - self.lo[1]
        return math.sqrt(w * w + h * h)

    def children(self, el):
        if self._kids is None:
            w = self.hi[0] - self.lo[0]
            h = self.hi[1] - self.lo[1]
            ax = 0 if w >= h else 1
            mid = 0.5 * (self.lo[ax] + self.hi[ax])
            c = (el["mx"] if ax == 0 else el["my"])[self.idx]
            up = c >= mid
            kids = []
            for sel, (lo, hi) in ((~up, (self.lo, list(self.hi))), (up, (list(self.lo), self.hi))):
                lo, hi = list(lo), list(hi)
                if sel is up:
                    lo[ax] = mid
                else:
                    hi[ax] = mid
                if sel.any():
                    kids.append(Cluster(tuple(lo), tuple(hi), self.idx[sel], self.level + 1))
            self._kids = kids
        return self._kids


def root_cluster(el):
    mx, my = el["mx"], el["my"]
    return Cluster((mx.min(), my.min()), (mx.max(), my.max()), np.arange(mx.shape[0]), 0)


def block_tree(el, p, maxdepth=64):
    """List of leaves: dicts with kind 'adm' / 'near', the two clusters and geometry."""
    if p.eta_scheme not in (0, 1) or (p.eta_scheme == 1 and not p.lmin > 0.0):
        raise ValueError("eta_scheme must be 0, or 1 with lmin > 0")
    root = root_cluster(el)
    lens = el["len"]
    leaves = []
    stack = [(root, root, 0)]
    while stack:
        tau, sig, depth = stack.pop()
        diag = max(tau.diag(), sig.diag())
        maxlen = max(lens[tau.idx].max(), lens[sig.idx].max())
        diam = diag + maxlen
        ct, cs_ = tau.centre(), sig.centre()
        rbar = math.sqrt((ct[0] - cs_[0]) * (ct[0] - cs_[0]) + (ct[1] - cs_[1]) * (ct[1] - cs_[1]))
        dist = rbar - diam
        if p.eta_scheme == 1:      # constant eta^2 dist scheme (Eq. 25)
            adm = p.eta > 0.0 and dist > 0.0 and diam < math.sqrt(p.eta * p.lmin * dist)
        else:                      # constant eta scheme (Eq. 8)
            adm = p.eta > 0.0 and diam < p.eta * dist
        if adm:
            leaves.append(dict(kind="adm", tau=tau, sig=sig, diam=diam, dist=dist, rbar=rbar))
        elif (tau.idx.size <= p.leaf and sig.idx.size <= p.leaf) or diam < p.lmin or depth >= maxdepth:
            leaves.append(dict(kind="near", tau=tau, sig=sig, diam=diam, dist=dist, rbar=rbar))
        else:
            kids = [(a, b) for a in tau.children(el) for b in sig.children(el)]
            for a, b in reversed(kids):
                stack.append((a, b, depth + 1))
    return leaves


# ----------------------------------------------------------------------------- LRA

def lra(A, eps):
    """Truncated SVD with minimal rank r: ||A - A_r||_F < eps ||A||_F.  Returns (A_r, r, exact)."""
    nr, ns = A.shape
    normA = np.linalg.norm(A)
    if normA == 0.0:
        return np.zeros_like(A), 0, False
    if eps <= 0.0:
        return A.copy(), min(nr, ns), True
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    tail = np.sqrt(np.cumsum((s * s)[::-1])[::-1])   # tail[r] = sqrt(sum_{l >= r} s_l^2)
    tail = np.append(tail, 0.0)
    r = int(np.argmax(tail < eps * normA))
    if r * (nr + ns) >= nr * ns:
        return A.copy(), min(nr, ns), True
    return (U[:, :r] * s[:r]) @ Vt[:r], r, False


# ----------------------------------------------------------------------------- plan

def _src(el, idx):
    return {k: el[k][idx] for k in ("ax", "ay", "tx", "ty", "len")}


def admissible_leaf(el, lf, p, nc, need_operator=True):
    """ART integers and compressed Domain F / S / transient data of one admissible leaf."""
    tau, sig = lf["tau"], lf["sig"]
    I, J = tau.idx, sig.idx
    istar, jstar = tau.centre(), sig.centre()
    rbar = lf["rbar"]
    cdt = p.cs * p.dt
    r_ijs = _dist(el["mx"][I], el["my"][I], jstar[0], jstar[1])
    r_isj = _dist(istar[0], istar[1], el["mx"][J], el["my"][J])
    half = 0.5 * el["len"][J]
    dm = np.floor((r_ijs - rbar) / cdt).astype(np.int64)
    phi = (r_ijs - rbar) / cdt - dm          # sub-step part of the receiver delay, in [0, 1)
    mbar = np.floor((r_isj - half) / cdt).astype(np.int64)
    Dm = (np.ceil((r_isj + half) / cdt).astype(np.int64) - mbar + nc)
    out = dict(I=I, J=J, dm=dm, mbar=mbar, Dm=Dm, phi=phi, causal=int((dm[:, None] + mbar[None, :]).min()))
    if not need_operator:
        return out
    mu, cs, dt = p.mu, p.cs, p.dt
    a = dm[:, None] + mbar[None, :]                     # Domain-F start of each pair
    kS = a + Dm[None, :]                                # Domain-S start of each pair
    srcJ = _src(el, J[None, :])
    PX = el["mx"][I][:, None]
    PY = el["my"][I][:, None]
    NX = el["nx"][I][:, None]
    NY = el["ny"][I][:, None]
    # --- Domain F amplitudes (per stress component) and waveforms at i*
    if p.amp_window == 1:
        # Eq. 28 as written: the integral over the pair's own Domain F (t-_ij, t+_ij), which is
        # the Domain F of the representative receiver i* (App. C.3: [mbar_j dt, (mbar_j + Dm_j) dt])
        # moved by the pair's travel-time difference (r_ij - r_{i* j}) / c
        r_ij = _dist(PX, PY, el["mx"][J][None, :], el["my"][J][None, :])
        t_lo = mbar[None, :] * dt + (r_ij - r_isj[None, :]) / cs
        t_hi = t_lo + Dm[None, :] * dt
        sxz, syz = kn.stress_jump(PX, PY, srcJ, np.maximum(t_lo, 0.0), t_hi, mu, cs)   # R = 0 before t = 0
        tS = t_hi                        # the pair's own Domain-S start: temporal pivot of the transient
    else:
        sxz, syz = kn.stress_jump(PX, PY, srcJ, a * dt, kS * dt, mu, cs)
        tS = kS * dt
    A = {"x": NX * sxz, "y": NY * syz}
    s1 = _src(el, J)
    hxz, hyz = kn.stress_jump(istar[0], istar[1], s1, mbar * dt, (mbar + Dm) * dt, mu, cs)
    amp = {"x": hxz, "y": hyz}
    Dmax = int(Dm.max())
    mm = np.arange(Dmax)[None, :]
    t1 = (mbar[:, None] + mm) * dt
    wxz, wyz = kn.stress_jump(istar[0], istar[1], _src(el, J[:, None]), t1, t1 + dt, mu, cs)
    live = mm < Dm[:, None]
    wav = {"x": np.where(live, wxz, 0.0), "y": np.where(live, wyz, 0.0)}
    h = {}
    # waveform of the stress vector at i* projected on its own impulse direction
    # (well conditioned: the denominator is |Khat|^2, not one component)
    nrm2 = amp["x"] * amp["x"] + amp["y"] * amp["y"]
    hproj = (amp["x"][:, None] * wav["x"] + amp["y"][:, None] * wav["y"]) / np.where(nrm2 > 0.0, nrm2, 1.0)[:, None]
    for c in ("x", "y"):
        own = np.abs(amp[c]) >= NODAL_TAU * np.sqrt(nrm2)
        own &= amp[c] != 0.0
        h[c] = np.where(own[:, None], wav[c] / np.where(own, amp[c], 1.0)[:, None], hproj)
    F = {}
    for c in ("x", "y"):
        Ar, r, ex = lra(A[c], p.eps)
        F[c] = dict(op=Ar, rank=r, exact=ex, h=h[c], raw=A[c])
    # --- Domain S static
    Ks = kn.static_kernel(el, mu, I, J)
    Sr, rS, exS = lra(Ks, p.eps)
    # --- Domain S transient (per stress component)
    thr = p.eps_tr * mu / (2.0 * cs)
    txz, tyz = kn.stress_tail(PX, PY, srcJ, tS, tS + dt, mu, cs)
    TR = {}
    for c, tc, Nc in (("x", txz, NX), ("y", tyz, NY)):
        flat = int(np.argmax(np.abs(tc)))
        pi, pj = divmod(flat, tc.shape[1])
        if tc[pi, pj] == 0.0:
            TR[c] = dict(op=np.zeros_like(tc), rank=0, exact=False, h=np.zeros(0), Dm=0, pivot=(pi, pj))
            continue
        t0 = float(tS[pi, pj])
        m = np.arange(p.M, dtype=np.float64)
        f1, f2 = kn.stress_tail(el["mx"][I[pi]], el["my"][I[pi]], _src(el, J[pj]),
                                t0 + m * dt, t0 + (m + 1.0) * dt, mu, cs)
        fib = f1 if c == "x" else f2
        big = np.nonzero(np.abs(fib) >= thr)[0]
        Dtr = 0 if big.size == 0 else int(big.max()) + 1
        Br, rT, exT = lra(Nc * tc, p.eps)
        h = fib[:Dtr] / fib[0]
        tail_fit = np.zeros(0)
        if p.soe_terms > 0:
            # extension (not the paper's): beyond the Dm_tr exact taps the normalised fibre is
            # carried by its least-squares fit on the exponential basis instead of being dropped
            Dtr = max(Dtr, 1)
            h = fib[:Dtr] / fib[0]
            if p.M - Dtr >= soe_min_len(Dtr):
                lam = soe_rates(p.M, p.soe_terms)
                B = np.exp(-lam[None, :] * np.arange(p.M - Dtr, dtype=np.float64)[:, None])
                coef, *_ = np.linalg.lstsq(B, fib[Dtr:] / fib[0], rcond=None)
                tail_fit = B @ coef
        if not p.transient:
            Br, rT, exT, h, Dtr, tail_fit = np.zeros_like(Br), 0, False, np.zeros(0), 0, np.zeros(0)
        qb = qh = None
        if p.eps_q > 0.0 and Dtr > 0:
            # App. A.1.1 on the normalised fibre: a staircase of constant values over ranges
            # [b_q, b_q+1) of the exact taps, evaluated by running window sums (Eq. A.4)
            qb, qh = qz.partitions(h, p.eps_q)
            h = qz.staircase(qb, qh, Dtr)
        TR[c] = dict(op=Br, rank=rT, exact=exT, h=h, Dm=Dtr, pivot=(pi, pj), tail=tail_fit, raw=Nc * tc, qb=qb, qh=qh)
    out.update(a=a, kS=kS, F=F, S=dict(op=Sr, rank=rS, exact=exS, raw=Ks), TR=TR)
    return out


def near_leaf(el, lf, p):
    """Exact kernel up to m_S(i, j), then the static kernel (App. E, App. H).

    With p.soe_terms = Q > 0 (an extension of this implementation, not the paper's): the exact
    kernel is kept for every pair of the leaf up to W = the leaf's longest wave passage (both end
    points' fronts + n_c steps), and beyond W the difference K - K_stat dt is represented by its
    least-squares fit on the exponentials exp(-lambda_q (k - W)), q < Q (soe_rates), instead of
    being dropped; m_S plays no part then.
    """
    I, J = lf["tau"].idx, lf["sig"].idx
    K = kn.discrete_kernel(el, p.dt, p.M, p.mu, p.cs, I, J)          # [M, nr, ns]
    Ks = kn.static_kernel(el, p.mu, I, J)
    tail = None
    if p.eps_st > 0.0 or p.soe_terms > 0:
        thr = p.eps_st * p.mu / (2.0 * p.cs)
        tail = kn.tail_kernel(el, p.dt, p.M, p.mu, p.cs, I, J)
        big = np.abs(tail) >= thr
        any_big = big.any(axis=0)
        last = p.M - 1 - np.argmax(big[::-1], axis=0)
        mS = np.where(any_big, last + 1, 0)
    else:
        mS = np.full((I.size, J.size), p.M, dtype=np.int64)
    out = dict(I=I, J=J, K=K, Ks=Ks, mS=mS)
    if p.soe_terms > 0:
        Q = p.soe_terms
        # the window covers the wave passage of every pair (both end points' fronts
        # plus the n_c extra steps of Domain F), since a fit on smooth exponentials cannot
        # represent a wavefront
        nc = default_extra_steps(el, p) if p.extra_steps < 0 else p.extra_steps
        far_end = np.maximum(_dist(el["mx"][I][:, None], el["my"][I][:, None], el["ax"][J][None, :], el["ay"][J][None, :]),
                             _dist(el["mx"][I][:, None], el["my"][I][:, None], el["bx"][J][None, :], el["by"][J][None, :]))
        passage = np.ceil(far_end / (p.cs * p.dt)).astype(np.int64) + nc
        W = int(passage.max())           # the fit takes over once the wave has passed (no m_S cut)
        if p.M - W < soe_min_len(W):     # too short a tail to fit well: keep the kernel exact
            W = p.M
        fit = np.zeros((p.M - W, I.size, J.size))
        if W < p.M:
            lam = soe_rates(p.M, Q)
            B = np.exp(-lam[None, :] * np.arange(p.M - W, dtype=np.float64)[:, None])   # [M-W, Q]
            Y = tail[W:].reshape(p.M - W, -1)
            coef, *_ = np.linalg.lstsq(B, Y, rcond=None)
            fit = (B @ coef).reshape(p.M - W, I.size, J.size)
        out.update(W=W, fit=fit)
    return out


def build_plan(el, p, receivers=None):
    """Plan restricted to the leaves whose receiver cluster meets `receivers` (all if None)."""
    nc = default_extra_steps(el, p) if p.extra_steps < 0 else p.extra_steps
    leaves = block_tree(el, p)
    sel = None if receivers is None else set(int(i) for i in receivers)
    adm, near = [], []
    for lf in leaves:
        if sel is not None and not sel.intersection(lf["tau"].idx.tolist()):
            continue
        if lf["kind"] == "adm":
            d = admissible_leaf(el, lf, p, nc)
            if d["causal"] < 1:
                raise ValueError("discretised causality violated (Sec. 5.2): min(dm + mbar) = %d" % d["causal"])
            adm.append(d)
        else:
            near.append(near_leaf(el, lf, p))
    return dict(nc=nc, leaves=leaves, adm=adm, near=near, p=p)


def operator_rows(el, plan, receivers):
    """Compressed operator Kc[k, r, j] (k < M) for the listed receivers, by brute force."""
    p = plan["p"]
    M, dt = p.M, p.dt
    N = el["len"].shape[0]
    receivers = np.asarray(receivers)
    pos = {int(i): r for r, i in enumerate(receivers)}
    Kc = np.zeros((M, receivers.size, N))
    k = np.arange(M)
    for d in plan["adm"]:
        rows = [(r_loc, pos[int(i)]) for r_loc, i in enumerate(d["I"]) if int(i) in pos]
        if not rows:
            continue
        for il, r in rows:
            for jl, j in enumerate(d["J"]):
                a = d["a"][il, jl]
                kS = d["kS"][il, jl]
                col = np.zeros(M)
                for c in ("x", "y"):
                    Fc = d["F"][c]
                    if Fc["rank"] > 0:
                        L = min(int(d["Dm"][jl]), max(M - a, 0))
                        col[a:a + L] += Fc["op"][il, jl] * Fc["h"][jl, :L]
                col[min(kS, M):] += d["S"]["op"][il, jl] * dt
                for c in ("x", "y"):
                    T = d["TR"][c]
                    if T["rank"] > 0 and T["Dm"] > 0:
                        L = min(T["Dm"], max(M - kS, 0))
                        col[kS:kS + L] += T["op"][il, jl] * T["h"][:L]
                        nt = T["tail"].size
                        if nt:
                            k1 = kS + T["Dm"]
                            L2 = min(nt, max(M - k1, 0))
                            col[k1:k1 + L2] += T["op"][il, jl] * T["tail"][:L2]
                if p.art_interp:
                    # extension (Sec. 4.3.1 suggests higher-order interpolation of the receiver
                    # delay): read the representative stress at the exact delay dm_i + phi_i by
                    # linear interpolation between the two neighbouring steps
                    ph = d["phi"][il]
                    col = (1.0 - ph) * col + ph * np.concatenate([[0.0], col[:-1]])
                Kc[:, r, j] += col
    for d in plan["near"]:
        for il, i in enumerate(d["I"]):
            if int(i) not in pos:
                continue
            r = pos[int(i)]
            for jl, j in enumerate(d["J"]):
                if "W" in d:     # exact window, then static + fitted exponential tail
                    W = d["W"]
                    Kc[:W, r, j] += d["K"][:W, il, jl]
                    Kc[W:, r, j] += d["Ks"][il, jl] * dt + d["fit"][:, il, jl]
                    continue
                mS = int(d["mS"][il, jl])
                Kc[:mS, r, j] += d["K"][:mS, il, jl]
                Kc[mS:, r, j] += d["Ks"][il, jl] * dt
    return Kc


def leaf_signature(el, plan):
    """Order-free, comparable description of the tree and integers (bit-exact checks)."""
    sig = []
    for lf in plan["leaves"]:
        sig.append((lf["kind"], tuple(sorted(lf["tau"].idx.tolist())), tuple(sorted(lf["sig"].idx.tolist()))))
    return sorted(sig)
