// plan.cpp -- host construction of the FDP=H operator (Secs. 2.3, 4, App. B.1, B.3, C.3, E, H).
//
// For every admissible leaf (receivers i, sources j, representative points i*, j* = box centres):
//   a_ij = dm_i + mbar_j          start of the pair's discrete Domain F (Eq. 31)
//   kS_ij = a_ij + Dm_j           start of Domain S
//   Domain F, per global stress component c (App. C.2, stress first, traction afterwards):
//     amplitude  Khat^c_ij = R^c_ij(kS dt) - R^c_ij(a dt) over the placed window, or (amp_window 1)
//                R^c_ij(t+_ij) - R^c_ij(t-_ij) over the pair's own Domain F (Eq. 28),
//                t-_ij = mbar_j dt + (r_ij - r_i*j) / c, t+_ij = t-_ij + Dm_j dt; low-rank after
//                the projection n^c_i                            (Eq. 13)
//     waveform   h^c_{j,m} = K^c_{i* j, mbar_j + m} / Khat^c_{i* j}  (Eq. 29), or, when
//                component c is nearly nodal at i*, the waveform of the stress vector
//                projected on its impulse direction
//   Domain S: static traction kernel per unit slip, low-rank, applied as dt * slip from kS on
//             (App. B.1; the App. C.3 integers make its second term vanish)
//   transient (App. B.3, App. H): K - Khat^S dt ~ Khat^tr h^tr with the temporal pivot at the start
//             of the pair's Domain S (kS dt, or t+_ij with amp_window 1) and the spatial pivot at
//             the largest |entry| of the leaf; Dm_tr from eps_st
// Inadmissible leaves only get their geometry here; their exact-kernel windows are computed on
// the device (fdph.cu) because they need O(pairs * M) kernel evaluations.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>

#include "kernel2d.cuh"
#include "plan.h"

namespace fdph {

namespace {

const double kNodalTau = 0.2;

struct LeafOut {
    ArtInts art;
    int r0, nr, s0, ns;
    int HM = 0;
    LowRank F[2], S, TR[2];
    std::vector<double> h[2];      // [HM][ns]
    std::vector<double> htr[2];    // exact taps
    std::vector<double> trc[2];    // exponential-tail coefficients of the fibre (if any)
    std::vector<int32_t> qb[2];    // eps_q > 0: quantized ranges of the taps (bounds) ...
    std::vector<double> qh[2];     // ... and their values
    int Dtr[2] = {0, 0};
    int trsoe[2] = {0, 0};
    bool ok = true;
};

Seg seg_of(const Elements& el, int e) {
    Seg s;
    s.ax = el.ax[e];
    s.ay = el.ay[e];
    s.tx = el.tx[e];
    s.ty = el.ty[e];
    s.len = el.len[e];
    return s;
}

}  // namespace

// App. A.1.1 (the oracle's reading): from b_q the range grows while |K_m - K_b_q| / 2 <=
// eps_q |(K_b_q + K_m) / 2|; b_q+1 is the first m that breaks it; khat_q = (K_b_q + K_b_q+1 - 1) / 2.
void quantize_partitions(const double* K, int n, double eps_q, std::vector<int32_t>& b, std::vector<double>& khat) {
    b.assign(1, 0);
    khat.clear();
    int q0 = 0;
    while (q0 < n) {
        int m = q0 + 1;
        while (m < n) {
            const double kh = 0.5 * (K[q0] + K[m]);
            if (0.5 * fabs(K[m] - K[q0]) > eps_q * fabs(kh)) break;
            ++m;
        }
        khat.push_back(0.5 * (K[q0] + K[m - 1]));
        b.push_back(m);
        q0 = m;
    }
}

namespace {

void admissible(const Elements& el, const Tree& tr, const Leaf& lf, const PlanInputs& in, LeafOut& o) {
    const ClusterNode& tn = tr.nodes[lf.tau];
    const ClusterNode& sn = tr.nodes[lf.sig];
    o.r0 = tn.lo;
    o.nr = tn.hi - tn.lo;
    o.s0 = sn.lo;
    o.ns = sn.hi - sn.lo;
    o.art = art_integers(el, tr, lf, in);
    if (o.art.causal < 1) {
        o.ok = false;
        return;
    }
    const int nr = o.nr, ns = o.ns;
    const double dt = in.dt, mu = in.mu, c = in.cs;
    const double ist[2] = {0.5 * (tn.box.lo[0] + tn.box.hi[0]), 0.5 * (tn.box.lo[1] + tn.box.hi[1])};
    // the pair's Domain-F window (Eq. 28 or the placed one, reading 5) and Domain-S start
    auto window = [&](int il, int jl, double& t_lo, double& t_hi) {
        const long a = (long)o.art.dm[il] + o.art.mbar[jl];
        const long kS = a + o.art.Dm[jl];
        t_lo = (double)a * dt;
        t_hi = (double)kS * dt;
        if (in.amp_window == 1) {
            // Eq. 28: the pair's own Domain F, the window of i* moved by r_ij - r_{i* j}
            const int ei = tr.perm[o.r0 + il], ej = tr.perm[o.s0 + jl];
            const double dxi = el.mx[ei] - el.mx[ej], dyi = el.my[ei] - el.my[ej];
            const double dxs = ist[0] - el.mx[ej], dys = ist[1] - el.my[ej];
            t_lo = (double)o.art.mbar[jl] * dt + (sqrt(dxi * dxi + dyi * dyi) - sqrt(dxs * dxs + dys * dys)) / c;
            t_hi = t_lo + (double)o.art.Dm[jl] * dt;
            t_lo = t_lo > 0.0 ? t_lo : 0.0;   // the ramp response is zero before t = 0
        }
    };
    // kind 0, 1: Domain-F amplitude of the x / y stress component on the receiver normal; 2: static
    // traction kernel; 3, 4: the remainder K - Khat^S dt of the x / y component at the Domain-S start
    auto entry = [&](int kind, int il, int jl) -> double {
        const int ei = tr.perm[o.r0 + il], ej = tr.perm[o.s0 + jl];
        const double px = el.mx[ei], py = el.my[ei];
        const Seg sg = seg_of(el, ej);
        double t_lo, t_hi;
        window(il, jl, t_lo, t_hi);
        if (kind < 2) {
            const Stress2 amp = stress_jump(px, py, sg, t_lo, t_hi, mu, c);
            return kind == 0 ? el.nx[ei] * amp.x : el.ny[ei] * amp.y;
        }
        if (kind == 2) {
            const Stress2 st = stress_static(px, py, sg, mu);
            return el.nx[ei] * st.x + el.ny[ei] * st.y;
        }
        const Stress2 tl = stress_tail(px, py, sg, t_hi, t_hi + dt, mu, c);
        return kind == 3 ? tl.x : tl.y;   // the stress component; factor() projects it on n_i
    };
    // large blocks: cross approximation from rows and columns computed on demand (low_rank_aca),
    // the dense block only if it does not converge; small blocks: all five blocks formed in one pass
    const bool aca = (long long)nr * ns >= in.aca_min;
    std::vector<double> D[5];   // dense blocks of the five kinds (empty on the cross-approximation path)
    size_t best[2] = {0, 0};    // transient pivots: the largest |remainder| of each stress component
    double bval[2] = {0.0, 0.0}, bt0[2] = {0.0, 0.0};
    auto pivot = [&](int il, int jl, double tx, double ty, double t_hi) {
        const double v[2] = {tx, ty};
        for (int cc = 0; cc < 2; ++cc)
            if (fabs(v[cc]) > fabs(bval[cc]) || (il == 0 && jl == 0)) {
                best[cc] = (size_t)il * ns + jl;
                bval[cc] = v[cc];
                bt0[cc] = t_hi;
            }
    };
    if (!aca) {
        for (int k = 0; k < 5; ++k) D[k].resize((size_t)nr * ns);
        for (int il = 0; il < nr; ++il) {
            const int ei = tr.perm[o.r0 + il];
            const double px = el.mx[ei], py = el.my[ei], nx = el.nx[ei], ny = el.ny[ei];
            for (int jl = 0; jl < ns; ++jl) {
                const Seg sg = seg_of(el, tr.perm[o.s0 + jl]);
                double t_lo, t_hi;
                window(il, jl, t_lo, t_hi);
                const Stress2 amp = stress_jump(px, py, sg, t_lo, t_hi, mu, c);
                const Stress2 st = stress_static(px, py, sg, mu);
                const Stress2 tl = stress_tail(px, py, sg, t_hi, t_hi + dt, mu, c);
                const size_t q = (size_t)il * ns + jl;
                D[0][q] = nx * amp.x;
                D[1][q] = ny * amp.y;
                D[2][q] = nx * st.x + ny * st.y;
                D[3][q] = nx * tl.x;
                D[4][q] = ny * tl.y;
                pivot(il, jl, tl.x, tl.y, t_hi);
            }
        }
    } else {
        // the largest entry by alternating row / column maxima (the partial pivoting of ACA),
        // O(N_r + N_s) evaluations per search instead of N_r N_s
        auto tail = [&](int il, int jl, int cc, double& t_hi) {
            const int ei = tr.perm[o.r0 + il];
            double t_lo;
            window(il, jl, t_lo, t_hi);
            const Stress2 tl = stress_tail(el.mx[ei], el.my[ei], seg_of(el, tr.perm[o.s0 + jl]), t_hi, t_hi + dt,
                                           mu, c);
            return cc == 0 ? tl.x : tl.y;
        };
        for (int cc = 0; cc < 2; ++cc) {
            int pi = 0, pj = -1;
            for (int round = 0; round < 8; ++round) {
                int bj = 0;
                double bv = -1.0;
                for (int jl = 0; jl < ns; ++jl) {
                    double th;
                    const double v = fabs(tail(pi, jl, cc, th));
                    if (v > bv) bv = v, bj = jl;
                }
                int bi = 0;
                bv = -1.0;
                for (int il = 0; il < nr; ++il) {
                    double th;
                    const double v = fabs(tail(il, bj, cc, th));
                    if (v > bv) bv = v, bi = il;
                }
                const bool same = bi == pi && bj == pj;
                pi = bi;
                pj = bj;
                if (same) break;
            }
            double th;
            bval[cc] = tail(pi, pj, cc, th);
            bt0[cc] = th;
            best[cc] = (size_t)pi * ns + pj;
        }
    }
    auto factor = [&](int kind, LowRank& out) {
        if (!aca) {
            low_rank(D[kind].data(), nr, ns, in.eps, out);
            return;
        }
        auto val = [&](int il, int jl) {
            const int ei = tr.perm[o.r0 + il];
            const double v = entry(kind, il, jl);
            return kind == 3 ? el.nx[ei] * v : kind == 4 ? el.ny[ei] * v : v;
        };
        auto row = [&](int il, double* out_r) {
            for (int jl = 0; jl < ns; ++jl) out_r[jl] = val(il, jl);
        };
        auto col = [&](int jl, double* out_c) {
            for (int il = 0; il < nr; ++il) out_c[il] = val(il, jl);
        };
        if (low_rank_aca(row, col, nr, ns, in.eps, out)) return;
        std::vector<double> A((size_t)nr * ns);
        for (int il = 0; il < nr; ++il) row(il, A.data() + (size_t)il * ns);
        low_rank(A.data(), nr, ns, in.eps, out);
    };
    // waveforms at i*
    int HM = 0;
    for (int jl = 0; jl < ns; ++jl) HM = std::max(HM, o.art.Dm[jl]);
    o.HM = HM;
    o.h[0].assign((size_t)HM * ns, 0.0);
    o.h[1].assign((size_t)HM * ns, 0.0);
    std::vector<double> wx(HM), wy(HM);
    for (int jl = 0; jl < ns; ++jl) {
        const int ej = tr.perm[o.s0 + jl];
        const Seg s = seg_of(el, ej);
        const int mb = o.art.mbar[jl], D = o.art.Dm[jl];
        const Stress2 amp = stress_jump(ist[0], ist[1], s, (double)mb * dt, (double)(mb + D) * dt, mu, c);
        for (int m = 0; m < D; ++m) {
            const double t1 = (double)(mb + m) * dt;
            const Stress2 w = stress_jump(ist[0], ist[1], s, t1, t1 + dt, mu, c);
            wx[m] = w.x;
            wy[m] = w.y;
        }
        const double nrm2 = amp.x * amp.x + amp.y * amp.y;
        const double nrm = sqrt(nrm2);
        const double den = nrm2 > 0.0 ? nrm2 : 1.0;
        for (int cc = 0; cc < 2; ++cc) {
            const double ac = cc == 0 ? amp.x : amp.y;
            const bool own = fabs(ac) >= kNodalTau * nrm && ac != 0.0;
            for (int m = 0; m < D; ++m) {
                const double v = own ? (cc == 0 ? wx[m] : wy[m]) / ac : (amp.x * wx[m] + amp.y * wy[m]) / den;
                o.h[cc][(size_t)m * ns + jl] = v;
            }
        }
    }
    factor(0, o.F[0]);
    factor(1, o.F[1]);
    factor(2, o.S);
    // transient, per component
    const double thr = in.eps_st * mu / (2.0 * c);
    for (int cc = 0; cc < 2; ++cc) {
        if (bval[cc] == 0.0) continue;
        const int pi = (int)(best[cc] / ns), pj = (int)(best[cc] % ns);
        const int ei = tr.perm[o.r0 + pi], ej = tr.perm[o.s0 + pj];
        const Seg s = seg_of(el, ej);
        const double t0 = bt0[cc];   // kS dt, or the pivot pair's own Domain-S start (amp_window 1)
        std::vector<double> fib(in.M, 0.0);
        int last = -1;
        for (int m = 0; m < in.M; ++m) {
            // without the tail fit only the taps above thr matter: none follows once the falling
            // tail bound is below thr / 2 (the factor 2 covers rounding)
            if (in.soe == 0 && stress_tail_bound(el.mx[ei], el.my[ei], s, t0 + (double)m * dt, dt, mu, c) < 0.5 * thr)
                break;
            const Stress2 v = stress_tail(el.mx[ei], el.my[ei], s, t0 + (double)m * dt, t0 + (double)(m + 1) * dt,
                                          mu, c);
            fib[m] = cc == 0 ? v.x : v.y;
            if (fabs(fib[m]) >= thr) last = m;
        }
        int Dtr = last + 1;
        int nsoe = 0;
        std::vector<double> coef;
        if (in.soe > 0) {
            // extension: beyond the exact taps the normalised fibre is kept as its fit on the
            // exponential basis rather than dropped
            Dtr = std::max(Dtr, 1);
            const int len = in.M - Dtr;
            if (len >= soe_min_len(Dtr)) {
                const std::vector<double> rho = soe_rho(in.M, in.soe);
                std::vector<double> g(in.soe, 0.0), pw(in.soe, 1.0);
                for (int k = 0; k < len; ++k) {
                    const double y = fib[Dtr + k] / fib[0];
                    for (int q = 0; q < in.soe; ++q) {
                        g[q] += pw[q] * y;
                        pw[q] *= rho[q];
                    }
                }
                coef.resize(in.soe);
                soe_solve(rho, len, g.data(), coef.data(), 1);
                nsoe = in.soe;
            }
        }
        if (Dtr == 0) continue;
        factor(3 + cc, o.TR[cc]);   // the remainder projected on the receiver normal
        o.Dtr[cc] = Dtr;
        o.trsoe[cc] = nsoe;
        o.htr[cc].resize(Dtr);
        for (int m = 0; m < Dtr; ++m) o.htr[cc][m] = fib[m] / fib[0];
        o.trc[cc] = coef;
        if (in.eps_q > 0.0) quantize_partitions(o.htr[cc].data(), Dtr, in.eps_q, o.qb[cc], o.qh[cc]);
    }
}

template <class T>
int64_t append(std::vector<T>& dst, const T* src, size_t n) {
    const int64_t off = (int64_t)dst.size();
    dst.insert(dst.end(), src, src + n);
    return off;
}

}  // namespace

int build_host_plan(const Elements& el, const PlanInputs& in, HostPlan& hp) {
    build_host_tree(el, in, hp);
    return build_host_far(el, in, hp);
}

int check_causality(const Elements& el, const PlanInputs& in, const Tree& tr) {
    for (const Leaf& lf : tr.leaves)
        if (lf.kind == 1 && art_integers(el, tr, lf, in).causal < 1) {
            set_error("discretised causality min(dm_i + mbar_j) >= 1 violated by an admissible leaf "
                      "(Sec. 5.2, App. D): increase l_min / eta or reduce dt");
            return -3;
        }
    return 0;
}

void build_host_tree(const Elements& el, const PlanInputs& in, HostPlan& hp) {
    hp.n = el.n;
    hp.M = in.M;
    hp.dt = in.dt;
    hp.mu = in.mu;
    hp.cs = in.cs;
    build_tree(el, in, hp.tree);
    const Tree& tr = hp.tree;
    const int n = el.n;
    hp.perm.assign(tr.perm.begin(), tr.perm.end());
    auto fill = [&](std::vector<double>& v, const std::vector<double>& src) {
        v.resize(n);
        for (int p = 0; p < n; ++p) v[p] = src[tr.perm[p]];
    };
    fill(hp.px, el.mx); fill(hp.py, el.my); fill(hp.pnx, el.nx); fill(hp.pny, el.ny);
    fill(hp.sax, el.ax); fill(hp.say, el.ay); fill(hp.sbx, el.bx); fill(hp.sby, el.by);
    fill(hp.stx, el.tx); fill(hp.sty, el.ty);
    fill(hp.slen, el.len);

    std::vector<const Leaf*> adm;
    for (const Leaf& lf : tr.leaves) {
        if (lf.kind == 1) adm.push_back(&lf);
        else {
            const ClusterNode& tn = tr.nodes[lf.tau];
            const ClusterNode& sn = tr.nodes[lf.sig];
            hp.near_r0.push_back(tn.lo);
            hp.near_nr.push_back(tn.hi - tn.lo);
            hp.near_s0.push_back(sn.lo);
            hp.near_ns.push_back(sn.hi - sn.lo);
        }
    }
    hp.n_adm = (int)adm.size();
    hp.n_near = (int)hp.near_r0.size();
    hp.soe = in.soe;
    hp.interp = in.interp;
    if (in.soe > 0) hp.rho = soe_rho(in.M, in.soe);
}

int build_host_far(const Elements& el, const PlanInputs& in, HostPlan& hp) {
    const Tree& tr = hp.tree;
    const int n = el.n;
    std::vector<const Leaf*> adm;
    for (const Leaf& lf : tr.leaves)
        if (lf.kind == 1) adm.push_back(&lf);
    std::vector<LeafOut> outs(adm.size());
    // largest blocks first, so that no big factorisation starts last (results stay in leaf order)
    std::vector<long> order(adm.size());
    for (long a = 0; a < (long)adm.size(); ++a) order[a] = a;
    auto size_of = [&](long a) {
        const ClusterNode& t = tr.nodes[adm[a]->tau];
        const ClusterNode& g = tr.nodes[adm[a]->sig];
        return (long)(t.hi - t.lo) * (g.hi - g.lo);
    };
    std::stable_sort(order.begin(), order.end(), [&](long x, long y) { return size_of(x) > size_of(y); });
#pragma omp parallel for schedule(dynamic, 1) num_threads(in.threads)
    for (long q = 0; q < (long)adm.size(); ++q) admissible(el, tr, *adm[order[q]], in, outs[order[q]]);
    for (const LeafOut& o : outs)
        if (!o.ok) {
            set_error("discretised causality min(dm_i + mbar_j) >= 1 violated by an admissible leaf");
            return -3;
        }

    // ---- assemble sub-blocks
    std::vector<std::vector<std::pair<int, int>>> recv(n);   // receiver -> (sb, il)
    double rank_sum = 0;
    int rank_cnt = 0;
    for (const LeafOut& o : outs) {
        const int64_t dm_off = append(hp.ints, o.art.dm.data(), o.art.dm.size());
        const int64_t phi_off = in.interp ? append(hp.phis, o.art.phi.data(), o.art.phi.size()) : 0;
        const int ex = in.interp ? 1 : 0;   // one more (older) slot read per receiver
        std::vector<int32_t> dF(o.ns), dS(o.ns);
        for (int j = 0; j < o.ns; ++j) {
            dF[j] = o.art.mbar[j];
            dS[j] = o.art.mbar[j] + o.art.Dm[j];
        }
        const int64_t dF_off = append(hp.ints, dF.data(), dF.size());
        const int64_t dS_off = append(hp.ints, dS.data(), dS.size());
        const int mindm = *std::min_element(o.art.dm.begin(), o.art.dm.end());
        const int maxdm = *std::max_element(o.art.dm.begin(), o.art.dm.end());
        auto add = [&](int kind, const LowRank& lr, const std::vector<int32_t>& dl, int64_t dl_off,
                       const std::vector<double>* h, int taps, int soe, const std::vector<double>* trc,
                       const std::vector<int32_t>* qb = nullptr, const std::vector<double>* qh = nullptr) {
            if (lr.rank <= 0) return;
            SubBlock sb;
            memset(&sb, 0, sizeof(sb));
            sb.kind = kind;
            sb.rank = lr.rank;
            sb.r0 = o.r0; sb.nr = o.nr; sb.s0 = o.s0; sb.ns = o.ns;
            sb.maxdelay = *std::max_element(dl.begin(), dl.end());
            sb.mindelay = *std::min_element(dl.begin(), dl.end());
            sb.mindm = mindm;
            sb.maxdm = maxdm;
            sb.taps = taps;
            sb.f = append(hp.fac, lr.F.data(), lr.F.size());
            sb.g = append(hp.fac, lr.G.data(), lr.G.size());
            const bool quant = qh && !qh->empty();   // the taps' staircase values replace the taps
            if (kind == SB_F && h) {
                // Domain-F waveforms source-major, [j][taps]: a FIR task reads its taps contiguously
                std::vector<double> hj((size_t)o.ns * taps);
                for (int j = 0; j < o.ns; ++j)
                    for (int m = 0; m < taps; ++m) hj[(size_t)j * taps + m] = (*h)[(size_t)m * o.ns + j];
                sb.h = append(hp.fac, hj.data(), hj.size());
            } else {
                sb.h = quant ? append(hp.fac, qh->data(), qh->size()) : h ? append(hp.fac, h->data(), h->size()) : 0;
            }
            sb.qn = quant ? (int32_t)qh->size() : 0;
            sb.qb = quant ? append(hp.ints, qb->data(), qb->size()) : 0;
            sb.delay = dl_off;
            sb.dm = dm_off;
            sb.phi = phi_off;
            sb.soe = soe;
            sb.trc = trc ? append(hp.trcoef, trc->data(), trc->size()) : 0;
            sb.ident = lr.exact ? (lr.m <= lr.n ? 1 : 2) : 0;
            sb.e0 = (int32_t)hp.far_nent;
            hp.far_nent += o.nr;
            sb.ustate = hp.ustate_len;   // [rank][soe + qn]: exponential-tail states, then running sums
            hp.ustate_len += (int64_t)sb.rank * (soe + sb.qn);
            if (kind == SB_TR) {
                // + the input Y(t - taps) of the tail and of the last running sum
                sb.L = sb.maxdelay + mindm + taps + (soe || sb.qn ? 1 : 0);
                sb.LZ = maxdm - mindm + 1 + ex;
            } else {
                sb.L = sb.maxdelay + maxdm + 1 + ex;
                sb.LZ = 0;
            }
            sb.ring = hp.ring_len;
            hp.ring_len += (int64_t)sb.rank * sb.L;
            sb.zring = hp.zring_len;
            hp.zring_len += (int64_t)sb.rank * sb.LZ;
            sb.dhat = hp.dhat_len;
            if (kind == SB_F) hp.dhat_len += o.ns;
            // scatter runs: sources sorted by delay
            std::vector<int> ord(o.ns);
            for (int j = 0; j < o.ns; ++j) ord[j] = j;
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return dl[a] < dl[b]; });
            const int32_t src0 = (int32_t)hp.src_order.size();
            for (int j : ord) hp.src_order.push_back(j);
            sb.run0 = (int32_t)hp.run_delay.size();
            int q = 0;
            while (q < o.ns) {
                int e = q;
                while (e < o.ns && dl[ord[e]] == dl[ord[q]]) ++e;
                hp.run_delay.push_back(dl[ord[q]]);
                hp.run_start.push_back(src0 + q);
                hp.run_len.push_back(e - q);
                q = e;
            }
            sb.nruns = (int32_t)hp.run_delay.size() - sb.run0;
            const int id = (int)hp.sbs.size();
            hp.sbs.push_back(sb);
            if (kind == SB_F)
                for (int j = 0; j < o.ns; ++j) {
                    hp.fir_sb.push_back(id);
                    hp.fir_j.push_back(j);
                }
            if (kind == SB_TR)
                for (int l = 0; l < sb.rank; ++l) {
                    hp.tr_sb.push_back(id);
                    hp.tr_l.push_back(l);
                }
            for (int il = 0; il < o.nr; ++il) recv[o.r0 + il].push_back({id, il});
            hp.max_rank = std::max(hp.max_rank, sb.rank);
            hp.max_taps = std::max(hp.max_taps, kind == SB_F ? taps : 0);
            rank_sum += sb.rank;
            rank_cnt += 1;
            hp.rank_w[kind] += (double)sb.rank * o.nr * o.ns;   // entry-weighted, as the paper's mean rank
            hp.ent_w[kind] += (double)o.nr * o.ns;
            hp.n_exact[kind] += lr.exact ? 1 : 0;
            hp.n_aca += lr.aca ? 1 : 0;
            hp.far_entries += (int64_t)lr.F.size() + lr.G.size() + (h ? h->size() : 0);
        };
        add(SB_F, o.F[0], dF, dF_off, &o.h[0], o.HM, 0, nullptr);
        add(SB_F, o.F[1], dF, dF_off, &o.h[1], o.HM, 0, nullptr);
        add(SB_S, o.S, dS, dS_off, nullptr, 0, 0, nullptr);
        for (int cc = 0; cc < 2; ++cc)
            if (o.Dtr[cc] > 0)
                add(SB_TR, o.TR[cc], dS, dS_off, &o.htr[cc], o.Dtr[cc], o.trsoe[cc], &o.trc[cc], &o.qb[cc], &o.qh[cc]);
    }
    hp.mean_rank = rank_cnt ? rank_sum / rank_cnt : 0.0;
    hp.g_ptr.assign(n + 1, 0);
    for (int p = 0; p < n; ++p) {
        hp.g_ptr[p + 1] = hp.g_ptr[p] + (int32_t)recv[p].size();
        for (auto& e : recv[p]) {
            hp.g_sb.push_back(e.first);
            hp.g_il.push_back(e.second);
        }
    }
    // the FIR tasks by source element (CSR, tasks of one source in task order) and each source's
    // longest waveform: a source's recent slip rates are read once for all its tasks
    hp.sfir_ptr.assign(n + 1, 0);
    hp.sfir_tmax.assign(n, 0);
    for (size_t q = 0; q < hp.fir_sb.size(); ++q) {
        const SubBlock& sb = hp.sbs[hp.fir_sb[q]];
        const int p = sb.s0 + hp.fir_j[q];
        hp.sfir_ptr[p + 1] += 1;
        hp.sfir_tmax[p] = std::max(hp.sfir_tmax[p], sb.taps);
    }
    for (int p = 0; p < n; ++p) hp.sfir_ptr[p + 1] += hp.sfir_ptr[p];
    hp.sfir_q.assign(hp.fir_sb.size(), 0);
    {
        std::vector<int32_t> fill(hp.sfir_ptr.begin(), hp.sfir_ptr.end() - 1);
        for (size_t q = 0; q < hp.fir_sb.size(); ++q) {
            const int p = hp.sbs[hp.fir_sb[q]].s0 + hp.fir_j[q];
            hp.sfir_q[fill[p]++] = (int32_t)q;
        }
    }
    // block-major list of the same entries; recv[p] was filled in increasing block order, so the
    // k-th visit of receiver p is its k-th CSR slot
    std::vector<int32_t> cnt(n, 0);
    for (int id = 0; id < (int)hp.sbs.size(); ++id) {
        const SubBlock& sb = hp.sbs[id];
        for (int il = 0; il < sb.nr; ++il) {
            const int p = sb.r0 + il;
            hp.e_pos.push_back(hp.g_ptr[p] + cnt[p]++);
        }
    }
    return 0;
}

void finish_near_layout(HostPlan& hp, const std::vector<int32_t>& W, const std::vector<char>& has_tail, int chunk,
                        int vec, int vec_aux, int aux_chunk) {
    const int nl = (int)hp.near_r0.size();
    hp.near.resize(nl);
    hp.items.clear();
    hp.near_tensor_len = 0;
    hp.near_aux_len = 0;
    hp.near_tail_len = 0;
    hp.vstate_len = 0;
    hp.max_W = 0;
    std::vector<std::vector<int32_t>> slots(hp.n);
    for (int l = 0; l < nl; ++l) {
        NearLeaf& L = hp.near[l];
        L.r0 = hp.near_r0[l];
        L.nr = hp.near_nr[l];
        L.s0 = hp.near_s0[l];
        L.ns = hp.near_ns[l];
        L.W = W[l];
        L.sl = (L.ns + vec - 1) / vec * vec * L.nr;
        L.sla = (L.ns + vec_aux - 1) / vec_aux * vec_aux * L.nr;
        L.tensor = hp.near_tensor_len;                     // stays a multiple of vec elements
        hp.near_tensor_len += (int64_t)L.W * L.sl;
        const bool tail = hp.soe > 0 && has_tail[l];
        L.naux = 1 + (tail ? hp.soe : 0);
        L.stat = hp.near_aux_len;                          // a multiple of vec_aux elements, like sla
        L.tail = tail ? L.stat + L.sla : -1;
        hp.near_aux_len += (int64_t)L.naux * L.sla;
        if (tail) hp.near_tail_len += (int64_t)hp.soe * L.sla;
        L.vstate = 0;
        if (tail) {
            L.vstate = hp.vstate_len;
            hp.vstate_len += (int64_t)hp.soe * L.ns;
        }
        hp.max_W = std::max(hp.max_W, L.W);
        // one work item per chunk of window steps, and per aux_chunk of the aux slices (static
        // term from step W on, exponential tail)
        auto add = [&](int kind, int k0, int k1) {
            NearItem it;
            it.leaf = l;
            it.kind = kind;
            it.k0 = k0;
            it.k1 = k1;
            const int id = (int)hp.items.size();
            hp.items.push_back(it);
            for (int il = 0; il < L.nr; ++il) slots[L.r0 + il].push_back(id * 32 + il);
        };
        for (int k0 = 0; k0 < L.W; k0 += chunk) add(0, k0, std::min(L.W, k0 + chunk));
        for (int k0 = 0; k0 < L.naux; k0 += aux_chunk) add(1, k0, std::min(L.naux, k0 + aux_chunk));
    }
    hp.np_ptr.assign(hp.n + 1, 0);
    hp.np_idx.clear();
    for (int p = 0; p < hp.n; ++p) {
        hp.np_ptr[p + 1] = hp.np_ptr[p] + (int32_t)slots[p].size();
        hp.np_idx.insert(hp.np_idx.end(), slots[p].begin(), slots[p].end());
    }
}

}  // namespace fdph
