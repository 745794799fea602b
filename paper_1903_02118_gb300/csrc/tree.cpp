// tree.cpp -- elements, bounding-box cluster tree, block-cluster tree, ART integers.
//
// Compiled with -ffp-contract=off: every decision here (box splits, admissibility, the
// integer delays) must be reproducible bit for bit, so no multiply-add is fused.
//
// Clustering (Sec. 2.3 and Sec. 4.2.2): the root box bounds the element midpoints; a box is
// cut at the middle of its longest side (x when the sides are equal) and never re-tightened,
// so all boxes of one level share their shape; an element goes to the child that holds its
// midpoint (a midpoint on the cut goes to the upper child); empty children are dropped.
// Elements are stored in the order of a stable recursive partition, which makes every
// cluster a contiguous range of internal positions.
//
// Block tree (Eqs. 8-9, Sec. 4.2.2): diam = largest box diagonal + largest element length of
// the two clusters, rbar = distance of the box centres, dist = rbar - diam; admissible when
// diam < eta dist (constant eta scheme) or diam < sqrt(eta l_min dist) (constant eta^2 dist
// scheme, Eq. 25), inadmissible when both clusters hold at most `leaf` elements (or
// diam < l_min), else both clusters are bisected.
#include <math.h>

#include <algorithm>
#include <functional>

#include "internal.h"

namespace fdph {

Elements make_elements(int n, const double* xy) {
    Elements e;
    e.n = n;
    auto rs = [&](std::vector<double>& v) { v.resize(n); };
    rs(e.ax); rs(e.ay); rs(e.bx); rs(e.by); rs(e.mx); rs(e.my);
    rs(e.len); rs(e.tx); rs(e.ty); rs(e.nx); rs(e.ny);
    for (int k = 0; k < n; ++k) {
        const double x0 = xy[4 * k], y0 = xy[4 * k + 1], x1 = xy[4 * k + 2], y1 = xy[4 * k + 3];
        const double ex = x1 - x0, ey = y1 - y0;
        const double L = sqrt(ex * ex + ey * ey);
        e.ax[k] = x0; e.ay[k] = y0; e.bx[k] = x1; e.by[k] = y1;
        e.mx[k] = 0.5 * (x0 + x1);
        e.my[k] = 0.5 * (y0 + y1);
        e.len[k] = L;
        e.tx[k] = ex / L;
        e.ty[k] = ey / L;
        e.nx[k] = -e.ty[k];
        e.ny[k] = e.tx[k];
    }
    return e;
}

static inline double box_diag(const Box& b) {
    const double w = b.hi[0] - b.lo[0];
    const double h = b.hi[1] - b.lo[1];
    return sqrt(w * w + h * h);
}

static inline void box_centre(const Box& b, double c[2]) {
    c[0] = 0.5 * (b.lo[0] + b.hi[0]);
    c[1] = 0.5 * (b.lo[1] + b.hi[1]);
}

// Split node `id` (stable partition of its range), creating its non-empty children.
static void split_node(const Elements& el, Tree& tr, int id) {
    ClusterNode nd = tr.nodes[id];
    if (nd.split_done) return;
    const double w = nd.box.hi[0] - nd.box.lo[0];
    const double h = nd.box.hi[1] - nd.box.lo[1];
    const int ax = (w >= h) ? 0 : 1;
    const double mid = 0.5 * (nd.box.lo[ax] + nd.box.hi[ax]);
    const std::vector<double>& c = ax == 0 ? el.mx : el.my;
    // stable partition: below the cut first
    std::vector<int> lower, upper;
    for (int p = nd.lo; p < nd.hi; ++p) {
        const int e = tr.perm[p];
        (c[e] >= mid ? upper : lower).push_back(e);
    }
    int p = nd.lo;
    for (int e : lower) tr.perm[p++] = e;
    for (int e : upper) tr.perm[p++] = e;
    const int nlow = (int)lower.size();
    int kids[2] = {-1, -1};
    int nk = 0;
    for (int side = 0; side < 2; ++side) {
        const int lo = side == 0 ? nd.lo : nd.lo + nlow;
        const int hi = side == 0 ? nd.lo + nlow : nd.hi;
        if (hi <= lo) continue;
        ClusterNode ch;
        ch.box = nd.box;
        if (side == 0) ch.box.hi[ax] = mid; else ch.box.lo[ax] = mid;
        ch.lo = lo;
        ch.hi = hi;
        ch.level = nd.level + 1;
        ch.kid[0] = ch.kid[1] = -1;
        ch.split_done = false;
        tr.nodes.push_back(ch);
        kids[nk++] = (int)tr.nodes.size() - 1;
    }
    tr.nodes[id].kid[0] = kids[0];
    tr.nodes[id].kid[1] = kids[1];
    tr.nodes[id].split_done = true;
}

static const int kMaxDepth = 64;

void build_tree(const Elements& el, const PlanInputs& in, Tree& tr) {
    const int n = el.n;
    tr.perm.resize(n);
    for (int k = 0; k < n; ++k) tr.perm[k] = k;
    tr.nodes.clear();
    tr.leaves.clear();
    ClusterNode root;
    root.box.lo[0] = root.box.hi[0] = el.mx[0];
    root.box.lo[1] = root.box.hi[1] = el.my[0];
    for (int k = 1; k < n; ++k) {
        root.box.lo[0] = std::min(root.box.lo[0], el.mx[k]);
        root.box.hi[0] = std::max(root.box.hi[0], el.mx[k]);
        root.box.lo[1] = std::min(root.box.lo[1], el.my[k]);
        root.box.hi[1] = std::max(root.box.hi[1], el.my[k]);
    }
    root.lo = 0;
    root.hi = n;
    root.level = 0;
    root.kid[0] = root.kid[1] = -1;
    root.split_done = false;
    tr.nodes.push_back(root);
    // Fix the permutation first: split every cluster with >= 2 elements (depth-capped).
    // Splitting one-element clusters never reorders, so those are split lazily below.
    {
        std::vector<int> stack{0};
        while (!stack.empty()) {
            const int id = stack.back();
            stack.pop_back();
            const ClusterNode& nd = tr.nodes[id];
            if (nd.hi - nd.lo < 2 || nd.level >= kMaxDepth) continue;
            split_node(el, tr, id);
            for (int s = 0; s < 2; ++s)
                if (tr.nodes[id].kid[s] >= 0) stack.push_back(tr.nodes[id].kid[s]);
        }
    }
    // maximum element length per cluster range is needed for diam
    auto maxlen = [&](const ClusterNode& nd) {
        double m = 0.0;
        for (int p = nd.lo; p < nd.hi; ++p) m = std::max(m, el.len[tr.perm[p]]);
        return m;
    };
    struct Item { int tau, sig, depth; };
    std::vector<Item> stack{{0, 0, 0}};
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        const ClusterNode tn = tr.nodes[it.tau];
        const ClusterNode sn = tr.nodes[it.sig];
        const double diag = std::max(box_diag(tn.box), box_diag(sn.box));
        const double diam = diag + std::max(maxlen(tn), maxlen(sn));
        double ct[2], cs[2];
        box_centre(tn.box, ct);
        box_centre(sn.box, cs);
        const double rbar = sqrt((ct[0] - cs[0]) * (ct[0] - cs[0]) + (ct[1] - cs[1]) * (ct[1] - cs[1]));
        const double dist = rbar - diam;
        const int nt = tn.hi - tn.lo, ns = sn.hi - sn.lo;
        const bool adm = in.eta_scheme == 1 ? (in.eta > 0.0 && dist > 0.0 && diam < sqrt(in.eta * in.lmin * dist))
                                            : (in.eta > 0.0 && diam < in.eta * dist);
        if (adm) {
            tr.leaves.push_back({1, it.tau, it.sig, diam, dist, rbar});
        } else if ((nt <= in.leaf && ns <= in.leaf) || diam < in.lmin || it.depth >= kMaxDepth) {
            tr.leaves.push_back({0, it.tau, it.sig, diam, dist, rbar});
        } else {
            split_node(el, tr, it.tau);
            split_node(el, tr, it.sig);
            const ClusterNode& t2 = tr.nodes[it.tau];
            const ClusterNode& s2 = tr.nodes[it.sig];
            int tk[2] = {t2.kid[0], t2.kid[1]}, sk[2] = {s2.kid[0], s2.kid[1]};
            for (int a = 1; a >= 0; --a)
                for (int b = 1; b >= 0; --b)
                    if (tk[a] >= 0 && sk[b] >= 0) stack.push_back({tk[a], sk[b], it.depth + 1});
        }
    }
    double lmax = 0.0;
    for (int k = 0; k < n; ++k) lmax = std::max(lmax, el.len[k]);
    tr.nc = in.extra_steps >= 0 ? in.extra_steps : (int)ceil(10.0 * lmax / (in.cs * in.dt) - 1e-9);
}

// ART integers of Eq. 30 and App. C.3 for one admissible leaf, receivers and sources in
// internal order: i* / j* are the box centres, c dt the step length of the wavefront.
ArtInts art_integers(const Elements& el, const Tree& tr, const Leaf& lf, const PlanInputs& in) {
    const ClusterNode& tn = tr.nodes[lf.tau];
    const ClusterNode& sn = tr.nodes[lf.sig];
    double ist[2], jst[2];
    box_centre(tn.box, ist);
    box_centre(sn.box, jst);
    const double cdt = in.cs * in.dt;
    ArtInts a;
    a.dm.resize(tn.hi - tn.lo);
    a.phi.resize(tn.hi - tn.lo);
    a.mbar.resize(sn.hi - sn.lo);
    a.Dm.resize(sn.hi - sn.lo);
    for (int p = tn.lo; p < tn.hi; ++p) {
        const int e = tr.perm[p];
        const double dx = el.mx[e] - jst[0], dy = el.my[e] - jst[1];
        const double r = sqrt(dx * dx + dy * dy);
        const double x = (r - lf.rbar) / cdt;
        a.dm[p - tn.lo] = (int)floor(x);
        a.phi[p - tn.lo] = x - floor(x);
    }
    for (int p = sn.lo; p < sn.hi; ++p) {
        const int e = tr.perm[p];
        const double dx = ist[0] - el.mx[e], dy = ist[1] - el.my[e];
        const double r = sqrt(dx * dx + dy * dy);
        const double half = 0.5 * el.len[e];
        const int mb = (int)floor((r - half) / cdt);
        a.mbar[p - sn.lo] = mb;
        a.Dm[p - sn.lo] = (int)ceil((r + half) / cdt) - mb + tr.nc;
    }
    int mn = 1 << 30;
    const int mnd = *std::min_element(a.dm.begin(), a.dm.end());
    const int mnb = *std::min_element(a.mbar.begin(), a.mbar.end());
    mn = mnd + mnb;
    a.causal = mn;
    return a;
}

}  // namespace fdph
