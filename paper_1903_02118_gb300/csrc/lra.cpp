// lra.cpp -- low-rank approximation of one H-matrix block (Sec. 2.3, Eq. 13).
//
// The criterion of the paper is |K_a - K_a,LRA|_F < eps |K_a|_F.  The best approximation of a
// given rank is the truncated SVD, so the rank chosen here is the smallest r whose discarded
// singular values satisfy the criterion.  The SVD is computed in two exact stages:
//   1. Householder QR with column pivoting (column norms downdated, recomputed on cancellation),
//      stopped once the trailing block is below
//      1e-11 |A|_F (A P = Q R + E): E changes the factors by at most 1e-11 relative, far
//      below any criterion eps used with the method, and it is counted in the discarded part
//      of the rank decision.  Rounding noise of the kernel values makes the numerical rank
//      at 1e-15 nearly full (512 x 512 blocks: ~490-514); at 1e-11 the mean k of the curved
//      N = 4096 plan is 16 (30 at 1e-12), and the Jacobi stage below costs O(n k^2) a sweep.
//      Blocks whose rounding noise itself sits above 1e-11 (the transient's spatial slices of
//      large blocks: 980 of 1024 singular values above 1e-11 on a planar fault) stop after 64
//      steps once the trailing block is below 1e-3 eps |A|_F;
//   2. SVD of the k x n row space B = R P^T: Householder QR of B^T, then one-sided (Hestenes)
//      Jacobi on the k x k triangular factor.
// Factors are balanced: F = U_r sqrt(S_r), G = V_r sqrt(S_r).  When the chosen rank would
// store at least as many numbers as the block (rank (m + n) >= m n) the block is kept exact
// (the fallback of Sec. 6.2): F = I, G = A^T (or F = A, G = I).
#include <math.h>

#include <algorithm>
#include <functional>
#include <numeric>
#include <vector>

#include "internal.h"

namespace fdph {

namespace {

// x . y over n entries with four partial sums (independent chains the compiler can pipeline)
inline double dot4(const double* x, const double* y, int n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 3 < n; i += 4) {
        s0 += x[i] * y[i];
        s1 += x[i + 1] * y[i + 1];
        s2 += x[i + 2] * y[i + 2];
        s3 += x[i + 3] * y[i + 3];
    }
    for (; i < n; ++i) s0 += x[i] * y[i];
    return (s0 + s1) + (s2 + s3);
}

// One-sided Jacobi on the columns of X (rows x cols, column-major), accumulating V.
// On return columns of X are mutually orthogonal: X_in = X_out V^T.
void hestenes(std::vector<double>& X, int rows, int cols, std::vector<double>& V) {
    V.assign((size_t)cols * cols, 0.0);
    for (int i = 0; i < cols; ++i) V[(size_t)i * cols + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < cols - 1; ++p) {
            for (int q = p + 1; q < cols; ++q) {
                double* xp = &X[(size_t)p * rows];
                double* xq = &X[(size_t)q * rows];
                double a = 0.0, b = 0.0, g = 0.0;
                for (int i = 0; i < rows; ++i) {
                    a += xp[i] * xp[i];
                    b += xq[i] * xq[i];
                    g += xp[i] * xq[i];
                }
                if (g == 0.0 || fabs(g) <= 1e-15 * sqrt(a * b)) continue;
                off = std::max(off, fabs(g) / sqrt(a * b));
                const double zeta = (b - a) / (2.0 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = c * t;
                for (int i = 0; i < rows; ++i) {
                    const double u = xp[i], v = xq[i];
                    xp[i] = c * u - s * v;
                    xq[i] = s * u + c * v;
                }
                double* vp = &V[(size_t)p * cols];
                double* vq = &V[(size_t)q * cols];
                for (int i = 0; i < cols; ++i) {
                    const double u = vp[i], v = vq[i];
                    vp[i] = c * u - s * v;
                    vq[i] = s * u + c * v;
                }
            }
        }
        if (off <= 1e-15) break;
    }
}

}  // namespace

void low_rank(const double* A, int m, int n, double eps, LowRank& out, bool allow_exact) {
    out.m = m;
    out.n = n;
    out.rank = 0;
    out.exact = false;
    out.aca = false;
    out.F.clear();
    out.G.clear();
    double norm2 = 0.0;
    for (long i = 0; i < (long)m * n; ++i) norm2 += A[i] * A[i];
    if (norm2 == 0.0) return;
    auto keep_exact = [&]() {
        out.exact = true;
        if (m <= n) {
            out.rank = m;
            out.F.assign((size_t)m * m, 0.0);
            for (int i = 0; i < m; ++i) out.F[(size_t)i * m + i] = 1.0;
            out.G.resize((size_t)n * m);
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < m; ++i) out.G[(size_t)j * m + i] = A[(size_t)i * n + j];
        } else {
            out.rank = n;
            out.F.assign(A, A + (size_t)m * n);
            out.G.assign((size_t)n * n, 0.0);
            for (int j = 0; j < n; ++j) out.G[(size_t)j * n + j] = 1.0;
        }
    };
    if (eps <= 0.0) {
        keep_exact();
        return;
    }
    // ---- stage 1: QR with column pivoting on a column-major copy
    std::vector<double> W((size_t)m * n);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) W[(size_t)j * m + i] = A[(size_t)i * n + j];
    std::vector<int> piv(n);
    std::iota(piv.begin(), piv.end(), 0);
    std::vector<double> tau;
    std::vector<std::vector<double>> hv;  // Householder vectors (length m - k)
    const int kmax = std::min(m, n);
    int k = 0;
    const double stop2 = 1e-22 * norm2;
    // A block still above the 1e-11 floor after kNoiseSteps steps is dominated by the rounding of
    // its entries (the Domain-S transient's spatial slice is a difference of nearly equal kernel
    // values, accurate to ~1e-11 relative: its numerical rank at 1e-11 is nearly full, and the QR
    // would run to m n min(m, n) work); from there the QR also stops at (1e-3 eps)^2 |A|^2, which
    // changes the rank decision by at most that share of the criterion (the remainder is counted
    // as discarded) and the factors by at most 1e-3 eps |A|
    const int kNoiseSteps = 64;
    const double stop2_eps = 1e-6 * eps * eps * norm2;
    // squared norms of the columns' trailing parts, downdated after each reflection (cn) and
    // recomputed from the column when the downdate has cancelled most of the value they had at
    // their last recomputation (cn0), as in the usual pivoted QR
    auto trailing = [&](int j, int from) {
        const double* col = &W[(size_t)j * m] + from;
        return dot4(col, col, m - from);
    };
    std::vector<double> cn(n), cn0(n);
    for (int j = 0; j < n; ++j) cn[j] = cn0[j] = trailing(j, 0);
    for (; k < kmax; ++k) {
        double trail = 0.0;
        for (int j = k; j < n; ++j) trail += cn[j];
        if (trail <= 4.0 * stop2) {   // near the stop: decide on exact norms
            trail = 0.0;
            for (int j = k; j < n; ++j) trail += (cn[j] = cn0[j] = trailing(j, k));
        }
        if (trail <= stop2 || (k >= kNoiseSteps && trail <= stop2_eps)) break;
        int best = k;
        for (int j = k + 1; j < n; ++j)
            if (cn[j] > cn[best]) best = j;
        if (best != k) {
            std::swap_ranges(&W[(size_t)k * m], &W[(size_t)k * m] + m, &W[(size_t)best * m]);
            std::swap(piv[k], piv[best]);
            std::swap(cn[k], cn[best]);
            std::swap(cn0[k], cn0[best]);
        }
        cn[k] = trailing(k, k);   // the pivot column's norm exactly (it defines the reflector)
        double* col = &W[(size_t)k * m];
        const double alpha = sqrt(cn[k]);
        const double beta = col[k] >= 0 ? -alpha : alpha;
        std::vector<double> v(col + k, col + m);
        v[0] -= beta;
        double vn2 = 0.0;
        for (double x : v) vn2 += x * x;
        if (vn2 > 0.0) {
            for (int j = k + 1; j < n; ++j) {
                double* cj = &W[(size_t)j * m];
                const double f = 2.0 * dot4(v.data(), cj + k, m - k) / vn2;
                for (int i = 0; i < m - k; ++i) cj[k + i] -= f * v[i];
            }
        }
        for (int j = k + 1; j < n; ++j) {   // row k of R leaves the trailing part
            const double r = W[(size_t)j * m + k];
            cn[j] -= r * r;
            if (!(cn[j] > 1e-8 * cn0[j])) cn[j] = cn0[j] = trailing(j, k + 1);
        }
        col[k] = beta;
        for (int i = k + 1; i < m; ++i) col[i] = 0.0;
        hv.push_back(v);
        tau.push_back(vn2);
    }
    const int kr = k;  // numerical rank of the QR stage
    double resid2 = 0.0;
    for (int j = kr; j < n; ++j) {
        const double* col = &W[(size_t)j * m];
        for (int i = kr; i < m; ++i) resid2 += col[i] * col[i];
    }
    if (kr == 0) return;
    // ---- stage 2: SVD of B = R P^T (kr x n): Householder QR B^T = Q2 R2 (n x kr), then Jacobi on
    // the kr x kr factor R2 (R2 V = U2 S), so that B^T V = Q2 U2 S and the Jacobi sweeps cost
    // O(kr^3) instead of O(n kr^2)
    std::vector<double> BT((size_t)n * kr, 0.0);
    for (int j = 0; j < n; ++j) {
        const double* col = &W[(size_t)j * m];
        for (int i = 0; i < std::min(kr, j + 1); ++i) BT[(size_t)i * n + piv[j]] = col[i];
    }
    std::vector<std::vector<double>> hv2;  // reflectors of the QR of B^T (length n - c)
    std::vector<double> tau2;
    for (int c = 0; c < kr; ++c) {
        double* col = &BT[(size_t)c * n];
        double a2 = 0.0;
        for (int i = c; i < n; ++i) a2 += col[i] * col[i];
        const double alpha = sqrt(a2);
        const double beta = col[c] >= 0 ? -alpha : alpha;
        std::vector<double> v(col + c, col + n);
        v[0] -= beta;
        double vn2 = 0.0;
        for (double x : v) vn2 += x * x;
        if (vn2 > 0.0) {
            for (int c2 = c + 1; c2 < kr; ++c2) {
                double* cj = &BT[(size_t)c2 * n];
                const double f = 2.0 * dot4(v.data(), cj + c, n - c) / vn2;
                for (int i = 0; i < n - c; ++i) cj[c + i] -= f * v[i];
            }
            col[c] = beta;
            for (int i = c + 1; i < n; ++i) col[i] = 0.0;
        }
        hv2.push_back(v);
        tau2.push_back(vn2);
    }
    std::vector<double> R2((size_t)kr * kr, 0.0);   // column-major, upper triangular
    for (int c = 0; c < kr; ++c)
        for (int i = 0; i <= c; ++i) R2[(size_t)c * kr + i] = BT[(size_t)c * n + i];
    std::vector<double> V;
    hestenes(R2, kr, kr, V);
    std::vector<double> sv(kr);
    for (int c = 0; c < kr; ++c) {
        double s = 0.0;
        for (int i = 0; i < kr; ++i) s += R2[(size_t)c * kr + i] * R2[(size_t)c * kr + i];
        sv[c] = sqrt(s);
    }
    std::vector<int> ord(kr);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
    // rank: smallest r with sqrt(sum_{l >= r} s_l^2 + resid) < eps |A|
    std::vector<double> tail(kr + 1, 0.0);
    tail[kr] = resid2;
    for (int l = kr - 1; l >= 0; --l) tail[l] = tail[l + 1] + sv[ord[l]] * sv[ord[l]];
    const double lim = eps * sqrt(norm2);
    int r = kr;
    for (int l = 0; l <= kr; ++l)
        if (sqrt(tail[l]) < lim) { r = l; break; }
    if (allow_exact && (long)r * (m + n) >= (long)m * n) {
        keep_exact();
        return;
    }
    out.rank = r;
    if (r == 0) return;
    // left vectors: Q * V[:, c]  (Q from the Householder reflectors, kr columns)
    // B = V S U^T with U columns = BT columns / s; A ~ Q B = (Q V) S U^T
    out.F.assign((size_t)m * r, 0.0);
    out.G.assign((size_t)n * r, 0.0);
    for (int l = 0; l < r; ++l) {
        const int c = ord[l];
        const double s = sv[c];
        const double rs = sqrt(s);
        // y = Q * e where e = V column c padded to length m
        std::vector<double> y(m, 0.0);
        for (int i = 0; i < kr; ++i) y[i] = V[(size_t)c * kr + i];
        for (int h = kr - 1; h >= 0; --h) {
            const std::vector<double>& v = hv[h];
            double d = 0.0;
            for (int i = 0; i < m - h; ++i) d += v[i] * y[h + i];
            const double f = 2.0 * d / tau[h];
            for (int i = 0; i < m - h; ++i) y[h + i] -= f * v[i];
        }
        for (int i = 0; i < m; ++i) out.F[(size_t)i * r + l] = y[i] * rs;
        // column c of B^T V = Q2 (R2 V)_c, applying the reflectors of Q2 in reverse
        std::vector<double> z(n, 0.0);
        for (int i = 0; i < kr; ++i) z[i] = R2[(size_t)c * kr + i];
        for (int h = kr - 1; h >= 0; --h) {
            if (!(tau2[h] > 0.0)) continue;
            const std::vector<double>& v = hv2[h];
            double d = 0.0;
            for (int i = 0; i < n - h; ++i) d += v[i] * z[h + i];
            const double f = 2.0 * d / tau2[h];
            for (int i = 0; i < n - h; ++i) z[h + i] -= f * v[i];
        }
        for (int j = 0; j < n; ++j) out.G[(size_t)j * r + l] = z[j] / s * rs;
    }
}

}  // namespace fdph

namespace fdph {

std::vector<double> soe_rho(int M, int Q) {
    std::vector<double> r(Q);
    const double a = log(0.5 / M), b = log(1.0);
    for (int q = 0; q < Q; ++q) r[q] = exp(-exp(a + (double)q / (Q - 1.0) * (b - a)));
    return r;
}

// Gram matrix G_pq = sum_{k < len} (rho_p rho_q)^k = (1 - (rho_p rho_q)^len) / (1 - rho_p rho_q),
// Cholesky-factored once, then `count` right-hand sides g (count x Q) are solved in place into c.
void soe_solve(const std::vector<double>& rho, int len, const double* g, double* c, int count) {
    const int Q = (int)rho.size();
    std::vector<double> G((size_t)Q * Q);
    for (int p = 0; p < Q; ++p)
        for (int q = 0; q < Q; ++q) {
            const double x = rho[p] * rho[q];
            G[(size_t)p * Q + q] = (1.0 - pow(x, (double)len)) / (1.0 - x);
        }
    // Cholesky G = L L^T (lower, in place); if a pivot is lost to rounding, retry with a small
    // ridge (relative 1e-13 of the diagonal), which only touches directions the data cannot fix
    const std::vector<double> G0 = G;
    double ridge = 0.0;
    for (int attempt = 0; attempt < 6; ++attempt) {
        G = G0;
        for (int j = 0; j < Q; ++j) G[(size_t)j * Q + j] *= 1.0 + ridge;
        bool ok = true;
        for (int j = 0; j < Q && ok; ++j) {
            double d = G[(size_t)j * Q + j];
            for (int k = 0; k < j; ++k) d -= G[(size_t)j * Q + k] * G[(size_t)j * Q + k];
            if (!(d > 0.0)) {
                ok = false;
                break;
            }
            d = sqrt(d);
            G[(size_t)j * Q + j] = d;
            for (int i = j + 1; i < Q; ++i) {
                double s = G[(size_t)i * Q + j];
                for (int k = 0; k < j; ++k) s -= G[(size_t)i * Q + k] * G[(size_t)j * Q + k];
                G[(size_t)i * Q + j] = s / d;
            }
        }
        if (ok) break;
        ridge = ridge == 0.0 ? 1e-13 : ridge * 100.0;
    }
    for (int r = 0; r < count; ++r) {
        const double* gr = g + (size_t)r * Q;
        double* cr = c + (size_t)r * Q;
        for (int i = 0; i < Q; ++i) {  // L z = g
            double s = gr[i];
            for (int k = 0; k < i; ++k) s -= G[(size_t)i * Q + k] * cr[k];
            cr[i] = s / G[(size_t)i * Q + i];
        }
        for (int i = Q - 1; i >= 0; --i) {  // L^T c = z
            double s = cr[i];
            for (int k = i + 1; k < Q; ++k) s -= G[(size_t)k * Q + i] * cr[k];
            cr[i] = s / G[(size_t)i * Q + i];
        }
    }
}

}  // namespace fdph

namespace fdph {

namespace {

// deterministic generator for the reference rows / columns of the cross approximation
struct Lcg {
    unsigned long long s;
    explicit Lcg(unsigned long long seed) : s(seed * 6364136223846793005ULL + 1442695040888963407ULL) {}
    int below(int n) {
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        return (int)((s >> 33) % (unsigned long long)n);
    }
};

// Q R of the columns of X (rows x k, column-major) by Gram-Schmidt applied twice per column; X is
// replaced by Q, R (k x k, column-major, upper) is returned.  A column that vanishes after its
// projections stays zero (its row of R is zero).
std::vector<double> cgs2(std::vector<double>& X, int rows, int k) {
    std::vector<double> R((size_t)k * k, 0.0);
    for (int c = 0; c < k; ++c) {
        double* x = &X[(size_t)c * rows];
        for (int pass = 0; pass < 2; ++pass)
            for (int p = 0; p < c; ++p) {
                const double* q = &X[(size_t)p * rows];
                const double d = dot4(q, x, rows);
                R[(size_t)c * k + p] += d;
                for (int i = 0; i < rows; ++i) x[i] -= d * q[i];
            }
        const double nx = sqrt(dot4(x, x, rows));
        R[(size_t)c * k + c] = nx;
        const double inv = nx > 0.0 ? 1.0 / nx : 0.0;
        for (int i = 0; i < rows; ++i) x[i] *= inv;
    }
    return R;
}

}  // namespace

bool low_rank_aca(const std::function<void(int, double*)>& row, const std::function<void(int, double*)>& col, int m,
                  int n, double eps, LowRank& out) {
    out.m = m;
    out.n = n;
    out.rank = 0;
    out.exact = false;
    out.aca = false;
    out.F.clear();
    out.G.clear();
    if (m < 2 || n < 2 || !(eps > 0.0)) return false;
    const double tol = 1e-3 * eps;
    const int kmax = std::min(std::min(m, n), 96);
    std::vector<std::vector<double>> U, V;            // A ~ sum_l U_l V_l^T
    std::vector<char> rused(m, 0), cused(n, 0);
    std::vector<double> r(n), c(m), rref(n), cref(m);
    Lcg rng(0x5eedULL + (unsigned long long)m * 131071ULL + (unsigned long long)n);
    auto resid_row = [&](int i, std::vector<double>& out_r) {
        row(i, out_r.data());
        for (size_t l = 0; l < U.size(); ++l) {
            const double f = U[l][i];
            for (int j = 0; j < n; ++j) out_r[j] -= f * V[l][j];
        }
    };
    auto resid_col = [&](int j, std::vector<double>& out_c) {
        col(j, out_c.data());
        for (size_t l = 0; l < U.size(); ++l) {
            const double f = V[l][j];
            for (int i = 0; i < m; ++i) out_c[i] -= f * U[l][i];
        }
    };
    auto argmax_free = [](const std::vector<double>& x, const std::vector<char>& used) {
        int best = -1;
        double bv = -1.0;
        for (size_t t = 0; t < x.size(); ++t)
            if (!used[t] && fabs(x[t]) > bv) {
                bv = fabs(x[t]);
                best = (int)t;
            }
        return best;
    };
    auto pick_free = [&](const std::vector<char>& used, int count) {
        for (int tries = 0; tries < 64; ++tries) {
            const int t = rng.below(count);
            if (!used[t]) return t;
        }
        for (int t = 0; t < count; ++t)
            if (!used[t]) return t;
        return -1;
    };
    int iref = pick_free(rused, m), jref = pick_free(cused, n);
    resid_row(iref, rref);
    resid_col(jref, cref);
    double norm2 = 0.0;
    int small = 0, vanished = 0;
    bool converged = false;
    for (int k = 0; k < kmax; ++k) {
        // pivot from the larger of the reference row's and the reference column's residuals (ACA+)
        const int j1 = argmax_free(rref, cused), i1 = argmax_free(cref, rused);
        if (j1 < 0 || i1 < 0) break;
        int is, js;
        if (fabs(rref[j1]) >= fabs(cref[i1])) {
            js = j1;
            resid_col(js, c);
            is = argmax_free(c, rused);
            resid_row(is, r);
        } else {
            is = i1;
            resid_row(is, r);
            js = argmax_free(r, cused);
            resid_col(js, c);
        }
        const double piv = r[js];
        if (!(fabs(piv) > 1e-300)) {
            // the residual vanished on the reference row and column and on the cross through their
            // largest entries: a few fresh references before concluding that the rest is zero
            if (++vanished > 3) {
                converged = true;
                break;
            }
            rused[iref] = 1;
            cused[jref] = 1;
            iref = pick_free(rused, m);
            jref = pick_free(cused, n);
            if (iref < 0 || jref < 0) {
                converged = true;
                break;
            }
            resid_row(iref, rref);
            resid_col(jref, cref);
            --k;
            continue;
        }
        std::vector<double> u(m), v(r);
        for (int i = 0; i < m; ++i) u[i] = c[i] / piv;
        rused[is] = 1;
        cused[js] = 1;
        // |S + u v^T|_F^2 = |S|_F^2 + 2 sum_l (u . U_l)(v . V_l) + |u|^2 |v|^2
        const double uu = dot4(u.data(), u.data(), m), vv = dot4(v.data(), v.data(), n);
        double cross = 0.0;
        for (size_t l = 0; l < U.size(); ++l) cross += dot4(u.data(), U[l].data(), m) * dot4(v.data(), V[l].data(), n);
        norm2 += 2.0 * cross + uu * vv;
        // the reference row and column lose the new cross
        const double ur = u[iref], vc = v[jref];
        U.push_back(std::move(u));
        V.push_back(std::move(v));
        for (int j = 0; j < n; ++j) rref[j] -= ur * V.back()[j];
        for (int i = 0; i < m; ++i) cref[i] -= vc * U.back()[i];
        if (rused[iref]) {
            iref = pick_free(rused, m);
            if (iref < 0) break;
            resid_row(iref, rref);
        }
        if (cused[jref]) {
            jref = pick_free(cused, n);
            if (jref < 0) break;
            resid_col(jref, cref);
        }
        small = sqrt(uu * vv) <= tol * sqrt(std::max(norm2, 0.0)) ? small + 1 : 0;
        if (small >= 2) {
            converged = true;
            break;
        }
    }
    if (!converged) return false;
    if (U.empty()) {   // rank 0: every sampled row and column vanished
        out.aca = true;
        return true;
    }
    // the reference row and column are residuals of unused random ones: their energy, scaled to the
    // whole block, must be within the tolerance, else the cross approximation missed a part
    const double rr = dot4(rref.data(), rref.data(), n) * m, cc = dot4(cref.data(), cref.data(), m) * n;
    if (std::max(rr, cc) > 100.0 * tol * tol * norm2) return false;
    // recompression: U = Qu Ru, V = Qv Rv, core Ru Rv^T truncated at eps (its Frobenius norm is the
    // approximation's), A ~ (Qu Fc)(Qv Gc)^T
    const int k = (int)U.size();
    std::vector<double> Qu((size_t)m * k), Qv((size_t)n * k);
    for (int l = 0; l < k; ++l) {
        std::copy(U[l].begin(), U[l].end(), Qu.begin() + (size_t)l * m);
        std::copy(V[l].begin(), V[l].end(), Qv.begin() + (size_t)l * n);
    }
    const std::vector<double> Ru = cgs2(Qu, m, k), Rv = cgs2(Qv, n, k);
    std::vector<double> core((size_t)k * k, 0.0);   // row-major k x k: (Ru Rv^T)[a][b]
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            double s = 0.0;
            for (int l = std::max(a, b); l < k; ++l) s += Ru[(size_t)l * k + a] * Rv[(size_t)l * k + b];
            core[(size_t)a * k + b] = s;
        }
    LowRank cr;
    low_rank(core.data(), k, k, eps, cr, false);
    const int rk = cr.rank;
    if ((long)rk * (m + n) >= (long)m * n) return false;   // the block is kept exact (Sec. 6.2)
    out.rank = rk;
    out.aca = true;
    if (rk == 0) return true;
    out.F.assign((size_t)m * rk, 0.0);
    out.G.assign((size_t)n * rk, 0.0);
    for (int a = 0; a < k; ++a)
        for (int l = 0; l < rk; ++l) {
            const double f = cr.F[(size_t)a * rk + l], g = cr.G[(size_t)a * rk + l];
            if (f != 0.0)
                for (int i = 0; i < m; ++i) out.F[(size_t)i * rk + l] += Qu[(size_t)a * m + i] * f;
            if (g != 0.0)
                for (int j = 0; j < n; ++j) out.G[(size_t)j * rk + l] += Qv[(size_t)a * n + j] * g;
        }
    return true;
}

}  // namespace fdph
