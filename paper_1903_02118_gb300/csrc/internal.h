// internal.h -- host-side plan structures shared by the plan builder and the CUDA code.
#pragma once
#include <stdint.h>

#include <string>
#include <climits>
#include <functional>
#include <vector>

namespace fdph {

struct Elements {
    int n = 0;
    std::vector<double> ax, ay, bx, by, mx, my, len, tx, ty, nx, ny;
};

struct Box {
    double lo[2], hi[2];
};

struct ClusterNode {
    Box box;
    int lo, hi;        // range of internal positions
    int level;
    int kid[2];        // child nodes (-1 = none)
    bool split_done;
};

struct Leaf {
    int kind;          // 1 admissible, 0 inadmissible
    int tau, sig;      // cluster nodes
    double diam, dist, rbar;
};

// Tree, permutation and ART integers (everything decided bit-exactly on the host).
struct Tree {
    std::vector<int> perm;            // perm[p] = geometry index of internal position p
    std::vector<ClusterNode> nodes;
    std::vector<Leaf> leaves;
    int nc = 0;                        // extra Domain-F steps
};

struct ArtInts {                      // per admissible leaf
    std::vector<int> dm, mbar, Dm;    // dm[nr], mbar[ns], Dm[ns]
    std::vector<double> phi;          // phi[nr]: sub-step part of the receiver delay, in [0, 1)
    int causal = 0;                   // min(dm + mbar)
};

struct PlanInputs {
    double mu, cs, dt, eps, eta, lmin, eps_st;
    int M, leaf, extra_steps;
    int soe;           // exponential-tail terms (0 = the paper's static cut)
    int interp;        // 1: receiver delays interpolated between steps (extension)
    int threads;       // host threads of the build (OpenMP), > 0
    int eta_scheme;    // 0: constant eta (Eq. 8); 1: constant eta^2 dist (Eq. 25)
    int amp_window;    // Domain-F amplitude window: 0 the placed discrete window, 1 the pair's own (Eq. 28)
    double eps_q;      // > 0: the transient's exact taps quantized (App. A)
    long long aca_min = LLONG_MAX;   // blocks of at least this many entries: cross approximation
};

// App. A.1.1 partitions of K[0, n): b (q + 1 entries, b[0] = 0, b[q] = n) and range values khat (q)
void quantize_partitions(const double* K, int n, double eps_q, std::vector<int32_t>& b, std::vector<double>& khat);

// Decay factors rho_q = exp(-lambda_q) of the exponential tail basis, lambda_q spaced
// geometrically in [0.5/M, 1] (q < Q).
std::vector<double> soe_rho(int M, int Q);
// Minimum fitted range of an exponential tail after an exact window of W steps.
inline int soe_min_len(int W) { return W * 2 > 512 ? W * 2 : 512; }
// Least-squares coefficients c (Q) of y(k') ~ sum_q c_q rho_q^k', k' < len, from the projections
// g_q = sum_k' rho_q^k' y(k') (normal equations, closed-form Gram matrix, Cholesky).
void soe_solve(const std::vector<double>& rho, int len, const double* g, double* c, int count);

Elements make_elements(int n, const double* xy);
void build_tree(const Elements& el, const PlanInputs& in, Tree& tr);
ArtInts art_integers(const Elements& el, const Tree& tr, const Leaf& lf, const PlanInputs& in);

// Truncated SVD low-rank approximation with the Frobenius criterion.
// A is m x n row-major.  On return: rank r, F (m x r, row-major), G (n x r, row-major) with
// A_r = F G^T; exact = true when the block is kept exact (rank * (m + n) >= m * n), which
// allow_exact = false turns off (the truncation is returned whatever its rank).
struct LowRank {
    int m = 0, n = 0, rank = 0;
    bool exact = false;
    bool aca = false;      // factorised by low_rank_aca
    std::vector<double> F, G;
};
void low_rank(const double* A, int m, int n, double eps, LowRank& out, bool allow_exact = true);
// Adaptive cross approximation with reference row and column (ACA+) to 1e-3 eps, entries computed on
// demand (row(i, out[n]), col(j, out[m])), then recompressed to the truncated SVD of the
// approximation at eps.  False when it did not converge within 96 crosses, the reference row /
// column show a missed part, or the rank would keep the block exact (the caller then forms the
// block and takes low_rank).
bool low_rank_aca(const std::function<void(int, double*)>& row, const std::function<void(int, double*)>& col, int m,
                  int n, double eps, LowRank& out);

void set_error(const std::string& msg);

}  // namespace fdph
