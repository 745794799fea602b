// fdph.cu -- device side of the FDP=H time step and the C ABI (include/fdph.h).
//
// One time step n (Eq. 4 evaluated through the plan's operator) runs these kernels in order
// on the plan's stream:
//   push     D_n -> slip-rate ring (internal order); cumulative slip C_j(n) = sum_{s<=n} D_j,s
//            with a compensated (Kahan) FP64 sum, -> cumulative-slip ring
//   fir      Domain F, formula 1 (Eq. 32): Dhat_j = sum_{m < Dm_j} h_{j,m} D_{j,n-m}
//   scatter  formula 2 (Eq. 42): Tbar'_l[n + delay_j] += g_{l,j} u_j for every run of sources
//            (rings are stored [slot][rank] so that one receiver's ranks share a sector)
//            with equal delay (no atomics: one writer per ring slot); u = Dhat (Domain F),
//            dt * C (Domain S, App. B.1 written on the cumulative slip), D (transient);
//            the ring is the shift operator M of Eq. 40 as a base-pointer increment
//   trconv   transient (App. B.3): Z_l(n - min dm) = sum_{m < Dm_tr} h^tr_m Y_l(n - min dm - m)
//   near     inadmissible leaves (App. E): sum_{k < W} K_{ij,k} D_{j,n-k} + Kstat_ij dt C_j(n-W),
//            per (leaf, chunk of k) work item into a partial-sum slot
//   gather   formula 3 (Eq. 39): T_i = sum_{blocks} sum_l f_{l,i} Tbar'_l[n - dm_i] + near
//            partials, written in the caller's element order
// Causality (min(dm + delay) >= 1, checked at plan time) guarantees that the ring slots read
// at step n were completed by steps < n and that the slots written at step n are not read.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <omp.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/fdph.h"
#include "internal.h"
#include "kernel2d.cuh"
#include "plan.h"

namespace fdph {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace fdph

using namespace fdph;

#define FDPH_CUDA(call)                                                                      \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
            return FDPH_E_CUDA;                                                              \
        }                                                                                    \
    } while (0)

static const int kChunk = 64;      // steps of exact kernel per near-field work item
static const int kNearThreads = 256;
static const int kStages = 4;      // shared-memory pipeline depth of the near-field kernel
static const int kStageBytes = 12288;
static const long long kWaitLimit = 1LL << 22;   // bounded mbarrier polls before giving up

// ------------------------------------------------------------------------------------------
// device-side views

struct SbDev {
    int kind, rank, r0, nr, s0, ns, L, LZ, taps, maxdelay, mindm, run0, soe, pad;
    long long f, g, h, ring, zring, dhat, delay, dm, ustate, trc, phi;
};

struct NearDev {
    int r0, nr, s0, ns, W, sl;
    long long tensor, stat, tail, vstate;
};

static const int kMaxSoe = 16;

template <class T>
struct StepArgs {
    int n, N, WD, WC;
    // graph replay: the step index is read from n_dev, and D_in / T_out advance by io_stride
    // elements per step past n_base (both unused when n_dev is null)
    const int* n_dev;
    int n_base;
    long long io_stride;
    double dt;
    const double* D_in;       // caller's D_n (geometry order)
    double* T_out;            // caller's T_n (geometry order)
    const int* perm;          // internal -> geometry
    double* Dring;            // [WD][N]
    double* Cring;            // [WC][N]
    double* C;                // [N] cumulative slip (rounded sum)
    double* Ccomp;            // [N] Kahan compensation
    // far field
    const SbDev* sbs;
    const T* fac;
    const int* ints;
    const int* run_delay;
    const int* run_start;
    const int* run_len;
    const int* src_order;
    const int* scat_sb;
    const int* scat_run;
    const int* scat_l;
    int n_scat;
    const int* e_sb;
    const int* e_il;
    const int* e_pos;
    int n_ent;
    double* fval;             // [n_ent] far-field value of each (block, receiver) entry, CSR order
    const int* fir_sb;
    const int* fir_j;
    int n_fir;
    const int* tr_sb;
    const int* tr_l;
    int n_tr;
    const int* g_ptr;
    const int* g_sb;
    const int* g_il;
    double* ring;
    double* zring;
    double* dhat;
    // near field
    const NearDev* near;
    const int4* items;
    int n_items;
    const T* tensor;
    const double* stat;
    double* partial;          // [n_items][32]
    const int* np_ptr;
    const int* np_idx;
    int* err;                 // device error word (1 = a bounded wait gave up)
    // exponential tails (extension; soe == 0: the paper's static cut)
    int soe;
    const double* rho;        // [soe] decay factors
    double* ustate;           // transient blocks: [rank][soe] per block
    const double* trcoef;     // transient blocks: [soe] tail coefficients per block (FP64)
    const double* phi;        // sub-step receiver delays (interpolated reading; null: rounded)
    double* vstate;           // inadmissible leaves: [soe][ns] per leaf
    const double* tail;       // inadmissible leaves: [soe][ns][nr] coefficients per leaf (FP64: the
                              // fitted coefficients partly cancel, so they are not rounded to FP32)
};

__device__ __forceinline__ int pmod(long long a, int L) {
    long long r = a % L;
    return (int)(r < 0 ? r + L : r);
}

template <class T>
__device__ __forceinline__ int step_index(const StepArgs<T>& a) {
    return a.n_dev ? *a.n_dev : a.n;
}

__global__ void advance_step_kernel(int* n_dev) { *n_dev += 1; }

__global__ void set_step_kernel(int* n_dev, int v) { *n_dev = v; }

template <class T>
__global__ void push_kernel(StepArgs<T> a) {
    const int n = step_index(a);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.N) return;
    if (!a.D_in) {   // rupture predictor: the unknown slip rate of this step is held at zero
        a.Dring[(size_t)pmod(n, a.WD) * a.N + p] = 0.0;
        return;
    }
    const double d = a.D_in[(a.n_dev ? (long long)(n - a.n_base) * a.io_stride : 0) + a.perm[p]];
    a.Dring[(size_t)pmod(n, a.WD) * a.N + p] = d;
    // compensated running sum of the slip (units of dt)
    const double y = d - a.Ccomp[p];
    const double c0 = a.C[p];
    const double t = c0 + y;
    a.Ccomp[p] = (t - c0) - y;
    a.C[p] = t;
    a.Cring[(size_t)pmod(n, a.WC) * a.N + p] = t;
}

template <class T>
__global__ void fir_kernel(StepArgs<T> a) {
    const int n = step_index(a);
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.n_fir) return;
    const SbDev sb = a.sbs[a.fir_sb[q]];
    const int jl = a.fir_j[q];
    const int col = sb.s0 + jl;
    double s = 0.0;
    const int taps = min(sb.taps, n + 1);
    for (int m = 0; m < taps; ++m)
        s += (double)a.fac[sb.h + (long long)m * sb.ns + jl] * a.Dring[(size_t)pmod(n - m, a.WD) * a.N + col];
    a.dhat[sb.dhat + jl] = s;
}

template <class T>
__global__ void scatter_kernel(StepArgs<T> a) {
    const int n = step_index(a);
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.n_scat) return;
    const SbDev sb = a.sbs[a.scat_sb[q]];
    const int run = a.scat_run[q];
    const int l = a.scat_l[q];
    const int delay = a.run_delay[run];
    const int st = a.run_start[run];
    const int len = a.run_len[run];
    const int slot = pmod((long long)n + delay, sb.L);
    const size_t dslot = (size_t)pmod(n, a.WD) * a.N;
    double s = 0.0;
    for (int u = 0; u < len; ++u) {
        const int jl = a.src_order[st + u];
        double v;
        if (sb.kind == SB_F) v = a.dhat[sb.dhat + jl];
        else if (sb.kind == SB_S) v = a.dt * a.C[sb.s0 + jl];
        else v = a.Dring[dslot + sb.s0 + jl];
        s += (double)a.fac[sb.g + (long long)jl * sb.rank + l] * v;
    }
    double* r = a.ring + sb.ring + (long long)slot * sb.rank + l;   // ring layout [slot][rank]
    *r = delay == sb.maxdelay ? s : *r + s;   // the newest slot starts fresh
}

// one warp per (transient block, rank index)
template <class T>
__global__ void trconv_kernel(StepArgs<T> a) {
    const int n = step_index(a);
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= a.n_tr) return;
    const SbDev sb = a.sbs[a.tr_sb[q]];
    const int l = a.tr_l[q];
    const long long t0 = (long long)n - sb.mindm;
    const double* Y = a.ring + sb.ring + l;
    double z = 0.0;
    for (int m = lane; m < sb.taps; m += 32)
        z += (double)a.fac[sb.h + m] * Y[(long long)pmod(t0 - m, sb.L) * sb.rank];
    if (lane < sb.soe) {
        // tail beyond the exact taps: U_q(t) = rho_q U_q(t - 1) + Y(t - taps), z += c_q U_q(t)
        double* u = a.ustate + sb.ustate + (long long)l * sb.soe + lane;
        const double un = a.rho[lane] * *u + Y[(long long)pmod(t0 - sb.taps, sb.L) * sb.rank];
        *u = un;
        z += a.trcoef[sb.trc + lane] * un;
    }
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) a.zring[sb.zring + (long long)pmod(t0, sb.LZ) * sb.rank + l] = z;
}

// ---- bulk-async copy + mbarrier helpers (PTX)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned phase) {
    const unsigned a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(a), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Near field: one CTA per work item (leaf, k in [k0, k1)).  The item's coefficients are one
// contiguous block [k][sl]; thread 0 streams it into a kStages-deep ring of shared-memory stages
// with cp.async.bulk + mbarrier, all four warps consume: warp w takes every 4th slice of a
// stage, lane i owns receiver i, the slip rates D_{n-k, j} are broadcast by shuffle.  Products
// and the sum over one item are formed in the storage type T; items are combined in FP64.
template <class T>
__global__ void __launch_bounds__(kNearThreads, 3) near_kernel(StepArgs<T> a) {
    const int n = step_index(a);
    extern __shared__ __align__(128) unsigned char stage_mem[];
    __shared__ __align__(8) unsigned long long bar[kStages];
    __shared__ double red[kNearThreads / 32][32];
    const int item = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 it = a.items[item];
    const NearDev L = a.near[it.x];
    const int k0 = it.y;
    const int nsl = min(it.z, n + 1) - k0;              // slices needed at this step
    const int per = max(1, kStageBytes / (L.sl * (int)sizeof(T)));
    const int nst = nsl > 0 ? (nsl + per - 1) / per : 0;  // stage loads
    T* sd = (T*)(stage_mem + kStages * kStageBytes);      // [kChunk][32] slip rates D_{n-k, j}
    T acc = (T)0;
    bool failed = false;
    if (nst > 0) {
        const T* src = a.tensor + L.tensor + (long long)k0 * L.sl;
        if (threadIdx.x == 0) {
            for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
            mbar_fence_init();
            for (int q = 0; q < min(kStages, nst); ++q) {
                const int cnt = min(per, nsl - q * per);
                const unsigned bytes = (unsigned)(cnt * L.sl * sizeof(T));
                mbar_expect_tx(&bar[q], bytes);
                bulk_g2s(stage_mem + q * kStageBytes, src + (long long)q * per * L.sl, bytes, &bar[q]);
            }
        }
        // slip-rate history of the item's sources, while the first stages are in flight
        for (int e = threadIdx.x; e < nsl * 32; e += kNearThreads) {
            const int kk = e >> 5, j = e & 31;
            sd[e] = j < L.ns ? (T)a.Dring[(size_t)pmod(n - (k0 + kk), a.WD) * a.N + L.s0 + j] : (T)0;
        }
        __syncthreads();
        for (int q = 0; q < nst; ++q) {
            const int s = q % kStages;
            const bool ok = mbar_wait_bounded(&bar[s], (unsigned)((q / kStages) & 1));
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            const T* buf = (const T*)(stage_mem + s * kStageBytes);
            const int cnt = min(per, nsl - q * per);
            if (lane < L.nr) {
                for (int kk = warp; kk < cnt; kk += kNearThreads / 32) {
                    const T* tile = buf + kk * L.sl + lane;
                    const T* d = sd + (q * per + kk) * 32;
                    T s0 = (T)0, s1 = (T)0;
                    int j = 0;
                    for (; j + 1 < L.ns; j += 2) {
                        s0 += tile[j * L.nr] * d[j];
                        s1 += tile[(j + 1) * L.nr] * d[j + 1];
                    }
                    if (j < L.ns) s0 += tile[j * L.nr] * d[j];
                    acc += s0 + s1;
                }
            }
            __syncthreads();
            const int nq = q + kStages;
            if (threadIdx.x == 0 && nq < nst) {
                fence_proxy_async();
                const int c2 = min(per, nsl - nq * per);
                const unsigned bytes = (unsigned)(c2 * L.sl * sizeof(T));
                mbar_expect_tx(&bar[s], bytes);
                bulk_g2s(stage_mem + s * kStageBytes, src + (long long)nq * per * L.sl, bytes, &bar[s]);
            }
        }
    }
    if (failed) {
        if (threadIdx.x == 0) atomicExch(a.err, 1);
        // give the copies still in flight a bounded chance to land before the CTA exits
        for (int s = 0; s < kStages; ++s) (void)mbar_wait_bounded(&bar[s], 0u);
        return;
    }
    double accd = (double)acc;
    if (k0 == 0 && warp == 0 && n - L.W >= 0) {
        const long long t = (long long)n - L.W;
        const double cv = lane < L.ns ? a.Cring[(size_t)pmod(t, a.WC) * a.N + L.s0 + lane] : 0.0;
        for (int j = 0; j < L.ns; ++j) {
            const double cj = __shfl_sync(0xffffffffu, cv, j);
            if (lane < L.nr) accd += a.stat[L.stat + j * L.nr + lane] * cj;
        }
    }
    if (k0 == 0 && L.tail >= 0) {
        // exponential tail beyond the window (extension): V_qj(n) = rho_q V_qj(n-1) + D_{j,n-W},
        // T_i += sum_qj c_qji V_qj(n); the state update is done once per step, by this CTA
        const long long t = (long long)n - L.W;
        const size_t slot = (size_t)pmod(t, a.WD) * a.N;
        for (int e = threadIdx.x; e < a.soe * L.ns; e += kNearThreads) {
            const int q = e / L.ns, j = e - q * L.ns;
            double* v = a.vstate + L.vstate + e;
            const double vn = a.rho[q] * *v + (t >= 0 ? a.Dring[slot + L.s0 + j] : 0.0);
            *v = vn;
        }
        __syncthreads();
        if (lane < L.nr)
            for (int q = warp; q < a.soe; q += kNearThreads / 32) {
                const double* c = a.tail + L.tail + (long long)q * L.ns * L.nr + lane;
                const double* v = a.vstate + L.vstate + (long long)q * L.ns;
                double s = 0.0;
                for (int j = 0; j < L.ns; ++j) s += c[j * L.nr] * v[j];
                accd += s;
            }
    }
    red[warp][lane] = accd;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int w = 0; w < kNearThreads / 32; ++w) s += red[w][lane];
        a.partial[(size_t)item * 32 + lane] = s;
    }
}

// Eq. 39, one thread per (block, receiver) entry, blocks in order: f_{l,i} Tbar'_l[n - dm_i]
template <class T>
__global__ void far_eval_kernel(StepArgs<T> a) {
    const int n = step_index(a);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.n_ent) return;
    const SbDev sb = a.sbs[a.e_sb[e]];
    const int il = a.e_il[e];
    const long long t = (long long)n - a.ints[sb.dm + il];
    const T* f = a.fac + sb.f + (long long)il * sb.rank;
    double s = 0.0;
    const bool tr = sb.kind == SB_TR;
    const double* base = tr ? a.zring + sb.zring : a.ring + sb.ring;
    const int len = tr ? sb.LZ : sb.L;
    const double* r = base + (long long)pmod(t, len) * sb.rank;
    if (a.phi) {   // exact delay dm_i + phi_i: linear interpolation with the next older step
        const double ph = a.phi[sb.phi + il];
        const double* r1 = base + (long long)pmod(t - 1, len) * sb.rank;
        for (int l = 0; l < sb.rank; ++l) s += (double)f[l] * ((1.0 - ph) * r[l] + ph * r1[l]);
    } else {
        for (int l = 0; l < sb.rank; ++l) s += (double)f[l] * r[l];
    }
    a.fval[a.e_pos[e]] = s;
}

// one warp per receiver: sum of its far entries and near-field partials, fixed order
template <class T>
__global__ void gather_kernel(StepArgs<T> a) {
    const int n = step_index(a);
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= a.N) return;
    double s = 0.0;
    for (int e = a.g_ptr[p] + lane; e < a.g_ptr[p + 1]; e += 32) s += a.fval[e];
    for (int e = a.np_ptr[p] + lane; e < a.np_ptr[p + 1]; e += 32) s += a.partial[a.np_idx[e]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) a.T_out[(a.n_dev ? (long long)(n - a.n_base) * a.io_stride : 0) + a.perm[p]] = s;
}

// Local friction solve (geometry order): T_pred holds the traction change with D_n = 0.
struct FrictionDev {
    const double* tau0;
    const double* k0;      // instantaneous self coefficient K_{ii,0} (< 0)
    double* slip;
    double sigma_n, mu_s, mu_d, Dc, dt;
};

__global__ void friction_kernel(FrictionDev f, int N, double* D, double* T) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const double tau = f.tau0[e] + T[e];
    const double u = f.slip[e];
    const double w = u < f.Dc ? u / f.Dc : 1.0;
    const double strength = f.sigma_n * (f.mu_s - (f.mu_s - f.mu_d) * w);
    const double eta = -f.k0[e];
    const double v = tau > strength ? (tau - strength) / eta : 0.0;
    D[e] = v;
    T[e] = tau + f.k0[e] * v;
    f.slip[e] = u + v * f.dt;
}

// ------------------------------------------------------------------------------------------
// plan-time device kernels: near-field windows and exact-kernel tensors

struct GeoDev {
    const double *px, *py, *nx, *ny, *ax, *ay, *tx, *ty, *len;
};

__device__ __forceinline__ Seg dev_seg(const GeoDev& g, int p) {
    Seg s;
    s.ax = g.ax[p];
    s.ay = g.ay[p];
    s.tx = g.tx[p];
    s.ty = g.ty[p];
    s.len = g.len[p];
    return s;
}

// m_S(i, j) = 1 + last k < M with |K_ijk - Kstat_ij dt| >= thr (App. H), 0 if none; M if thr == 0
__global__ void near_ms_kernel(GeoDev g, const int* pr, const int* pnr, const int* ps, const int* pns,
                               const long long* pair0, long long npairs, int nleaf, int M, double dt,
                               double mu, double c, double thr, int* ms) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    int lo = 0, hi = nleaf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pair0[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const long long loc = q - pair0[lo];
    const int il = (int)(loc / pns[lo]), jl = (int)(loc % pns[lo]);
    const int pi = pr[lo] + il, pj = ps[lo] + jl;
    if (thr <= 0.0) {
        ms[q] = M;
        return;
    }
    const Seg s = dev_seg(g, pj);
    int res = 0;
    for (int k = M - 1; k >= 0; --k) {
        const Stress2 v = stress_tail(g.px[pi], g.py[pi], s, (double)k * dt, (double)(k + 1) * dt, mu, c);
        const double tval = g.nx[pi] * v.x + g.ny[pi] * v.y;
        if (fabs(tval) >= thr) {
            res = k + 1;
            break;
        }
    }
    ms[q] = res;
}

// coefficients [k][j][i] for k < W: exact kernel below m_S(i, j), static * dt above
template <class T>
__global__ void near_fill_kernel(GeoDev g, NearDev L, const int* ms_leaf, double dt, double mu, double c,
                                 T* tensor, double* stat) {
    const long long total = (long long)L.W * L.ns * L.nr;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int il = (int)(q % L.nr);
        const long long r = q / L.nr;
        const int jl = (int)(r % L.ns);
        const int k = (int)(r / L.ns);
        const int pi = L.r0 + il, pj = L.s0 + jl;
        const Seg s = dev_seg(g, pj);
        double v;
        const int mS = ms_leaf[il * L.ns + jl];
        if (k < mS) {
            const Stress2 w = stress_jump(g.px[pi], g.py[pi], s, (double)k * dt, (double)(k + 1) * dt, mu, c);
            v = g.nx[pi] * w.x + g.ny[pi] * w.y;
        } else {
            const Stress2 w = stress_static(g.px[pi], g.py[pi], s, mu);
            v = (g.nx[pi] * w.x + g.ny[pi] * w.y) * dt;
        }
        tensor[L.tensor + (long long)k * L.sl + (q % ((long long)L.ns * L.nr))] = (T)v;
        if (k == 0) {
            const Stress2 w = stress_static(g.px[pi], g.py[pi], s, mu);
            stat[L.stat + (long long)jl * L.nr + il] = (g.nx[pi] * w.x + g.ny[pi] * w.y) * dt;
        }
    }
}

// projections g_q = sum_{k' < M - W} rho_q^k' (K_ij,W+k' - Kstat_ij dt) of every pair of the
// inadmissible leaves with a tail, on the exponential basis (least-squares right-hand sides);
// one thread per pair, pairs of leaf l at [pair0[l], pair0[l + 1])
__global__ void near_soe_proj_kernel(GeoDev g, const NearDev* leaves, const long long* pair0, int nleaf,
                                     long long npairs, int M, double dt, double mu, double c, int Q,
                                     const double* rho, double* out) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    int lo = 0, hi = nleaf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pair0[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const NearDev L = leaves[lo];
    const long long loc = q - pair0[lo];
    const int il = (int)(loc / L.ns), jl = (int)(loc % L.ns);
    const int pi = L.r0 + il, pj = L.s0 + jl;
    const Seg s = dev_seg(g, pj);
    double acc[kMaxSoe], pw[kMaxSoe];
#pragma unroll
    for (int r = 0; r < kMaxSoe; ++r) {
        acc[r] = 0.0;
        pw[r] = 1.0;
    }
    for (int k = L.W; k < M; ++k) {
        const Stress2 v = stress_tail(g.px[pi], g.py[pi], s, (double)k * dt, (double)(k + 1) * dt, mu, c);
        const double y = g.nx[pi] * v.x + g.ny[pi] * v.y;
#pragma unroll
        for (int r = 0; r < kMaxSoe; ++r)
            if (r < Q) {
                acc[r] += pw[r] * y;
                pw[r] *= rho[r];
            }
    }
#pragma unroll
    for (int r = 0; r < kMaxSoe; ++r)
        if (r < Q) out[(size_t)q * Q + r] = acc[r];
}

// ------------------------------------------------------------------------------------------
// the plan object

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct fdph_plan_s {
    int device = 0;
    int precision = FDPH_FP64;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int N = 0, M = 0, n = 0, WD = 1, WC = 1;
    double dt = 0;
    HostPlan hp;
    fdph_stats st;
    // device memory
    std::vector<void*> allocs;
    int* perm = nullptr;
    SbDev* sbs = nullptr;
    void* fac = nullptr;
    int *ints = nullptr, *run_delay = nullptr, *run_start = nullptr, *run_len = nullptr, *src_order = nullptr;
    int *scat_l = nullptr, *e_sb = nullptr, *e_il = nullptr, *e_pos = nullptr;
    double* fval = nullptr;
    int *scat_sb = nullptr, *scat_run = nullptr, *fir_sb = nullptr, *fir_j = nullptr, *tr_sb = nullptr,
        *tr_l = nullptr, *g_ptr = nullptr, *g_sb = nullptr, *g_il = nullptr;
    NearDev* near = nullptr;
    int4* items = nullptr;
    void* tensor = nullptr;
    double* stat = nullptr;
    int *np_ptr = nullptr, *np_idx = nullptr;
    int* err = nullptr;
    double* rho = nullptr;
    void* tail = nullptr;
    // rupture state
    bool rupture = false;
    FrictionDev fr;
    double *ustate = nullptr, *vstate = nullptr, *trcoef = nullptr, *phi = nullptr;
    // state
    double *Dring = nullptr, *Cring = nullptr, *C = nullptr, *Ccomp = nullptr;
    double *ring = nullptr, *zring = nullptr, *dhat = nullptr, *partial = nullptr;
    size_t state_bytes = 0;
    // host staging for fdph_step_host
    double *hD = nullptr, *hT = nullptr, *dD = nullptr, *dT = nullptr;
    // per-kernel event timing
    bool prof = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
    double prof_ms[FDPH_NUM_KERNELS] = {0};
    int64_t prof_n[FDPH_NUM_KERNELS] = {0};
    // graph of one step for fdph_run (replayed with the step index in n_dev)
    cudaGraphExec_t graph = nullptr;
    int* n_dev = nullptr;
};

template <class T>
static int dalloc(fdph_plan_t P, T** out, size_t count) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        return FDPH_E_OOM;
    }
    P->allocs.push_back(p);
    *out = (T*)p;
    return FDPH_OK;
}

template <class T>
static int upload(fdph_plan_t P, T** out, const std::vector<T>& v) {
    int rc = dalloc(P, out, v.size());
    if (rc) return rc;
    if (!v.empty()) FDPH_CUDA(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FDPH_OK;
}

template <class T>
static StepArgs<T> make_args(fdph_plan_t P, const double* D, double* T_) {
    StepArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.n = P->n;
    a.n_dev = nullptr;
    a.N = P->N;
    a.WD = P->WD;
    a.WC = P->WC;
    a.dt = P->dt;
    a.D_in = D;
    a.T_out = T_;
    a.perm = P->perm;
    a.Dring = P->Dring;
    a.Cring = P->Cring;
    a.C = P->C;
    a.Ccomp = P->Ccomp;
    a.sbs = P->sbs;
    a.fac = (const T*)P->fac;
    a.ints = P->ints;
    a.run_delay = P->run_delay;
    a.run_start = P->run_start;
    a.run_len = P->run_len;
    a.src_order = P->src_order;
    a.scat_sb = P->scat_sb;
    a.scat_run = P->scat_run;
    a.scat_l = P->scat_l;
    a.e_sb = P->e_sb;
    a.e_il = P->e_il;
    a.e_pos = P->e_pos;
    a.n_ent = (int)P->hp.e_sb.size();
    a.fval = P->fval;
    a.n_scat = (int)P->hp.scat_sb.size();
    a.fir_sb = P->fir_sb;
    a.fir_j = P->fir_j;
    a.n_fir = (int)P->hp.fir_sb.size();
    a.tr_sb = P->tr_sb;
    a.tr_l = P->tr_l;
    a.n_tr = (int)P->hp.tr_sb.size();
    a.g_ptr = P->g_ptr;
    a.g_sb = P->g_sb;
    a.g_il = P->g_il;
    a.ring = P->ring;
    a.zring = P->zring;
    a.dhat = P->dhat;
    a.near = P->near;
    a.items = P->items;
    a.n_items = (int)P->hp.items.size();
    a.tensor = (const T*)P->tensor;
    a.stat = P->stat;
    a.partial = P->partial;
    a.np_ptr = P->np_ptr;
    a.np_idx = P->np_idx;
    a.err = P->err;
    a.soe = P->hp.soe;
    a.rho = P->rho;
    a.ustate = P->ustate;
    a.trcoef = P->trcoef;
    a.phi = P->hp.interp ? P->phi : nullptr;
    a.vstate = P->vstate;
    a.tail = (const double*)P->tail;
    return a;
}

static inline int blocks(long long n, int t) { return (int)std::max<long long>(1, (n + t - 1) / t); }

struct ProfScope {
    fdph_plan_t P;
    int id;
    cudaEvent_t b = nullptr, e = nullptr;
    ProfScope(fdph_plan_t P_, int id_);
    ~ProfScope();
};

template <class T>
static void enqueue_step(fdph_plan_t P, const StepArgs<T>& a, cudaStream_t s) {
    { ProfScope ps(P, 0); push_kernel<T><<<blocks(a.N, 256), 256, 0, s>>>(a); }
    if (a.n_fir) { ProfScope ps(P, 1); fir_kernel<T><<<blocks(a.n_fir, 128), 128, 0, s>>>(a); }
    if (a.n_scat) { ProfScope ps(P, 2); scatter_kernel<T><<<blocks(a.n_scat, 128), 128, 0, s>>>(a); }
    if (a.n_tr) { ProfScope ps(P, 3); trconv_kernel<T><<<blocks((long long)a.n_tr * 32, 128), 128, 0, s>>>(a); }
    if (a.n_items) {
        ProfScope ps(P, 4);
        near_kernel<T><<<a.n_items, kNearThreads, kStages * kStageBytes + kChunk * 32 * sizeof(T), s>>>(a);
    }
    {
        ProfScope ps(P, 5);
        if (a.n_ent) far_eval_kernel<T><<<blocks(a.n_ent, 128), 128, 0, s>>>(a);
        gather_kernel<T><<<blocks((long long)a.N * 32, 128), 128, 0, s>>>(a);
    }
}

template <class T>
static int launch_step(fdph_plan_t P, const double* D, double* Tout) {
    StepArgs<T> a = make_args<T>(P, D, Tout);
    enqueue_step<T>(P, a, P->stream);
    FDPH_CUDA(cudaGetLastError());
    return FDPH_OK;
}

// `steps` steps as replays of one captured step graph; kernels read the step index from n_dev
// (advanced by the last node) and offset D / T by one row per step
template <class T>
static int run_graph(fdph_plan_t P, int steps, const double* D, double* Tout) {
    if (!P->n_dev) {
        int rc = dalloc(P, &P->n_dev, 1);
        if (rc) return rc;
    }
    cudaStream_t s = P->stream;
    StepArgs<T> a = make_args<T>(P, D, Tout);
    a.n_dev = P->n_dev;
    a.n_base = P->n;
    a.io_stride = P->N;
    set_step_kernel<<<1, 1, 0, s>>>(P->n_dev, P->n);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    FDPH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    enqueue_step<T>(P, a, s);
    advance_step_kernel<<<1, 1, 0, s>>>(P->n_dev);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
        set_error(std::string("graph capture: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    for (int k = 0; k < steps; ++k) {
        e = cudaGraphLaunch(ex, s);
        if (e != cudaSuccess) break;
    }
    cudaGraphExecDestroy(ex);
    if (e != cudaSuccess) {
        set_error(std::string("graph launch: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    P->n += steps;
    return FDPH_OK;
}

ProfScope::ProfScope(fdph_plan_t P_, int id_) : P(P_), id(id_) {
    if (!P->prof) return;
    cudaEventCreate(&b);
    cudaEventCreate(&e);
    cudaEventRecord(b, P->stream);
}

ProfScope::~ProfScope() {
    if (!P->prof || !b) return;
    cudaEventRecord(e, P->stream);
    P->prof_ev.push_back({id, {b, e}});
}

static void prof_drain(fdph_plan_t P) {
    for (auto& q : P->prof_ev) {
        float ms = 0.f;
        cudaEventSynchronize(q.second.second);
        cudaEventElapsedTime(&ms, q.second.first, q.second.second);
        P->prof_ms[q.first] += ms;
        P->prof_n[q.first] += 1;
        cudaEventDestroy(q.second.first);
        cudaEventDestroy(q.second.second);
    }
    P->prof_ev.clear();
}

// after a stream synchronisation: report a bounded device wait that gave up
static int check_device_error(fdph_plan_t P) {
    int e = 0;
    if (!P->err) return FDPH_OK;
    FDPH_CUDA(cudaMemcpy(&e, P->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        set_error("a bounded mbarrier wait in the near-field kernel gave up; results of the step are invalid");
        cudaMemset(P->err, 0, sizeof(int));
        return FDPH_E_TIMEOUT;
    }
    return FDPH_OK;
}

static int step_impl(fdph_plan_t P, const double* D, double* T_) {
    int rc = P->precision == FDPH_FP32 ? launch_step<float>(P, D, T_) : launch_step<double>(P, D, T_);
    if (rc == FDPH_OK) P->n += 1;
    return rc;
}

template <class T>
static int launch_rupture_step(fdph_plan_t P, double* D, double* Tout) {
    StepArgs<T> a = make_args<T>(P, nullptr, Tout);
    cudaStream_t s = P->stream;
    { ProfScope ps(P, 0); push_kernel<T><<<blocks(a.N, 256), 256, 0, s>>>(a); }          // D_n = 0
    if (a.n_tr) { ProfScope ps(P, 3); trconv_kernel<T><<<blocks((long long)a.n_tr * 32, 128), 128, 0, s>>>(a); }
    if (a.n_items) {
        ProfScope ps(P, 4);
        near_kernel<T><<<a.n_items, kNearThreads, kStages * kStageBytes + kChunk * 32 * sizeof(T), s>>>(a);
    }
    {
        ProfScope ps(P, 5);
        if (a.n_ent) far_eval_kernel<T><<<blocks(a.n_ent, 128), 128, 0, s>>>(a);
        gather_kernel<T><<<blocks((long long)a.N * 32, 128), 128, 0, s>>>(a);
    }
    friction_kernel<<<blocks(a.N, 256), 256, 0, s>>>(P->fr, a.N, D, Tout);
    a.D_in = D;                                                                                // commit D_n
    { ProfScope ps(P, 0); push_kernel<T><<<blocks(a.N, 256), 256, 0, s>>>(a); }
    if (a.n_fir) { ProfScope ps(P, 1); fir_kernel<T><<<blocks(a.n_fir, 128), 128, 0, s>>>(a); }
    if (a.n_scat) { ProfScope ps(P, 2); scatter_kernel<T><<<blocks(a.n_scat, 128), 128, 0, s>>>(a); }
    FDPH_CUDA(cudaGetLastError());
    return FDPH_OK;
}

template <class T>
static int build_near(fdph_plan_t P, const PlanInputs& in) {
    HostPlan& hp = P->hp;
    const int nl = (int)hp.near_r0.size();
    GeoDev g;
    double *px, *py, *nx, *ny, *ax, *ay, *tx, *ty, *ln;
    int rc;
    if ((rc = upload(P, &px, hp.px)) || (rc = upload(P, &py, hp.py)) || (rc = upload(P, &nx, hp.pnx)) ||
        (rc = upload(P, &ny, hp.pny)) || (rc = upload(P, &ax, hp.sax)) || (rc = upload(P, &ay, hp.say)) ||
        (rc = upload(P, &tx, hp.stx)) || (rc = upload(P, &ty, hp.sty)) || (rc = upload(P, &ln, hp.slen)))
        return rc;
    g.px = px; g.py = py; g.nx = nx; g.ny = ny; g.ax = ax; g.ay = ay; g.tx = tx; g.ty = ty; g.len = ln;
    std::vector<long long> pair0(nl + 1, 0);
    for (int l = 0; l < nl; ++l) pair0[l + 1] = pair0[l] + (long long)hp.near_nr[l] * hp.near_ns[l];
    const long long npairs = pair0[nl];
    std::vector<int32_t> W(nl, 0);
    std::vector<int> ms;
    int *d_ms = nullptr, *d_r = nullptr, *d_nr = nullptr, *d_s = nullptr, *d_ns = nullptr;
    long long* d_p0 = nullptr;
    if (nl > 0) {
        if ((rc = dalloc(P, &d_ms, npairs)) || (rc = upload(P, &d_r, hp.near_r0)) ||
            (rc = upload(P, &d_nr, hp.near_nr)) || (rc = upload(P, &d_s, hp.near_s0)) ||
            (rc = upload(P, &d_ns, hp.near_ns)))
            return rc;
        std::vector<long long> p0(pair0.begin(), pair0.end() - 1);
        if ((rc = upload(P, &d_p0, p0))) return rc;
        const double thr = in.eps_st * in.mu / (2.0 * in.cs);
        near_ms_kernel<<<blocks(npairs, 128), 128>>>(g, d_r, d_nr, d_s, d_ns, d_p0, npairs, nl, in.M, in.dt,
                                                      in.mu, in.cs, thr, d_ms);
        FDPH_CUDA(cudaGetLastError());
        ms.resize(npairs);
        FDPH_CUDA(cudaMemcpy(ms.data(), d_ms, npairs * sizeof(int), cudaMemcpyDeviceToHost));
        for (int l = 0; l < nl; ++l)
            for (long long q = pair0[l]; q < pair0[l + 1]; ++q) W[l] = std::max(W[l], ms[q]);
    }
    std::vector<char> has_tail(nl, 0);
    if (in.soe > 0) {
        // exponential tails: the window also covers every pair's wave passage (both end-point
        // fronts + n_c steps); the exact kernel is kept for all pairs up to the leaf's window
        const double cdt = in.cs * in.dt;
        for (int l = 0; l < nl; ++l) {
            for (int il = 0; il < hp.near_nr[l]; ++il) {
                const int pi = hp.near_r0[l] + il;
                for (int jl = 0; jl < hp.near_ns[l]; ++jl) {
                    const int pj = hp.near_s0[l] + jl;
                    double dx = hp.px[pi] - hp.sax[pj], dy = hp.py[pi] - hp.say[pj];
                    const double da = sqrt(dx * dx + dy * dy);
                    dx = hp.px[pi] - hp.sbx[pj];
                    dy = hp.py[pi] - hp.sby[pj];
                    const double db = sqrt(dx * dx + dy * dy);
                    const int pass = (int)ceil(std::max(da, db) / cdt) + hp.tree.nc;
                    W[l] = std::max(W[l], pass);
                }
            }
            if (in.M - W[l] < soe_min_len(W[l])) W[l] = in.M;
            else has_tail[l] = 1;
            for (long long q = pair0[l]; q < pair0[l + 1]; ++q) ms[q] = W[l];   // exact over the window
        }
        FDPH_CUDA(cudaMemcpy(d_ms, ms.data(), npairs * sizeof(int), cudaMemcpyHostToDevice));
    }
    // work-item length: the longest chunk (kChunk) that still yields about four waves of
    // resident CTAs (152 SMs x 3), so small problems (the plain config) fill the device too
    long long slices = 0;
    for (int l = 0; l < nl; ++l) slices += std::max(W[l], 1);
    int chunk = kChunk;
    while (chunk > 8 && slices / chunk < 4LL * 152 * 3) chunk /= 2;
    finish_near_layout(hp, W, has_tail, chunk);
    std::vector<NearDev> nd(nl);
    for (int l = 0; l < nl; ++l) {
        const NearLeaf& L = hp.near[l];
        nd[l] = {L.r0, L.nr, L.s0, L.ns, L.W, L.sl, (long long)L.tensor, (long long)L.stat, (long long)L.tail,
                 (long long)L.vstate};
    }
    if ((rc = upload(P, &P->near, nd))) return rc;
    T* tens = nullptr;
    if ((rc = dalloc(P, &tens, hp.near_tensor_len)) || (rc = dalloc(P, &P->stat, hp.near_stat_len))) return rc;
    P->tensor = tens;
    if (hp.near_tensor_len) FDPH_CUDA(cudaMemset(tens, 0, hp.near_tensor_len * sizeof(T)));  // slice padding
    for (int l = 0; l < nl; ++l) {
        const long long tot = (long long)nd[l].W * nd[l].ns * nd[l].nr;
        if (tot == 0 && nd[l].ns * nd[l].nr == 0) continue;
        // static tile is written by k == 0 entries; a leaf with W == 0 still needs it
        NearDev L = nd[l];
        if (L.W == 0) {
            // temporarily fill one k-slice into a scratch to get the static tile
            T* tmp = nullptr;
            if ((rc = dalloc(P, &tmp, (size_t)L.ns * L.nr))) return rc;
            NearDev L1 = L;
            L1.W = 1;
            L1.tensor = 0;
            L1.sl = L.ns * L.nr;
            near_fill_kernel<T><<<blocks((long long)L.ns * L.nr, 128), 128>>>(g, L1, d_ms + pair0[l], in.dt,
                                                                            in.mu, in.cs, tmp, P->stat);
        } else {
            near_fill_kernel<T><<<std::min<long long>(blocks(tot, 256), 4096), 256>>>(
                g, L, d_ms + pair0[l], in.dt, in.mu, in.cs, tens, P->stat);
        }
        FDPH_CUDA(cudaGetLastError());
    }
    if (in.soe > 0 && hp.near_tail_len > 0) {
        // all tail leaves in one launch, then one Cholesky solve per leaf on the host
        std::vector<NearDev> tl;
        std::vector<int> tl_id;
        std::vector<long long> tp0{0};
        for (int l = 0; l < nl; ++l)
            if (has_tail[l]) {
                tl.push_back(nd[l]);
                tl_id.push_back(l);
                tp0.push_back(tp0.back() + (long long)nd[l].nr * nd[l].ns);
            }
        const long long ntp = tp0.back();
        NearDev* d_tl = nullptr;
        long long* d_tp0 = nullptr;
        double* d_g = nullptr;
        std::vector<long long> tp0s(tp0.begin(), tp0.end() - 1);
        if ((rc = upload(P, &d_tl, tl)) || (rc = upload(P, &d_tp0, tp0s)) || (rc = dalloc(P, &d_g, (size_t)ntp * in.soe)))
            return rc;
        near_soe_proj_kernel<<<blocks(ntp, 128), 128>>>(g, d_tl, d_tp0, (int)tl.size(), ntp, in.M, in.dt, in.mu, in.cs,
                                                        in.soe, P->rho, d_g);
        FDPH_CUDA(cudaGetLastError());
        std::vector<double> gh((size_t)ntp * in.soe), ch((size_t)ntp * in.soe);
        FDPH_CUDA(cudaMemcpy(gh.data(), d_g, gh.size() * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<double> tail_h(hp.near_tail_len);
#pragma omp parallel for schedule(dynamic, 8)
        for (long t = 0; t < (long)tl.size(); ++t) {
            const NearDev& L = tl[t];
            const size_t b = (size_t)tp0[t] * in.soe;
            soe_solve(hp.rho, in.M - L.W, gh.data() + b, ch.data() + b, L.nr * L.ns);
            for (int il = 0; il < L.nr; ++il)
                for (int jl = 0; jl < L.ns; ++jl)
                    for (int q = 0; q < in.soe; ++q)
                        tail_h[L.tail + ((size_t)q * L.ns + jl) * L.nr + il] =
                            ch[b + ((size_t)il * L.ns + jl) * in.soe + q];
        }
        double* dt_ = nullptr;
        if ((rc = upload(P, &dt_, tail_h))) return rc;
        P->tail = dt_;
    }
    std::vector<int4> it(hp.items.size());
    for (size_t q = 0; q < it.size(); ++q) it[q] = make_int4(hp.items[q].leaf, hp.items[q].k0, hp.items[q].k1, 0);
    if ((rc = upload(P, &P->items, it)) || (rc = upload(P, &P->np_ptr, hp.np_ptr)) ||
        (rc = upload(P, &P->np_idx, hp.np_idx)))
        return rc;
    FDPH_CUDA(cudaDeviceSynchronize());
    return FDPH_OK;
}

static void fill_stats(fdph_plan_t P) {
    HostPlan& hp = P->hp;
    fdph_stats& s = P->st;
    const double ps = P->precision == FDPH_FP32 ? 4.0 : 8.0;
    s.n = hp.n;
    s.M = hp.M;
    s.n_admissible = hp.n_adm;
    s.n_near = hp.n_near;
    s.n_subblocks = (int)hp.sbs.size();
    s.max_rank = hp.max_rank;
    s.mean_rank = hp.mean_rank;
    s.extra_steps = hp.tree.nc;
    s.max_window = hp.max_W;
    s.near_entries = hp.near_tensor_len;
    s.far_entries = hp.far_entries;
    // algorithmic bytes of one steady-state step
    double near_b = 0, far_b = 0, flops = 0;
    for (const NearLeaf& L : hp.near) {
        near_b += (double)L.W * L.ns * L.nr * ps + (double)L.ns * L.nr * 8.0;  // tensor + static tile
        near_b += (double)(L.W + 1) * L.ns * 8.0;                              // slip history read
        flops += 2.0 * ((double)L.W + 1) * L.ns * L.nr;
        if (L.tail >= 0) {                                                     // tail coefficients + states
            near_b += (double)hp.soe * L.ns * L.nr * ps + (double)hp.soe * L.ns * 16.0;
            flops += 2.0 * hp.soe * L.ns * (L.nr + 1.0);
        }
    }
    for (const SubBlock& sb : hp.sbs) {
        const double r = sb.rank;
        far_b += (sb.nr + sb.ns) * r * ps + (sb.nr + sb.ns) * 4.0;          // f, g, delays
        far_b += sb.nr * r * 8.0 + sb.nruns * r * 16.0;                     // ring reads / RMW
        flops += 2.0 * (sb.nr + sb.ns) * r;
        if (sb.kind == SB_F) {
            far_b += (double)sb.taps * sb.ns * (ps + 8.0) + sb.ns * 16.0;   // h, D history, Dhat
            flops += 2.0 * sb.taps * sb.ns;
        }
        if (sb.kind == SB_TR) {
            far_b += r * (sb.taps * 8.0 + sb.taps * ps + 8.0) + r * sb.soe * 24.0;
            flops += 2.0 * r * (sb.taps + 2.0 * sb.soe);
        }
    }
    const double push_b = hp.n * (8.0 + 8.0 + 32.0 + 8.0 + 4.0);           // D in, ring, C/comp, Cring, perm
    const double out_b = hp.n * (8.0 + 4.0) + (double)hp.np_idx.size() * 12.0;
    s.bytes_per_step = near_b + far_b + push_b + out_b;
    s.near_bytes_per_step = near_b;
    s.flops_per_step = flops;
    s.state_bytes = (long long)P->state_bytes;
    long long arena = 0;
    arena += (long long)(hp.fac.size() * ps) + hp.ints.size() * 4 + hp.sbs.size() * sizeof(SbDev);
    arena += (long long)(hp.near_tensor_len * ps) + hp.near_stat_len * 8 + (long long)(hp.near_tail_len * ps);
    s.arena_bytes = arena;
}

// ------------------------------------------------------------------------------------------
// C ABI

extern "C" {

void fdph_default_params(fdph_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->eta = 0.5;
    p->lmin = 0.0;
    p->eps_st = 1e-6;
    p->leaf_size = 32;
    p->extra_steps = -1;
    p->precision = FDPH_FP64;
    p->device = 0;
    p->cuda_stream = nullptr;
}

const char* fdph_strerror(int s) {
    switch (s) {
        case FDPH_OK: return "ok";
        case FDPH_E_ARG: return "invalid argument";
        case FDPH_E_OOM: return "out of memory";
        case FDPH_E_CAUSALITY: return "discretised causality violated (increase l_min/eta or reduce dt)";
        case FDPH_E_CUDA: return "CUDA error";
        case FDPH_E_TIMEOUT: return "device wait timed out";
        case FDPH_E_NAN: return "non-finite value";
        case FDPH_E_STATE: return "invalid plan state";
        default: return "unknown status";
    }
}

const char* fdph_last_error(void) { return g_last_error.c_str(); }

static int check_inputs(const fdph_geometry* g, const fdph_material* m, double dt, const fdph_params* p) {
    if (!g || !m || !g->xy || g->n <= 0 || !(dt > 0.0) || !(m->mu > 0.0) || !(m->cs > 0.0)) {
        set_error("geometry, material and dt must be given, n > 0, dt, mu, cs > 0");
        return FDPH_E_ARG;
    }
    if (p && (p->leaf_size < 1 || p->leaf_size > 32 || p->eta < 0.0 || p->eps_st < 0.0 ||
              (p->precision != FDPH_FP64 && p->precision != FDPH_FP32) ||
              (p->soe_terms != 0 && (p->soe_terms < 4 || p->soe_terms > kMaxSoe)))) {
        set_error("params: leaf_size in [1, 32], eta >= 0, eps_st >= 0, precision FP64 or FP32, "
                  "soe_terms 0 or in [4, 16]");
        return FDPH_E_ARG;
    }
    for (int k = 0; k < 4 * g->n; ++k)
        if (!std::isfinite(g->xy[k])) {
            set_error("geometry holds a non-finite coordinate");
            return FDPH_E_NAN;
        }
    for (int e = 0; e < g->n; ++e) {
        const double dx = g->xy[4 * e + 2] - g->xy[4 * e], dy = g->xy[4 * e + 3] - g->xy[4 * e + 1];
        if (dx * dx + dy * dy == 0.0) {
            set_error("element " + std::to_string(e) + " has zero length");
            return FDPH_E_ARG;
        }
    }
    return FDPH_OK;
}

static PlanInputs make_inputs(const fdph_material* m, double dt, int M, double eps, const fdph_params& p) {
    PlanInputs in;
    in.mu = m->mu;
    in.cs = m->cs;
    in.dt = dt;
    in.M = M;
    in.eps = eps;
    in.eta = p.eta;
    in.lmin = p.lmin;
    in.eps_st = p.eps_st;
    in.leaf = p.leaf_size;
    in.extra_steps = p.extra_steps;
    in.soe = p.soe_terms;
    in.interp = p.art_interp ? 1 : 0;
    return in;
}

int fdph_tree_export(const fdph_geometry* geometry, const fdph_material* material, double dt,
                     const fdph_params* params, int32_t* buf, int64_t cap, int64_t* len) {
    int rc = check_inputs(geometry, material, dt, params);
    if (rc) return rc;
    if (!len) return FDPH_E_ARG;
    fdph_params p;
    fdph_default_params(&p);
    if (params) p = *params;
    PlanInputs in = make_inputs(material, dt, 1, 0.0, p);
    Elements el = make_elements(geometry->n, geometry->xy);
    Tree tr;
    build_tree(el, in, tr);
    std::vector<int32_t> out;
    out.push_back(el.n);
    out.insert(out.end(), tr.perm.begin(), tr.perm.end());
    out.push_back((int32_t)tr.leaves.size());
    for (const Leaf& lf : tr.leaves) {
        const ClusterNode& tn = tr.nodes[lf.tau];
        const ClusterNode& sn = tr.nodes[lf.sig];
        out.push_back(lf.kind);
        out.push_back(tn.lo);
        out.push_back(tn.hi - tn.lo);
        out.push_back(sn.lo);
        out.push_back(sn.hi - sn.lo);
        if (lf.kind == 1) {
            ArtInts a = art_integers(el, tr, lf, in);
            if (a.causal < 1) {
                set_error("discretised causality violated");
                return FDPH_E_CAUSALITY;
            }
            out.insert(out.end(), a.dm.begin(), a.dm.end());
            out.insert(out.end(), a.mbar.begin(), a.mbar.end());
            out.insert(out.end(), a.Dm.begin(), a.Dm.end());
        }
    }
    *len = (int64_t)out.size();
    if (buf) {
        if (cap < (int64_t)out.size()) {
            set_error("buffer too small");
            return FDPH_E_ARG;
        }
        memcpy(buf, out.data(), out.size() * sizeof(int32_t));
    }
    return FDPH_OK;
}

int fdph_plan(const fdph_geometry* geometry, const fdph_material* material, double dt, int32_t M, double eps,
              const fdph_params* params, fdph_plan_t* out) {
    if (!out) return FDPH_E_ARG;
    *out = nullptr;
    int rc = check_inputs(geometry, material, dt, params);
    if (rc) return rc;
    if (M <= 0) {
        set_error("M must be positive");
        return FDPH_E_ARG;
    }
    const auto t0 = std::chrono::steady_clock::now();
    fdph_params p;
    fdph_default_params(&p);
    if (params) p = *params;
    fdph_plan_s* P = new (std::nothrow) fdph_plan_s();
    if (!P) return FDPH_E_OOM;
    P->device = p.device;
    P->precision = p.precision;
    P->N = geometry->n;
    P->M = M;
    P->dt = dt;
    auto fail = [&](int code) {
        fdph_destroy(P);
        return code;
    };
    if (cudaSetDevice(p.device) != cudaSuccess) {
        set_error("cudaSetDevice failed");
        return fail(FDPH_E_CUDA);
    }
    if (p.cuda_stream) {
        P->stream = (cudaStream_t)p.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("cudaStreamCreate failed");
            return fail(FDPH_E_CUDA);
        }
        P->own_stream = true;
    }
    PlanInputs in = make_inputs(material, dt, M, eps, p);
    Elements el = make_elements(geometry->n, geometry->xy);
    HostPlan& hp = P->hp;
    const bool verbose = getenv("FDPH_VERBOSE") != nullptr;
    auto stamp = [&](const char* what) {
        if (verbose)
            fprintf(stderr, "[fdph_plan] %-28s %8.3f s\n", what,
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    };
    rc = build_host_plan(el, in, hp);
    if (verbose) fprintf(stderr, "[fdph_plan] host threads %d\n", omp_get_max_threads());
    stamp("host plan (tree, LRA)");
    if (rc == -3) return fail(FDPH_E_CAUSALITY);
    if (rc) return fail(FDPH_E_ARG);
    // ---- upload the far-field operator
    std::vector<SbDev> sd(hp.sbs.size());
    for (size_t q = 0; q < sd.size(); ++q) {
        const SubBlock& b = hp.sbs[q];
        sd[q] = {b.kind, b.rank, b.r0, b.nr, b.s0, b.ns, b.L, b.LZ, b.taps, b.maxdelay, b.mindm, b.run0,
                 b.soe, 0, (long long)b.f, (long long)b.g, (long long)b.h, (long long)b.ring, (long long)b.zring,
                 (long long)b.dhat, (long long)b.delay, (long long)b.dm, (long long)b.ustate, (long long)b.trc,
                 (long long)b.phi};
    }
    if ((rc = upload(P, &P->perm, hp.perm)) || (rc = upload(P, &P->sbs, sd)) || (rc = upload(P, &P->ints, hp.ints)) ||
        (rc = upload(P, &P->run_delay, hp.run_delay)) || (rc = upload(P, &P->run_start, hp.run_start)) ||
        (rc = upload(P, &P->run_len, hp.run_len)) || (rc = upload(P, &P->src_order, hp.src_order)) ||
        (rc = upload(P, &P->scat_sb, hp.scat_sb)) || (rc = upload(P, &P->scat_run, hp.scat_run)) ||
        (rc = upload(P, &P->scat_l, hp.scat_l)) || (rc = upload(P, &P->e_sb, hp.e_sb)) ||
        (rc = upload(P, &P->e_il, hp.e_il)) || (rc = upload(P, &P->e_pos, hp.e_pos)) ||
        (rc = upload(P, &P->fir_sb, hp.fir_sb)) || (rc = upload(P, &P->fir_j, hp.fir_j)) ||
        (rc = upload(P, &P->tr_sb, hp.tr_sb)) || (rc = upload(P, &P->tr_l, hp.tr_l)) ||
        (rc = upload(P, &P->g_ptr, hp.g_ptr)) || (rc = upload(P, &P->g_sb, hp.g_sb)) ||
        (rc = upload(P, &P->g_il, hp.g_il)))
        return fail(rc);
    if (P->precision == FDPH_FP32) {
        std::vector<float> f(hp.fac.begin(), hp.fac.end());
        float* d = nullptr;
        if ((rc = upload(P, &d, f))) return fail(rc);
        P->fac = d;
    } else {
        double* d = nullptr;
        if ((rc = upload(P, &d, hp.fac))) return fail(rc);
        P->fac = d;
    }
    if (hp.soe > 0 && ((rc = upload(P, &P->rho, hp.rho)) || (rc = upload(P, &P->trcoef, hp.trcoef)))) return fail(rc);
    if (hp.interp && (rc = upload(P, &P->phi, hp.phis))) return fail(rc);
    stamp("far-field upload");
    // ---- near field (device-evaluated kernel windows)
    rc = P->precision == FDPH_FP32 ? build_near<float>(P, in) : build_near<double>(P, in);
    if (rc) return fail(rc);
    stamp("near field (windows, tails)");
    FDPH_CUDA(cudaFuncSetAttribute(near_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kStages * kStageBytes + kChunk * 32 * (int)sizeof(double)));
    FDPH_CUDA(cudaFuncSetAttribute(near_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kStages * kStageBytes + kChunk * 32 * (int)sizeof(float)));
    if ((rc = dalloc(P, &P->err, 1))) return fail(rc);
    FDPH_CUDA(cudaMemset(P->err, 0, sizeof(int)));
    // ---- state
    P->WD = std::max(std::max(hp.max_W + (hp.soe > 0 ? 1 : 0), hp.max_taps), 1);
    P->WC = hp.max_W + 1;
    size_t sb = 0;
    auto st = [&](double** p, size_t cnt) {
        sb += std::max<size_t>(cnt, 1) * 8;
        return dalloc(P, p, cnt);
    };
    if ((rc = st(&P->Dring, (size_t)P->WD * P->N)) || (rc = st(&P->Cring, (size_t)P->WC * P->N)) ||
        (rc = st(&P->C, P->N)) || (rc = st(&P->Ccomp, P->N)) || (rc = st(&P->ring, hp.ring_len)) ||
        (rc = st(&P->zring, hp.zring_len)) || (rc = st(&P->dhat, hp.dhat_len)) ||
        (rc = st(&P->partial, hp.items.size() * 32)) || (rc = st(&P->fval, hp.e_sb.size())) ||
        (rc = st(&P->ustate, hp.ustate_len)) || (rc = st(&P->vstate, hp.vstate_len)))
        return fail(rc);
    P->state_bytes = sb;
    if ((rc = fdph_reset(P))) return fail(rc);
    fill_stats(P);
    P->st.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return FDPH_OK;
}

int fdph_reset(fdph_plan_t P) {
    if (!P) return FDPH_E_ARG;
    cudaSetDevice(P->device);
    double* bufs[] = {P->Dring, P->Cring, P->C, P->Ccomp, P->ring, P->zring, P->dhat, P->partial,
                      P->ustate, P->vstate};
    size_t cnt[] = {(size_t)P->WD * P->N, (size_t)P->WC * P->N, (size_t)P->N, (size_t)P->N,
                    (size_t)P->hp.ring_len, (size_t)P->hp.zring_len, (size_t)P->hp.dhat_len,
                    P->hp.items.size() * 32, (size_t)P->hp.ustate_len, (size_t)P->hp.vstate_len};
    for (int q = 0; q < 10; ++q)
        if (bufs[q] && cnt[q]) FDPH_CUDA(cudaMemsetAsync(bufs[q], 0, cnt[q] * sizeof(double), P->stream));
    if (P->rupture) FDPH_CUDA(cudaMemsetAsync(P->fr.slip, 0, P->N * sizeof(double), P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    P->n = 0;
    return FDPH_OK;
}

int fdph_step(fdph_plan_t P, const double* D_n, double* T_n) {
    if (!P || !D_n || !T_n) return FDPH_E_ARG;
    if (P->n >= P->M) {
        set_error("the plan has already taken M steps");
        return FDPH_E_STATE;
    }
    return step_impl(P, D_n, T_n);
}

int fdph_run(fdph_plan_t P, int32_t steps, const double* D, double* T) {
    if (!P || !D || !T || steps < 0) return FDPH_E_ARG;
    if (P->n + steps > P->M) {
        set_error("run would pass step M");
        return FDPH_E_STATE;
    }
    if (steps >= 8 && !P->prof)   // launch-bound steps: replay a captured graph of one step
        return P->precision == FDPH_FP32 ? run_graph<float>(P, steps, D, T) : run_graph<double>(P, steps, D, T);
    for (int s = 0; s < steps; ++s) {
        int rc = step_impl(P, D + (size_t)s * P->N, T + (size_t)s * P->N);
        if (rc) return rc;
    }
    return FDPH_OK;
}

int fdph_step_host(fdph_plan_t P, const double* D_n_host, double* T_n_host) {
    if (!P || !D_n_host || !T_n_host) return FDPH_E_ARG;
    if (!P->dD) {
        int rc;
        if ((rc = dalloc(P, &P->dD, P->N)) || (rc = dalloc(P, &P->dT, P->N))) return rc;
    }
    FDPH_CUDA(cudaMemcpyAsync(P->dD, D_n_host, P->N * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    int rc = fdph_step(P, P->dD, P->dT);
    if (rc) return rc;
    FDPH_CUDA(cudaMemcpyAsync(T_n_host, P->dT, P->N * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    return check_device_error(P);
}

int fdph_current_step(fdph_plan_t P, int32_t* n) {
    if (!P || !n) return FDPH_E_ARG;
    *n = P->n;
    return FDPH_OK;
}

int fdph_synchronize(fdph_plan_t P) {
    if (!P) return FDPH_E_ARG;
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    return check_device_error(P);
}

int fdph_get_stats(fdph_plan_t P, fdph_stats* s) {
    if (!P || !s) return FDPH_E_ARG;
    *s = P->st;
    return FDPH_OK;
}

int fdph_save_state(fdph_plan_t P, void* buf, size_t* len) {
    if (!P || !len) return FDPH_E_ARG;
    double* bufs[] = {P->Dring, P->Cring, P->C, P->Ccomp, P->ring, P->zring, P->ustate, P->vstate};
    size_t cnt[] = {(size_t)P->WD * P->N, (size_t)P->WC * P->N, (size_t)P->N, (size_t)P->N,
                    (size_t)P->hp.ring_len, (size_t)P->hp.zring_len, (size_t)P->hp.ustate_len,
                    (size_t)P->hp.vstate_len};
    size_t need = sizeof(int32_t) * 2;
    for (int q = 0; q < 8; ++q) need += cnt[q] * sizeof(double);
    if (!buf) {
        *len = need;
        return FDPH_OK;
    }
    if (*len < need) return FDPH_E_ARG;
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    char* o = (char*)buf;
    int32_t hdr[2] = {P->n, P->N};
    memcpy(o, hdr, sizeof(hdr));
    o += sizeof(hdr);
    for (int q = 0; q < 8; ++q) {
        if (cnt[q]) FDPH_CUDA(cudaMemcpy(o, bufs[q], cnt[q] * sizeof(double), cudaMemcpyDeviceToHost));
        o += cnt[q] * sizeof(double);
    }
    *len = need;
    return FDPH_OK;
}

int fdph_load_state(fdph_plan_t P, const void* buf, size_t len) {
    if (!P || !buf) return FDPH_E_ARG;
    size_t need = 0;
    int rc = fdph_save_state(P, nullptr, &need);
    if (rc) return rc;
    if (len != need) {
        set_error("state buffer size does not match this plan");
        return FDPH_E_ARG;
    }
    const char* o = (const char*)buf;
    int32_t hdr[2];
    memcpy(hdr, o, sizeof(hdr));
    if (hdr[1] != P->N || hdr[0] < 0 || hdr[0] > P->M) {
        set_error("state buffer belongs to another plan");
        return FDPH_E_ARG;
    }
    o += sizeof(hdr);
    double* bufs[] = {P->Dring, P->Cring, P->C, P->Ccomp, P->ring, P->zring, P->ustate, P->vstate};
    size_t cnt[] = {(size_t)P->WD * P->N, (size_t)P->WC * P->N, (size_t)P->N, (size_t)P->N,
                    (size_t)P->hp.ring_len, (size_t)P->hp.zring_len, (size_t)P->hp.ustate_len,
                    (size_t)P->hp.vstate_len};
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    for (int q = 0; q < 8; ++q) {
        if (cnt[q]) FDPH_CUDA(cudaMemcpy(bufs[q], o, cnt[q] * sizeof(double), cudaMemcpyHostToDevice));
        o += cnt[q] * sizeof(double);
    }
    P->n = hdr[0];
    return FDPH_OK;
}

int fdph_rupture_init(fdph_plan_t P, const fdph_friction* f) {
    if (!P || !f || !f->tau0 || !(f->sigma_n > 0.0) || !(f->Dc > 0.0) || f->mu_d > f->mu_s) {
        set_error("fdph_rupture_init: friction with tau0, sigma_n > 0, Dc > 0, mu_d <= mu_s required");
        return FDPH_E_ARG;
    }
    const HostPlan& hp = P->hp;
    double minlen = 1e300;
    for (int p = 0; p < P->N; ++p) minlen = std::min(minlen, hp.slen[p]);
    if (hp.cs * P->dt > 0.5 * minlen * (1.0 + 1e-12)) {
        set_error("fdph_rupture_init: cs dt exceeds half the shortest element; the instantaneous term is not local");
        return FDPH_E_STATE;
    }
    // K_{ii,0}: jump of the ramp response of each element at its own midpoint over [0, dt]
    std::vector<double> k0(P->N);
    for (int p = 0; p < P->N; ++p) {
        Seg sg;
        sg.ax = hp.sax[p];
        sg.ay = hp.say[p];
        sg.tx = hp.stx[p];
        sg.ty = hp.sty[p];
        sg.len = hp.slen[p];
        const Stress2 w = stress_jump(hp.px[p], hp.py[p], sg, 0.0, P->dt, hp.mu, hp.cs);
        k0[hp.perm[p]] = hp.pnx[p] * w.x + hp.pny[p] * w.y;
    }
    if (!P->rupture) {
        double *tau0 = nullptr, *kk = nullptr, *slip = nullptr;
        int rc;
        if ((rc = dalloc(P, &tau0, P->N)) || (rc = dalloc(P, &kk, P->N)) || (rc = dalloc(P, &slip, P->N))) return rc;
        P->fr.tau0 = tau0;
        P->fr.k0 = kk;
        P->fr.slip = slip;
    }
    FDPH_CUDA(cudaMemcpy((void*)P->fr.tau0, f->tau0, P->N * sizeof(double), cudaMemcpyDeviceToDevice));
    FDPH_CUDA(cudaMemcpy((void*)P->fr.k0, k0.data(), P->N * sizeof(double), cudaMemcpyHostToDevice));
    FDPH_CUDA(cudaMemset(P->fr.slip, 0, P->N * sizeof(double)));
    P->fr.sigma_n = f->sigma_n;
    P->fr.mu_s = f->mu_s;
    P->fr.mu_d = f->mu_d;
    P->fr.Dc = f->Dc;
    P->fr.dt = P->dt;
    P->rupture = true;
    return FDPH_OK;
}

int fdph_rupture_step(fdph_plan_t P, double* D_n, double* T_n) {
    if (!P || !D_n || !T_n) return FDPH_E_ARG;
    if (!P->rupture) {
        set_error("fdph_rupture_init has not been called on this plan");
        return FDPH_E_STATE;
    }
    if (P->n >= P->M) {
        set_error("the plan has already taken M steps");
        return FDPH_E_STATE;
    }
    int rc = P->precision == FDPH_FP32 ? launch_rupture_step<float>(P, D_n, T_n) : launch_rupture_step<double>(P, D_n, T_n);
    if (rc == FDPH_OK) P->n += 1;
    return rc;
}

int fdph_rupture_run(fdph_plan_t P, int32_t steps, double* D, double* T) {
    if (!P || !D || !T || steps < 0) return FDPH_E_ARG;
    if (P->n + steps > P->M) {
        set_error("run would pass step M");
        return FDPH_E_STATE;
    }
    for (int s = 0; s < steps; ++s) {
        int rc = fdph_rupture_step(P, D + (size_t)s * P->N, T + (size_t)s * P->N);
        if (rc) return rc;
    }
    return FDPH_OK;
}

int fdph_rupture_slip(fdph_plan_t P, double* slip) {
    if (!P || !slip) return FDPH_E_ARG;
    if (!P->rupture) return FDPH_E_STATE;
    FDPH_CUDA(cudaMemcpyAsync(slip, P->fr.slip, P->N * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
    return FDPH_OK;
}

int fdph_set_profiling(fdph_plan_t P, int enable) {
    if (!P) return FDPH_E_ARG;
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    prof_drain(P);
    for (int k = 0; k < FDPH_NUM_KERNELS; ++k) {
        P->prof_ms[k] = 0.0;
        P->prof_n[k] = 0;
    }
    P->prof = enable != 0;
    return FDPH_OK;
}

int fdph_kernel_times(fdph_plan_t P, double* ms, int64_t* launches) {
    if (!P || !ms || !launches) return FDPH_E_ARG;
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    prof_drain(P);
    for (int k = 0; k < FDPH_NUM_KERNELS; ++k) {
        ms[k] = P->prof_ms[k];
        launches[k] = P->prof_n[k];
    }
    return FDPH_OK;
}

void fdph_destroy(fdph_plan_t P) {
    if (!P) return;
    cudaSetDevice(P->device);
    if (P->stream) cudaStreamSynchronize(P->stream);
    prof_drain(P);
    if (P->graph) cudaGraphExecDestroy(P->graph);
    for (void* p : P->allocs) cudaFree(p);
    if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
    delete P;
}

}  // extern "C"
