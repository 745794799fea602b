// fdph.cu -- device side of the FDP=H time step and the C ABI (include/fdph.h).
//
// One time step n (Eq. 4 evaluated through the plan's operator) runs these kernels (captured
// as one CUDA graph: FIR + scatter and transient + Eq. 39 on two side streams, concurrently with
// the near field, all joined before gather; several right-hand sides go through one launch, the
// far-field kernels taking all of them in a thread or warp):
//   push     D_n -> slip-rate ring (internal order); cumulative slip C_j(n) = sum_{s<=n} D_j,s
//            with a compensated (Kahan) FP64 sum, -> cumulative-slip ring; with the tensor-core
//            near field (FP16 window, several right-hand sides) also the ring row's scaled FP16
//            (hi, lo) copy (tc_rows)
//   fir      Domain F, formula 1 (Eq. 32): Dhat_j = sum_{m < Dm_j} h_{j,m} D_{j,n-m}, per F block
//            and source (fir), or per source for all its F blocks (sfir), in the factor type
//   scatter  formula 2 (Eq. 42): Tbar'_l[n + delay_j] += g_{l,j} u_j for every run of sources
//            (rings are stored [slot][rank] so that one receiver's ranks share a sector)
//            with equal delay (no atomics: one writer per ring slot); u = Dhat (Domain F),
//            dt * C (Domain S, App. B.1 written on the cumulative slip), D (transient);
//            the ring is the shift operator M of Eq. 40 as a base-pointer increment
//   trconv   transient (App. B.3): Z_l(n - min dm) = sum_{m < Dm_tr} h^tr_m Y_l(n - min dm - m)
//   near     inadmissible leaves (App. E): sum_{k < W} K_{ij,k} D_{j,n-k} + Kstat_ij dt C_j(n-W),
//            per (leaf, chunk of k) work item into a partial-sum slot
//   far_eval + far_sum  formula 3 (Eq. 39): Tfar_i = sum_{blocks} sum_l f_{l,i} Tbar'_l[n - dm_i]
//            (far-field branch)
//   gather   T_i = Tfar_i + the receiver's near partials, written in the caller's element order
// Causality (min(dm + delay) >= 1, checked at plan time) guarantees that the ring slots read
// at step n were completed by steps < n and that the slots written at step n are not read.
// A rupture step (Sec. 6.2) predicts with D_n = 0, solves the friction law per element and
// then commits D_n; a batch of plans runs each of these kernels as one launch over all plans.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <omp.h>
#include <stdlib.h>

#include <algorithm>
#include <climits>
#include <type_traits>
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

// Bounded-index debug build (-DFDPH_CHECK, libfdph_check.so): every ring, state, partial-sum and
// near-slice access of the step kernels is checked against the extent of its array; a failing
// check records kErrIndex in the plan's error word and skips the access (no trap: the kernel
// carries on and finishes), and the next synchronising call returns FDPH_E_CHECK.  In the normal
// build FDPH_IDX is the constant true and costs nothing.
static const int kErrTimeout = 1;   // error word: a bounded wait gave up
static const int kErrIndex = 2;     // error word: an index check failed (FDPH_CHECK builds)
__device__ __forceinline__ bool fdph_idx_check(bool ok, int* err) {
    if (!ok && err) atomicExch(err, kErrIndex);
    return ok;
}
#ifdef FDPH_CHECK
#define FDPH_IDX(cond, err) fdph_idx_check((cond), (err))
#else
#define FDPH_IDX(cond, err) true
#endif

static const int kChunk = 64;      // steps of exact kernel per near-field work item
static const int kNearConsumers = 4;                       // consumer warps of the near-field kernel
static const int kNearThreads = 32 * (kNearConsumers + 1);  // + one producer warp
static const int kNearStageBytes = 16384;                  // one pipeline stage
static const int kMaxPer = kChunk;                         // slices per stage at most
static const int kTaskCache = 48;                          // work items per CTA kept in shared memory
static_assert(kNearStageBytes >= 32 * 32 * 8, "a stage holds at least one FP64 slice of a 32 x 32 leaf");
static const long long kWaitLimit = 1LL << 22;   // bounded mbarrier polls before giving up

// ------------------------------------------------------------------------------------------
// device-side views

struct SbDev {
    int kind, rank, r0, nr, s0, ns, L, LZ, taps, maxdelay, mindm, run0, soe, ident, e0, LH;
    long long f, g, h, ring, zring, dhat, delay, dm, ustate, trc, phi;
    long long uhist;    // delayed-history form: [LH][ns] source values u_j of the last LH steps
    int mindelay, qn;   // qn: quantized ranges of a transient's taps (0: exact taps)
    long long qb;       // offset of their qn + 1 bounds in ints
};

struct NearDev {
    int r0, nr, s0, ns, W, sl, sla, pad;
    long long tensor, stat, tail, vstate;
};

// one near-field work item as the persistent kernel reads it (one 64-byte load)
struct __align__(16) NearTask {
    long long off;       // element offset of the item's first slice (tensor, or aux for kind 1)
    int item, k0, k1, kind, nr, ns, sl, s0, W, vstate;
    int scen;            // plan of the item in a batch (0 otherwise)
    int pad;
};
static_assert(sizeof(NearTask) == 64, "one work item is four 16-byte loads");

static const int kMaxSoe = 16;
static const int kMaxRhs = 8;    // right-hand sides of one plan at most (1, 2, 4 or 8)

template <class T>
struct StepArgs {
    int n, N, WD, WC;
    // graph replay: the step index is read from n_dev[0], and D_in / T_out advance by io_stride
    // elements per step past the step n_dev[1] of the call's first row (unused when n_dev is null)
    const int* n_dev;
    long long io_stride;
    int io_ring;              // > 0: D_in / T_out rows are a ring of io_ring staging slots
    double dt;
    const double* D_in;       // caller's D_n (geometry order)
    double* T_out;            // caller's T_n (geometry order)
    const int* perm;          // internal -> geometry
    double* Dring;            // [WD][N]
    float* Dring32;           // [WD][N] FP32 copy of Dring (plans whose near-field rows are FP32)
    __half2* Dring16;         // [2 WD][nrhs][NP] scaled FP16 (hi, lo) pairs of Dring (FP16 plans, nrhs >= 2):
                              // slot s is stored at s and s + WD (a window of <= WD slots never wraps),
                              // all right-hand sides of a slot side by side, rows padded to NP (multiple of 4)
    float* Dscale;            // [2 WD][SR] inverse power-of-two scale of each Dring16 row, mirrored like
                              // Dring16, SR = max(nrhs, 4) floats a slot (16-byte rows for the TMA)
    const void* tmap16;       // TMA tensor maps (device memory): [0] Dring16, box 36 sources x nrhs x
                              // item slots; [1] Dscale, box SR x item slots
    int NP;
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
    const int4* sc_tasks;     // scatter warp tasks {block, first run, runs, log2 lanes per run}
    int n_sct;
    const int4* ev_tasks;     // Eq. 39 warp tasks {block, first receiver, receivers, log2 lanes per receiver}
    int n_evt;
    const int* e_pos;         // CSR slot of each (block, receiver) entry, block-major
    double* fval;             // [entries] far-field value of each (block, receiver) entry, CSR order
    double* tfar;             // [N] far-field traction of each receiver (sum of its entries)
    const int* fir_sb;
    const int* fir_j;
    int n_fir;
    const int* sfir_ptr;      // [N + 1] the FIR tasks by source element (CSR into sfir_q)
    const int* sfir_q;
    const int* sfir_tmax;     // [N] longest waveform of the source's tasks
    int sfir_taps;            // longest waveform of all (shared-memory rows of a warp)
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
    const NearTask* tasks;    // near-field work items in per-CTA order
    const int* cta_ptr;       // [n_cta + 1]: CTA c owns tasks [cta_ptr[c], cta_ptr[c+1])
    int n_cta;
    int n_items;
    const void* tensor;       // near-field window slices (window storage type)
    float kinv;               // inverse of the window coefficients' storage scale (FP16: 2^-e, else 1)
    const void* stat;         // aux slices: static tiles, exponential-tail coefficients (aux storage type)
    long long len_tensor, len_aux;   // elements of tensor and stat (index checks of FDPH_CHECK builds)
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
    // right-hand sides: every time-stepping state array above is [nrhs][...] with these strides
    // (elements); the caller's rows D_n, T_n are [nrhs][N] (io_stride = nrhs N per step)
    int nrhs;
    long long rs_D, rs_C, rs_ring, rs_zring, rs_dhat, rs_fval, rs_ustate, rs_vstate, rs_partial;
    // delayed-history form of Eq. 42 (far_mode 1)
    double* uhist;            // [blocks][LH][ns] source values
    long long rs_uhist;
    const int2* rec_tasks;    // (block, source) recorded per step
    const int2* gat_tasks;    // (block, rank index) gathered per step
    int n_rec, n_gat;
};

// ring slot of step a (a may be negative; |a| < 2^31)
__device__ __forceinline__ int wrap(int a, int L) {
    const int r = a % L;
    return r < 0 ? r + L : r;
}

template <class T>
__device__ __forceinline__ int step_index(const StepArgs<T>& a) {
    return a.n_dev ? *a.n_dev : a.n;
}

// element offset of step n's row of D_in / T_out
template <class T>
__device__ __forceinline__ long long io_offset(const StepArgs<T>& a, int n) {
    if (!a.n_dev) return 0;
    const int k = n - a.n_dev[1];
    return (long long)(a.io_ring > 0 ? k % a.io_ring : k) * a.io_stride;
}

// the arguments of right-hand side r (grid y of the per-step kernels)
template <class T>
__device__ __forceinline__ StepArgs<T> rhs_args(const StepArgs<T>& a0, int r) {
    StepArgs<T> a = a0;
    if (r) {
        const long long rN = (long long)r * a0.N;
        if (a0.D_in) a.D_in = a0.D_in + rN;
        if (a0.T_out) a.T_out = a0.T_out + rN;
        a.Dring = a0.Dring + r * a0.rs_D;
        if (a0.Dring32) a.Dring32 = a0.Dring32 + r * a0.rs_D;
        a.Cring = a0.Cring + r * a0.rs_C;
        a.C = a0.C + rN;
        a.Ccomp = a0.Ccomp + rN;
        a.ring = a0.ring + r * a0.rs_ring;
        a.zring = a0.zring + r * a0.rs_zring;
        a.dhat = a0.dhat + r * a0.rs_dhat;
        a.fval = a0.fval + r * a0.rs_fval;
        a.tfar = a0.tfar + rN;
        if (a0.ustate) a.ustate = a0.ustate + r * a0.rs_ustate;
        if (a0.vstate) a.vstate = a0.vstate + r * a0.rs_vstate;
        a.partial = a0.partial + r * a0.rs_partial;
        if (a0.uhist) a.uhist = a0.uhist + r * a0.rs_uhist;
    }
    return a;
}

__global__ void advance_step_kernel(int* n_dev) { *n_dev += 1; }

// FP32 copy of a restored slip-rate ring
__global__ void ring_to_float_kernel(const double* x, float* y, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}

// Slip-rate rows for the tensor-core near field (FP16 window, nrhs >= 2): ring row (slot, RHS) as
// (hi, lo) FP16 pairs of x 2^sh, sh = 14 - e for the row's largest |x| = f 2^e, f in [0.5, 1)
// (e from the exponent field; a zero or subnormal row takes the largest shift), hi = fp16(x 2^sh),
// lo = fp16(x 2^sh - hi), and Dscale = 2^-sh.  One CTA per row: the row of step n (all_slots 0,
// after push), or every slot (all_slots 1, after a state restore).  grid (slots or 1, nrhs).
// The near kernel fetches a work item's rows of all right-hand sides with one TMA tensor copy.
constexpr int kRowThreads = 256;

__device__ __forceinline__ int row_shift(float m) {
    const int e = m > 0.f ? (int)((__float_as_uint(m) >> 23) & 0xffu) - 126 : -126;
    return min(max(14 - e, -100), 100);
}

// 2^k as a float, k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(127 + k) << 23); }

template <class T>
__global__ void __launch_bounds__(kRowThreads) tc_rows_kernel(StepArgs<T> a0, int all_slots) {
    __shared__ float wmax[kRowThreads / 32];
    const StepArgs<T> a = rhs_args(a0, blockIdx.y);
    const int slot = all_slots ? blockIdx.x : wrap(step_index(a), a.WD);
    const double* row = a.Dring + (size_t)slot * a.N;
    float m = 0.f;
    for (int p = threadIdx.x; p < a.N; p += kRowThreads) m = fmaxf(m, fabsf((float)row[p]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < kRowThreads / 32; ++w) m = fmaxf(m, wmax[w]);
    const int sh = row_shift(m);
    const float s = pow2f(sh);
    // slot s of right-hand side q at rows (s, q) and (s + WD, q) of the mirrored [2 WD][nrhs][NP] layout
    __half2* out0 = a.Dring16 + ((size_t)slot * a.nrhs + blockIdx.y) * a.NP;
    __half2* out1 = out0 + (size_t)a.WD * a.nrhs * a.NP;
    for (int p = threadIdx.x; p < a.N; p += kRowThreads) {
        const float y = (float)row[p] * s;
        const __half hi = __float2half_rn(y);
        const __half2 v = __halves2half2(hi, __float2half_rn(y - __half2float(hi)));
        out0[p] = v;
        out1[p] = v;
    }
    if (threadIdx.x == 0) {
        const int sr = a.nrhs > 4 ? a.nrhs : 4;
        a.Dscale[(size_t)slot * sr + blockIdx.y] = pow2f(-sh);
        a.Dscale[(size_t)(slot + a.WD) * sr + blockIdx.y] = pow2f(-sh);
    }
}

__global__ void set_step_kernel(int* n_dev, int v) {
    n_dev[0] = v;   // step index
    n_dev[1] = v;   // step of the call's first row of D / T
}

// Every per-step kernel is a body over one work index of one plan (element, task or warp task),
// launched either for one plan (grid y = right-hand side) or for a batch of plans (one launch
// over the work of all plans; the plan of a work index from the prefix sums of their counts).
template <class T>
__device__ __forceinline__ void push_body(const StepArgs<T>& a, int p, bool zero) {
    const int n = step_index(a);
    const size_t slot = (size_t)wrap(n, a.WD) * a.N + p;
    if (!FDPH_IDX(p < a.N && (long long)slot < a.rs_D, a.err)) return;
    if (zero || !a.D_in) {   // rupture predictor: the unknown slip rate of this step is held at zero
        a.Dring[slot] = 0.0;
        if (a.Dring32) a.Dring32[slot] = 0.f;
        return;
    }
    const double d = a.D_in[io_offset(a, n) + a.perm[p]];
    a.Dring[slot] = d;
    if (a.Dring32) a.Dring32[slot] = (float)d;
    // compensated running sum of the slip (units of dt)
    const double y = d - a.Ccomp[p];
    const double c0 = a.C[p];
    const double t = c0 + y;
    a.Ccomp[p] = (t - c0) - y;
    a.C[p] = t;
    a.Cring[(size_t)wrap(n, a.WC) * a.N + p] = t;
}

template <class T>
__global__ void push_kernel(StepArgs<T> a0) {
    const StepArgs<T> a = rhs_args(a0, blockIdx.y);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < a.N) push_body(a, p, false);
}

// The slip-rate history and the sums in the factor type: FP32 plans read the FP32 copy of the ring
// and add in FP32 (this GPU's FP64 rate is a small fraction of its FP32 rate, and the ~27 taps of
// a waveform lose ~2^-24 sqrt(27) relative), FP64 plans stay in FP64
template <class T>
__device__ __forceinline__ const T* fir_ring(const StepArgs<T>& a) {
    if constexpr (sizeof(T) == 4) return a.Dring32; else return a.Dring;
}

template <class T>
__device__ __forceinline__ void fir_body(const StepArgs<T>& a, int q) {
    const int n = step_index(a);
    const SbDev& sb = a.sbs[a.fir_sb[q]];
    const int jl = a.fir_j[q];
    const T* h = a.fac + sb.h + (long long)jl * sb.taps;   // the source's taps, contiguous
    const T* D = fir_ring(a) + sb.s0 + jl;
    const int taps = min(sb.taps, n + 1);   // taps <= WD, so one wrap-around at most
    const int slot = wrap(n, a.WD);
    if (!FDPH_IDX(taps <= a.WD && sb.s0 + jl < a.N && (long long)sb.dhat + jl < a.rs_dhat, a.err)) return;
    T s0 = 0, s1 = 0;
    int m = 0;
    for (; m + 1 < taps; m += 2) {
        int t0 = slot - m, t1 = slot - m - 1;
        t0 += t0 < 0 ? a.WD : 0;
        t1 += t1 < 0 ? a.WD : 0;
        s0 += h[m] * D[(size_t)t0 * a.N];
        s1 += h[m + 1] * D[(size_t)t1 * a.N];
    }
    if (m < taps) {
        int t0 = slot - m;
        t0 += t0 < 0 ? a.WD : 0;
        s0 += h[m] * D[(size_t)t0 * a.N];
    }
    a.dhat[sb.dhat + jl] = (double)(s0 + s1);
}

// The same for NR right-hand sides at once: the taps are read once and feed the NR slip-rate rows
// (per right-hand side the single-RHS order of operations, so the results are the same bits)
template <class T, int NR>
__device__ __forceinline__ void fir_body_nr(const StepArgs<T>& a, int q) {
    const int n = step_index(a);
    const SbDev& sb = a.sbs[a.fir_sb[q]];
    const int jl = a.fir_j[q];
    const T* h = a.fac + sb.h + (long long)jl * sb.taps;
    const T* D = fir_ring(a) + sb.s0 + jl;
    const int taps = min(sb.taps, n + 1);
    const int slot = wrap(n, a.WD);
    if (!FDPH_IDX(taps <= a.WD && sb.s0 + jl < a.N && (long long)sb.dhat + jl < a.rs_dhat, a.err)) return;
    T s0[NR], s1[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) s0[r] = s1[r] = 0;
    int m = 0;
    for (; m + 1 < taps; m += 2) {
        int t0 = slot - m, t1 = slot - m - 1;
        t0 += t0 < 0 ? a.WD : 0;
        t1 += t1 < 0 ? a.WD : 0;
        const T h0 = h[m], h1 = h[m + 1];
        const T* d0 = D + (size_t)t0 * a.N;
        const T* d1 = D + (size_t)t1 * a.N;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            s0[r] += h0 * d0[r * a.rs_D];
            s1[r] += h1 * d1[r * a.rs_D];
        }
    }
    if (m < taps) {
        int t0 = slot - m;
        t0 += t0 < 0 ? a.WD : 0;
        const T h0 = h[m];
        const T* d0 = D + (size_t)t0 * a.N;
#pragma unroll
        for (int r = 0; r < NR; ++r) s0[r] += h0 * d0[r * a.rs_D];
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) a.dhat[r * a.rs_dhat + sb.dhat + jl] = (double)(s0[r] + s1[r]);
}

// NR = 1: one grid row per right-hand side; NR > 1: all of them in one thread
template <class T, int NR>
__global__ void fir_kernel(StepArgs<T> a0) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (NR == 1) {
        const StepArgs<T> a = rhs_args(a0, blockIdx.y);
        if (q < a.n_fir) fir_body(a, q);
    } else {
        if (q < a0.n_fir) fir_body_nr<T, NR>(a0, q);
    }
}

// Eq. 32 source-major (the single-plan step): one warp per source element j, which copies its
// last taps slip rates of every right-hand side to shared memory once, then its lanes take j's
// FIR tasks (one per F block containing j, ~10^2 at large N) and sum each task's contiguous taps
// against the shared rows.  The sub-block-major kernel above reads a source's slip rates once
// per task; this reads them once per step.  Per task and right-hand side the sums run in the
// same order (even and odd taps apart), so the results are the same bits.
constexpr int kSfirWarps = 4;

template <class T, int NR>
__global__ void __launch_bounds__(32 * kSfirWarps) sfir_kernel(StepArgs<T> a) {
    extern __shared__ __align__(8) unsigned char sfir_smem[];
    T* sfir_rows = (T*)sfir_smem;           // per warp [sfir_taps][NR]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kSfirWarps + warp;
    if (p >= a.N) return;   // warp-uniform
    const int e0 = a.sfir_ptr[p], e1 = a.sfir_ptr[p + 1];
    if (e0 == e1) return;
    const int n = step_index(a);
    const int tmax = min(a.sfir_tmax[p], n + 1);
    T* sd = sfir_rows + (size_t)warp * a.sfir_taps * NR;
    const T* ring = fir_ring(a);
    if (!FDPH_IDX(tmax <= a.WD && a.sfir_tmax[p] <= a.sfir_taps, a.err)) return;
    const int slot = wrap(n, a.WD);
    for (int m = lane; m < tmax; m += 32) {
        int t = slot - m;
        t += t < 0 ? a.WD : 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) sd[m * NR + r] = ring[r * a.rs_D + (size_t)t * a.N + p];
    }
    __syncwarp();
    for (int e = e0 + lane; e < e1; e += 32) {
        const int q = a.sfir_q[e];
        const SbDev& sb = a.sbs[a.fir_sb[q]];
        const int jl = a.fir_j[q];
        const int taps = min(sb.taps, n + 1);
        if (!FDPH_IDX(taps <= tmax && (long long)sb.dhat + jl < a.rs_dhat, a.err)) continue;
        const T* h = a.fac + sb.h + (long long)jl * sb.taps;
        T s0[NR], s1[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) s0[r] = s1[r] = 0;
        int m = 0;
        for (; m + 1 < taps; m += 2) {
            const T h0 = h[m], h1 = h[m + 1];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                s0[r] += h0 * sd[m * NR + r];
                s1[r] += h1 * sd[(m + 1) * NR + r];
            }
        }
        if (m < taps) {
            const T h0 = h[m];
#pragma unroll
            for (int r = 0; r < NR; ++r) s0[r] += h0 * sd[m * NR + r];
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) a.dhat[r * a.rs_dhat + sb.dhat + jl] = (double)(s0[r] + s1[r]);
    }
}

// source quantity u_j of Eq. 42 for block kind: Dhat (Domain F), dt * cumulative slip (Domain S,
// App. B.1), slip rate (transient)
template <class T>
__device__ __forceinline__ double source_value(const StepArgs<T>& a, const SbDev& sb, int jl, int dslot) {
    if (sb.kind == SB_F) return a.dhat[sb.dhat + jl];
    if (sb.kind == SB_S) return a.dt * a.C[sb.s0 + jl];
    return a.Dring[(size_t)dslot * a.N + sb.s0 + jl];
}

// Eq. 42: one warp per task of runs (sources of equal delay) of one block; 2^lg lanes per run
// cover the rank index l, so a run writes its ring slot row [slot][0, rank) in one coalesced pass.
// One writer per (slot, l): the runs of a block have distinct delays.
template <class T>
__device__ __forceinline__ void scatter_body(const StepArgs<T>& a, int w, int lane) {
    const int n = step_index(a);
    const int4 tk = a.sc_tasks[w];
    const SbDev& sb = a.sbs[tk.x];
    const int lg = tk.w, G = 1 << lg;
    const int gi = lane >> lg, lj = lane & (G - 1);
    if (gi >= tk.z) return;
    const int run = tk.y + gi;
    const int delay = a.run_delay[run], st = a.run_start[run], len = a.run_len[run];
    const int rank = sb.rank;
    double* r = a.ring + sb.ring + (long long)wrap(n + delay, sb.L) * rank;
    const int dslot = sb.kind == SB_TR ? wrap(n, a.WD) : 0;
    if (!FDPH_IDX(sb.ring + (long long)(wrap(n + delay, sb.L) + 1) * rank <= a.rs_ring &&
                  (sb.ident != 2 || sb.ns <= rank), a.err))
        return;
    if (sb.ident == 2) {
        // G is the identity: column j of a slot receives source j only, once
        for (int u = lj; u < len; u += G) {
            const int jl = a.src_order[st + u];
            r[jl] = source_value(a, sb, jl, dslot);
        }
        return;
    }
    const bool fresh = delay == sb.maxdelay;   // the newest slot of the ring starts from zero
    const T* g = a.fac + sb.g;
    if (len == 1) {
        const int jl = a.src_order[st];
        const double u = source_value(a, sb, jl, dslot);
        const T* gj = g + (long long)jl * rank;
        for (int l = lj; l < rank; l += G) r[l] = fresh ? (double)gj[l] * u : r[l] + (double)gj[l] * u;
        return;
    }
    for (int l = lj; l < rank; l += G) {
        double s = 0.0;
        for (int u = 0; u < len; ++u) {
            const int jl = a.src_order[st + u];
            s += (double)g[(long long)jl * rank + l] * source_value(a, sb, jl, dslot);
        }
        r[l] = fresh ? s : r[l] + s;
    }
}

// The same for NR right-hand sides at once: g and the task's indices are read once (per right-hand
// side the single-RHS order of operations)
template <class T, int NR>
__device__ __forceinline__ void scatter_body_nr(const StepArgs<T>& a, int w, int lane) {
    const int n = step_index(a);
    const int4 tk = a.sc_tasks[w];
    const SbDev& sb = a.sbs[tk.x];
    const int lg = tk.w, G = 1 << lg;
    const int gi = lane >> lg, lj = lane & (G - 1);
    if (gi >= tk.z) return;
    const int run = tk.y + gi;
    const int delay = a.run_delay[run], st = a.run_start[run], len = a.run_len[run];
    const int rank = sb.rank;
    double* r0 = a.ring + sb.ring + (long long)wrap(n + delay, sb.L) * rank;
    const int dslot = sb.kind == SB_TR ? wrap(n, a.WD) : 0;
    if (!FDPH_IDX(sb.ring + (long long)(wrap(n + delay, sb.L) + 1) * rank <= a.rs_ring &&
                  (sb.ident != 2 || sb.ns <= rank), a.err))
        return;
    auto sv = [&](int jl, int r) -> double {   // source_value of right-hand side r
        if (sb.kind == SB_F) return a.dhat[r * a.rs_dhat + sb.dhat + jl];
        if (sb.kind == SB_S) return a.dt * a.C[(long long)r * a.N + sb.s0 + jl];
        return a.Dring[r * a.rs_D + (size_t)dslot * a.N + sb.s0 + jl];
    };
    if (sb.ident == 2) {
        for (int u = lj; u < len; u += G) {
            const int jl = a.src_order[st + u];
#pragma unroll
            for (int r = 0; r < NR; ++r) r0[r * a.rs_ring + jl] = sv(jl, r);
        }
        return;
    }
    const bool fresh = delay == sb.maxdelay;
    const T* g = a.fac + sb.g;
    if (len == 1) {
        const int jl = a.src_order[st];
        double u[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) u[r] = sv(jl, r);
        const T* gj = g + (long long)jl * rank;
        for (int l = lj; l < rank; l += G) {
            const double gl = (double)gj[l];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                double* rr = r0 + r * a.rs_ring;
                rr[l] = fresh ? gl * u[r] : rr[l] + gl * u[r];
            }
        }
        return;
    }
    for (int l = lj; l < rank; l += G) {
        double sum[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) sum[r] = 0.0;
        for (int u = 0; u < len; ++u) {
            const int jl = a.src_order[st + u];
            const double gl = (double)g[(long long)jl * rank + l];
#pragma unroll
            for (int r = 0; r < NR; ++r) sum[r] += gl * sv(jl, r);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            double* rr = r0 + r * a.rs_ring;
            rr[l] = fresh ? sum[r] : rr[l] + sum[r];
        }
    }
}

template <class T, int NR>
__global__ void scatter_kernel(StepArgs<T> a0) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if constexpr (NR == 1) {
        const StepArgs<T> a = rhs_args(a0, blockIdx.y);
        if (w < a.n_sct) scatter_body(a, w, threadIdx.x & 31);
    } else {
        if (w < a0.n_sct) scatter_body_nr<T, NR>(a0, w, threadIdx.x & 31);
    }
}

// Delayed-history form of Eq. 42 (the gather variant of Sec. 5.3): instead of adding g_{l,j} u_j
// to the future slots n + delay_j, every step records u_j(n) in the block's history of the last
// LH = maxdelay - mindelay + 1 steps and computes the one slot that the step completes,
//     Tbar'_l[n + mindelay] = sum_j g_{l,j} u_j(n + mindelay - delay_j),
// by causality (min(dm + delay) >= 1) a slot no evaluation of step n reads yet.
template <class T>
__device__ __forceinline__ void record_body(const StepArgs<T>& a, int q) {
    const int n = step_index(a);
    const int2 t = a.rec_tasks[q];
    const SbDev& sb = a.sbs[t.x];
    const int dslot = sb.kind == SB_TR ? wrap(n, a.WD) : 0;
    a.uhist[sb.uhist + (long long)wrap(n, sb.LH) * sb.ns + t.y] = source_value(a, sb, t.y, dslot);
}

template <class T>
__global__ void record_kernel(StepArgs<T> a0) {
    const StepArgs<T> a = rhs_args(a0, blockIdx.y);
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < a.n_rec) record_body(a, q);
}

// one warp per (block, rank index l), lanes over the sources
template <class T>
__device__ __forceinline__ void hgather_body(const StepArgs<T>& a, int w, int lane) {
    const int n = step_index(a);
    const int2 t = a.gat_tasks[w];
    const SbDev& sb = a.sbs[t.x];
    const int l = t.y;
    const int s = n + sb.mindelay;
    const int* dl = a.ints + sb.delay;
    const double* u = a.uhist + sb.uhist;
    double acc = 0.0;
    if (sb.ident == 2) {   // G is the identity: rank index l is source l
        if (lane == 0) acc = u[(long long)wrap(s - dl[l], sb.LH) * sb.ns + l];
    } else {
        const T* g = a.fac + sb.g;
        for (int j = lane; j < sb.ns; j += 32)
            acc += (double)g[(long long)j * sb.rank + l] * u[(long long)wrap(s - dl[j], sb.LH) * sb.ns + j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    if (lane == 0) a.ring[sb.ring + (long long)wrap(s, sb.L) * sb.rank + l] = acc;
}

template <class T>
__global__ void hgather_kernel(StepArgs<T> a0) {
    const StepArgs<T> a = rhs_args(a0, blockIdx.y);
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w < a.n_gat) hgather_body(a, w, threadIdx.x & 31);   // warp-uniform
}

// one warp per (transient block, rank index)
template <class T>
__device__ __forceinline__ void trconv_body(const StepArgs<T>& a, int q, int lane) {
    const int n = step_index(a);
    const SbDev sb = a.sbs[a.tr_sb[q]];
    const int l = a.tr_l[q];
    const int t0 = n - sb.mindm;
    const double* Y = a.ring + sb.ring + l;
    if (!FDPH_IDX(sb.ring + (long long)sb.L * sb.rank <= a.rs_ring && l < sb.rank &&
                  sb.zring + (long long)sb.LZ * sb.rank <= a.rs_zring &&
                  (!(sb.soe + sb.qn) || sb.ustate + (long long)sb.rank * (sb.soe + sb.qn) <= a.rs_ustate), a.err))
        return;
    double z = 0.0;
    const int su = sb.soe + sb.qn;   // states of one rank index: exponential tail, then running sums
    if (sb.qn) {
        // quantized taps (App. A): z = sum_q hhat_q Yhat_q, Yhat_q(t) = Yhat_q(t - 1) + Y(t - b_q)
        // - Y(t - b_q+1) (Eq. A.4), the running window sums kept in the block's states
        for (int q = lane; q < sb.qn; q += 32) {
            const int b0 = a.ints[sb.qb + q], b1 = a.ints[sb.qb + q + 1];
            double* u = a.ustate + sb.ustate + (long long)l * su + sb.soe + q;
            const double y = *u + Y[(long long)wrap(t0 - b0, sb.L) * sb.rank] - Y[(long long)wrap(t0 - b1, sb.L) * sb.rank];
            *u = y;
            z += (double)a.fac[sb.h + q] * y;
        }
    } else {
        for (int m = lane; m < sb.taps; m += 32)
            z += (double)a.fac[sb.h + m] * Y[(long long)wrap(t0 - m, sb.L) * sb.rank];
    }
    if (lane < sb.soe) {
        // tail beyond the exact taps: U_q(t) = rho_q U_q(t - 1) + Y(t - taps), z += c_q U_q(t)
        double* u = a.ustate + sb.ustate + (long long)l * su + lane;
        const double un = a.rho[lane] * *u + Y[(long long)wrap(t0 - sb.taps, sb.L) * sb.rank];
        *u = un;
        z += a.trcoef[sb.trc + lane] * un;
    }
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) a.zring[sb.zring + (long long)wrap(t0, sb.LZ) * sb.rank + l] = z;
}

template <class T>
__global__ void trconv_kernel(StepArgs<T> a0) {
    const StepArgs<T> a = rhs_args(a0, blockIdx.y);
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q < a.n_tr) trconv_body(a, q, threadIdx.x & 31);
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

// as bulk_g2s, with an L2 cache policy (evict-first for data read once per step)
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                              unsigned long long policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// 2-D TMA tile load of the box at (x, y) of the tensor map (global memory) into shared memory
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 3-D TMA tile load of the box at (x, y, z) of the tensor map (global memory) into shared memory,
// completing `bytes` of the mbarrier's transaction count
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}



__device__ __forceinline__ bool mbar_wait_limit(unsigned long long* bar, unsigned phase, long long limit) {
    const unsigned a = smem_u32(bar);
    for (long long it = 0; it < limit; ++it) {
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

// every pipeline wait of the library: at most kWaitLimit polls, then the caller records a timeout
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned phase) {
    return mbar_wait_limit(bar, phase, kWaitLimit);
}

// Self-test of the bounded wait: one CTA waits on an mbarrier that no thread ever completes; the
// wait gives up after `limit` polls and records the timeout in err, and the kernel returns (no
// copy is in flight), so the context stays usable.
__global__ void wait_selftest_kernel(long long limit, int* err) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_limit(&bar, 0u, limit)) atomicExch(err, 1);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// asynchronous 4- / 8-byte copy global -> shared (cp.async); src_bytes = 0 zero-fills the destination
__device__ __forceinline__ void cp_async_4(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_8(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// this thread's cp.async copies have landed (a barrier then publishes them to the block)
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void consumer_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(kNearConsumers * 32) : "memory");
}

template <class T>
__device__ __forceinline__ int near_slices(const NearTask& tk, int n) {
    return tk.kind ? tk.k1 - tk.k0 : min(tk.k1, n + 1) - tk.k0;
}

// What a near-field work item reads of its plan (the plan of the launch, or for a batch of
// plans the item's own plan), with the plan's step index n.
struct NearView {
    const double* Dring;
    const float* Dring32;
    const __half2* Dring16;
    const float* Dscale;
    const void* tmap16;
    const double* Cring;
    double* vstate;
    const double* rho;
    const void* tensor;
    const void* stat;
    double* partial;
    int* err;
    float kinv;
    int N, WD, WC, n, nrhs;
    long long rs_D, rs_C, rs_vstate, rs_partial;
    long long len_tensor, len_aux;
};

template <class T>
__device__ __forceinline__ NearView near_view(const StepArgs<T>& a) {
    NearView v;
    v.Dring = a.Dring;
    v.Dring32 = a.Dring32;
    v.Dring16 = a.Dring16;
    v.Dscale = a.Dscale;
    v.tmap16 = a.tmap16;
    v.Cring = a.Cring;
    v.vstate = a.vstate;
    v.rho = a.rho;
    v.tensor = a.tensor;
    v.kinv = a.kinv;
    v.stat = a.stat;
    v.partial = a.partial;
    v.err = a.err;
    v.N = a.N;
    v.WD = a.WD;
    v.WC = a.WC;
    v.n = step_index(a);
    v.nrhs = a.nrhs;
    v.rs_D = a.rs_D;
    v.rs_C = a.rs_C;
    v.rs_vstate = a.rs_vstate;
    v.rs_partial = a.rs_partial;
    v.len_tensor = a.len_tensor;
    v.len_aux = a.len_aux;
    return v;
}

// The vectors of one work item (rows of 32 in the row type; with NR right-hand sides row
// k * NR + r holds slice k of right-hand side r) are gathered by the consumer warps, this warp
// taking rows w, w + C, ...: window rows D_{n - k0 - k, j} are copied from the slip-rate ring in
// the row type straight to shared memory (cp.async, issued one item ahead, awaited before the
// item's closing barrier); aux rows go through registers in two halves, near_issue loading
// them and near_commit (one item later, so that the loads are in flight meanwhile) forming the
// values and storing them.  Aux row a = k0 + k: a = 0, C_j(n - W) (the
// static tile carries dt); a = q + 1, the tail state V_qj(n) = rho_q V_qj(n - 1) + D_{j, n-W},
// updated here by its only reader.
constexpr int kRowsPerWarp = kChunk / kNearConsumers;
static_assert(kRowsPerWarp * kNearConsumers == kChunk, "vector rows are dealt evenly over the consumer warps");

// tensor-core window rows travel with the window slices: each pipeline stage carries kTcPer slices
// (8 x 32 x 32 FP16 = one 16 KB stage) followed by their rows as one TMA box lands,
// [slot][right-hand side][kTcBox] (hi, lo) words, slots from the stage's oldest, and then the rows'
// scales [slot][max(NR, 4)]
constexpr int kTcBox = 36;
constexpr int kTcPer = 8;
// vector rows of the aux items of a tensor-core plan (static tile and tail slices, NR per slice)
constexpr int kTcVecRows = 32;

template <class R, int NR, int VR, bool TC>
__device__ __forceinline__ void near_issue(const NearView& a, const NearTask& tk, int warp, int lane,
                                           double (&r)[kRowsPerWarp], double (&dW)[NR], unsigned char* vb) {
    const int n = a.n;
    const int nsl = near_slices<double>(tk, n);
    const bool on = lane < tk.ns;
    const size_t col = (size_t)tk.s0 + (on ? lane : 0);   // lanes past ns zero-fill from a valid address
    if constexpr (TC) {
        if (!tk.kind) return;   // the window rows come with the slices' pipeline stages (producer)
    }
    if (!tk.kind) {
        const int b0 = wrap(n - tk.k0, a.WD);
#pragma unroll
        for (int m = 0; m < VR / kNearConsumers; ++m) {
            const int v = warp + m * kNearConsumers;
            const int k = v / NR, q = v % NR;
            int slot = b0 - k;                         // k < W < WD: one wrap at most
            slot += slot < 0 ? a.WD : 0;
            if (k < nsl && FDPH_IDX(slot >= 0 && slot < a.WD && col < (size_t)a.N, a.err)) {
                const size_t off = q * a.rs_D + (size_t)slot * a.N + col;
                if constexpr (sizeof(R) == 4) {
                    cp_async_4((R*)vb + v * 32 + lane, a.Dring32 + off, on ? 4 : 0);
                } else {
                    cp_async_8((R*)vb + v * 32 + lane, a.Dring + off, on ? 8 : 0);
                }
            }
        }
    } else {
        const int t = n - tk.W;
#pragma unroll
        for (int q = 0; q < NR; ++q)
            dW[q] = (on && t >= 0 && tk.k1 > 1) ? a.Dring[q * a.rs_D + (size_t)wrap(t, a.WD) * a.N + col] : 0.0;
#pragma unroll
        for (int m = 0; m < kRowsPerWarp; ++m) {
            const int v = warp + m * kNearConsumers;
            const int k = v / NR, q = v % NR, ai = tk.k0 + k;
            double x = 0.0;
            if (on && k < nsl) {
                if (ai == 0) x = t >= 0 ? a.Cring[q * a.rs_C + (size_t)wrap(t, a.WC) * a.N + col] : 0.0;
                else if (FDPH_IDX(tk.vstate + (long long)(ai - 1) * tk.ns + lane < a.rs_vstate, a.err))
                    x = a.vstate[q * a.rs_vstate + tk.vstate + (size_t)(ai - 1) * tk.ns + lane];
            }
            r[m] = x;
        }
    }
}

template <class R, int NR>
__device__ __forceinline__ void near_commit(const NearView& a, const NearTask& tk, int warp, int lane,
                                            const double (&r)[kRowsPerWarp], const double (&dW)[NR],
                                            unsigned char* vb) {
    if (!tk.kind) return;   // window rows: asynchronous copies, awaited by cp_async_wait_all
    const int nsl = near_slices<double>(tk, a.n);
#pragma unroll
    for (int m = 0; m < kRowsPerWarp; ++m) {
        const int v = warp + m * kNearConsumers;
        const int k = v / NR, q = v % NR, ai = tk.k0 + k;
        if (k < nsl) {
            double x = r[m];
            if (tk.kind && ai > 0) {
                x = 0.0;
                if (lane < tk.ns) {
                    x = a.rho[ai - 1] * r[m] + dW[q];
                    if (FDPH_IDX(tk.vstate + (long long)(ai - 1) * tk.ns + lane < a.rs_vstate, a.err))
                        a.vstate[q * a.rs_vstate + tk.vstate + (size_t)(ai - 1) * tk.ns + lane] = x;
                }
            }
            ((R*)vb)[v * 32 + lane] = (R)x;
        }
    }
}

// Near-field storage: window slices in H; aux slices (static tile, tail coefficients) in the aux
// type (FP32 when the window is FP16: the static term multiplies the cumulative slip, so its
// coefficients keep FP32); slip-rate vectors and products in the row type R.
template <class H> struct NearTypes { using Aux = H; using Row = H; };
template <> struct NearTypes<__half> { using Aux = float; using Row = float; };

template <class H, int NR = 1>
struct NearCfg {
    using R = typename NearTypes<H>::Row;
    // tensor-core window slices (FP16 window, several right-hand sides): their rows and scales ride
    // in the slices' stages (kTcPer slices a stage), so the vector buffers only hold aux rows
    static constexpr bool tc = std::is_same<H, __half>::value && NR >= 2;
    // vector rows of one item: 64, or 128 for several right-hand sides in FP32 rows (their window
    // rows go by cp.async, without registers), so that items stay 128 / NR slices long
    static constexpr int vec_rows = tc ? kTcVecRows : NR >= 2 && sizeof(R) == 4 ? 2 * kChunk : kChunk;
    static constexpr int tc_rows_bytes = kTcPer * NR * kTcBox * 4;
    static constexpr int tc_scale_bytes = kTcPer * (NR > 4 ? NR : 4) * 4;
    // one stage: the slices, then (tensor cores) a 128-byte aligned TMA landing zone for rows + scales
    static constexpr int stage_bytes =
        tc ? kNearStageBytes + (tc_rows_bytes + tc_scale_bytes + 127) / 128 * 128 : kNearStageBytes;
    // shared-memory pipeline depth, within two CTAs per SM next to the vector buffers and the
    // partial sums of the right-hand sides
    static constexpr int stages = NR >= 8 ? 3 : NR >= 2 ? 4 : sizeof(R) == 4 ? 5 : 4;
    static constexpr int vec_bytes = vec_rows * 32 * (int)sizeof(R);
    // (+ 128 bytes of room to align the stages for the TMA boxes)
    static constexpr int smem = stages * stage_bytes + 2 * vec_bytes + (tc ? 128 : 0);
};

// the longest work item (window slices) of a plan: the item's vector rows over its right-hand sides
static inline int near_max_chunk(int nrhs, int precision) {
    if (nrhs >= 2 && precision == FDPH_FP16) return kChunk;   // tensor cores: rows ride in the stages
    return (nrhs >= 2 && precision != FDPH_FP64 ? 2 * kChunk : kChunk) / nrhs;
}

// the longest aux item (static tile and tail slices): its NR rows a slice fill the vector buffer
static inline int near_aux_chunk(int nrhs, int precision) {
    return (nrhs >= 2 && precision == FDPH_FP16 ? kTcVecRows : kChunk) / nrhs;
}

// slice . vector for one receiver lane: 16-byte loads of the source-interleaved slice (plan.h)
// and of the vector row; products and the sum in the row type
__device__ __forceinline__ float slice_dot(const float* buf, const float* vrow, int ns, int nr, int li) {
    const float4* tile = (const float4*)buf + li;
    const float4* d = (const float4*)vrow;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    const int nb = (ns + 3) >> 2;
    if (nb == 8 && nr == 32) {
#pragma unroll
        for (int jb = 0; jb < 8; ++jb) {
            const float4 x = tile[jb * 32];
            const float4 y = d[jb];
            s0 = fmaf(x.x, y.x, s0);
            s1 = fmaf(x.y, y.y, s1);
            s2 = fmaf(x.z, y.z, s2);
            s3 = fmaf(x.w, y.w, s3);
        }
    } else {
        for (int jb = 0; jb < nb; ++jb) {
            const float4 x = tile[jb * nr];
            const float4 y = d[jb];
            s0 = fmaf(x.x, y.x, s0);
            s1 = fmaf(x.y, y.y, s1);
            s2 = fmaf(x.z, y.z, s2);
            s3 = fmaf(x.w, y.w, s3);
        }
    }
    return (s0 + s1) + (s2 + s3);
}

__device__ __forceinline__ double slice_dot(const double* buf, const double* vrow, int ns, int nr, int li) {
    const double2* tile = (const double2*)buf + li;
    const double2* d = (const double2*)vrow;
    double s0 = 0.0, s1 = 0.0;
    const int nb = (ns + 1) >> 1;
    for (int jb = 0; jb < nb; ++jb) {
        const double2 x = tile[jb * nr];
        const double2 y = d[jb];
        s0 = fma(x.x, y.x, s0);
        s1 = fma(x.y, y.y, s1);
    }
    return s0 + s1;
}

__device__ __forceinline__ float half8_dot(const uint4 x, const float4 y0, const float4 y1, float acc) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&x.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&x.y));
    const float2 c = __half22float2(*reinterpret_cast<const __half2*>(&x.z));
    const float2 e = __half22float2(*reinterpret_cast<const __half2*>(&x.w));
    acc = fmaf(a.x, y0.x, acc);
    acc = fmaf(a.y, y0.y, acc);
    acc = fmaf(b.x, y0.z, acc);
    acc = fmaf(b.y, y0.w, acc);
    acc = fmaf(c.x, y1.x, acc);
    acc = fmaf(c.y, y1.y, acc);
    acc = fmaf(e.x, y1.z, acc);
    return fmaf(e.y, y1.w, acc);
}

// FP16 slices: 8 sources per 16-byte load, converted to FP32
__device__ __forceinline__ float slice_dot(const __half* buf, const float* vrow, int ns, int nr, int li) {
    const uint4* tile = (const uint4*)buf + li;
    const float4* d = (const float4*)vrow;
    float s0 = 0.f, s1 = 0.f;
    const int nb = (ns + 7) >> 3;
    if (nb == 4 && nr == 32) {
#pragma unroll
        for (int jb = 0; jb < 4; jb += 2) {
            s0 = half8_dot(tile[jb * 32], d[2 * jb], d[2 * jb + 1], s0);
            s1 = half8_dot(tile[(jb + 1) * 32], d[2 * jb + 2], d[2 * jb + 3], s1);
        }
    } else {
        for (int jb = 0; jb < nb; ++jb) s0 = half8_dot(tile[jb * nr], d[2 * jb], d[2 * jb + 1], s0);
    }
    return s0 + s1;
}
static_assert(17 <= kChunk, "aux vectors (1 + 16 tail terms) fit a vector buffer");

// The same slice products for NR right-hand sides (vector rows vrows, vrows + 32, ...): each
// coefficient load serves the NR vectors; per right-hand side the operations and their order are
// those of slice_dot, so every right-hand side gets the single-RHS result bit for bit.
template <int NR>
__device__ __forceinline__ void slice_dot_nr(const float* buf, const float* vrows, int ns, int nr, int li,
                                             float (&out)[NR]) {
    const float4* tile = (const float4*)buf + li;
    float s0[NR], s1[NR], s2[NR], s3[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) s0[q] = s1[q] = s2[q] = s3[q] = 0.f;
    const int nb = (ns + 3) >> 2;
    const int stride = nb == 8 && nr == 32 ? 32 : nr;
    for (int jb = 0; jb < nb; ++jb) {
        const float4 x = tile[jb * stride];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const float4 y = ((const float4*)(vrows + q * 32))[jb];
            s0[q] = fmaf(x.x, y.x, s0[q]);
            s1[q] = fmaf(x.y, y.y, s1[q]);
            s2[q] = fmaf(x.z, y.z, s2[q]);
            s3[q] = fmaf(x.w, y.w, s3[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) out[q] = (s0[q] + s1[q]) + (s2[q] + s3[q]);
}

template <int NR>
__device__ __forceinline__ void slice_dot_nr(const double* buf, const double* vrows, int ns, int nr, int li,
                                             double (&out)[NR]) {
    const double2* tile = (const double2*)buf + li;
    double s0[NR], s1[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) s0[q] = s1[q] = 0.0;
    const int nb = (ns + 1) >> 1;
    for (int jb = 0; jb < nb; ++jb) {
        const double2 x = tile[jb * nr];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const double2 y = ((const double2*)(vrows + q * 32))[jb];
            s0[q] = fma(x.x, y.x, s0[q]);
            s1[q] = fma(x.y, y.y, s1[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) out[q] = s0[q] + s1[q];
}

template <int NR>
__device__ __forceinline__ void slice_dot_nr(const __half* buf, const float* vrows, int ns, int nr, int li,
                                             float (&out)[NR]) {
    const uint4* tile = (const uint4*)buf + li;
    float s0[NR], s1[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) s0[q] = s1[q] = 0.f;
    const int nb = (ns + 7) >> 3;
    if (nb == 4 && nr == 32) {
        for (int jb = 0; jb < 4; jb += 2) {
            const uint4 x0 = tile[jb * 32], x1 = tile[(jb + 1) * 32];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const float4* d = (const float4*)(vrows + q * 32);
                s0[q] = half8_dot(x0, d[2 * jb], d[2 * jb + 1], s0[q]);
                s1[q] = half8_dot(x1, d[2 * jb + 2], d[2 * jb + 3], s1[q]);
            }
        }
    } else {
        for (int jb = 0; jb < nb; ++jb) {
            const uint4 x = tile[jb * nr];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const float4* d = (const float4*)(vrows + q * 32);
                s0[q] = half8_dot(x, d[2 * jb], d[2 * jb + 1], s0[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) out[q] = s0[q] + s1[q];
}

// ---- several right-hand sides on the tensor cores (FP16 window, NR >= 2)
//
// One slice is a 32 x 32 (receivers x sources) FP16 tile times the slip rates of the NR right-hand
// sides, a dense (32 x 32) x (32 x NR) contraction: warp-level mma.sync m16n8k16 (FP16 inputs, FP32
// accumulation), two 16-receiver tiles x two 16-source steps.  The A fragments come straight from
// the stage with ldmatrix (the source-interleaved slice layout of plan.h puts 8 sources of one
// receiver in 16 contiguous bytes, the rows of an 8 x 8 ldmatrix tile).  The slip rates come from
// the ring's FP16 (hi, lo) copy (tc_rows_kernel: each ring row scaled by a power of two that puts
// its largest entry in [2^13, 2^14), hi + lo carrying it to ~2^-22 relative, 2^-39 of the row's
// largest entry absolute), so that the only rounding of the FP16 path remains that of the stored
// coefficients.  hi and lo are separate B columns: one 8-column pass holds both for NR <= 4
// (columns q and q + NR), NR = 8 takes a hi pass and a lo pass into the same accumulator; the B
// fragments are packed from the (hi, lo) pairs with byte permutes.  Each slice's products are
// scaled back per column by its row's 2^-sh and added to the item's FP32 sums.
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_16816(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// S window slices at once (sl[s]: stage copy; rows[s]: their NR (hi, lo) rows of kTcBox words from
// the source s0; sc[s]: their scales, right-hand side q at sc[s][q sstride]) into the warp's
// accumulators acc[m-tile][fragment] (rows g,
// g + 8 of each 16-receiver tile, columns 2t, 2t + 1, with g = lane / 4, t = lane % 4).  All
// fragments are loaded first and the MMAs of the S slices and two receiver tiles interleave, so
// that 2 S independent accumulator chains are in flight.
template <int NR, int S>
__device__ __forceinline__ void tc_slices(const __half* const (&sl)[S], const unsigned* const (&rows)[S],
                                          const float* const (&sc)[S], int sstride, int nr, int ns, int lane,
                                          float (&acc)[2][4]) {
    static_assert(NR == 2 || NR == 4 || NR == 8, "tensor-core slices take 2, 4 or 8 right-hand sides");
    const int ng = (ns + 7) >> 3;          // 8-source groups of the slice (zero-padded)
    const int nks = (ng + 1) >> 1;         // 16-source steps
    const int nmt = nr > 16 ? 2 : 1;       // 16-receiver tiles
    constexpr int npass = (2 * NR + 7) / 8;
    const int g = lane >> 2, t = lane & 3;
    const int mq = lane >> 3, mr = lane & 7;   // ldmatrix: lane gives row mr of matrix mq
    float c[S][2][4];
#pragma unroll
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int f = 0; f < 4; ++f) c[q][mt][f] = 0.f;
    for (int kk = 0; kk < nks; ++kk) {
        // B column g of pass p: virtual row 8 p + g = right-hand side (8p + g) % NR, part
        // ((8p + g) / NR) & 1 (0 hi, 1 lo; NR = 2 repeats its four columns, unused); sources
        // 16 kk + 2t, + 1 (b[0]) and 16 kk + 8 + 2t, + 1 (b[1]), zero past ns
        unsigned b[S][npass][2], a[S][2][4];
#pragma unroll
        for (int q = 0; q < S; ++q) {
#pragma unroll
            for (int p = 0; p < npass; ++p) {
                const int vr = 8 * p + g;
                // (32-bit loads: the row starts at the remainder of s0, not 8-byte aligned in general)
                const unsigned* br = rows[q] + (vr % NR) * kTcBox + 2 * t + 16 * kk;
                const unsigned sel = ((vr / NR) & 1) ? 0x7632u : 0x5410u;   // high or low halves of two pairs
                b[q][p][0] = __byte_perm(br[0], br[1], sel);
                b[q][p][1] = __byte_perm(br[8], br[9], sel);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                // receivers past nr read valid rows of the slice (their products land in unused
                // rows); a source group past ng (the upper half of the last 16-source step) is
                // zeroed, since the TMA box carries the next elements' slip rates there (sources
                // past ns inside the last group meet the slice's zero padding)
                const int i = min(16 * mt + 8 * (mq & 1) + mr, nr - 1);
                const int gg = min(2 * kk + (mq >> 1), ng - 1);
                if (mt < nmt) {
                    ldsm_x4(a[q][mt], sl[q] + ((size_t)gg * nr + i) * 8);
                    if (2 * kk + 1 >= ng) a[q][mt][2] = a[q][mt][3] = 0u;
                }
            }
        }
#pragma unroll
        for (int p = 0; p < npass; ++p)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int q = 0; q < S; ++q)
                    if (mt < nmt) mma_16816(c[q][mt], a[q][mt], b[q][p]);
    }
    // column v holds right-hand side v % NR
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const float s0 = sc[q][((2 * t) % NR) * sstride], s1 = sc[q][((2 * t + 1) % NR) * sstride];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            acc[mt][0] = fmaf(c[q][mt][0], s0, acc[mt][0]);
            acc[mt][1] = fmaf(c[q][mt][1], s1, acc[mt][1]);
            acc[mt][2] = fmaf(c[q][mt][2], s0, acc[mt][2]);
            acc[mt][3] = fmaf(c[q][mt][3], s1, acc[mt][3]);
        }
    }
}

// The item's sums of one warp into red[q][receiver] (FP64): the hi and lo columns of a right-hand
// side are added first (NR <= 4), then scaled by the window's storage scale kinv.
template <int NR>
__device__ __forceinline__ void tc_item_to_red(float (&acc)[2][4], int lane, int nr, float kinv, double (*red)[32]) {
    if constexpr (NR < 8) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int f = 0; f < 4; ++f) acc[mt][f] += __shfl_xor_sync(0xffffffffu, acc[mt][f], NR / 2);
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int v = 2 * t + (f & 1), r = 16 * mt + g + 8 * (f >> 1);
            if (v < NR) red[v][r] = r < nr ? (double)(acc[mt][f] * kinv) : 0.0;
        }
}

// Near field (App. E), persistent and warp-specialised.  Each CTA owns a list of work items
// (window slices [k0, k1) of a leaf, or the leaf's aux slices: static tile and exponential
// tail).  One producer thread streams the items' slices through a ring of shared-memory stages
// (cp.async.bulk, full/empty mbarriers), continuing across item boundaries.  The consumer warps
// load the vectors of the next item into a second shared buffer while they consume the current
// one; consumer warp w takes slices w, w + kNearConsumers, ... of each stage, lane i = receiver i,
// reading its coefficients and the vector 16 bytes at a time.  At the end of an item the
// consumers' sums are combined in FP64 into the item's partial-sum slot.  kBatch: the items of
// several plans in one launch (fdph_batch_run); item tk belongs to plan scen[tk.scen].  NR: the
// plan's right-hand sides, consumed together (each coefficient read once per step, the vectors
// of all right-hand sides in the item's vector buffer).
// (one right-hand side: registers bounded as for three CTAs per SM, ~128 per thread, although
// shared memory admits two: the far-field kernels of the step then find room beside it and
// finish alongside it instead of after it)
template <class T, class H, bool kBatch, int NR>
__global__ void __launch_bounds__(kNearThreads, NR == 1 ? 3 : 2) near_kernel(StepArgs<T> a, const StepArgs<T>* scen) {
    using C = NearCfg<H, NR>;
    using A = typename NearTypes<H>::Aux;
    using R = typename NearTypes<H>::Row;
    // FP16 windows with several right-hand sides: window slices on the tensor cores (tc_slice)
    constexpr bool kTC = std::is_same<H, __half>::value && NR >= 2 && !kBatch;
    extern __shared__ __align__(128) unsigned char near_smem[];
    __shared__ __align__(8) unsigned long long full[C::stages], empty[C::stages];
    __shared__ double red[2][kNearConsumers][NR][32];
    __shared__ __align__(16) NearTask tcache[kTaskCache];   // this CTA's first work items
    __shared__ int abort_flag;
    const NearView v0 = kBatch ? NearView{} : near_view(a);
    auto view = [&](const NearTask& tk) -> NearView { return kBatch ? near_view(scen[tk.scen]) : v0; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t0 = a.cta_ptr[blockIdx.x], t1 = a.cta_ptr[blockIdx.x + 1];
    unsigned char* stage0 = near_smem;
    if constexpr (C::tc)   // TMA boxes land on 128-byte boundaries (the configuration reserves the room)
        stage0 = (unsigned char*)(((unsigned long long)near_smem + 127) & ~127ull);
    unsigned char* vbuf = stage0 + C::stages * C::stage_bytes;
    {
        const int nt = min(t1 - t0, kTaskCache) * (int)(sizeof(NearTask) / sizeof(int4));
        for (int e = threadIdx.x; e < nt; e += blockDim.x)
            ((int4*)tcache)[e] = ((const int4*)(a.tasks + t0))[e];
    }
    auto task = [&](int ti) -> NearTask { return ti - t0 < kTaskCache ? tcache[ti - t0] : a.tasks[ti]; };
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kNearConsumers);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    int g = 0;   // running stage counter, identical in producer and consumers
    if (warp == kNearConsumers) {
        // ---------------- producer (one thread)
        if (lane == 0) {
            const unsigned long long policy = l2_evict_first_policy();   // coefficients are read once
            for (int ti = t0; ti < t1; ++ti) {
                const NearTask tk = task(ti);
                const NearView v = view(tk);
                const int esz = tk.kind ? (int)sizeof(A) : (int)sizeof(H);
                const int nsl = near_slices<T>(tk, v.n);
                const bool tcw = kTC && !tk.kind;   // tensor-core window item: rows ride in the stages
                const int per = tcw ? kTcPer : min(kMaxPer, max(1, kNearStageBytes / (tk.sl * esz)));
                const int nst = nsl > 0 ? (nsl + per - 1) / per : 0;
                const unsigned char* src = tk.kind ? (const unsigned char*)((const A*)v.stat + tk.off)
                                                   : (const unsigned char*)((const H*)v.tensor + tk.off);
                for (int q = 0; q < nst; ++q, ++g) {
                    const int s = g % C::stages;
                    if (!mbar_wait_bounded(&empty[s], (unsigned)(((g / C::stages) & 1) ^ 1))) {
                        abort_flag = 1;
                        atomicExch(v.err, kErrTimeout);
                    }
                    const int cnt = min(per, nsl - q * per);
                    const unsigned bytes = (unsigned)(cnt * tk.sl * esz);
                    // (index check: the stage's slices lie inside the stored coefficients; a failed
                    // check completes the stage without data)
                    const bool ok = FDPH_IDX(tk.off + (long long)(q * per + cnt) * tk.sl <= (tk.kind ? v.len_aux : v.len_tensor),
                                             v.err);
                    unsigned char* stage = stage0 + s * C::stage_bytes;
                    fence_proxy_async();
                    mbar_expect_tx(&full[s], (ok ? bytes : 0u) + (tcw ? (unsigned)(C::tc_rows_bytes + C::tc_scale_bytes) : 0u));
                    if (ok)
                        bulk_g2s_hint(stage, src + (size_t)q * per * tk.sl * esz, bytes, &full[s], policy);
                    if constexpr (kTC) {
                        if (tcw) {
                            // the stage's window rows of every right-hand side with one TMA tensor copy: a
                            // box of kTcBox sources from s0 rounded down to a multiple of 4 (the 16-byte
                            // rule of the innermost coordinate; the consumers index from the remainder) x
                            // nrhs x kTcPer slots from the oldest the stage may hold (the mirrored ring
                            // keeps them contiguous; past it the box reads zeros), then their scales
                            const int z0 = wrap(v.n - tk.k0 - (q * kTcPer + kTcPer - 1), v.WD);
                            tma_load_3d(stage + kNearStageBytes, v.tmap16, tk.s0 & ~3, 0, z0, &full[s]);
                            tma_load_2d(stage + kNearStageBytes + C::tc_rows_bytes,
                                        (const unsigned char*)v.tmap16 + sizeof(CUtensorMap), 0, z0, &full[s]);
                        }
                    }
                }
            }
        }
    } else {
        // ---------------- consumers
        // Vector rows are staged one item ahead (registers for aux rows, cp.async for window rows).
        // Tensor-core plans stage nothing: their window rows ride in the stages, and their few aux
        // items load their rows when they start, so that no staged aux rows stay live in
        // registers across the MMA loop of a window item
        constexpr bool kAhead = !kTC;
        NearTask nxt;
        NearView vn;
        if (t0 < t1) {
            nxt = task(t0);
            vn = view(nxt);
            if constexpr (kAhead) {
                double rows[kRowsPerWarp], dW[NR];
                near_issue<R, NR, C::vec_rows, kTC>(vn, nxt, warp, lane, rows, dW, vbuf);
                near_commit<R, NR>(vn, nxt, warp, lane, rows, dW, vbuf);
            }
        }
        cp_async_wait_all();
        consumer_barrier();
        [[maybe_unused]] double rows[kAhead ? kRowsPerWarp : 1], dW[kAhead ? NR : 1];
        int par = 0;
        for (int ti = t0; ti < t1; ++ti, par ^= 1) {
            const NearTask tk = nxt;
            const NearView v = vn;
            // the next item's vector loads stay in flight while this item is consumed
            if (ti + 1 < t1) {
                nxt = task(ti + 1);
                vn = view(nxt);
                if constexpr (kAhead)
                    near_issue<R, NR, C::vec_rows, kTC>(vn, nxt, warp, lane, rows, dW, vbuf + (par ^ 1) * C::vec_bytes);
            }
            if constexpr (!kAhead) {
                if (tk.kind) {   // an aux item of a tensor-core plan: its rows now
                    double ar[kRowsPerWarp], adw[NR];
                    near_issue<R, NR, C::vec_rows, kTC>(v, tk, warp, lane, ar, adw, vbuf + par * C::vec_bytes);
                    near_commit<R, NR>(v, tk, warp, lane, ar, adw, vbuf + par * C::vec_bytes);
                    consumer_barrier();
                }
            }
            const unsigned char* vrows = vbuf + par * C::vec_bytes;
            const int esz = tk.kind ? (int)sizeof(A) : (int)sizeof(H);
            const int nsl = near_slices<T>(tk, v.n);
            // leaves of at most 16 receivers: the warp splits into 32 / span lane groups of span
            // lanes, each taking its own slices (lane = group * span + receiver); tensor-core
            // slices take the whole warp
            const bool tc = kTC && !tk.kind;
            const int per = tc ? kTcPer : min(kMaxPer, max(1, kNearStageBytes / (tk.sl * esz)));
            const int nst = nsl > 0 ? (nsl + per - 1) / per : 0;
            const int span = tc || tk.nr > 16 ? 32 : tk.nr > 8 ? 16 : tk.nr > 4 ? 8 : tk.nr > 2 ? 4 : tk.nr > 1 ? 2 : 1;
            const int ngrp = 32 / span, grp = lane / span, ri = lane - grp * span;
            const int li = ri < tk.nr ? ri : 0;         // lanes past nr read a valid element, unused
            R acc[NR];
            double accd[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                acc[r] = (R)0;
                accd[r] = 0.0;
            }
            float tacc[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int f = 0; f < 4; ++f) tacc[mt][f] = 0.f;
            for (int q = 0; q < nst; ++q, ++g) {
                const int s = g % C::stages;
                const int cnt = min(per, nsl - q * per);
                if (!mbar_wait_bounded(&full[s], (unsigned)((g / C::stages) & 1))) {
                    abort_flag = 1;
                    atomicExch(v.err, kErrTimeout);
                }
                const unsigned char* buf = stage0 + s * C::stage_bytes;
                for (int kk = warp * ngrp + grp; kk < cnt; kk += kNearConsumers * ngrp) {
                    const R* vrow = (const R*)(vrows + (size_t)(q * per + kk) * NR * 32 * sizeof(R));
                    if constexpr (kTC) {
                        if (tc) {
                            // this warp's slices kk and kk + kNearConsumers of the stage together;
                            // stage slice kk (ring slot of step n - k0 - q kTcPer - kk): box slot
                            // kTcPer - 1 - kk of the rows and scales that came with the stage
                            const unsigned* rw = (const unsigned*)(buf + kNearStageBytes) + (tk.s0 & 3);
                            auto rows_of = [&](int k) { return rw + (size_t)(kTcPer - 1 - k) * NR * kTcBox; };
                            constexpr int SR = NR > 4 ? NR : 4;
                            const float* scl = (const float*)(buf + kNearStageBytes + C::tc_rows_bytes);
                            auto scale_of = [&](int k) { return scl + (kTcPer - 1 - k) * SR; };
                            if (kk + kNearConsumers < cnt) {
                                const __half* const sl2[2] = {(const __half*)buf + (size_t)kk * tk.sl,
                                                              (const __half*)buf + (size_t)(kk + kNearConsumers) * tk.sl};
                                const unsigned* const rw2[2] = {rows_of(kk), rows_of(kk + kNearConsumers)};
                                const float* const sc2[2] = {scale_of(kk), scale_of(kk + kNearConsumers)};
                                tc_slices<NR, 2>(sl2, rw2, sc2, 1, tk.nr, tk.ns, lane, tacc);
                                kk += kNearConsumers;
                            } else {
                                const __half* const sl1[1] = {(const __half*)buf + (size_t)kk * tk.sl};
                                const unsigned* const rw1[1] = {rows_of(kk)};
                                const float* const sc1[1] = {scale_of(kk)};
                                tc_slices<NR, 1>(sl1, rw1, sc1, 1, tk.nr, tk.ns, lane, tacc);
                            }
                            continue;
                        }
                    }
                    if constexpr (NR == 1) {
                        if (tk.kind)   // static and tail slices: FP64 across slices
                            accd[0] += (double)slice_dot((const A*)buf + (size_t)kk * tk.sl, vrow, tk.ns, tk.nr, li);
                        else
                            acc[0] += slice_dot((const H*)buf + (size_t)kk * tk.sl, vrow, tk.ns, tk.nr, li);
                    } else {
                        R t[NR];
                        if (tk.kind) {
                            slice_dot_nr<NR>((const A*)buf + (size_t)kk * tk.sl, vrow, tk.ns, tk.nr, li, t);
#pragma unroll
                            for (int r = 0; r < NR; ++r) accd[r] += (double)t[r];
                        } else if constexpr (!kTC) {   // (with kTC window slices took tc_slice)
                            slice_dot_nr<NR>((const H*)buf + (size_t)kk * tk.sl, vrow, tk.ns, tk.nr, li, t);
#pragma unroll
                            for (int r = 0; r < NR; ++r) acc[r] += t[r];
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if constexpr (kAhead)
                if (ti + 1 < t1) near_commit<R, NR>(vn, nxt, warp, lane, rows, dW, vbuf + (par ^ 1) * C::vec_bytes);
            if (tc) {
                if constexpr (kTC) tc_item_to_red<NR>(tacc, lane, tk.nr, v.kinv, red[par][warp]);
            } else {
                // window sums carry the storage scale of the window (FP16), aux sums none
                const double ks = tk.kind ? 1.0 : (double)v.kinv;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    double tot = (double)acc[r] * ks + accd[r];
                    for (int o = span; o < 32; o <<= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
                    red[par][warp][r][lane] = lane < tk.nr ? tot : 0.0;
                }
            }
            cp_async_wait_all();
            consumer_barrier();   // also publishes the next item's vectors
            if (warp == 0 && FDPH_IDX((long long)tk.item * 32 + 32 <= v.rs_partial, v.err)) {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    double sum = 0.0;
                    for (int w = 0; w < kNearConsumers; ++w) sum += red[par][w][r][lane];
                    v.partial[r * v.rs_partial + (size_t)tk.item * 32 + lane] = sum;
                }
            }
        }
    }
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) {
        // a wait gave up: give the copies that may still be in flight a bounded chance to land
        for (int s = 0; s < C::stages; ++s) {
            (void)mbar_wait_bounded(&full[s], 0u);
            (void)mbar_wait_bounded(&full[s], 1u);
        }
    }
}

// Eq. 39: one warp per task of receivers of one block; 2^lg lanes per receiver split the rank
// index l, so the receiver's factor row f_{i, .} and ring slot row are read coalesced; the value
// f_{., i} . Tbar'[n - dm_i] goes to the receiver's CSR slot.  A block kept exact with F = I
// reads one ring entry per receiver (2^lg = 1).
template <class T>
__device__ __forceinline__ void far_eval_body(const StepArgs<T>& a, int w, int lane) {
    const int n = step_index(a);
    const int4 tk = a.ev_tasks[w];
    const SbDev& sb = a.sbs[tk.x];
    const int lg = tk.w, G = 1 << lg;
    const int gi = lane >> lg, lj = lane & (G - 1);
    const int il = tk.y + gi;
    bool valid = gi < tk.z;
    double s = 0.0;
    if (valid)   // (a failed index check leaves this receiver's lanes out; the shuffles take all lanes)
        valid = FDPH_IDX((sb.kind == SB_TR ? sb.zring + (long long)sb.LZ * sb.rank <= a.rs_zring
                                           : sb.ring + (long long)sb.L * sb.rank <= a.rs_ring) &&
                             (sb.ident != 1 || il < sb.rank) && a.e_pos[sb.e0 + il] < a.rs_fval,
                         a.err);
    if (valid) {
        const bool tr = sb.kind == SB_TR;
        const double* base = tr ? a.zring + sb.zring : a.ring + sb.ring;
        const int len = tr ? sb.LZ : sb.L;
        const int rank = sb.rank;
        const int t = n - a.ints[sb.dm + il];
        const double* r = base + (long long)wrap(t, len) * rank;
        if (a.phi) {   // exact delay dm_i + phi_i: linear interpolation with the next older step
            const double ph = a.phi[sb.phi + il];
            const double* r1 = base + (long long)wrap(t - 1, len) * rank;
            if (sb.ident == 1) {
                s = (1.0 - ph) * r[il] + ph * r1[il];
            } else {
                const T* f = a.fac + sb.f + (long long)il * rank;
                for (int l = lj; l < rank; l += G) s += (double)f[l] * ((1.0 - ph) * r[l] + ph * r1[l]);
            }
        } else if (sb.ident == 1) {
            s = r[il];
        } else {
            const T* f = a.fac + sb.f + (long long)il * rank;
            for (int l = lj; l < rank; l += G) s += (double)f[l] * r[l];
        }
    }
    for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (valid && lj == 0) a.fval[a.e_pos[sb.e0 + il]] = s;
}

// The same for NR right-hand sides at once: the task, delays and factor row are read once (per
// right-hand side the single-RHS order of operations)
template <class T, int NR>
__device__ __forceinline__ void far_eval_body_nr(const StepArgs<T>& a, int w, int lane) {
    const int n = step_index(a);
    const int4 tk = a.ev_tasks[w];
    const SbDev& sb = a.sbs[tk.x];
    const int lg = tk.w, G = 1 << lg;
    const int gi = lane >> lg, lj = lane & (G - 1);
    const int il = tk.y + gi;
    bool valid = gi < tk.z;
    double s[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) s[r] = 0.0;
    if (valid)
        valid = FDPH_IDX((sb.kind == SB_TR ? sb.zring + (long long)sb.LZ * sb.rank <= a.rs_zring
                                           : sb.ring + (long long)sb.L * sb.rank <= a.rs_ring) &&
                             (sb.ident != 1 || il < sb.rank) && a.e_pos[sb.e0 + il] < a.rs_fval,
                         a.err);
    if (valid) {
        const bool tr = sb.kind == SB_TR;
        const double* base = tr ? a.zring + sb.zring : a.ring + sb.ring;
        const long long rs = tr ? a.rs_zring : a.rs_ring;
        const int len = tr ? sb.LZ : sb.L;
        const int rank = sb.rank;
        const int t = n - a.ints[sb.dm + il];
        const double* rw = base + (long long)wrap(t, len) * rank;
        if (a.phi) {
            const double ph = a.phi[sb.phi + il];
            const double* rw1 = base + (long long)wrap(t - 1, len) * rank;
            if (sb.ident == 1) {
#pragma unroll
                for (int r = 0; r < NR; ++r) s[r] = (1.0 - ph) * rw[r * rs + il] + ph * rw1[r * rs + il];
            } else {
                const T* f = a.fac + sb.f + (long long)il * rank;
                for (int l = lj; l < rank; l += G) {
                    const double fl = (double)f[l];
#pragma unroll
                    for (int r = 0; r < NR; ++r) s[r] += fl * ((1.0 - ph) * rw[r * rs + l] + ph * rw1[r * rs + l]);
                }
            }
        } else if (sb.ident == 1) {
#pragma unroll
            for (int r = 0; r < NR; ++r) s[r] = rw[r * rs + il];
        } else {
            const T* f = a.fac + sb.f + (long long)il * rank;
            for (int l = lj; l < rank; l += G) {
                const double fl = (double)f[l];
#pragma unroll
                for (int r = 0; r < NR; ++r) s[r] += fl * rw[r * rs + l];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r)
        for (int o = G >> 1; o > 0; o >>= 1) s[r] += __shfl_xor_sync(0xffffffffu, s[r], o);
    if (valid && lj == 0) {
        const long long pos = a.e_pos[sb.e0 + il];
#pragma unroll
        for (int r = 0; r < NR; ++r) a.fval[r * a.rs_fval + pos] = s[r];
    }
}

template <class T, int NR>
__global__ void far_eval_kernel(StepArgs<T> a0) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if constexpr (NR == 1) {
        const StepArgs<T> a = rhs_args(a0, blockIdx.y);
        if (w < a.n_evt) far_eval_body(a, w, threadIdx.x & 31);   // warp-uniform
    } else {
        if (w < a0.n_evt) far_eval_body_nr<T, NR>(a0, w, threadIdx.x & 31);
    }
}

// Eq. 39 summed per receiver: one warp per receiver adds its far entries (fixed order) into
// tfar; this runs on the far-field branch, beside the near field
template <class T>
__device__ __forceinline__ void far_sum_body(const StepArgs<T>& a, int p, int lane) {
    double s = 0.0;
    for (int e = a.g_ptr[p] + lane; e < a.g_ptr[p + 1]; e += 32)
        if (FDPH_IDX(e < a.rs_fval, a.err)) s += a.fval[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) a.tfar[p] = s;
}

template <class T, int NR>
__device__ __forceinline__ void far_sum_body_nr(const StepArgs<T>& a, int p, int lane) {
    double s[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) s[r] = 0.0;
    for (int e = a.g_ptr[p] + lane; e < a.g_ptr[p + 1]; e += 32)
        if (FDPH_IDX(e < a.rs_fval, a.err)) {
#pragma unroll
            for (int r = 0; r < NR; ++r) s[r] += a.fval[r * a.rs_fval + e];
        }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        for (int o = 16; o > 0; o >>= 1) s[r] += __shfl_xor_sync(0xffffffffu, s[r], o);
        if (lane == 0) a.tfar[(long long)r * a.N + p] = s[r];
    }
}

template <class T, int NR>
__global__ void far_sum_kernel(StepArgs<T> a0) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if constexpr (NR == 1) {
        const StepArgs<T> a = rhs_args(a0, blockIdx.y);
        if (p < a.N) far_sum_body(a, p, threadIdx.x & 31);   // warp-uniform
    } else {
        if (p < a0.N) far_sum_body_nr<T, NR>(a0, p, threadIdx.x & 31);
    }
}

// the step's output: far-field traction + the receiver's near-field partial sums (a few per
// receiver, fixed order), one thread per receiver, written in the caller's element order
template <class T>
__device__ __forceinline__ void gather_body(const StepArgs<T>& a, int p) {
    const int n = step_index(a);
    double s = a.tfar[p];
    for (int e = a.np_ptr[p]; e < a.np_ptr[p + 1]; ++e)
        if (FDPH_IDX(a.np_idx[e] < a.rs_partial, a.err)) s += a.partial[a.np_idx[e]];
    a.T_out[io_offset(a, n) + a.perm[p]] = s;
}

template <class T>
__global__ void gather_kernel(StepArgs<T> a0) {
    const StepArgs<T> a = rhs_args(a0, blockIdx.y);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < a.N) gather_body(a, p);
}

// Local friction solve (geometry order): T_pred holds the traction change with D_n = 0.
struct FrictionDev {
    const double* tau0;
    const double* k0;      // instantaneous self coefficient K_{ii,0} (< 0)
    double* slip;
    double sigma_n, mu_s, mu_d, Dc, dt;
    int law;               // 0: linear slip weakening, 1: exponential (Sec. 6.2)
};

// D, T: this step's rows (graph replay: row n_dev[0] - n_dev[1] of a step-major array)
__device__ __forceinline__ void friction_body(const FrictionDev& f, int N, int e, double* D, double* T,
                                              const int* n_dev) {
    if (n_dev) {
        const long long off = (long long)(n_dev[0] - n_dev[1]) * N;
        D += off;
        T += off;
    }
    const double tau = f.tau0[e] + T[e];
    const double u = f.slip[e];
    double strength;
    if (f.law == 1) {
        strength = f.sigma_n * (f.mu_d + (f.mu_s - f.mu_d) * exp(-u / f.Dc));
    } else {
        const double w = u < f.Dc ? u / f.Dc : 1.0;
        strength = f.sigma_n * (f.mu_s - (f.mu_s - f.mu_d) * w);
    }
    const double eta = -f.k0[e];
    const double v = tau > strength ? (tau - strength) / eta : 0.0;
    D[e] = v;
    T[e] = tau + f.k0[e] * v;
    f.slip[e] = u + v * f.dt;
}

__global__ void friction_kernel(FrictionDev f, int N, double* D, double* T, const int* n_dev) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < N) friction_body(f, N, e, D, T, n_dev);
}

// ---- the per-step kernels over a batch of plans: one launch covers the work of every plan;
// pre[0..np] are the prefix sums of the plans' work counts (elements, FIR tasks, ...)

// plan of global work index t: the largest p with pre[p] <= t
__device__ __forceinline__ int plan_of(const int* pre, int np, int t) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class T>
__global__ void push_batch(const StepArgs<T>* scen, const int* pre, int np, int zero) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pre[np]) return;
    const int p = plan_of(pre, np, t);
    push_body(scen[p], t - pre[p], zero != 0);
}

template <class T>
__global__ void fir_batch(const StepArgs<T>* scen, const int* pre, int np) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pre[np]) return;
    const int p = plan_of(pre, np, t);
    fir_body(scen[p], t - pre[p]);
}

template <class T>
__global__ void scatter_batch(const StepArgs<T>* scen, const int* pre, int np) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= pre[np]) return;   // warp-uniform
    const int p = plan_of(pre, np, w);
    scatter_body(scen[p], w - pre[p], threadIdx.x & 31);
}

template <class T>
__global__ void trconv_batch(const StepArgs<T>* scen, const int* pre, int np) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= pre[np]) return;
    const int p = plan_of(pre, np, w);
    trconv_body(scen[p], w - pre[p], threadIdx.x & 31);
}

template <class T>
__global__ void far_eval_batch(const StepArgs<T>* scen, const int* pre, int np) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= pre[np]) return;
    const int p = plan_of(pre, np, w);
    far_eval_body(scen[p], w - pre[p], threadIdx.x & 31);
}

template <class T>
__global__ void far_sum_batch(const StepArgs<T>* scen, const int* pre, int np) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= pre[np]) return;
    const int p = plan_of(pre, np, w);
    far_sum_body(scen[p], w - pre[p], threadIdx.x & 31);
}

template <class T>
__global__ void gather_batch(const StepArgs<T>* scen, const int* pre, int np) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pre[np]) return;
    const int p = plan_of(pre, np, t);
    gather_body(scen[p], t - pre[p]);
}

template <class T>
__global__ void friction_batch(const FrictionDev* fr, const StepArgs<T>* scen, const int* pre, int np) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pre[np]) return;
    const int p = plan_of(pre, np, t);
    const StepArgs<T>& a = scen[p];
    friction_body(fr[p], a.N, t - pre[p], const_cast<double*>(a.D_in), a.T_out, a.n_dev);
}

template <class T>
__global__ void advance_batch(const StepArgs<T>* scen, int np) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) *const_cast<int*>(scen[p].n_dev) += 1;
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

// m_S(i, j) = 1 + last k < M with |K_ijk - Kstat_ij dt| >= thr (App. H), 0 if none; M if thr == 0.
// The scan covers only the steps before the tail bound (stress_tail_bound) falls below thr / 2, so it
// costs the pair's wave passage plus its decay to thr rather than M steps.
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
    // steps from the first k whose tail bound is below thr / 2 on cannot reach thr (the bound falls
    // with k; the factor 2 covers rounding): the backward scan starts below that k
    int k_lo = 0, k_hi = M;
    while (k_lo < k_hi) {
        const int mid = (k_lo + k_hi) >> 1;
        if (stress_tail_bound(g.px[pi], g.py[pi], s, (double)mid * dt, dt, mu, c) < 0.5 * thr)
            k_hi = mid;
        else
            k_lo = mid + 1;
    }
    int res = 0;
    for (int k = k_lo - 1; k >= 0; --k) {
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
template <class H, class A>
__global__ void near_fill_kernel(GeoDev g, NearDev L, const int* ms_leaf, double dt, double mu, double c,
                                 double kscale, H* tensor, A* stat) {
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
        constexpr int vh = 16 / (int)sizeof(H), va = 16 / (int)sizeof(A);   // source-interleaved slices (plan.h)
        tensor[L.tensor + (long long)k * L.sl + ((jl / vh) * L.nr + il) * vh + jl % vh] = (H)(v * kscale);
        if (k == 0) {
            const Stress2 w = stress_static(g.px[pi], g.py[pi], s, mu);
            stat[L.stat + ((jl / va) * L.nr + il) * va + jl % va] = (A)((g.nx[pi] * w.x + g.ny[pi] * w.y) * dt);
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
    int nrhs = 1;             // right-hand sides (slip-rate histories) stepped together
    int far_mode = 0;         // 0: Eq. 42 as scatter into delay rings; 1: delayed-history gather
    long long uhist_len = 0;  // far_mode 1: source-value histories (doubles per right-hand side)
    int2 *rec_tasks = nullptr, *gat_tasks = nullptr;
    int n_rec = 0, n_gat = 0;
    double* uhist = nullptr;
    double dt = 0;
    HostPlan hp;
    fdph_stats st;
    // device memory
    std::vector<void*> allocs;
    int* perm = nullptr;
    SbDev* sbs = nullptr;
    void* fac = nullptr;
    int *ints = nullptr, *run_delay = nullptr, *run_start = nullptr, *run_len = nullptr, *src_order = nullptr;
    int* e_pos = nullptr;
    int4 *sc_tasks = nullptr, *ev_tasks = nullptr;
    int n_sct = 0, n_evt = 0;
    double* fval = nullptr;
    int *sfir_ptr = nullptr, *sfir_q = nullptr, *sfir_tmax = nullptr;
    bool sfir = false;        // Eq. 32 source-major (sfir_kernel) rather than sub-block-major
    int *fir_sb = nullptr, *fir_j = nullptr, *tr_sb = nullptr,
        *tr_l = nullptr, *g_ptr = nullptr, *g_sb = nullptr, *g_il = nullptr;
    NearDev* near = nullptr;
    NearTask* tasks = nullptr;
    int* cta_ptr = nullptr;
    int n_cta = 0;
    void* tensor = nullptr;
    void* stat = nullptr;     // aux slices, storage type
    int *np_ptr = nullptr, *np_idx = nullptr;
    int* err = nullptr;
    double* rho = nullptr;
    // rupture state
    bool rupture = false;
    bool predicted = false;   // fdph_predict issued for step n, fdph_commit pending
    FrictionDev fr;
    double *ustate = nullptr, *vstate = nullptr, *trcoef = nullptr, *phi = nullptr;
    // state
    double *Dring = nullptr, *Cring = nullptr, *C = nullptr, *Ccomp = nullptr;
    float* Dring32 = nullptr;   // FP32 copy of Dring (FP32 / FP16 plans)
    __half2* Dring16 = nullptr; // scaled FP16 (hi, lo) copy of Dring (tensor-core near field)
    void* tmap16 = nullptr;     // its TMA tensor map (device memory)
    int NP = 0;                 // Dring16 row length (N rounded up to a multiple of 4)
    double* tfar = nullptr;     // [nrhs][N] far-field traction of the step (scratch)
    std::vector<std::pair<unsigned char*, size_t>> canaries;   // FDPH_CHECK builds: allocation ends
    float* Dscale = nullptr;    // its per-row inverse scales
    double *ring = nullptr, *zring = nullptr, *dhat = nullptr, *partial = nullptr;
    size_t state_bytes = 0;
    // host staging for fdph_step_host
    double *hD = nullptr, *hT = nullptr, *dD = nullptr, *dT = nullptr;
    // per-kernel event timing
    bool prof = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
    double prof_ms[FDPH_NUM_KERNELS] = {0};
    int64_t prof_n[FDPH_NUM_KERNELS] = {0};
    // graphs of one step (fdph_run, fdph_run_host, fdph_rupture_run), replayed with the step index
    // and the call's first step in n_dev[0..1]; kept per (kind, D, T) so that repeated calls on
    // the same buffers reuse them
    struct GraphEntry {
        int kind;
        const void* D;
        const void* T;
        cudaGraphExec_t ex;
    };
    std::vector<GraphEntry> graphs;
    int* n_dev = nullptr;
    int near_priority = 0;    // greatest stream priority of the device
    // near-field schedule inputs (kept so that the work-item length can be changed later)
    std::vector<int32_t> near_W;
    std::vector<char> near_tail;
    int chunk = 0;            // steps of exact kernel per near-field work item
    double kscale = 1.0;      // FP16 window coefficients are stored as K * kscale (a power of two)
    int sched_version = 0;    // bumped whenever the near-field items are rebuilt
    size_t partial_cap = 0;   // capacity of `partial`, in doubles
    // branches of a step that run concurrently with the near field: [0] FIR + scatter,
    // [1] transient convolution + Eq. 39 evaluation (fork after push, join before gather)
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    // fdph_run_host: device staging ring, copy streams and their events
    static const int kIoSlots = 8;
    double *io_D = nullptr, *io_T = nullptr;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in[kIoSlots] = {}, ev_out[kIoSlots] = {}, ev_free[kIoSlots] = {};
};

#ifdef FDPH_CHECK
// FDPH_CHECK builds: every device allocation of a plan ends in kCanaryBytes of a known pattern,
// compared with the pattern whenever the plan synchronises (check_canaries)
static const size_t kCanaryBytes = 256;
static const unsigned char kCanary = 0xA5;
#endif

template <class T>
static int dalloc(fdph_plan_t P, T** out, size_t count) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
#ifdef FDPH_CHECK
    const size_t extra = kCanaryBytes;
#else
    const size_t extra = 0;
#endif
    cudaError_t e = cudaMalloc(&p, bytes + extra);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        return FDPH_E_OOM;
    }
    P->allocs.push_back(p);
#ifdef FDPH_CHECK
    P->canaries.push_back({(unsigned char*)p + bytes, extra});
    if (cudaMemsetAsync((unsigned char*)p + bytes, kCanary, extra, P->stream) != cudaSuccess) return FDPH_E_CUDA;
#endif
    *out = (T*)p;
    return FDPH_OK;
}

#ifdef FDPH_CHECK
// FDPH_CHECK builds: FDPH_E_CHECK if a write ran past the end of a device allocation
static int check_canaries(fdph_plan_t P) {
    std::vector<unsigned char> h;
    for (const auto& c : P->canaries) {
        h.assign(c.second, 0);
        FDPH_CUDA(cudaMemcpyAsync(h.data(), c.first, c.second, cudaMemcpyDeviceToHost, P->stream));
        FDPH_CUDA(cudaStreamSynchronize(P->stream));
        for (unsigned char b : h)
            if (b != kCanary) {
                set_error("a device write ran past the end of a plan allocation (canary overwritten)");
                return FDPH_E_CHECK;
            }
    }
    return FDPH_OK;
}
#endif

template <class T>
static int upload(fdph_plan_t P, T** out, const std::vector<T>& v) {
    int rc = dalloc(P, out, v.size());
    if (rc) return rc;
    // ordered on the plan's stream (a pageable source is staged before the call returns)
    if (!v.empty())
        FDPH_CUDA(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, P->stream));
    return FDPH_OK;
}

// TMA tensor map of the mirrored (hi, lo) ring Dring16 [2 WD][nrhs][NP] (4-byte elements): box =
// kTcBox sources x nrhs x one stage's kTcPer slots, no swizzle, zero fill outside; encoded
// through the driver entry point (no link against the driver library) and kept in device memory
static int make_row_tensor_map(fdph_plan_t P) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    FDPH_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess) {
        set_error("cuTensorMapEncodeTiled is not available");
        return FDPH_E_CUDA;
    }
    alignas(64) CUtensorMap map[2];
    const cuuint32_t chunk = (cuuint32_t)kTcPer;   // one stage's slots
    const cuuint64_t dims[3] = {(cuuint64_t)P->NP, (cuuint64_t)P->nrhs, (cuuint64_t)2 * P->WD};
    const cuuint64_t strides[2] = {(cuuint64_t)P->NP * 4, (cuuint64_t)P->nrhs * P->NP * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kTcBox, (cuuint32_t)P->nrhs, chunk};
    const cuuint32_t estr[3] = {1, 1, 1};
    auto encode = ((PFN_cuTensorMapEncodeTiled_v12000)fn);
    CUresult r = encode(&map[0], CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, (void*)P->Dring16, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    // the rows' scales: [2 WD][SR] floats, SR = max(nrhs, 4) (16-byte rows), box SR x chunk
    const cuuint64_t sr = (cuuint64_t)std::max(P->nrhs, 4);
    const cuuint64_t sdims[2] = {sr, (cuuint64_t)2 * P->WD};
    const cuuint64_t sstrides[1] = {sr * 4};
    const cuuint32_t sbox[2] = {(cuuint32_t)sr, chunk};
    if (r == CUDA_SUCCESS)
        r = encode(&map[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)P->Dscale, sdims, sstrides, sbox, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
        return FDPH_E_CUDA;
    }
    unsigned char* d = nullptr;
    int rc = dalloc(P, &d, sizeof(map));
    if (rc) return rc;
    FDPH_CUDA(cudaMemcpyAsync(d, map, sizeof(map), cudaMemcpyHostToDevice, P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    P->tmap16 = d;
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
    a.Dring32 = P->Dring32;
    a.Dring16 = P->Dring16;
    a.Dscale = P->Dscale;
    a.tmap16 = P->tmap16;
    a.NP = P->NP;
    a.tfar = P->tfar;
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
    a.sc_tasks = P->sc_tasks;
    a.n_sct = P->n_sct;
    a.ev_tasks = P->ev_tasks;
    a.n_evt = P->n_evt;
    a.e_pos = P->e_pos;
    a.fval = P->fval;
    a.fir_sb = P->fir_sb;
    a.fir_j = P->fir_j;
    a.n_fir = (int)P->hp.fir_sb.size();
    a.sfir_ptr = P->sfir ? P->sfir_ptr : nullptr;   // (null: the sub-block-major FIR)
    a.sfir_q = P->sfir_q;
    a.sfir_tmax = P->sfir_tmax;
    a.sfir_taps = P->hp.max_taps;
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
    a.tasks = P->tasks;
    a.cta_ptr = P->cta_ptr;
    a.n_cta = P->n_cta;
    a.n_items = (int)P->hp.items.size();
    a.tensor = P->tensor;
    a.kinv = (float)(1.0 / P->kscale);
    a.stat = P->stat;
    a.len_tensor = P->hp.near_tensor_len;
    a.len_aux = P->hp.near_aux_len;
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
    a.nrhs = P->nrhs;
    a.rs_D = (long long)P->WD * P->N;
    a.rs_C = (long long)P->WC * P->N;
    a.rs_ring = std::max<long long>(P->hp.ring_len, 1);
    a.rs_zring = std::max<long long>(P->hp.zring_len, 1);
    a.rs_dhat = std::max<long long>(P->hp.dhat_len, 1);
    a.rs_fval = std::max<long long>((long long)P->hp.e_pos.size(), 1);
    a.rs_ustate = std::max<long long>(P->hp.ustate_len, 1);
    a.rs_vstate = std::max<long long>(P->hp.vstate_len, 1);
    a.rs_partial = std::max<long long>((long long)P->partial_cap, 1);
    a.uhist = P->uhist;
    a.rs_uhist = std::max<long long>(P->uhist_len, 1);
    a.rec_tasks = P->rec_tasks;
    a.gat_tasks = P->gat_tasks;
    a.n_rec = P->n_rec;
    a.n_gat = P->n_gat;
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

// Launches of the far-field kernels: one grid row per right-hand side for one of them, one thread
// (or warp) for all of them otherwise, so that factors and indices are read once per step
#define FDPH_LAUNCH_NR(K, grid, threads, st, a)                                          \
    switch ((a).nrhs) {                                                                  \
        case 2: K<T, 2><<<(grid), (threads), 0, (st)>>>(a); break;                     \
        case 4: K<T, 4><<<(grid), (threads), 0, (st)>>>(a); break;                     \
        case 8: K<T, 8><<<(grid), (threads), 0, (st)>>>(a); break;                     \
        default: K<T, 1><<<dim3((grid), (a).nrhs), (threads), 0, (st)>>>(a); break;    \
    }

template <class T>
static void launch_fir(const StepArgs<T>& a, cudaStream_t s) {
    const size_t smem = (size_t)kSfirWarps * a.sfir_taps * a.nrhs * sizeof(T);
    if (a.sfir_ptr && a.sfir_taps > 0 && smem <= 48 * 1024) {   // source-major (no opt-in shared memory)
        const unsigned g = blocks(a.N, kSfirWarps);
        switch (a.nrhs) {
            case 2: sfir_kernel<T, 2><<<g, 32 * kSfirWarps, smem, s>>>(a); break;
            case 4: sfir_kernel<T, 4><<<g, 32 * kSfirWarps, smem, s>>>(a); break;
            case 8: sfir_kernel<T, 8><<<g, 32 * kSfirWarps, smem, s>>>(a); break;
            default: sfir_kernel<T, 1><<<g, 32 * kSfirWarps, smem, s>>>(a); break;
        }
        return;
    }
    FDPH_LAUNCH_NR(fir_kernel, blocks(a.n_fir, 128), 128, s, a)
}
template <class T>
static void launch_scatter(const StepArgs<T>& a, cudaStream_t s) {
    FDPH_LAUNCH_NR(scatter_kernel, blocks((long long)a.n_sct * 32, 128), 128, s, a)
}
template <class T>
static void launch_far_eval(const StepArgs<T>& a, cudaStream_t s) {
    FDPH_LAUNCH_NR(far_eval_kernel, blocks((long long)a.n_evt * 32, 128), 128, s, a)
}
template <class T>
static void launch_far_sum(const StepArgs<T>& a, cudaStream_t s) {
    FDPH_LAUNCH_NR(far_sum_kernel, blocks((long long)a.N * 32, 128), 128, s, a)
}

// Eq. 42 of a step: scatter into the delay rings, or (far_mode 1) record the source values and
// gather the completed slot from the histories
template <class T>
static void eq42(const StepArgs<T>& a, cudaStream_t s) {
    if (a.n_rec) {
        record_kernel<T><<<dim3(blocks(a.n_rec, 128), a.nrhs), 128, 0, s>>>(a);
        if (a.n_gat) hgather_kernel<T><<<dim3(blocks((long long)a.n_gat * 32, 128), a.nrhs), 128, 0, s>>>(a);
    } else if (a.n_sct) {
        launch_scatter<T>(a, s);
    }
}

template <class T, class H, int NR>
static void launch_near_nr(cudaLaunchConfig_t& cfg, const StepArgs<T>& a) {
    cfg.dynamicSmemBytes = NearCfg<H, NR>::smem;
    cudaLaunchKernelEx(&cfg, near_kernel<T, H, false, NR>, a, (const StepArgs<T>*)nullptr);
}

// the instantiation for the plan's right-hand sides (1, 2, 4 or 8)
template <class T, class H>
static void launch_near_h(cudaLaunchConfig_t& cfg, const StepArgs<T>& a, int nrhs) {
    switch (nrhs) {
        case 2: launch_near_nr<T, H, 2>(cfg, a); break;
        case 4: launch_near_nr<T, H, 4>(cfg, a); break;
        case 8: launch_near_nr<T, H, 8>(cfg, a); break;
        default: launch_near_nr<T, H, 1>(cfg, a);
    }
}

// The near-field kernel is persistent with a static schedule (one CTA pair per SM), so it is
// launched at the greatest stream priority: when it shares the GPU with the far-field branches of
// the same step its CTAs are placed first and none starts late.
template <class T>
static void launch_near(fdph_plan_t P, const StepArgs<T>& a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.n_cta);
    cfg.blockDim = dim3(kNearThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = P->near_priority;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (sizeof(T) == 4) {
        if (P->precision == FDPH_FP16) {
            launch_near_h<T, __half>(cfg, a, P->nrhs);
            return;
        }
    }
    launch_near_h<T, T>(cfg, a, P->nrhs);
}

template <class T>
static void enqueue_step(fdph_plan_t P, const StepArgs<T>& a, cudaStream_t s) {
    {
        ProfScope ps(P, 0);
        push_kernel<T><<<dim3(blocks(a.N, 256), a.nrhs), 256, 0, s>>>(a);
        if (a.Dring16) tc_rows_kernel<T><<<dim3(1, a.nrhs), kRowThreads, 0, s>>>(a, 0);
    }
    if (!P->prof && P->side[0]) {
        // Within a step, FIR + scatter (writes ring slots n + delay >= n + 1), the transient
        // convolution + Eq. 39 (read slots <= n - min dm, completed by earlier steps; causality
        // min(dm + delay) >= 1) and the near field touch disjoint data once push is done.
        cudaEventRecord(P->ev_fork, s);
        cudaStreamWaitEvent(P->side[0], P->ev_fork, 0);
        cudaStreamWaitEvent(P->side[1], P->ev_fork, 0);
        if (a.n_fir) launch_fir<T>(a, P->side[0]);
        eq42<T>(a, P->side[0]);
        if (a.n_tr) trconv_kernel<T><<<dim3(blocks((long long)a.n_tr * 32, 128), a.nrhs), 128, 0, P->side[1]>>>(a);
        if (a.n_evt) launch_far_eval<T>(a, P->side[1]);
        launch_far_sum<T>(a, P->side[1]);
        if (a.n_cta) launch_near<T>(P, a, s);
        cudaEventRecord(P->ev_join[0], P->side[0]);
        cudaEventRecord(P->ev_join[1], P->side[1]);
        cudaStreamWaitEvent(s, P->ev_join[0], 0);
        cudaStreamWaitEvent(s, P->ev_join[1], 0);
        gather_kernel<T><<<dim3(blocks(a.N, 128), a.nrhs), 128, 0, s>>>(a);
        return;
    }
    // serial order (per-kernel timing)
    if (a.n_fir) { ProfScope ps(P, 1); launch_fir<T>(a, s); }
    { ProfScope ps(P, 2); eq42<T>(a, s); }
    if (a.n_tr) { ProfScope ps(P, 3); trconv_kernel<T><<<dim3(blocks((long long)a.n_tr * 32, 128), a.nrhs), 128, 0, s>>>(a); }
    if (a.n_cta) {
        ProfScope ps(P, 4);
        launch_near<T>(P, a, s);
    }
    {
        ProfScope ps(P, 5);
        if (a.n_evt) launch_far_eval<T>(a, s);
        launch_far_sum<T>(a, s);
        gather_kernel<T><<<dim3(blocks(a.N, 128), a.nrhs), 128, 0, s>>>(a);
    }
}

template <class T>
static int launch_step(fdph_plan_t P, const double* D, double* Tout) {
    StepArgs<T> a = make_args<T>(P, D, Tout);
    enqueue_step<T>(P, a, P->stream);
    FDPH_CUDA(cudaGetLastError());
    return FDPH_OK;
}

// kinds of cached step graphs
enum { GRAPH_RUN = 0, GRAPH_RUN_HOST = 1, GRAPH_RUPTURE = 2 };

template <class T>
static void enqueue_rupture_step(fdph_plan_t P, StepArgs<T> a, double* D, cudaStream_t s);

// The cached graph of one step of `kind` on buffers (D, T) (rows modulo io_ring when > 0),
// captured on first use; the step index and the first row's step are set on the device before
// the replays.
template <class T>
static int step_graph(fdph_plan_t P, int kind, const double* D, double* Tout, int io_ring, cudaGraphExec_t* ex) {
    if (!P->n_dev) {
        int rc = dalloc(P, &P->n_dev, 2);
        if (rc) return rc;
    }
    cudaStream_t s = P->stream;
    set_step_kernel<<<1, 1, 0, s>>>(P->n_dev, P->n);
    for (const auto& ge : P->graphs)
        if (ge.kind == kind && ge.D == (const void*)D && ge.T == (const void*)Tout) {
            *ex = ge.ex;
            return FDPH_OK;
        }
    StepArgs<T> a = make_args<T>(P, kind == GRAPH_RUPTURE ? nullptr : D, Tout);
    a.n_dev = P->n_dev;
    a.io_stride = (long long)P->N * P->nrhs;
    a.io_ring = io_ring;
    cudaGraph_t g = nullptr;
    FDPH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    if (kind == GRAPH_RUPTURE) enqueue_rupture_step<T>(P, a, (double*)D, s);
    else enqueue_step<T>(P, a, s);
    advance_step_kernel<<<1, 1, 0, s>>>(P->n_dev);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
        set_error(std::string("graph capture: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    e = cudaGraphInstantiate(ex, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    if (P->graphs.size() >= 8) {   // bounded cache: drop the oldest graph
        cudaStreamSynchronize(s);
        cudaGraphExecDestroy(P->graphs.front().ex);
        P->graphs.erase(P->graphs.begin());
    }
    P->graphs.push_back({kind, (const void*)D, (const void*)Tout, *ex});
    return FDPH_OK;
}

// `steps` steps as replays of one captured step graph
template <class T>
static int run_graph(fdph_plan_t P, int steps, const double* D, double* Tout) {
    cudaGraphExec_t ex = nullptr;
    int rc = step_graph<T>(P, GRAPH_RUN, D, Tout, 0, &ex);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps; ++k) {
        e = cudaGraphLaunch(ex, P->stream);
        if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
        set_error(std::string("graph launch: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    P->n += steps;
    return FDPH_OK;
}

// Host-buffer steps: step k's D row goes host -> staging slot k % S on the h2d stream, the
// step graph runs on the plan stream once that copy is done, and its T row goes back on the
// d2h stream; slot k is reused by step k + S after T of step k has left it.
template <class T>
static int run_host(fdph_plan_t P, int steps, const double* D_host, double* T_host) {
    const int S = fdph_plan_s::kIoSlots;
    const size_t row = (size_t)P->N * P->nrhs;
    if (!P->io_D) {
        int rc;
        if ((rc = dalloc(P, &P->io_D, S * row)) || (rc = dalloc(P, &P->io_T, S * row))) return rc;
        FDPH_CUDA(cudaStreamCreateWithFlags(&P->h2d, cudaStreamNonBlocking));
        FDPH_CUDA(cudaStreamCreateWithFlags(&P->d2h, cudaStreamNonBlocking));
        for (int q = 0; q < S; ++q) {
            FDPH_CUDA(cudaEventCreateWithFlags(&P->ev_in[q], cudaEventDisableTiming));
            FDPH_CUDA(cudaEventCreateWithFlags(&P->ev_out[q], cudaEventDisableTiming));
            FDPH_CUDA(cudaEventCreateWithFlags(&P->ev_free[q], cudaEventDisableTiming));
        }
    }
    // the staging slots must not be reused before work still queued from an earlier call is done
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->d2h));
    cudaGraphExec_t ex = nullptr;
    int rc = step_graph<T>(P, GRAPH_RUN_HOST, P->io_D, P->io_T, S, &ex);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        const int q = k % S;
        if (k >= S) e = cudaStreamWaitEvent(P->h2d, P->ev_free[q], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(P->io_D + q * row, D_host + (size_t)k * row, row * sizeof(double),
                                cudaMemcpyHostToDevice, P->h2d);
        if (e == cudaSuccess) e = cudaEventRecord(P->ev_in[q], P->h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ev_in[q], 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(ex, P->stream);
        if (e == cudaSuccess) e = cudaEventRecord(P->ev_out[q], P->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->d2h, P->ev_out[q], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(T_host + (size_t)k * row, P->io_T + q * row, row * sizeof(double),
                                cudaMemcpyDeviceToHost, P->d2h);
        if (e == cudaSuccess) e = cudaEventRecord(P->ev_free[q], P->d2h);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->d2h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
        set_error(std::string("fdph_run_host: ") + cudaGetErrorString(e));
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
    FDPH_CUDA(cudaMemcpyAsync(&e, P->err, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    if (e) {
        cudaMemsetAsync(P->err, 0, sizeof(int), P->stream);
        if (e == kErrIndex) {
            set_error("a device index check failed (bounded-index debug build); results of the step are invalid");
            return FDPH_E_CHECK;
        }
        set_error("a bounded mbarrier wait in the near-field kernel gave up; results of the step are invalid");
        return FDPH_E_TIMEOUT;
    }
#ifdef FDPH_CHECK
    return check_canaries(P);
#else
    return FDPH_OK;
#endif
}

static int step_impl(fdph_plan_t P, const double* D, double* T_) {
    int rc = P->precision != FDPH_FP64 ? launch_step<float>(P, D, T_) : launch_step<double>(P, D, T_);
    if (rc == FDPH_OK) P->n += 1;
    return rc;
}

// Prediction of step n (Sec. 6.2): the traction with D_n = 0 (push of a zero row, transient,
// near field, Eq. 39, gather) into a.T_out.  Advances the transient and exponential-tail states,
// so it runs once per step, followed by enqueue_commit.
template <class T>
static void enqueue_predict(fdph_plan_t P, StepArgs<T> a, cudaStream_t s) {
    a.D_in = nullptr;
    { ProfScope ps(P, 0); push_kernel<T><<<dim3(blocks(a.N, 256), a.nrhs), 256, 0, s>>>(a); }          // D_n = 0
    if (!P->prof && P->side[1]) {
        // the transient convolution and Eq. 39 read ring slots completed by earlier steps and the
        // near field reads the slip-rate rows: the two branches run concurrently after push
        cudaEventRecord(P->ev_fork, s);
        cudaStreamWaitEvent(P->side[1], P->ev_fork, 0);
        if (a.n_tr) trconv_kernel<T><<<dim3(blocks((long long)a.n_tr * 32, 128), a.nrhs), 128, 0, P->side[1]>>>(a);
        if (a.n_evt) launch_far_eval<T>(a, P->side[1]);
        launch_far_sum<T>(a, P->side[1]);
        if (a.n_cta) launch_near<T>(P, a, s);
        cudaEventRecord(P->ev_join[1], P->side[1]);
        cudaStreamWaitEvent(s, P->ev_join[1], 0);
        gather_kernel<T><<<dim3(blocks(a.N, 128), a.nrhs), 128, 0, s>>>(a);
        return;
    }
    if (a.n_tr) { ProfScope ps(P, 3); trconv_kernel<T><<<dim3(blocks((long long)a.n_tr * 32, 128), a.nrhs), 128, 0, s>>>(a); }
    if (a.n_cta) {
        ProfScope ps(P, 4);
        launch_near<T>(P, a, s);
    }
    {
        ProfScope ps(P, 5);
        if (a.n_evt) launch_far_eval<T>(a, s);
        launch_far_sum<T>(a, s);
        gather_kernel<T><<<dim3(blocks(a.N, 128), a.nrhs), 128, 0, s>>>(a);
    }
}

// Commit of step n: push D_n into the history (overwriting the zero row of the prediction), FIR,
// scatter.
template <class T>
static void enqueue_commit(fdph_plan_t P, StepArgs<T> a, const double* D, cudaStream_t s) {
    a.D_in = D;
    { ProfScope ps(P, 0); push_kernel<T><<<dim3(blocks(a.N, 256), a.nrhs), 256, 0, s>>>(a); }
    if (a.n_fir) { ProfScope ps(P, 1); launch_fir<T>(a, s); }
    { ProfScope ps(P, 2); eq42<T>(a, s); }
}

// One rupture step (Sec. 6.2): predict, solve the friction law element by element, commit D_n.
// `a` carries the step-index source (direct: a.n; graph: n_dev).
template <class T>
static void enqueue_rupture_step(fdph_plan_t P, StepArgs<T> a, double* D, cudaStream_t s) {
    enqueue_predict<T>(P, a, s);
    friction_kernel<<<blocks(a.N, 256), 256, 0, s>>>(P->fr, a.N, D, a.T_out, a.n_dev);
    enqueue_commit<T>(P, a, D, s);
}

template <class T>
static int launch_predict(fdph_plan_t P, double* T_pred) {
    StepArgs<T> a = make_args<T>(P, nullptr, T_pred);
    enqueue_predict<T>(P, a, P->stream);
    FDPH_CUDA(cudaGetLastError());
    return FDPH_OK;
}

template <class T>
static int launch_commit(fdph_plan_t P, const double* D_n) {
    StepArgs<T> a = make_args<T>(P, D_n, nullptr);
    enqueue_commit<T>(P, a, D_n, P->stream);
    FDPH_CUDA(cudaGetLastError());
    return FDPH_OK;
}

template <class T>
static int launch_rupture_step(fdph_plan_t P, double* D, double* Tout) {
    StepArgs<T> a = make_args<T>(P, nullptr, Tout);
    enqueue_rupture_step<T>(P, a, D, P->stream);
    FDPH_CUDA(cudaGetLastError());
    return FDPH_OK;
}

// `steps` rupture steps as replays of one captured step graph (rows of D, T advance per step)
template <class T>
static int rupture_graph(fdph_plan_t P, int steps, double* D, double* Tout) {
    cudaGraphExec_t ex = nullptr;
    int rc = step_graph<T>(P, GRAPH_RUPTURE, D, Tout, 0, &ex);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(ex, P->stream);
    if (e != cudaSuccess) {
        set_error(std::string("rupture graph: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    P->n += steps;
    return FDPH_OK;
}

// The plan's near-field work items as the persistent kernel reads them, with their steady-state
// cost in bytes (+ a fixed per-item overhead).
template <class T, class H>
static void near_tasks(fdph_plan_t P, int scen, std::vector<NearTask>& tasks, std::vector<double>& cost) {
    using A = typename NearTypes<H>::Aux;
    const HostPlan& hp = P->hp;
    const int ni = (int)hp.items.size();
    for (int q = 0; q < ni; ++q) {
        const NearItem& it = hp.items[q];
        const NearLeaf& L = hp.near[it.leaf];
        NearTask t;
        memset(&t, 0, sizeof(t));
        t.off = it.kind ? (long long)L.stat + (long long)it.k0 * L.sla : (long long)L.tensor + (long long)it.k0 * L.sl;
        t.item = q;
        t.k0 = it.k0;
        t.k1 = it.k1;
        t.kind = it.kind;
        t.nr = L.nr;
        t.ns = L.ns;
        t.sl = it.kind ? L.sla : L.sl;
        t.s0 = L.s0;
        t.W = L.W;
        t.vstate = (int)L.vstate;
        t.scen = scen;
        tasks.push_back(t);
        cost.push_back((double)(it.k1 - it.k0) * t.sl * (double)(it.kind ? sizeof(A) : sizeof(H)) + 4096.0);
    }
}

// Work items dealt largest first to the least-loaded of ncta CTAs; per-CTA task lists in CTA
// order and their offsets.
static void deal_tasks(const std::vector<NearTask>& all, const std::vector<double>& cost, int ncta,
                       std::vector<NearTask>& tasks, std::vector<int>& cptr) {
    const int ni = (int)all.size();
    std::vector<int> order(ni);
    for (int q = 0; q < ni; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<std::vector<int>> own(ncta);
    std::vector<std::pair<double, int>> heap;
    for (int c = 0; c < ncta; ++c) heap.push_back({0.0, c});
    auto cmp = [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
        return x.first > y.first || (x.first == y.first && x.second > y.second);
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (int q : order) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        heap.back().first += cost[q];
        own[heap.back().second].push_back(q);
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    tasks.clear();
    cptr.assign(1, 0);
    for (int c = 0; c < ncta; ++c) {
        for (int q : own[c]) tasks.push_back(all[q]);
        cptr.push_back((int)tasks.size());
    }
}

// CTAs of the persistent near-field grid: SMs x resident CTAs per SM of the kernel
template <class T, class H, bool kBatch, int NR>
static int near_grid(int device, int* ncta_max) {
    FDPH_CUDA(cudaFuncSetAttribute(near_kernel<T, H, kBatch, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   NearCfg<H, NR>::smem));
    int sms = 0, per_sm = 0;
    FDPH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    FDPH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, near_kernel<T, H, kBatch, NR>, kNearThreads,
                                                            NearCfg<H, NR>::smem));
    *ncta_max = sms * std::max(per_sm, 1);
    return FDPH_OK;
}

// Persistent near-field grid of one plan: work items dealt over the CTAs (steady-state bytes);
// uploads the task lists and the receiver -> partial-slot map of the current items.
template <class T, class H>
static int build_schedule(fdph_plan_t P) {
    HostPlan& hp = P->hp;
    int rc, ncta_max = 1;
    rc = P->nrhs == 8   ? near_grid<T, H, false, 8>(P->device, &ncta_max)
         : P->nrhs == 4 ? near_grid<T, H, false, 4>(P->device, &ncta_max)
         : P->nrhs == 2 ? near_grid<T, H, false, 2>(P->device, &ncta_max)
                        : near_grid<T, H, false, 1>(P->device, &ncta_max);
    if (rc) return rc;
    std::vector<NearTask> all, tasks;
    std::vector<double> cost;
    std::vector<int> cptr;
    near_tasks<T, H>(P, 0, all, cost);
    const int ni = (int)all.size();
    const int ncta = std::max(1, std::min(ni, ncta_max));
    deal_tasks(all, cost, ncta, tasks, cptr);
    P->n_cta = ni ? ncta : 0;
    P->sched_version += 1;
    if ((rc = upload(P, &P->tasks, tasks)) || (rc = upload(P, &P->cta_ptr, cptr)) ||
        (rc = upload(P, &P->np_ptr, hp.np_ptr)) || (rc = upload(P, &P->np_idx, hp.np_idx)))
        return rc;
    return FDPH_OK;
}

// Near-field build in two phases around the host factorisation of the admissible blocks, which
// it does not need: build_near_begin (windows, exact tensors, tail projections launched on the
// device) and build_near_finish (tail fits on the host, upload, persistent schedule).
struct NearBuild {
    std::vector<NearDev> tl;        // leaves with an exponential tail
    std::vector<long long> tp0;     // their first pair
    double* d_g = nullptr;          // projections on the device
    long long ntp = 0;
    bool tails = false;
};

// T: far-field / step type; H: near-field window storage type (aux slices: NearTypes<H>::Aux)
template <class T, class H>
static int build_near_begin(fdph_plan_t P, const PlanInputs& in, NearBuild& nb) {
    using A = typename NearTypes<H>::Aux;
    HostPlan& hp = P->hp;
    const int nl = (int)hp.near_r0.size();
    const bool verbose = getenv("FDPH_VERBOSE") != nullptr;
    const auto t_start = std::chrono::steady_clock::now();
    auto stamp = [&](const char* what) {   // stage times of the near-field build
        if (!verbose) return;
        fprintf(stderr, "[fdph_plan]   %-26s %8.3f s\n", what,
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
    };
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
        ms.assign(npairs, 0);
        if (in.soe == 0) {   // the paper's cut: exact kernel up to each pair's m_S (App. H)
            const double thr = in.eps_st * in.mu / (2.0 * in.cs);
            near_ms_kernel<<<blocks(npairs, 128), 128, 0, P->stream>>>(g, d_r, d_nr, d_s, d_ns, d_p0, npairs, nl, in.M, in.dt,
                                                          in.mu, in.cs, thr, d_ms);
            FDPH_CUDA(cudaGetLastError());
            FDPH_CUDA(cudaMemcpyAsync(ms.data(), d_ms, npairs * sizeof(int), cudaMemcpyDeviceToHost, P->stream));
            FDPH_CUDA(cudaStreamSynchronize(P->stream));
            for (int l = 0; l < nl; ++l)
                for (long long q = pair0[l]; q < pair0[l + 1]; ++q) W[l] = std::max(W[l], ms[q]);
        }
        stamp("near: windows");
    }
    std::vector<char> has_tail(nl, 0);
    if (in.soe > 0) {
        // exponential tails: the window covers every pair's wave passage (both end-point fronts +
        // n_c steps), the exact kernel is kept for all pairs up to the leaf's window, and the
        // smooth remainder beyond it is fitted (no m_S cut is needed)
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
        FDPH_CUDA(cudaMemcpyAsync(d_ms, ms.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, P->stream));
    }
    // work-item length: the longest chunk (kChunk) that still yields about four waves of
    // resident CTAs (152 SMs x 3), so small problems (the plain N = 256 march) fill the device too
    long long slices = 0;
    for (int l = 0; l < nl; ++l) slices += std::max(W[l], 1);
    // (with nrhs right-hand sides an item's vectors, nrhs per slice, fill the same buffer)
    int chunk = near_max_chunk(P->nrhs, P->precision);
    while (chunk > std::max(1, 8 / P->nrhs) && slices / chunk < 4LL * 152 * 3) chunk /= 2;
    finish_near_layout(hp, W, has_tail, chunk, 16 / (int)sizeof(H), 16 / (int)sizeof(A),
                       near_aux_chunk(P->nrhs, P->precision));
    P->near_W = W;
    P->near_tail = has_tail;
    P->chunk = chunk;
    std::vector<NearDev> nd(nl);
    for (int l = 0; l < nl; ++l) {
        const NearLeaf& L = hp.near[l];
        nd[l] = {L.r0, L.nr, L.s0, L.ns, L.W, L.sl, L.sla, 0, (long long)L.tensor, (long long)L.stat, (long long)L.tail,
                 (long long)L.vstate};
    }
    if ((rc = upload(P, &P->near, nd))) return rc;
    // FP16 windows: coefficients are stored times 2^e, e = 13 - ceil(log2(mu / (2 cs))), so that
    // the radiation-damping self term mu / (2 cs), the largest coefficient, sits near 2^13: far
    // from the FP16 overflow (65504) whatever the units, and small coefficients keep the normal
    // FP16 range; the products are scaled back by 2^-e
    P->kscale = std::is_same<H, __half>::value ? std::ldexp(1.0, 13 - (int)std::ceil(std::log2(in.mu / (2.0 * in.cs))))
                                                : 1.0;
    H* tens = nullptr;
    A* aux = nullptr;
    if ((rc = dalloc(P, &tens, hp.near_tensor_len)) || (rc = dalloc(P, &aux, hp.near_aux_len))) return rc;
    P->tensor = tens;
    P->stat = aux;
    if (hp.near_tensor_len) FDPH_CUDA(cudaMemsetAsync(tens, 0, hp.near_tensor_len * sizeof(H), P->stream));  // padding
    if (hp.near_aux_len) FDPH_CUDA(cudaMemsetAsync(aux, 0, hp.near_aux_len * sizeof(A), P->stream));
    for (int l = 0; l < nl; ++l) {
        const long long tot = (long long)nd[l].W * nd[l].ns * nd[l].nr;
        if (tot == 0 && nd[l].ns * nd[l].nr == 0) continue;
        // static tile is written by k == 0 entries; a leaf with W == 0 still needs it
        NearDev L = nd[l];
        if (L.W == 0) {
            // temporarily fill one k-slice into a scratch to get the static tile
            H* tmp = nullptr;
            if ((rc = dalloc(P, &tmp, (size_t)L.sl))) return rc;
            NearDev L1 = L;
            L1.W = 1;
            L1.tensor = 0;
            near_fill_kernel<H, A><<<blocks((long long)L.ns * L.nr, 128), 128, 0, P->stream>>>(g, L1, d_ms + pair0[l], in.dt,
                                                                            in.mu, in.cs, P->kscale, tmp, aux);
        } else {
            near_fill_kernel<H, A><<<std::min<long long>(blocks(tot, 256), 4096), 256, 0, P->stream>>>(
                g, L, d_ms + pair0[l], in.dt, in.mu, in.cs, P->kscale, tens, aux);
        }
        FDPH_CUDA(cudaGetLastError());
    }
    stamp("near: exact windows filled");
    if (in.soe > 0 && hp.near_tail_len > 0) {
        // all tail leaves in one launch (here), then one Cholesky solve per leaf on the host (finish)
        std::vector<NearDev>& tl = nb.tl;
        std::vector<int> tl_id;
        std::vector<long long>& tp0 = nb.tp0;
        tp0.assign(1, 0);
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
        near_soe_proj_kernel<<<blocks(ntp, 128), 128, 0, P->stream>>>(g, d_tl, d_tp0, (int)tl.size(), ntp, in.M, in.dt, in.mu, in.cs,
                                                        in.soe, P->rho, d_g);
        FDPH_CUDA(cudaGetLastError());
        nb.d_g = d_g;
        nb.ntp = ntp;
        nb.tails = true;
    }
    stamp("near: tail projections launched");
    return FDPH_OK;
}

template <class T, class H>
static int build_near_finish(fdph_plan_t P, const PlanInputs& in, NearBuild& nb) {
    using A = typename NearTypes<H>::Aux;
    HostPlan& hp = P->hp;
    A* aux = (A*)P->stat;
    int rc;
    const bool verbose = getenv("FDPH_VERBOSE") != nullptr;
    const auto t_start = std::chrono::steady_clock::now();
    auto stamp = [&](const char* what) {
        if (!verbose) return;
        fprintf(stderr, "[fdph_plan]   %-26s %8.3f s\n", what,
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
    };
    if (nb.tails) {
        const std::vector<NearDev>& tl = nb.tl;
        const std::vector<long long>& tp0 = nb.tp0;
        const long long ntp = nb.ntp;
        double* d_g = nb.d_g;
        std::vector<double> gh((size_t)ntp * in.soe), ch((size_t)ntp * in.soe);
        FDPH_CUDA(cudaMemcpyAsync(gh.data(), d_g, gh.size() * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
        FDPH_CUDA(cudaStreamSynchronize(P->stream));
        stamp("near: tail projections done");
        // tail slices q = 1..Q of each leaf's aux block, [q][ns][nr] with slice stride sl
        std::vector<size_t> toff(tl.size() + 1, 0);
        for (size_t t = 0; t < tl.size(); ++t) toff[t + 1] = toff[t] + (size_t)in.soe * tl[t].sla;
        std::vector<A> tail_h(toff.back(), (A)0);
        constexpr int v4 = 16 / (int)sizeof(A);
#pragma omp parallel for schedule(dynamic, 8) num_threads(in.threads)
        for (long t = 0; t < (long)tl.size(); ++t) {
            const NearDev& L = tl[t];
            const size_t b = (size_t)tp0[t] * in.soe;
            soe_solve(hp.rho, in.M - L.W, gh.data() + b, ch.data() + b, L.nr * L.ns);
            for (int il = 0; il < L.nr; ++il)
                for (int jl = 0; jl < L.ns; ++jl)
                    for (int q = 0; q < in.soe; ++q)
                        tail_h[toff[t] + (size_t)q * L.sla + ((size_t)(jl / v4) * L.nr + il) * v4 + jl % v4] =
                            (A)ch[b + ((size_t)il * L.ns + jl) * in.soe + q];
        }
        for (size_t t = 0; t < tl.size(); ++t)
            FDPH_CUDA(cudaMemcpyAsync(aux + tl[t].tail, tail_h.data() + toff[t], (toff[t + 1] - toff[t]) * sizeof(A),
                                      cudaMemcpyHostToDevice, P->stream));
    }
    stamp("near: tail fits");
    if ((rc = build_schedule<T, H>(P))) return rc;
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    return FDPH_OK;
}

static void fill_stats(fdph_plan_t P) {
    HostPlan& hp = P->hp;
    fdph_stats& s = P->st;
    const double ps = P->precision != FDPH_FP64 ? 4.0 : 8.0;   // far factors and near aux slices
    const double pw = P->precision == FDPH_FP16 ? 2.0 : ps;    // near window coefficients
    s.n = hp.n;
    s.M = hp.M;
    s.n_admissible = hp.n_adm;
    s.n_near = hp.n_near;
    s.n_subblocks = (int)hp.sbs.size();
    s.max_rank = hp.max_rank;
    s.mean_rank = hp.mean_rank;
    s.n_exact = hp.n_exact[0] + hp.n_exact[1] + hp.n_exact[2];
    s.n_aca = hp.n_aca;
    s.mean_rank_f = hp.ent_w[SB_F] > 0 ? hp.rank_w[SB_F] / hp.ent_w[SB_F] : 0.0;
    s.mean_rank_s = hp.ent_w[SB_S] > 0 ? hp.rank_w[SB_S] / hp.ent_w[SB_S] : 0.0;
    s.mean_rank_tr = hp.ent_w[SB_TR] > 0 ? hp.rank_w[SB_TR] / hp.ent_w[SB_TR] : 0.0;
    s.extra_steps = hp.tree.nc;
    s.max_window = hp.max_W;
    s.near_entries = hp.near_tensor_len;
    s.far_entries = hp.far_entries;
    // algorithmic bytes of one steady-state step
    double near_b = 0, far_b = 0, flops = 0;
    // slip-rate window rows are read from the FP32 copy of the ring unless the plan is FP64;
    // every right-hand side reads its own rows and keeps its own tail states
    const double prow = P->precision != FDPH_FP64 ? 4.0 : 8.0;
    const double R = P->nrhs;
    for (const NearLeaf& L : hp.near) {
        near_b += (double)L.W * L.ns * L.nr * pw + (double)L.ns * L.nr * ps;   // tensor + static tile
        near_b += R * ((double)L.W * L.ns * prow + L.ns * 8.0);                // window rows + C row
        flops += 2.0 * R * ((double)L.W + 1) * L.ns * L.nr;
        if (L.tail >= 0) {                                                     // tail coefficients + states
            near_b += (double)hp.soe * L.ns * L.nr * ps + R * hp.soe * L.ns * 16.0;
            flops += 2.0 * R * hp.soe * L.ns * (L.nr + 1.0);
        }
    }
    for (const SubBlock& sb : hp.sbs) {
        const double r = sb.rank;
        far_b += (sb.nr + sb.ns) * 4.0;                                        // delays
        if (sb.ident == 1) {          // F = I: one ring read per receiver
            far_b += sb.nr * 8.0 + sb.ns * r * ps + sb.nruns * r * 16.0;
            flops += 2.0 * sb.ns * r;
        } else if (sb.ident == 2) {   // G = I: one ring store per source
            far_b += sb.nr * r * (ps + 8.0) + sb.ns * 8.0;
            flops += 2.0 * sb.nr * r;
        } else {
            far_b += (sb.nr + sb.ns) * r * ps;                                 // f, g
            far_b += sb.nr * r * 8.0 + sb.nruns * r * 16.0;                    // ring reads / RMW
            flops += 2.0 * (sb.nr + sb.ns) * r;
        }
        if (sb.kind == SB_F) {
            far_b += (double)sb.taps * sb.ns * ps + sb.ns * 8.0;   // h, Dhat (the D history below)
            flops += 2.0 * sb.taps * sb.ns;
        }
        if (sb.kind == SB_TR) {
            if (sb.qn)   // two ring reads, a running-sum update and a value per quantized range
                far_b += r * (sb.qn * (16.0 + 16.0 + ps) + 8.0) + r * sb.soe * 24.0;
            else
                far_b += r * (sb.taps * 8.0 + sb.taps * ps + 8.0) + r * sb.soe * 24.0;
            flops += 2.0 * r * ((sb.qn ? 2.0 * sb.qn : sb.taps) + 2.0 * sb.soe);
        }
    }
    for (int32_t t : hp.sfir_tmax) far_b += t * 8.0;                          // each source's D history, once
    const double push_b = hp.n * (8.0 + 8.0 + 32.0 + 8.0 + 4.0);           // D in, ring, C/comp, Cring, perm
    const double out_b = hp.n * (8.0 + 4.0) + (double)hp.np_idx.size() * 12.0;
    s.bytes_per_step = near_b + far_b + push_b + out_b;
    s.near_bytes_per_step = near_b;
    s.flops_per_step = flops;
    s.state_bytes = (long long)P->state_bytes;
    long long arena = 0;
    arena += (long long)(hp.fac.size() * ps) + hp.ints.size() * 4 + hp.sbs.size() * sizeof(SbDev);
    arena += (long long)(hp.near_tensor_len * pw + hp.near_aux_len * ps);
    s.arena_bytes = arena;
}

// Near-field work items of `chunk` kernel steps (1..kChunk): new items, partial slots and
// persistent schedule; the stored coefficients do not move.  Cached step graphs refer to the old
// schedule and are dropped.
template <class T, class H>
static int set_chunk(fdph_plan_t P, int chunk) {
    using A = typename NearTypes<H>::Aux;
    HostPlan& hp = P->hp;
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    for (auto& ge : P->graphs) cudaGraphExecDestroy(ge.ex);
    P->graphs.clear();
    const int64_t tens0 = hp.near_tensor_len, aux0 = hp.near_aux_len, vst0 = hp.vstate_len;
    finish_near_layout(hp, P->near_W, P->near_tail, chunk, 16 / (int)sizeof(H), 16 / (int)sizeof(A),
                       near_aux_chunk(P->nrhs, P->precision));
    if (hp.near_tensor_len != tens0 || hp.near_aux_len != aux0 || hp.vstate_len != vst0) {
        // the stored coefficients and states must keep their places (only the items change)
        set_error("set_chunk: near-field layout changed; the plan is unusable");
        return FDPH_E_STATE;
    }
    const size_t need = hp.items.size() * 32;
    if (need > P->partial_cap) {
        int rc = dalloc(P, &P->partial, need * P->nrhs);
        if (rc) return rc;
        FDPH_CUDA(cudaMemsetAsync(P->partial, 0, need * P->nrhs * sizeof(double), P->stream));
        P->partial_cap = need;
    }
    int rc = build_schedule<T, H>(P);
    if (rc) return rc;
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    P->chunk = chunk;
    return FDPH_OK;
}

static int set_chunk_any(fdph_plan_t P, int chunk) {
    return P->precision == FDPH_FP16   ? set_chunk<float, __half>(P, chunk)
           : P->precision == FDPH_FP32 ? set_chunk<float, float>(P, chunk)
                                       : set_chunk<double, double>(P, chunk);
}

// a step split by fdph_predict must be completed by fdph_commit before anything else steps or
// copies the state
static int pending_commit(fdph_plan_t P) {
    if (!P->predicted) return FDPH_OK;
    set_error("step predicted by fdph_predict awaits fdph_commit");
    return FDPH_E_STATE;
}

// ------------------------------------------------------------------------------------------
// Batches of plans: one near-field launch per step for all of them

// work kinds of a batch's prefix sums
enum { BW_ELEM = 0, BW_FIR = 1, BW_SCT = 2, BW_TR = 3, BW_EVT = 4, BW_KINDS = 5 };

// A set of plans (same device, same precision) stepped together: each kernel of a step is ONE
// launch over the work of all plans (the persistent near-field kernel over the work items of
// all plans, dealt together over the CTAs; the others over the concatenated elements and warp
// tasks).  Graphs of one batch step are captured per (kind, buffers) and replayed.
struct fdph_batch_s {
    int device = 0, precision = 0;
    std::vector<fdph_plan_t> plans;
    std::vector<int> version;            // each plan's near-field schedule at creation
    cudaStream_t stream = nullptr;
    cudaStream_t side[2] = {nullptr, nullptr};   // FIR + scatter | transient + Eq. 39
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr}, ev_end = nullptr;
    std::vector<cudaEvent_t> ev_ready;           // per plan: its queued work before a batch call
    NearTask* tasks = nullptr;
    int* cta_ptr = nullptr;
    int n_cta = 0;
    int near_priority = 0;
    int* pre = nullptr;                          // device prefix sums [BW_KINDS][np + 1]
    int tot[5] = {0, 0, 0, 0, 0};                // their totals
    FrictionDev* fr_dev = nullptr;               // friction of every plan (rupture batches)
    std::vector<FrictionDev> fr_host;
    struct Entry {
        int kind;
        std::vector<const void*> D, T;
        void* scen;                      // device StepArgs of every plan for this entry
        cudaGraphExec_t ex;
    };
    std::vector<Entry> graphs;
};

template <class T>
static void launch_near_batch(fdph_batch_t B, const StepArgs<T>* scen, cudaStream_t s) {
    StepArgs<T> ab;
    memset(&ab, 0, sizeof(ab));
    ab.tasks = B->tasks;
    ab.cta_ptr = B->cta_ptr;
    ab.n_cta = B->n_cta;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(B->n_cta);
    cfg.blockDim = dim3(kNearThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = B->near_priority;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (sizeof(T) == 4) {
        if (B->precision == FDPH_FP16) {
            cfg.dynamicSmemBytes = NearCfg<__half>::smem;
            cudaLaunchKernelEx(&cfg, near_kernel<T, __half, true, 1>, ab, scen);
            return;
        }
    }
    cfg.dynamicSmemBytes = NearCfg<T>::smem;
    cudaLaunchKernelEx(&cfg, near_kernel<T, T, true, 1>, ab, scen);
}

// One step of every plan of the batch (kind GRAPH_RUN or GRAPH_RUPTURE), for capture on the
// batch stream; scen: every plan's arguments on the device (step index from its n_dev; D_in the
// plan's D rows, the rupture outputs for GRAPH_RUPTURE).
template <class T>
static void enqueue_batch_step(fdph_batch_t B, int kind, const StepArgs<T>* scen) {
    cudaStream_t bs = B->stream;
    const int np = (int)B->plans.size();
    auto pre = [&](int k) { return (const int*)B->pre + k * (np + 1); };
    const int* tot = B->tot;
    auto fir = [&](cudaStream_t s) {
        if (tot[BW_FIR]) fir_batch<T><<<blocks(tot[BW_FIR], 128), 128, 0, s>>>(scen, pre(BW_FIR), np);
        if (tot[BW_SCT])
            scatter_batch<T><<<blocks((long long)tot[BW_SCT] * 32, 128), 128, 0, s>>>(scen, pre(BW_SCT), np);
    };
    auto far = [&](cudaStream_t s) {
        if (tot[BW_TR]) trconv_batch<T><<<blocks((long long)tot[BW_TR] * 32, 128), 128, 0, s>>>(scen, pre(BW_TR), np);
        if (tot[BW_EVT])
            far_eval_batch<T><<<blocks((long long)tot[BW_EVT] * 32, 128), 128, 0, s>>>(scen, pre(BW_EVT), np);
        far_sum_batch<T><<<blocks((long long)tot[BW_ELEM] * 32, 128), 128, 0, s>>>(scen, pre(BW_ELEM), np);
    };
    auto gather = [&]() {
        gather_batch<T><<<blocks(tot[BW_ELEM], 128), 128, 0, bs>>>(scen, pre(BW_ELEM), np);
    };
    if (kind == GRAPH_RUN) {
        push_batch<T><<<blocks(tot[BW_ELEM], 256), 256, 0, bs>>>(scen, pre(BW_ELEM), np, 0);
        cudaEventRecord(B->ev_fork, bs);
        cudaStreamWaitEvent(B->side[0], B->ev_fork, 0);
        cudaStreamWaitEvent(B->side[1], B->ev_fork, 0);
        fir(B->side[0]);
        far(B->side[1]);
        if (B->n_cta) launch_near_batch<T>(B, scen, bs);
        cudaEventRecord(B->ev_join[0], B->side[0]);
        cudaEventRecord(B->ev_join[1], B->side[1]);
        cudaStreamWaitEvent(bs, B->ev_join[0], 0);
        cudaStreamWaitEvent(bs, B->ev_join[1], 0);
        gather();
    } else {   // rupture: predict with D_n = 0 (far field beside the near field), friction, commit D_n
        push_batch<T><<<blocks(tot[BW_ELEM], 256), 256, 0, bs>>>(scen, pre(BW_ELEM), np, 1);
        cudaEventRecord(B->ev_fork, bs);
        cudaStreamWaitEvent(B->side[1], B->ev_fork, 0);
        far(B->side[1]);
        if (B->n_cta) launch_near_batch<T>(B, scen, bs);
        cudaEventRecord(B->ev_join[1], B->side[1]);
        cudaStreamWaitEvent(bs, B->ev_join[1], 0);
        gather();
        friction_batch<T><<<blocks(tot[BW_ELEM], 256), 256, 0, bs>>>(B->fr_dev, scen, pre(BW_ELEM), np);
        push_batch<T><<<blocks(tot[BW_ELEM], 256), 256, 0, bs>>>(scen, pre(BW_ELEM), np, 0);
        fir(bs);
    }
    advance_batch<T><<<blocks(np, 128), 128, 0, bs>>>(scen, np);
}

// `steps` steps of every plan of the batch as replays of one captured batch-step graph
template <class T>
static int batch_run(fdph_batch_t B, int kind, int steps, const double* const* D, double* const* Tt) {
    const size_t np = B->plans.size();
    cudaStream_t bs = B->stream;
    // ordered after the work already queued on every plan's stream; step indices on the device
    for (size_t p = 0; p < np; ++p) {
        fdph_plan_t P = B->plans[p];
        if (!P->n_dev) {
            int rc = dalloc(P, &P->n_dev, 2);
            if (rc) return rc;
        }
        FDPH_CUDA(cudaEventRecord(B->ev_ready[p], P->stream));
        FDPH_CUDA(cudaStreamWaitEvent(bs, B->ev_ready[p], 0));
    }
    for (size_t p = 0; p < np; ++p) set_step_kernel<<<1, 1, 0, bs>>>(B->plans[p]->n_dev, B->plans[p]->n);
    if (kind == GRAPH_RUPTURE) {   // the friction of every plan as it is now (pageable copy: staged at once)
        for (size_t p = 0; p < np; ++p) B->fr_host[p] = B->plans[p]->fr;
        FDPH_CUDA(cudaMemcpyAsync(B->fr_dev, B->fr_host.data(), np * sizeof(FrictionDev), cudaMemcpyHostToDevice, bs));
    }
    cudaGraphExec_t ex = nullptr;
    for (const auto& ge : B->graphs) {
        if (ge.kind != kind) continue;
        bool same = true;
        for (size_t p = 0; p < np && same; ++p) same = ge.D[p] == (const void*)D[p] && ge.T[p] == (const void*)Tt[p];
        if (same) {
            ex = ge.ex;
            break;
        }
    }
    if (!ex) {
        std::vector<StepArgs<T>> av(np);
        for (size_t p = 0; p < np; ++p) {
            fdph_plan_t P = B->plans[p];
            av[p] = make_args<T>(P, D[p], Tt[p]);
            av[p].n_dev = P->n_dev;
            av[p].io_stride = P->N;
            av[p].io_ring = 0;
        }
        void* scen = nullptr;
        FDPH_CUDA(cudaMalloc(&scen, np * sizeof(StepArgs<T>)));
        cudaError_t e = cudaMemcpy(scen, av.data(), np * sizeof(StepArgs<T>), cudaMemcpyHostToDevice);
        cudaGraph_t g = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_batch_step<T>(B, kind, (const StepArgs<T>*)scen);
            e = cudaStreamEndCapture(bs, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaFree(scen);
            set_error(std::string("batch graph: ") + cudaGetErrorString(e));
            return FDPH_E_CUDA;
        }
        if (B->graphs.size() >= 4) {   // bounded cache: drop the oldest graph
            cudaStreamSynchronize(bs);
            cudaGraphExecDestroy(B->graphs.front().ex);
            cudaFree(B->graphs.front().scen);
            B->graphs.erase(B->graphs.begin());
        }
        fdph_batch_s::Entry en;
        en.kind = kind;
        en.D.assign(D, D + np);
        en.T.assign(Tt, Tt + np);
        en.scen = scen;
        en.ex = ex;
        B->graphs.push_back(en);
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(ex, bs);
    if (e == cudaSuccess) e = cudaEventRecord(B->ev_end, bs);
    for (size_t p = 0; p < np && e == cudaSuccess; ++p) e = cudaStreamWaitEvent(B->plans[p]->stream, B->ev_end, 0);
    if (e != cudaSuccess) {
        set_error(std::string("batch run: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    for (size_t p = 0; p < np; ++p) B->plans[p]->n += steps;
    return FDPH_OK;
}

template <class T, class H>
static int batch_schedule(fdph_batch_t B) {
    int ncta_max = 1, rc;
    if ((rc = near_grid<T, H, true, 1>(B->device, &ncta_max))) return rc;
    std::vector<NearTask> all, tasks;
    std::vector<double> cost;
    std::vector<int> cptr;
    for (size_t p = 0; p < B->plans.size(); ++p) near_tasks<T, H>(B->plans[p], (int)p, all, cost);
    const int ni = (int)all.size();
    const int ncta = std::max(1, std::min(ni, ncta_max));
    deal_tasks(all, cost, ncta, tasks, cptr);
    B->n_cta = ni ? ncta : 0;
    FDPH_CUDA(cudaMalloc(&B->tasks, std::max<size_t>(1, tasks.size()) * sizeof(NearTask)));
    FDPH_CUDA(cudaMalloc(&B->cta_ptr, cptr.size() * sizeof(int)));
    if (!tasks.empty())
        FDPH_CUDA(cudaMemcpy(B->tasks, tasks.data(), tasks.size() * sizeof(NearTask), cudaMemcpyHostToDevice));
    FDPH_CUDA(cudaMemcpy(B->cta_ptr, cptr.data(), cptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    // prefix sums of the plans' work counts, per kind
    const int np = (int)B->plans.size();
    std::vector<int> pre((size_t)BW_KINDS * (np + 1), 0);
    for (int k = 0; k < BW_KINDS; ++k) {
        long long acc = 0;
        for (int p = 0; p < np; ++p) {
            const fdph_plan_t P = B->plans[p];
            const long long c = k == BW_ELEM ? P->N
                                : k == BW_FIR ? (long long)P->hp.fir_sb.size()
                                : k == BW_SCT ? P->n_sct
                                : k == BW_TR ? (long long)P->hp.tr_sb.size()
                                             : P->n_evt;
            pre[(size_t)k * (np + 1) + p] = (int)acc;
            acc += c;
        }
        if (acc > INT32_MAX / 32) {
            set_error("fdph_batch_create: the plans' work exceeds the batch index range");
            return FDPH_E_ARG;
        }
        pre[(size_t)k * (np + 1) + np] = (int)acc;
        B->tot[k] = (int)acc;
    }
    FDPH_CUDA(cudaMalloc(&B->pre, pre.size() * sizeof(int)));
    FDPH_CUDA(cudaMemcpy(B->pre, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice));
    FDPH_CUDA(cudaMalloc(&B->fr_dev, np * sizeof(FrictionDev)));
    B->fr_host.assign(np, FrictionDev{});
    return FDPH_OK;
}

static void batch_free(fdph_batch_t B) {
    if (!B) return;
    cudaSetDevice(B->device);
    if (B->stream) cudaStreamSynchronize(B->stream);
    for (auto& ge : B->graphs) {
        cudaGraphExecDestroy(ge.ex);
        cudaFree(ge.scen);
    }
    if (B->tasks) cudaFree(B->tasks);
    if (B->cta_ptr) cudaFree(B->cta_ptr);
    if (B->pre) cudaFree(B->pre);
    if (B->fr_dev) cudaFree(B->fr_dev);
    for (cudaEvent_t e : B->ev_ready) if (e) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (B->ev_join[k]) cudaEventDestroy(B->ev_join[k]);
        if (B->side[k]) cudaStreamDestroy(B->side[k]);
    }
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->ev_end) cudaEventDestroy(B->ev_end);
    if (B->stream) cudaStreamDestroy(B->stream);
    delete B;
}

// batch calls: every plan still has the schedule the batch was built on and no pending predict
static int batch_check(fdph_batch_t B, int steps) {
    for (size_t p = 0; p < B->plans.size(); ++p) {
        fdph_plan_t P = B->plans[p];
        if (P->predicted) return pending_commit(P);
        if (P->sched_version != B->version[p]) {
            set_error("a plan of the batch has rebuilt its near-field items (fdph_autotune): create the batch again");
            return FDPH_E_STATE;
        }
        if (P->prof) {
            set_error("batch run: profiling is on for a plan of the batch");
            return FDPH_E_STATE;
        }
        if (P->n + steps > P->M) {
            set_error("batch run would pass step M of a plan");
            return FDPH_E_STATE;
        }
    }
    return FDPH_OK;
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
    p->nrhs = 1;
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
        case FDPH_E_CHECK: return "device index check failed (bounded-index debug build)";
        default: return "unknown status";
    }
}

const char* fdph_last_error(void) { return g_last_error.c_str(); }

static int check_inputs(const fdph_geometry* g, const fdph_material* m, double dt, const fdph_params* p) {
    if (!g || !m || !g->xy || g->n <= 0 || !(dt > 0.0) || !(m->mu > 0.0) || !(m->cs > 0.0)) {
        set_error("geometry, material and dt must be given, n > 0, dt, mu, cs > 0");
        return FDPH_E_ARG;
    }
    if (p && (p->leaf_size < 1 || p->leaf_size > 32 || p->eta < 0.0 || p->eps_st < 0.0 || p->host_threads < 0 ||
              (p->eta_scheme != 0 && p->eta_scheme != 1) || (p->eta_scheme == 1 && !(p->lmin > 0.0)) ||
              (p->nrhs != 0 && p->nrhs != 1 && p->nrhs != 2 && p->nrhs != 4 && p->nrhs != kMaxRhs) ||
              (p->far_mode != 0 && p->far_mode != 1) || (p->amp_window != 0 && p->amp_window != 1) ||
              !(p->eps_q >= 0.0 && p->eps_q < 1.0) ||
              (p->precision != FDPH_FP64 && p->precision != FDPH_FP32 && p->precision != FDPH_FP16) ||
              (p->soe_terms != 0 && (p->soe_terms < 4 || p->soe_terms > kMaxSoe)))) {
        set_error("params: leaf_size in [1, 32], eta >= 0, eps_st >= 0, host_threads >= 0, eta_scheme 0 or 1 (1 needs "
                  "lmin > 0), nrhs 1, 2, 4 or 8 (0: 1), far_mode 0 or 1, amp_window 0 or 1, eps_q in [0, 1), precision "
                  "FP64, FP32 or "
                  "FP16, "
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
    in.threads = p.host_threads > 0 ? p.host_threads : omp_get_max_threads();
    in.eta_scheme = p.eta_scheme;
    in.amp_window = p.amp_window;
    in.eps_q = p.eps_q;
    in.aca_min = p.aca_min > 0 ? (long long)p.aca_min : LLONG_MAX;
    return in;
}

int fdph_low_rank(const double* A, int32_t m, int32_t n, double eps, double* F, double* G, int32_t* rank,
                  int32_t* exact) {
    if (!A || !F || !G || !rank || !exact || m < 1 || n < 1) return FDPH_E_ARG;
    for (long long q = 0; q < (long long)m * n; ++q)
        if (!std::isfinite(A[q])) {
            set_error("fdph_low_rank: non-finite entry");
            return FDPH_E_NAN;
        }
    LowRank lr;
    low_rank(A, m, n, eps, lr);
    *rank = lr.rank;
    *exact = lr.exact ? 1 : 0;
    std::copy(lr.F.begin(), lr.F.end(), F);
    std::copy(lr.G.begin(), lr.G.end(), G);
    return FDPH_OK;
}

int fdph_low_rank_aca(const double* A, int32_t m, int32_t n, double eps, double* F, double* G, int32_t* rank,
                      int32_t* converged, int64_t* evaluated) {
    if (!A || !F || !G || !rank || !converged || !evaluated || m < 1 || n < 1 || !(eps > 0.0)) {
        set_error("fdph_low_rank_aca: null pointer, m or n < 1 or eps <= 0");
        return FDPH_E_ARG;
    }
    for (long long q = 0; q < (long long)m * n; ++q)
        if (!std::isfinite(A[q])) {
            set_error("fdph_low_rank_aca: non-finite entry");
            return FDPH_E_NAN;
        }
    long long count = 0;
    auto row = [&](int i, double* out) {
        std::copy(A + (size_t)i * n, A + (size_t)(i + 1) * n, out);
        count += n;
    };
    auto col = [&](int j, double* out) {
        for (int i = 0; i < m; ++i) out[i] = A[(size_t)i * n + j];
        count += m;
    };
    LowRank lr;
    const bool ok = low_rank_aca(row, col, m, n, eps, lr);
    *converged = ok ? 1 : 0;
    *rank = ok ? lr.rank : 0;
    *evaluated = count;
    if (ok) {
        std::copy(lr.F.begin(), lr.F.end(), F);
        std::copy(lr.G.begin(), lr.G.end(), G);
    }
    return FDPH_OK;
}

int fdph_kernel_tail(const double* p, const double* seg, double t1, double dt, double mu, double cs, double* out) {
    if (!p || !seg || !out || !(dt > 0.0) || !(t1 >= 0.0) || !(mu > 0.0) || !(cs > 0.0) || !(seg[4] > 0.0)) {
        set_error("fdph_kernel_tail: null pointer, dt, mu, cs or the length <= 0, or t1 < 0");
        return FDPH_E_ARG;
    }
    const Seg s{seg[0], seg[1], seg[2], seg[3], seg[4]};
    const Stress2 v = stress_tail(p[0], p[1], s, t1, t1 + dt, mu, cs);
    out[0] = v.x;
    out[1] = v.y;
    out[2] = stress_tail_bound(p[0], p[1], s, t1, dt, mu, cs);
    return FDPH_OK;
}

int fdph_quantize(const double* K, int32_t n, double eps_q, int32_t* b, double* khat, int32_t* q) {
    if (!K || !b || !khat || !q || n < 1 || !(eps_q > 0.0)) {
        set_error("fdph_quantize: null pointer, n < 1 or eps_q <= 0");
        return FDPH_E_ARG;
    }
    for (int m = 0; m < n; ++m)
        if (!std::isfinite(K[m])) {
            set_error("fdph_quantize: non-finite value");
            return FDPH_E_NAN;
        }
    std::vector<int32_t> bb;
    std::vector<double> kh;
    quantize_partitions(K, n, eps_q, bb, kh);
    std::copy(bb.begin(), bb.end(), b);
    std::copy(kh.begin(), kh.end(), khat);
    *q = (int32_t)kh.size();
    return FDPH_OK;
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
    P->nrhs = std::max(p.nrhs, 1);
    P->far_mode = p.far_mode;
    P->N = geometry->n;
    P->M = M;
    P->dt = dt;
    auto fail = [&](int code) {
        fdph_destroy(P);
        return code;
    };
    // host trees and the discretised causality of every admissible leaf first: a plan that
    // violates it is refused before any device resource is taken
    PlanInputs in = make_inputs(material, dt, M, eps, p);
    Elements el = make_elements(geometry->n, geometry->xy);
    HostPlan& hp = P->hp;
    build_host_tree(el, in, hp);
    if (check_causality(el, in, hp.tree)) return fail(FDPH_E_CAUSALITY);
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
    for (int k = 0; k < 2; ++k)
        if (cudaStreamCreateWithFlags(&P->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->ev_join[k], cudaEventDisableTiming) != cudaSuccess) {
            set_error("cudaStreamCreate / cudaEventCreate failed");
            return fail(FDPH_E_CUDA);
        }
    if (cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
        set_error("cudaEventCreate failed");
        return fail(FDPH_E_CUDA);
    }
    {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess) P->near_priority = greatest;
    }
    const bool verbose = getenv("FDPH_VERBOSE") != nullptr;
    auto stamp = [&](const char* what) {
        if (verbose)
            fprintf(stderr, "[fdph_plan] %-28s %8.3f s\n", what,
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    };
    stamp("cluster and block trees");
    // near field on the device (exact windows, tail projections) while the host factorises the
    // admissible blocks
    NearBuild nb;
    if (hp.soe > 0 && (rc = upload(P, &P->rho, hp.rho))) return fail(rc);
    rc = P->precision == FDPH_FP16   ? build_near_begin<float, __half>(P, in, nb)
         : P->precision == FDPH_FP32 ? build_near_begin<float, float>(P, in, nb)
                                     : build_near_begin<double, double>(P, in, nb);
    if (rc) return fail(rc);
    rc = build_host_far(el, in, hp);
    if (verbose) fprintf(stderr, "[fdph_plan] host threads %d\n", in.threads);
    stamp("host plan (admissible blocks)");
    if (rc == -3) return fail(FDPH_E_CAUSALITY);
    if (rc) return fail(FDPH_E_ARG);
    // ---- upload the far-field operator
    std::vector<SbDev> sd(hp.sbs.size());
    for (size_t q = 0; q < sd.size(); ++q) {
        const SubBlock& b = hp.sbs[q];
        const int LH = b.maxdelay - b.mindelay + 1;
        sd[q] = {b.kind, b.rank, b.r0, b.nr, b.s0, b.ns, b.L, b.LZ, b.taps, b.maxdelay, b.mindm, b.run0,
                 b.soe, b.ident, b.e0, LH, (long long)b.f, (long long)b.g, (long long)b.h, (long long)b.ring, (long long)b.zring,
                 (long long)b.dhat, (long long)b.delay, (long long)b.dm, (long long)b.ustate, (long long)b.trc,
                 (long long)b.phi, 0, b.mindelay, b.qn, (long long)b.qb};
    }
    // delayed-history form of Eq. 42 (far_mode 1): per block a history [LH][ns] of the source
    // values, recorded every step, and one gather task per (block, rank index)
    std::vector<int2> rec, gat;
    if (P->far_mode == 1)
        for (size_t q = 0; q < sd.size(); ++q) {
            sd[q].uhist = P->uhist_len;
            P->uhist_len += (long long)sd[q].LH * sd[q].ns;
            for (int j = 0; j < sd[q].ns; ++j) rec.push_back(make_int2((int)q, j));
            for (int l = 0; l < sd[q].rank; ++l) gat.push_back(make_int2((int)q, l));
        }
    P->n_rec = (int)rec.size();
    P->n_gat = (int)gat.size();
    if ((rc = upload(P, &P->rec_tasks, rec)) || (rc = upload(P, &P->gat_tasks, gat))) return fail(rc);
    // warp tasks: 2^lg lanes per run (scatter) / per receiver (Eq. 39), 2^lg the rank rounded up
    // to a power of two (at most 32); identity factors need one lane
    std::vector<int4> sct, evt;
    for (size_t q = 0; q < hp.sbs.size(); ++q) {
        const SubBlock& b = hp.sbs[q];
        int lg = 0;
        while ((1 << lg) < std::min(b.rank, 32)) ++lg;
        const int lg_s = b.ident == 2 ? 0 : lg, lg_e = b.ident == 1 ? 0 : lg;
        for (int r = 0; r < b.nruns; r += 32 >> lg_s)
            sct.push_back(make_int4((int)q, b.run0 + r, std::min(32 >> lg_s, b.nruns - r), lg_s));
        for (int i = 0; i < b.nr; i += 32 >> lg_e)
            evt.push_back(make_int4((int)q, i, std::min(32 >> lg_e, b.nr - i), lg_e));
    }
    P->n_sct = (int)sct.size();
    P->n_evt = (int)evt.size();
    if ((rc = upload(P, &P->sc_tasks, sct)) || (rc = upload(P, &P->ev_tasks, evt))) return fail(rc);
    if ((rc = upload(P, &P->perm, hp.perm)) || (rc = upload(P, &P->sbs, sd)) || (rc = upload(P, &P->ints, hp.ints)) ||
        (rc = upload(P, &P->run_delay, hp.run_delay)) || (rc = upload(P, &P->run_start, hp.run_start)) ||
        (rc = upload(P, &P->run_len, hp.run_len)) || (rc = upload(P, &P->src_order, hp.src_order)) ||
        (rc = upload(P, &P->e_pos, hp.e_pos)) ||
        (rc = upload(P, &P->fir_sb, hp.fir_sb)) || (rc = upload(P, &P->fir_j, hp.fir_j)) ||
        (rc = upload(P, &P->sfir_ptr, hp.sfir_ptr)) || (rc = upload(P, &P->sfir_q, hp.sfir_q)) ||
        (rc = upload(P, &P->sfir_tmax, hp.sfir_tmax)) ||
        (rc = upload(P, &P->tr_sb, hp.tr_sb)) || (rc = upload(P, &P->tr_l, hp.tr_l)) ||
        (rc = upload(P, &P->g_ptr, hp.g_ptr)) || (rc = upload(P, &P->g_sb, hp.g_sb)) ||
        (rc = upload(P, &P->g_il, hp.g_il)))
        return fail(rc);
    // the source-major FIR where sources sit in many F blocks (large N; fdph_autotune times both)
    P->sfir = hp.fir_sb.size() >= (size_t)100 * hp.n;
    if (P->precision != FDPH_FP64) {
        std::vector<float> f(hp.fac.begin(), hp.fac.end());
        float* d = nullptr;
        if ((rc = upload(P, &d, f))) return fail(rc);
        P->fac = d;
    } else {
        double* d = nullptr;
        if ((rc = upload(P, &d, hp.fac))) return fail(rc);
        P->fac = d;
    }
    if (hp.soe > 0 && (rc = upload(P, &P->trcoef, hp.trcoef))) return fail(rc);
    if (hp.interp && (rc = upload(P, &P->phi, hp.phis))) return fail(rc);
    stamp("far-field upload");
    // ---- near field (device-evaluated kernel windows)
    rc = P->precision == FDPH_FP16   ? build_near_finish<float, __half>(P, in, nb)
         : P->precision == FDPH_FP32 ? build_near_finish<float, float>(P, in, nb)
                                     : build_near_finish<double, double>(P, in, nb);
    if (rc) return fail(rc);
    stamp("near field (windows, tails)");

    if ((rc = dalloc(P, &P->err, 1))) return fail(rc);
    FDPH_CUDA(cudaMemsetAsync(P->err, 0, sizeof(int), P->stream));
    // ---- state
    P->WD = std::max(std::max(hp.max_W + (hp.soe > 0 ? 1 : 0), hp.max_taps), 1);
    P->WC = hp.max_W + 1;
    size_t sb = 0;
    auto st = [&](double** p, size_t cnt) {   // one copy per right-hand side
        const size_t c = std::max<size_t>(cnt, 1) * P->nrhs;
        sb += c * 8;
        return dalloc(P, p, c);
    };
    if ((rc = st(&P->Dring, (size_t)P->WD * P->N)) || (rc = st(&P->Cring, (size_t)P->WC * P->N)) ||
        (rc = st(&P->C, P->N)) || (rc = st(&P->Ccomp, P->N)) || (rc = st(&P->ring, hp.ring_len)) ||
        (rc = st(&P->zring, hp.zring_len)) || (rc = st(&P->dhat, hp.dhat_len)) ||
        (rc = st(&P->partial, hp.items.size() * 32)) || (rc = st(&P->fval, hp.e_pos.size())) ||
        (rc = st(&P->ustate, hp.ustate_len)) || (rc = st(&P->vstate, hp.vstate_len)) ||
        (rc = st(&P->uhist, (size_t)P->uhist_len)))
        return fail(rc);
    if (P->precision != FDPH_FP64) {   // FP32 copy of the slip-rate ring for the near-field rows
        const size_t c = (size_t)P->WD * P->N * P->nrhs;
        if ((rc = dalloc(P, &P->Dring32, c))) return fail(rc);
        sb += c * 4;
    }
    if ((rc = dalloc(P, &P->tfar, (size_t)P->N * P->nrhs))) return fail(rc);   // far-field traction (scratch)
    if (P->precision == FDPH_FP16 && P->nrhs >= 2) {   // (hi, lo) FP16 rows of the tensor-core near field
        P->NP = (P->N + 3) & ~3;
        const size_t c = (size_t)2 * P->WD * P->nrhs * P->NP;
        const size_t cs = (size_t)2 * P->WD * std::max(P->nrhs, 4);
        if ((rc = dalloc(P, &P->Dring16, c)) || (rc = dalloc(P, &P->Dscale, cs))) return fail(rc);
        sb += c * 4 + cs * 4;
        if ((rc = make_row_tensor_map(P))) return fail(rc);
    }
    P->state_bytes = sb;
    P->partial_cap = std::max<size_t>(hp.items.size() * 32, 1);
    if ((rc = fdph_reset(P))) return fail(rc);
    fill_stats(P);
    P->st.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return FDPH_OK;
}

int fdph_reset(fdph_plan_t P) {
    if (!P) return FDPH_E_ARG;
    P->predicted = false;
    cudaSetDevice(P->device);
    double* bufs[] = {P->Dring, P->Cring, P->C, P->Ccomp, P->ring, P->zring, P->dhat, P->partial,
                      P->ustate, P->vstate, P->uhist};
    size_t cnt[] = {(size_t)P->WD * P->N, (size_t)P->WC * P->N, (size_t)P->N, (size_t)P->N,
                    (size_t)P->hp.ring_len, (size_t)P->hp.zring_len, (size_t)P->hp.dhat_len,
                    P->partial_cap, (size_t)P->hp.ustate_len, (size_t)P->hp.vstate_len, (size_t)P->uhist_len};
    for (int q = 0; q < 11; ++q)   // every right-hand side: [nrhs][max(count, 1)]
        if (bufs[q])
            FDPH_CUDA(cudaMemsetAsync(bufs[q], 0, std::max<size_t>(cnt[q], 1) * P->nrhs * sizeof(double), P->stream));
    if (P->Dring32)
        FDPH_CUDA(cudaMemsetAsync(P->Dring32, 0, (size_t)P->WD * P->N * P->nrhs * sizeof(float), P->stream));
    if (P->Dring16) {
        FDPH_CUDA(cudaMemsetAsync(P->Dring16, 0, (size_t)2 * P->WD * P->NP * P->nrhs * sizeof(__half2), P->stream));
        FDPH_CUDA(cudaMemsetAsync(P->Dscale, 0, (size_t)2 * P->WD * std::max(P->nrhs, 4) * sizeof(float), P->stream));
    }
    if (P->rupture) FDPH_CUDA(cudaMemsetAsync(P->fr.slip, 0, P->N * sizeof(double), P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    P->n = 0;
    return FDPH_OK;
}

int fdph_step(fdph_plan_t P, const double* D_n, double* T_n) {
    if (!P || !D_n || !T_n) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
    if (P->n >= P->M) {
        set_error("the plan has already taken M steps");
        return FDPH_E_STATE;
    }
    return step_impl(P, D_n, T_n);
}

int fdph_run(fdph_plan_t P, int32_t steps, const double* D, double* T) {
    if (!P || !D || !T || steps < 0) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
    if (P->n + steps > P->M) {
        set_error("run would pass step M");
        return FDPH_E_STATE;
    }
    if (steps >= 8 && !P->prof)   // launch-bound steps: replay a captured graph of one step
        return P->precision != FDPH_FP64 ? run_graph<float>(P, steps, D, T) : run_graph<double>(P, steps, D, T);
    for (int s = 0; s < steps; ++s) {
        const size_t row = (size_t)P->N * P->nrhs;
        int rc = step_impl(P, D + s * row, T + s * row);
        if (rc) return rc;
    }
    return FDPH_OK;
}

int fdph_run_host(fdph_plan_t P, int32_t steps, const double* D_host, double* T_host) {
    if (!P || !D_host || !T_host || steps < 0) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
    if (P->n + steps > P->M) {
        set_error("run would pass step M");
        return FDPH_E_STATE;
    }
    if (steps == 0) return FDPH_OK;
    int rc;
    if (P->prof) {   // per-kernel timing: plain launches, one staging row
        const size_t row = (size_t)P->N * P->nrhs;
        if (!P->dD && ((rc = dalloc(P, &P->dD, row)) || (rc = dalloc(P, &P->dT, row)))) return rc;
        for (int k = 0; k < steps; ++k) {
            FDPH_CUDA(cudaMemcpyAsync(P->dD, D_host + k * row, row * sizeof(double),
                                      cudaMemcpyHostToDevice, P->stream));
            if ((rc = step_impl(P, P->dD, P->dT))) return rc;
            FDPH_CUDA(cudaMemcpyAsync(T_host + k * row, P->dT, row * sizeof(double),
                                      cudaMemcpyDeviceToHost, P->stream));
        }
        FDPH_CUDA(cudaStreamSynchronize(P->stream));
        return check_device_error(P);
    }
    rc = P->precision != FDPH_FP64 ? run_host<float>(P, steps, D_host, T_host)
                                   : run_host<double>(P, steps, D_host, T_host);
    if (rc) return rc;
    return check_device_error(P);
}

int fdph_step_host(fdph_plan_t P, const double* D_n_host, double* T_n_host) {
    if (!P || !D_n_host || !T_n_host) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
    const size_t row = (size_t)P->N * P->nrhs;
    if (!P->dD) {
        int rc;
        if ((rc = dalloc(P, &P->dD, row)) || (rc = dalloc(P, &P->dT, row))) return rc;
    }
    FDPH_CUDA(cudaMemcpyAsync(P->dD, D_n_host, row * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    int rc = fdph_step(P, P->dD, P->dT);
    if (rc) return rc;
    FDPH_CUDA(cudaMemcpyAsync(T_n_host, P->dT, row * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    return check_device_error(P);
}

int fdph_selftest_wait_timeout(int32_t device, int64_t polls) {
    if (polls < 1 || polls > (1LL << 24)) {
        set_error("fdph_selftest_wait_timeout: polls in [1, 2^24]");
        return FDPH_E_ARG;
    }
    FDPH_CUDA(cudaSetDevice(device));
    int* err = nullptr;
    FDPH_CUDA(cudaMalloc(&err, sizeof(int)));
    int h = 0;
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32>>>(polls, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) {
        set_error(std::string("fdph_selftest_wait_timeout: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    if (h) {
        set_error("bounded mbarrier wait gave up after " + std::to_string(polls) + " polls (self-test)");
        return FDPH_E_TIMEOUT;
    }
    return FDPH_OK;
}

int fdph_autotune(fdph_plan_t P, int32_t steps, int32_t* chunk_out) {
    if (!P || steps < 1 || steps > 1024) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
    if (P->prof) {
        set_error("fdph_autotune: profiling is on");
        return FDPH_E_STATE;
    }
    if (P->hp.items.empty()) {
        if (chunk_out) *chunk_out = P->chunk;
        return FDPH_OK;
    }
    const int M = P->M;
    if (steps + 2 > M) {
        set_error("fdph_autotune: the plan has fewer than steps + 2 steps");
        return FDPH_E_ARG;
    }
    // the state is saved and restored around the trials
    size_t len = 0;
    int rc = fdph_save_state(P, nullptr, &len);
    if (rc) return rc;
    std::vector<char> saved(len);
    if ((rc = fdph_save_state(P, saved.data(), &len))) return rc;
    double *Dz = nullptr, *Tz = nullptr;
    const size_t rows = (size_t)(steps + 2) * P->N * P->nrhs;   // steps of nrhs rows of N
    if ((rc = dalloc(P, &Dz, rows)) || (rc = dalloc(P, &Tz, rows))) return rc;
    FDPH_CUDA(cudaMemsetAsync(Dz, 0, rows * sizeof(double), P->stream));
    // trials at a steady-state step index (every window full); the values stepped are irrelevant
    const int n0 = std::max(0, std::min(P->hp.max_W, M - steps - 2));
    cudaEvent_t e0, e1;
    FDPH_CUDA(cudaEventCreate(&e0));
    FDPH_CUDA(cudaEventCreate(&e1));
    const int cmax = near_max_chunk(P->nrhs, P->precision);
    const int cands[3] = {cmax, cmax / 2, cmax / 4};
    int best = P->chunk;
    float best_ms = 1e30f;
    for (int c : cands) {
        if ((rc = set_chunk_any(P, c))) break;
        P->n = n0;
        rc = P->precision != FDPH_FP64 ? run_graph<float>(P, 2, Dz, Tz) : run_graph<double>(P, 2, Dz, Tz);   // capture
        if (rc) break;
        cudaEventRecord(e0, P->stream);
        rc = P->precision != FDPH_FP64 ? run_graph<float>(P, steps, Dz, Tz) : run_graph<double>(P, steps, Dz, Tz);
        if (rc) break;
        cudaEventRecord(e1, P->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    if (!rc) rc = set_chunk_any(P, best);
    // then the other form of Eq. 32 (source-major or sub-block-major) at that item length
    if (!rc && P->sfir_ptr && P->hp.max_taps > 0) {
        const bool first = P->sfir;
        P->sfir = !first;
        FDPH_CUDA(cudaStreamSynchronize(P->stream));
        for (auto& ge : P->graphs) cudaGraphExecDestroy(ge.ex);   // they hold the old launches
        P->graphs.clear();
        P->n = n0;
        rc = P->precision != FDPH_FP64 ? run_graph<float>(P, 2, Dz, Tz) : run_graph<double>(P, 2, Dz, Tz);
        float ms = 1e30f;
        if (!rc) {
            cudaEventRecord(e0, P->stream);
            rc = P->precision != FDPH_FP64 ? run_graph<float>(P, steps, Dz, Tz) : run_graph<double>(P, steps, Dz, Tz);
            cudaEventRecord(e1, P->stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (rc || !(ms < best_ms)) {
            P->sfir = first;
            FDPH_CUDA(cudaStreamSynchronize(P->stream));
            for (auto& ge : P->graphs) cudaGraphExecDestroy(ge.ex);
            P->graphs.clear();
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2 = fdph_load_state(P, saved.data(), saved.size());
    if (rc) return rc;
    if (rc2) return rc2;
    if ((rc = check_device_error(P))) return rc;
    if (chunk_out) *chunk_out = best;
    return FDPH_OK;
}

int fdph_plan_stream(fdph_plan_t P, void** stream) {
    if (!P || !stream) return FDPH_E_ARG;
    *stream = (void*)P->stream;
    return FDPH_OK;
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
    if (P->predicted) return pending_commit(P);
    double* bufs[] = {P->Dring, P->Cring, P->C, P->Ccomp, P->ring, P->zring, P->ustate, P->vstate, P->uhist,
                      P->rupture ? P->fr.slip : nullptr};
    size_t cnt[] = {(size_t)P->WD * P->N, (size_t)P->WC * P->N, (size_t)P->N, (size_t)P->N,
                    (size_t)P->hp.ring_len, (size_t)P->hp.zring_len, (size_t)P->hp.ustate_len,
                    (size_t)P->hp.vstate_len, (size_t)P->uhist_len, 0};
    for (size_t& c : cnt) c = c ? c * P->nrhs : 0;   // [nrhs][count] (a zero count stays empty)
    if (P->rupture) cnt[9] = (size_t)P->N;             // the friction law's accumulated slip
    size_t need = sizeof(int32_t) * 2;
    for (int q = 0; q < 10; ++q) need += cnt[q] * sizeof(double);
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
    for (int q = 0; q < 10; ++q) {
        if (cnt[q]) FDPH_CUDA(cudaMemcpyAsync(o, bufs[q], cnt[q] * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
        o += cnt[q] * sizeof(double);
    }
    FDPH_CUDA(cudaStreamSynchronize(P->stream));   // the caller's buffer is complete on return
    *len = need;
    return FDPH_OK;
}

int fdph_load_state(fdph_plan_t P, const void* buf, size_t len) {
    if (!P || !buf) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
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
    double* bufs[] = {P->Dring, P->Cring, P->C, P->Ccomp, P->ring, P->zring, P->ustate, P->vstate, P->uhist,
                      P->rupture ? P->fr.slip : nullptr};
    size_t cnt[] = {(size_t)P->WD * P->N, (size_t)P->WC * P->N, (size_t)P->N, (size_t)P->N,
                    (size_t)P->hp.ring_len, (size_t)P->hp.zring_len, (size_t)P->hp.ustate_len,
                    (size_t)P->hp.vstate_len, (size_t)P->uhist_len, 0};
    for (size_t& c : cnt) c = c ? c * P->nrhs : 0;   // [nrhs][count] (a zero count stays empty)
    if (P->rupture) cnt[9] = (size_t)P->N;             // the friction law's accumulated slip
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    for (int q = 0; q < 10; ++q) {
        if (cnt[q]) FDPH_CUDA(cudaMemcpyAsync(bufs[q], o, cnt[q] * sizeof(double), cudaMemcpyHostToDevice, P->stream));
        o += cnt[q] * sizeof(double);
    }
    if (P->Dring32) {
        const long long c = (long long)P->WD * P->N * P->nrhs;
        ring_to_float_kernel<<<blocks(c, 256), 256, 0, P->stream>>>(P->Dring, P->Dring32, c);
        FDPH_CUDA(cudaGetLastError());
    }
    if (P->Dring16) {   // every slot of the (hi, lo) FP16 rows from the restored ring
        if (P->precision == FDPH_FP16) {
            const StepArgs<float> a = make_args<float>(P, nullptr, nullptr);
            tc_rows_kernel<float><<<dim3(P->WD, P->nrhs), kRowThreads, 0, P->stream>>>(a, 1);
        }
        FDPH_CUDA(cudaGetLastError());
    }
    FDPH_CUDA(cudaStreamSynchronize(P->stream));   // the caller may reuse the buffer on return
    P->n = hdr[0];
    return FDPH_OK;
}

// K_{ii,0} in geometry order: jump of the ramp response of each element at its own midpoint over
// [0, dt] (Eq. 4 with m = 0).  FDPH_E_STATE when the instantaneous term is not local
// (cs dt > half the shortest element: K_{ij,0} != 0 for neighbours).
static int self_coefficients(fdph_plan_t P, std::vector<double>& k0) {
    const HostPlan& hp = P->hp;
    double minlen = 1e300;
    for (int p = 0; p < P->N; ++p) minlen = std::min(minlen, hp.slen[p]);
    if (hp.cs * P->dt > 0.5 * minlen * (1.0 + 1e-12)) {
        set_error("cs dt exceeds half the shortest element; the instantaneous term is not local");
        return FDPH_E_STATE;
    }
    k0.assign(P->N, 0.0);
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
    return FDPH_OK;
}

int fdph_rupture_init(fdph_plan_t P, const fdph_friction* f) {
    if (!P || !f || !f->tau0 || !(f->sigma_n > 0.0) || !(f->Dc > 0.0) || f->mu_d > f->mu_s ||
        (f->law != 0 && f->law != 1)) {
        set_error("fdph_rupture_init: friction with tau0, sigma_n > 0, Dc > 0, mu_d <= mu_s, law 0 or 1 required");
        return FDPH_E_ARG;
    }
    if (P->predicted) return pending_commit(P);
    if (P->nrhs != 1) {
        set_error("fdph_rupture_init: dynamic rupture takes plans of one right-hand side (nrhs = 1)");
        return FDPH_E_ARG;
    }
    std::vector<double> k0;
    int rc0 = self_coefficients(P, k0);
    if (rc0) return rc0;
    if (!P->rupture) {
        double *tau0 = nullptr, *kk = nullptr, *slip = nullptr;
        int rc;
        if ((rc = dalloc(P, &tau0, P->N)) || (rc = dalloc(P, &kk, P->N)) || (rc = dalloc(P, &slip, P->N))) return rc;
        P->fr.tau0 = tau0;
        P->fr.k0 = kk;
        P->fr.slip = slip;
    }
    // ordered after the caller's work on the plan's stream (tau0 may have been written there)
    FDPH_CUDA(cudaMemcpyAsync((void*)P->fr.tau0, f->tau0, P->N * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
    FDPH_CUDA(cudaMemcpyAsync((void*)P->fr.k0, k0.data(), P->N * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    FDPH_CUDA(cudaMemsetAsync(P->fr.slip, 0, P->N * sizeof(double), P->stream));
    FDPH_CUDA(cudaStreamSynchronize(P->stream));
    P->fr.sigma_n = f->sigma_n;
    P->fr.mu_s = f->mu_s;
    P->fr.mu_d = f->mu_d;
    P->fr.Dc = f->Dc;
    P->fr.dt = P->dt;
    P->fr.law = f->law;
    P->rupture = true;
    return FDPH_OK;
}

int fdph_rupture_step(fdph_plan_t P, double* D_n, double* T_n) {
    if (!P || !D_n || !T_n) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
    if (!P->rupture) {
        set_error("fdph_rupture_init has not been called on this plan");
        return FDPH_E_STATE;
    }
    if (P->n >= P->M) {
        set_error("the plan has already taken M steps");
        return FDPH_E_STATE;
    }
    int rc = P->precision != FDPH_FP64 ? launch_rupture_step<float>(P, D_n, T_n) : launch_rupture_step<double>(P, D_n, T_n);
    if (rc == FDPH_OK) P->n += 1;
    return rc;
}

int fdph_rupture_run(fdph_plan_t P, int32_t steps, double* D, double* T) {
    if (!P || !D || !T || steps < 0) return FDPH_E_ARG;
    if (P->predicted) return pending_commit(P);
    if (P->n + steps > P->M) {
        set_error("run would pass step M");
        return FDPH_E_STATE;
    }
    if (!P->rupture) {
        set_error("fdph_rupture_init has not been called on this plan");
        return FDPH_E_STATE;
    }
    if (steps >= 8 && !P->prof)   // replay a captured graph of one rupture step
        return P->precision != FDPH_FP64 ? rupture_graph<float>(P, steps, D, T) : rupture_graph<double>(P, steps, D, T);
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

int fdph_predict(fdph_plan_t P, double* T_pred) {
    if (!P || !T_pred) return FDPH_E_ARG;
    if (P->nrhs != 1) {
        set_error("this call takes plans of one right-hand side (nrhs = 1)");
        return FDPH_E_ARG;
    }
    if (P->predicted) return pending_commit(P);
    if (P->n >= P->M) {
        set_error("the plan has already taken M steps");
        return FDPH_E_STATE;
    }
    int rc = P->precision != FDPH_FP64 ? launch_predict<float>(P, T_pred) : launch_predict<double>(P, T_pred);
    if (rc == FDPH_OK) P->predicted = true;
    return rc;
}

int fdph_commit(fdph_plan_t P, const double* D_n) {
    if (!P || !D_n) return FDPH_E_ARG;
    if (P->nrhs != 1) {
        set_error("this call takes plans of one right-hand side (nrhs = 1)");
        return FDPH_E_ARG;
    }
    if (!P->predicted) {
        set_error("fdph_commit without a preceding fdph_predict of this step");
        return FDPH_E_STATE;
    }
    int rc = P->precision != FDPH_FP64 ? launch_commit<float>(P, D_n) : launch_commit<double>(P, D_n);
    if (rc == FDPH_OK) {
        P->predicted = false;
        P->n += 1;
    }
    return rc;
}

int fdph_self(fdph_plan_t P, double* diag) {
    if (!P || !diag) return FDPH_E_ARG;
    std::vector<double> k0;
    int rc = self_coefficients(P, k0);
    if (rc) return rc;
    memcpy(diag, k0.data(), k0.size() * sizeof(double));
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

int fdph_batch_create(const fdph_plan_t* plans, int32_t count, fdph_batch_t* out) {
    if (!plans || !out || count < 1 || count > 1024) return FDPH_E_ARG;
    *out = nullptr;
    for (int p = 0; p < count; ++p) {
        if (!plans[p]) return FDPH_E_ARG;
        for (int q = 0; q < p; ++q)
            if (plans[q] == plans[p]) {
                set_error("fdph_batch_create: a plan appears twice");
                return FDPH_E_ARG;
            }
        if (plans[p]->device != plans[0]->device || plans[p]->precision != plans[0]->precision) {
            set_error("fdph_batch_create: plans of one batch share the device and the precision");
            return FDPH_E_ARG;
        }
        if (plans[p]->predicted) return pending_commit(plans[p]);
        if (plans[p]->nrhs != 1 || plans[p]->far_mode != 0) {
            set_error("fdph_batch_create: batches take plans of one right-hand side (nrhs = 1) and far_mode 0");
            return FDPH_E_ARG;
        }
    }
    fdph_batch_t B = new fdph_batch_s;
    B->device = plans[0]->device;
    B->precision = plans[0]->precision;
    B->plans.assign(plans, plans + count);
    for (int p = 0; p < count; ++p) B->version.push_back(plans[p]->sched_version);
    B->near_priority = plans[0]->near_priority;
    if (cudaSetDevice(B->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->side[0], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->side[1], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_join[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_join[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_end, cudaEventDisableTiming) != cudaSuccess) {
        set_error("fdph_batch_create: stream / event creation failed");
        batch_free(B);
        return FDPH_E_CUDA;
    }
    B->ev_ready.assign(count, nullptr);
    for (int p = 0; p < count; ++p)
        if (cudaEventCreateWithFlags(&B->ev_ready[p], cudaEventDisableTiming) != cudaSuccess) {
            set_error("fdph_batch_create: event creation failed");
            batch_free(B);
            return FDPH_E_CUDA;
        }
    int rc = B->precision == FDPH_FP16   ? batch_schedule<float, __half>(B)
             : B->precision == FDPH_FP32 ? batch_schedule<float, float>(B)
                                         : batch_schedule<double, double>(B);
    if (rc) {
        batch_free(B);
        return rc;
    }
    *out = B;
    return FDPH_OK;
}

int fdph_batch_run(fdph_batch_t B, int32_t steps, const double* const* D, double* const* T) {
    if (!B || !D || !T || steps < 0) return FDPH_E_ARG;
    for (size_t p = 0; p < B->plans.size(); ++p)
        if (!D[p] || !T[p]) return FDPH_E_ARG;
    int rc = batch_check(B, steps);
    if (rc || steps == 0) return rc;
    cudaSetDevice(B->device);
    return B->precision != FDPH_FP64 ? batch_run<float>(B, GRAPH_RUN, steps, D, T)
                                     : batch_run<double>(B, GRAPH_RUN, steps, D, T);
}

int fdph_batch_rupture_run(fdph_batch_t B, int32_t steps, double* const* D, double* const* T) {
    if (!B || !D || !T || steps < 0) return FDPH_E_ARG;
    for (size_t p = 0; p < B->plans.size(); ++p) {
        if (!D[p] || !T[p]) return FDPH_E_ARG;
        if (!B->plans[p]->rupture) {
            set_error("fdph_rupture_init has not been called on a plan of the batch");
            return FDPH_E_STATE;
        }
    }
    int rc = batch_check(B, steps);
    if (rc || steps == 0) return rc;
    cudaSetDevice(B->device);
    return B->precision != FDPH_FP64 ? batch_run<float>(B, GRAPH_RUPTURE, steps, (const double* const*)D, T)
                                     : batch_run<double>(B, GRAPH_RUPTURE, steps, (const double* const*)D, T);
}

int fdph_batch_synchronize(fdph_batch_t B) {
    if (!B) return FDPH_E_ARG;
    FDPH_CUDA(cudaStreamSynchronize(B->stream));
    for (fdph_plan_t P : B->plans) {
        FDPH_CUDA(cudaStreamSynchronize(P->stream));
        int rc = check_device_error(P);
        if (rc) return rc;
    }
    return FDPH_OK;
}

void fdph_batch_destroy(fdph_batch_t B) { batch_free(B); }

void fdph_destroy(fdph_plan_t P) {
    if (!P) return;
    cudaSetDevice(P->device);
    if (P->stream) cudaStreamSynchronize(P->stream);
    prof_drain(P);
    for (auto& ge : P->graphs) cudaGraphExecDestroy(ge.ex);
    for (int k = 0; k < 2; ++k) {
        if (P->side[k]) cudaStreamDestroy(P->side[k]);
        if (P->ev_join[k]) cudaEventDestroy(P->ev_join[k]);
    }
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->h2d) cudaStreamSynchronize(P->h2d);
    if (P->d2h) cudaStreamSynchronize(P->d2h);
    if (P->h2d) cudaStreamDestroy(P->h2d);
    if (P->d2h) cudaStreamDestroy(P->d2h);
    for (int q = 0; q < fdph_plan_s::kIoSlots; ++q) {
        if (P->ev_in[q]) cudaEventDestroy(P->ev_in[q]);
        if (P->ev_out[q]) cudaEventDestroy(P->ev_out[q]);
        if (P->ev_free[q]) cudaEventDestroy(P->ev_free[q]);
    }
    for (void* p : P->allocs) cudaFree(p);
    if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
    delete P;
}

}  // extern "C"
