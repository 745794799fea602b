// plan.h -- flat, device-ready description of an FDP=H operator (built on the host).
#pragma once
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace fdph {

enum SubKind { SB_F = 0, SB_S = 1, SB_TR = 2 };

// One low-rank operator: admissible leaf x domain (F / S / transient) x stress component.
// Receivers [r0, r0 + nr), sources [s0, s0 + ns) in internal order.
struct SubBlock {
    int32_t kind, rank, r0, nr, s0, ns;
    int32_t L;         // ring length (F, S: representative-stress ring; TR: source-sum ring Y)
    int32_t LZ;        // TR: length of the convolved ring Z
    int32_t taps;      // F: waveform taps (max Dm of the leaf); TR: Dm_tr
    int32_t maxdelay, mindelay, mindm, maxdm;
    int64_t f, g, h;   // offsets into the factor array (f: nr x rank, g: ns x rank, h: taps x ns or taps)
    int64_t ring, zring, dhat;   // offsets into state arrays
    int64_t delay, dm; // offsets into the int array (delay[ns], dm[nr])
    int32_t run0, nruns;
    int32_t soe;       // TR: exponential-tail terms after the `taps` exact taps (0 = none)
    int64_t trc;       // TR: offset of their FP64 coefficients in HostPlan::trcoef
    int64_t ustate;    // TR: offset of the [rank][soe] recursive tail states
    int64_t phi;       // offset of the receivers' sub-step delays in HostPlan::phis (interp only)
    int32_t ident;     // block kept exact: 1 = F is the identity (rank nr), 2 = G is the identity
                       // (rank ns), 0 = low-rank factors
    int32_t e0;        // index of the block's first (block, receiver) entry in block-major order
    int32_t qn;        // TR with eps_q > 0: quantized ranges of the taps (h then holds their qn values)
    int64_t qb;        // TR: offset of the qn + 1 range bounds in the int array
};

struct NearLeaf {
    int32_t r0, nr, s0, ns, W;   // W = window of exact kernel steps stored
    // Slices are stored source-interleaved: element (j, i) of a slice at ((j / v) * nr + i) * v + j % v
    // with v = 16 bytes / element size, the sources padded with zeros to a multiple of v, so that a
    // receiver reads v sources with one 16-byte load.
    int32_t sl;                  // window slice stride: ceil(ns / v) v nr (v of the window storage type)
    int32_t sla;                 // aux slice stride, the same with v of the aux storage type
    int64_t tensor;              // offset of [W][sl] coefficients
    // "aux" slices of the leaf (aux storage type, same layout), [naux][sla] at `stat`: slice 0
    // the static tile (x dt), slices 1..Q the exponential-tail coefficients (`tail`, -1: none)
    int64_t stat;
    int64_t tail;
    int32_t naux;
    int64_t vstate;              // offset of the [Q][ns] recursive tail states
};

// A near-field work item: window slices [k0, k1) of a leaf (kind 0), or its aux slices (kind 1).
// a work item: window slices [k0, k1) of a leaf (kind 0), or its aux slices [k0, k1) (kind 1:
// slice 0 the static tile, slice 1 + q the exponential-tail coefficients of term q)
struct NearItem {
    int32_t leaf, k0, k1, kind;
};

struct HostPlan {
    int n = 0, M = 0;
    double dt = 0, mu = 0, cs = 0;
    Tree tree;
    std::vector<int32_t> perm;                       // internal -> geometry index
    // internal-order geometry for the device near-field builder
    std::vector<double> px, py, pnx, pny, sax, say, sbx, sby, stx, sty, slen;
    // far field
    std::vector<SubBlock> sbs;
    std::vector<double> fac;                         // f, g, h, htr (FP64 master copy)
    std::vector<double> trcoef;                      // transient-fibre tail coefficients (FP64)
    std::vector<double> phis;                        // sub-step receiver delays per leaf
    int interp = 0;
    std::vector<int32_t> ints;                       // delays, dm
    std::vector<int32_t> run_delay, run_start, run_len, src_order;
    std::vector<int32_t> fir_sb, fir_j;              // FIR tasks
    std::vector<int32_t> sfir_ptr, sfir_q, sfir_tmax; // FIR tasks by source element, longest taps
    std::vector<int32_t> tr_sb, tr_l;                // transient convolution tasks
    std::vector<int32_t> g_ptr, g_sb, g_il;          // gather CSR (receiver-major)
    std::vector<int32_t> e_pos;                      // CSR slot of each entry, block-major order
    int64_t ring_len = 0, zring_len = 0, dhat_len = 0, ustate_len = 0;
    int soe = 0;                                     // exponential-tail terms (0: paper's cut)
    std::vector<double> rho;                         // their decay factors
    int32_t max_taps = 0;
    // near field
    std::vector<NearLeaf> near;
    std::vector<int32_t> near_r0, near_nr, near_s0, near_ns;   // for the m_S kernel
    std::vector<NearItem> items;
    std::vector<int32_t> np_ptr, np_idx;             // receiver -> partial slots
    int64_t near_tensor_len = 0, near_aux_len = 0, near_tail_len = 0, vstate_len = 0;
    int32_t max_W = 0;
    // stats
    int n_adm = 0, n_near = 0, max_rank = 0;
    double mean_rank = 0;
    double rank_w[3] = {0, 0, 0}, ent_w[3] = {0, 0, 0};   // per SubKind: sum rank * entries, sum entries
    int n_exact[3] = {0, 0, 0};                          // per SubKind: sub-blocks kept exact
    int n_aca = 0;                                       // sub-blocks from cross approximation
    int64_t far_entries = 0;
    int64_t far_nent = 0;                            // (block, receiver) entries
};

// Everything except the near-field windows (which need the device). Returns status.
int build_host_plan(const Elements& el, const PlanInputs& in, HostPlan& hp);
// The same in two stages: the cluster and block trees (with the near-leaf lists), then the
// admissible blocks (ART integers, low-rank factors, waveforms, transients).  The near-field
// build needs only the first stage, so the device can work on it during the second.
void build_host_tree(const Elements& el, const PlanInputs& in, HostPlan& hp);
// Discretised causality of every admissible leaf of the tree (Sec. 5.2): -3 if one violates it.
int check_causality(const Elements& el, const PlanInputs& in, const Tree& tr);
int build_host_far(const Elements& el, const PlanInputs& in, HostPlan& hp);
// Second stage once the near-field windows W are known (fills offsets, items, CSR).
// vec, vec_aux: sources per 16 bytes of the window and aux storage types (8 FP16, 4 FP32, 2 FP64);
// chunk, aux_chunk: window and aux slices per work item at most.
void finish_near_layout(HostPlan& hp, const std::vector<int32_t>& W, const std::vector<char>& has_tail, int chunk,
                        int vec, int vec_aux, int aux_chunk);

}  // namespace fdph
