/*
 * fdph.h -- C ABI of the FDP=H space-time BIEM hot path (2-D antiplane, GB300 / sm_103a).
 *
 * The library evaluates, one time step at a time, the discretised space-time
 * boundary integral equation of Sato & Ando (arXiv 1903.02118), Sec. 2.1.2, Eq. 4:
 *
 *     T_n = sum_{m >= 0} K_m D_{n-m}
 *
 * for N piecewise-constant fault elements, where D_n is the slip rate of step n
 * and T_n the traction at the element midpoints at time (n + 1) dt.  The kernel
 * tensor is never stored densely: the plan splits it into
 *   - admissible leaves of the H-matrix block tree (Sec. 2.3, Eq. 8), whose
 *     wavefront part (Domain F, Sec. 2.2) is a low-rank amplitude (Eqs. 12-13)
 *     times a per-source normalised waveform placed by the ART integers
 *     (Eqs. 29-31, App. C.3), followed by the static part (Domain S, App. B.1)
 *     and the 2-D transient of Domain S (App. B.3, App. H);
 *   - inadmissible leaves (Eq. 9, App. E): the exact kernel up to the start of
 *     Domain S, then the static kernel.
 * eta = 0 and eps_st = 0 give back the plain (dense) ST-BIEM of Eq. 4.
 *
 * Conventions common to every call:
 *   - Status: 0 = FDPH_OK, negative = error (see fdph_status); no exception
 *     crosses the ABI.  fdph_strerror gives a message; fdph_last_error gives the
 *     detail of the last failure in this thread.
 *   - Ownership: the caller owns every buffer it passes; the library owns the
 *     plan, its device arena and its time-stepping state.
 *   - Threads / streams: a plan is bound to one CUDA device and one stream and is
 *     not thread safe.  Distinct plans are independent.
 *   - Element order: D and T are indexed in the order of the geometry given to
 *     fdph_plan (the library's internal cluster order is hidden).
 */
#ifndef FDPH_H
#define FDPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fdph_status {
    FDPH_OK = 0,
    FDPH_E_ARG = -1,       /* invalid argument (null pointer, n <= 0, dt <= 0, ...) */
    FDPH_E_OOM = -2,       /* host or device allocation failed */
    FDPH_E_CAUSALITY = -3, /* discretised causality min(dm_i + mbar_j) >= 1 fails (Sec. 5.2, App. D) */
    FDPH_E_CUDA = -4,      /* a CUDA runtime call failed */
    FDPH_E_TIMEOUT = -5,   /* a bounded device wait gave up */
    FDPH_E_NAN = -6,       /* non-finite value found where the call checks for one */
    FDPH_E_STATE = -7,     /* call not valid in the plan's current state (e.g. past M steps) */
    FDPH_E_CHECK = -8      /* bounded-index debug build (libfdph_check.so, compiled with -DFDPH_CHECK)
                              only: a ring, state, partial-sum or near-slice index of a step kernel
                              fell outside its array (the access was skipped and the step's results
                              are invalid), or a write ran past the end of a plan allocation */
} fdph_status;

typedef enum fdph_precision {
    FDPH_FP64 = 0,         /* factors, waveforms and near-field tensor stored and multiplied in FP64 */
    FDPH_FP32 = 1,         /* stored in FP32; near-field products summed in FP32 within one work
                              item (<= 64 steps x 32 sources) and in FP64 across items; far-field
                              sums, rings and accumulators stay FP64 */
    FDPH_FP16 = 2          /* as FDPH_FP32, but the near-field window coefficients (the exact
                              kernel of the inadmissible leaves, the bulk of the bytes) are stored
                              in FP16 and converted to FP32 for the products; the near-field static
                              and tail coefficients stay FP32.  Adds a rounding error of at most
                              2^-11 of each stored coefficient (about 1e-3 relative on the test
                              faults); BF16 (2^-8) was measured at 6e-3 to 9e-3 and is not offered */
} fdph_precision;

typedef struct fdph_plan_s* fdph_plan_t;
typedef struct fdph_batch_s* fdph_batch_t;   /* opaque set of plans stepped together */

/* Fault geometry: n straight elements, host memory, xy[4*e + (0,1,2,3)] = (x0, y0, x1, y1)
 * of element e.  Collocation point = midpoint; normal = tangent rotated by +90 degrees
 * (Sec. 2.1.2).  Read during fdph_plan only. */
typedef struct fdph_geometry {
    int32_t n;
    const double* xy;
} fdph_geometry;

/* Homogeneous full space: shear modulus mu and S-wave speed cs (Sec. 2.1.1). */
typedef struct fdph_material {
    double mu;
    double cs;
} fdph_material;

/* Plan parameters (Sec. 6 / Sec. 7.1 names).  Fill with fdph_default_params first. */
typedef struct fdph_params {
    double eta;           /* admissibility diam < eta * dist (Eq. 8); 0 => no admissible leaf */
    double lmin;          /* inadmissibility diam < l_min (Eq. 9); default 0 */
    double eps_st;        /* Domain-S start: absolute kernel error bound, in units of mu/(2 cs)
                             (App. H); 0 => the exact kernel is kept for all M steps */
    int32_t leaf_size;    /* a block whose two clusters have at most leaf_size elements is an
                             inadmissible leaf (default 32) */
    int32_t extra_steps;  /* additional Domain-F width n_c in steps (App. H); < 0 => default
                             ceil(10 * max element length / (cs dt)) */
    int32_t precision;    /* fdph_precision, default FDPH_FP64 */
    int32_t device;       /* CUDA device ordinal, default 0 */
    int32_t soe_terms;    /* 0 (default): the paper's Domain-S cut -- beyond eps_st the kernel is
                             the static kernel alone.  Q in [4, 16]: extension of this library --
                             beyond the exact window, the remainder K - Kstat dt of each
                             inadmissible pair and of each transient fibre is kept as its
                             least-squares fit on Q decaying exponentials, evaluated by Q
                             recursive filter states per source; inadmissible windows then also
                             cover each pair's wave passage (+ extra_steps) */
    int32_t art_interp;   /* 0 (default): receiver delays rounded down to whole steps (Eq. 30).
                             1: extension -- the representative stress is read at the exact
                             delay dm_i + phi_i by linear interpolation between steps n - dm_i and
                             n - dm_i - 1 (the higher-order interpolation Sec. 4.3.1 mentions) */
    void* cuda_stream;    /* cudaStream_t the plan runs on; NULL => a stream the plan creates */
    int32_t host_threads; /* host threads of the plan build (OpenMP); 0 (default) => the OpenMP
                             default.  Callers that build several plans at once (a serving loop
                             with planner threads) give each a share of the cores */
    int32_t eta_scheme;   /* admissibility: 0 (default) the constant eta scheme, diam < eta dist
                             (Eq. 8); 1 the constant eta^2 dist scheme of Eq. 25, diam <
                             sqrt(eta lmin dist) (eta = eta_0, lmin > 0 required), which bounds the
                             travel-time error of the plane-wave approximation by eta lmin / (4 c)
                             (Eq. 26) at a cost that grows like N^(3/2) */
    int32_t nrhs;         /* right-hand sides: independent slip-rate histories stepped together on
                             the one operator (1, 2, 4 or 8; 0 => 1).  D_n and T_n of fdph_step,
                             fdph_run, fdph_step_host and fdph_run_host are then nrhs rows of n
                             (RHS-major: row r, element i at r * n + i) per step, and the state is
                             kept per RHS; each near-field coefficient is read once per step and
                             multiplied with the slip rates of all RHS (near-field work items
                             are nrhs times shorter).  Rupture, fdph_predict / fdph_commit and
                             batches take nrhs = 1 (FDPH_E_ARG otherwise) */
    int32_t far_mode;     /* Eq. 42 of the admissible blocks: 0 (default) scatter -- each step adds
                             g_{l,j} u_j into the delay-ring slots n + delay_j; 1 the delayed-history
                             gather of Sec. 5.3 -- each step records u_j(n) in a history of the last
                             maxdelay - mindelay + 1 steps per block and computes the one slot it
                             completes, Tbar'_l[n + mindelay] = sum_j g_{l,j} u_j(n + mindelay -
                             delay_j).  Same arithmetic (up to summation order) with more memory
                             (the histories); batches take far_mode 0 */
    int32_t amp_window;   /* time window of the Domain-F amplitude Khat^F_ij (Eq. 12 / Eq. 28):
                             0 (default) the pair's discrete window as the operator places it,
                             steps [dm_i + mbar_j, dm_i + mbar_j + Dm_j), so that amplitude, waveform
                             and the following static part add up to the exact kernel's impulse;
                             1 Eq. 28 as written, the pair's own continuous Domain F
                             (t^-_ij, t^+_ij) = mbar_j dt + (r_ij - r_{i* j}) / c + (0, Dm_j dt),
                             the window of the representative receiver i* (App. C.3) moved by the
                             pair's travel-time difference: smooth in i and j, hence low rank on
                             curved faults, at the price of an O(dt Kstat) mismatch at the start
                             of Domain S */
    double eps_q;         /* 0 (default): the Domain-S transient (App. B.3) keeps its Dm_tr exact taps.
                             > 0: those taps are quantized (App. A, applied to the transient as App. B.3
                             and App. A.3 do): a staircase of constant values over ranges [b_q, b_q+1)
                             grown while |h_m - h_b_q| / 2 <= eps_q |(h_b_q + h_m) / 2|, each value the
                             mean of its range's end taps, evaluated every step by running window sums
                             Yhat_q(n) = Yhat_q(n - 1) + Y(n - b_q) - Y(n - b_q+1) (Eq. A.4) */
    int64_t aca_min;      /* how the admissible blocks are factorised (Sec. 4, Sec. 6.2).  0 (default):
                             every block formed densely and factorised by pivoted QR + SVD, the
                             truncated SVD of minimal rank (the definition the LRA approximates).
                             > 0: a block of at least aca_min entries by adaptive cross approximation
                             with partial pivoting and reference row / column (ACA+, the H-matrix
                             construction Sec. 4 names) from rows and columns computed on demand,
                             recompressed to the rank eps needs: O(rank (N_r + N_s)) kernel
                             evaluations per block instead of N_r N_s, for plans too large to form
                             every block (N >= ~32768); a block whose cross approximation does not
                             converge is formed densely.  The transient's spatial pivot (App. H) on
                             such a block is the largest entry of alternating row / column searches.
                             Each block then meets |K - F G^T|_F < eps |K|_F up to the cross
                             approximation's own error (estimated at 1e-3 eps), but its factors are
                             not the truncated SVD's.  4096 is a good value */
} fdph_params;

/* Per-plan statistics (host copy). Bytes are algorithmic: what one step must move. */
typedef struct fdph_stats {
    int32_t n;                 /* elements */
    int32_t M;                 /* planned steps */
    int32_t n_admissible;      /* admissible leaves */
    int32_t n_near;            /* inadmissible leaves */
    int32_t n_subblocks;       /* low-rank operators (leaf x domain x stress component) */
    int32_t max_rank;
    int32_t extra_steps;       /* n_c used */
    int32_t max_window;        /* largest inadmissible-leaf window (steps of exact kernel) */
    double mean_rank;
    int64_t near_entries;      /* stored kernel coefficients of the inadmissible leaves */
    int64_t far_entries;       /* stored factor / waveform coefficients */
    int64_t arena_bytes;       /* device bytes of the plan (operator data) */
    int64_t state_bytes;       /* device bytes of the time-stepping state (rings, accumulators) */
    double bytes_per_step;     /* algorithmic HBM bytes of one full step at steady state */
    double near_bytes_per_step;/* of which the near-field kernel: coefficients, slip-rate window rows, tail states */
    double flops_per_step;     /* multiply-adds x 2 of one full step */
    double plan_seconds;       /* wall time of fdph_plan */
    int32_t n_exact;           /* low-rank operators kept exact (Sec. 6.2 fallback) */
    int32_t n_aca;             /* low-rank operators factorised by cross approximation (aca_min) */
    double mean_rank_f;        /* Domain-F amplitude ranks, weighted by the blocks' entries (the
                                  paper's "mean rank", Sec. 6.4.1); exact blocks count at full rank */
    double mean_rank_s;        /* the same for the Domain-S static blocks */
    double mean_rank_tr;       /* the same for the 2-D Domain-S transient blocks */
} fdph_stats;

/* Fill *p with the defaults above. Never fails. */
void fdph_default_params(fdph_params* p);

/* Build the plan of the FDP=H operator for `geometry` (Secs. 2.3, 4, App. C.3, App. E, App. H)
 * and upload it to the device.  dt: time step; M: number of steps the plan will be run
 * for (kernel windows and Domain-S cuts are evaluated up to M); eps: low-rank tolerance
 * eps_H of the Frobenius criterion |K_a - K_a,LRA| < eps |K_a| (Sec. 2.3), eps <= 0 keeps
 * every admissible block exact.  params may be NULL (defaults).  On success *out is a new
 * plan positioned at step 0.  Errors: FDPH_E_ARG, FDPH_E_OOM, FDPH_E_CAUSALITY, FDPH_E_CUDA. */
int fdph_plan(const fdph_geometry* geometry, const fdph_material* material, double dt, int32_t M,
              double eps, const fdph_params* params, fdph_plan_t* out);

/* One time step of Eq. 4: consumes D_n (device, n doubles) and writes T_n (device, n doubles),
 * n being the plan's current step, then advances to n + 1.  Asynchronous on the plan's stream;
 * D_n may be reused once the stream has passed this call.  Errors: FDPH_E_ARG (null plan or
 * pointer), FDPH_E_STATE (n == M), FDPH_E_CUDA (launch failure). */
int fdph_step(fdph_plan_t plan, const double* D_n, double* T_n);

/* `steps` consecutive steps: D (device, steps * n doubles, step-major) -> T (device, same shape).
 * Equivalent to `steps` calls of fdph_step; from 8 steps on (and with profiling off) the call
 * replays a CUDA graph of one step, which removes the per-kernel launch cost; the graph is kept
 * with the plan (at most 8 per plan) and reused by later calls on the same D, T buffers.
 * Errors as fdph_step; FDPH_E_STATE if the plan would pass step M. */
int fdph_run(fdph_plan_t plan, int32_t steps, const double* D, double* T);

/* Dynamic rupture (Sec. 6.2): the slip rate is not prescribed but follows from a friction law
 * at every element.  The unruptured element keeps zero slip rate; it ruptures when the shear
 * traction reaches its strength, then the traction equals the strength, with slip weakening of
 * the accumulated slip u, linear (law 0) or the paper's exponential form (law 1):
 *     law 0: strength(u) = sigma_n * (mu_s - (mu_s - mu_d) * min(u / Dc, 1))
 *     law 1: strength(u) = sigma_n * (mu_d + (mu_s - mu_d) * exp(-u / Dc))
 * (Sec. 6.2 writes law 1 with T_th = sigma_n mu_s and T_dy = sigma_n mu_d).
 * The instantaneous term of Eq. 4 is local (K_{ij,0} = 0 for j != i when cs dt <= dx/2,
 * K_{ii,0} = -mu/(2 cs) the radiation damping), so each step is: predict the traction with
 * D_n = 0, solve D_n >= 0 element by element (explicit strength at the slip of the previous
 * step), then commit D_n to the history. */
typedef struct fdph_friction {
    const double* tau0;   /* device, n doubles (geometry order): background shear traction */
    double sigma_n;       /* normal stress (compression positive) */
    double mu_s, mu_d;    /* static and dynamic friction coefficients */
    double Dc;            /* slip-weakening distance */
    int32_t law;          /* 0: linear slip weakening, 1: exponential slip weakening */
} fdph_friction;

/* Attach a friction law to a plan (copies tau0; zero slip).  Errors: FDPH_E_ARG, FDPH_E_OOM,
 * FDPH_E_CUDA, FDPH_E_STATE (instantaneous term not local: cs dt > min element length / 2). */
int fdph_rupture_init(fdph_plan_t plan, const fdph_friction* friction);

/* One rupture step: writes the solved slip rate D_n and the total shear traction
 * tau0 + T_n (both device, n doubles, geometry order) and advances to n + 1. */
int fdph_rupture_step(fdph_plan_t plan, double* D_n, double* T_n);

/* `steps` rupture steps into D, T (device, steps * n doubles, step-major).  From 8 steps on
 * (profiling off) one rupture step is captured as a CUDA graph and replayed; the graph is kept
 * with the plan for later calls on the same D, T buffers. */
int fdph_rupture_run(fdph_plan_t plan, int32_t steps, double* D, double* T);

/* Copy the accumulated slip (device, n doubles, geometry order). */
int fdph_rupture_slip(fdph_plan_t plan, double* slip);

/* One step of Eq. 4 split in two for a caller's own local solve (any friction law or boundary
 * condition, Sec. 6.2 / Sec. 2.1), the way the rupture step splits internally:
 *   fdph_predict writes T_pred = sum_{m >= 1} K_m D_{n-m} (device, n doubles, geometry order),
 *     the traction of the current step n with D_n = 0;
 *   the caller computes D_n (with T_n = T_pred + K_0 D_n; K_0 is diagonal when cs dt <= half the
 *     shortest element, its diagonal given by fdph_self);
 *   fdph_commit(D_n) (device, n doubles) appends D_n to the history and advances to n + 1.
 * fdph_predict advances the transient and exponential-tail states of step n, so each step takes
 * exactly one predict and one commit; between the two every other stepping or state call
 * returns FDPH_E_STATE (fdph_reset discards the pending step).  Both are asynchronous on the
 * plan's stream.  Errors: FDPH_E_ARG (null plan or pointer), FDPH_E_STATE (n == M, a predict
 * already pending, a commit with none pending), FDPH_E_CUDA. */
int fdph_predict(fdph_plan_t plan, double* T_pred);
int fdph_commit(fdph_plan_t plan, const double* D_n);

/* Batches (no counterpart in the paper; the serving pattern of independent scenarios): plans
 * that share the device and the precision, stepped together.  Every kernel of a batch step is
 * ONE launch over the work of all plans: push, FIR and scatter (Eqs. 32, 42), transient and
 * Eq. 39 over the concatenated elements and warp tasks, and the persistent near-field kernel
 * (App. E) over the work items of all plans, dealt largest first over the SMs; the step is
 * captured once per (kind, buffers) as a CUDA graph and replayed.  Each plan keeps its own state
 * and step index, and its results are bit-identical to stepping it alone.
 *
 * fdph_batch_create: `plans` (count >= 1, distinct, host array, copied) must outlive the batch.
 *   Errors: FDPH_E_ARG (null, duplicate, mixed device or precision), FDPH_E_STATE (a predict
 *   pending), FDPH_E_CUDA.  fdph_autotune on a member plan invalidates the batch (later batch
 *   calls return FDPH_E_STATE; create it again).
 * fdph_batch_run: `steps` steps of every plan; D[p], T[p] (host arrays of device pointers):
 *   plan p's rows, steps * n_p doubles, step-major, as fdph_run.  Asynchronous; every plan's
 *   stream is ordered after the batch's work.  Errors as fdph_run for any plan.
 * fdph_batch_rupture_run: the same for rupture steps (fdph_rupture_init on every plan) with the
 *   outputs of fdph_rupture_run.
 * fdph_batch_synchronize: wait for the batch and its plans; reports a near-field wait that gave
 *   up (FDPH_E_TIMEOUT).  fdph_batch_destroy: release the batch (not its plans); NULL ignored. */
int fdph_batch_create(const fdph_plan_t* plans, int32_t count, fdph_batch_t* out);
int fdph_batch_run(fdph_batch_t batch, int32_t steps, const double* const* D, double* const* T);
int fdph_batch_rupture_run(fdph_batch_t batch, int32_t steps, double* const* D, double* const* T);
int fdph_batch_synchronize(fdph_batch_t batch);
void fdph_batch_destroy(fdph_batch_t batch);

/* Instantaneous self coefficients K_{ii,0} (Eq. 4 with m = 0; -mu/(2 cs) on a straight fault at
 * cs dt = dx/2, the radiation damping) into diag (HOST, n doubles, geometry order).
 * FDPH_E_STATE when cs dt exceeds half the shortest element (K_0 is then not diagonal). */
int fdph_self(fdph_plan_t plan, double* diag);

/* Like fdph_step but D_n and T_n are HOST buffers; the call copies D_n in, steps, copies T_n
 * out and returns when T_n is ready (synchronous). */
int fdph_step_host(fdph_plan_t plan, const double* D_n_host, double* T_n_host);

/* `steps` consecutive steps with HOST buffers: D_host (steps * n doubles, step-major) ->
 * T_host (same shape).  Every step's D_n is copied to the device and its T_n back to the host
 * (page-locked buffers let the copies run asynchronously); the copies of later and earlier steps
 * overlap the step in progress through a ring of device staging slots, and the steps replay
 * one captured step graph.  Returns when T_host is complete.  Errors as fdph_run. */
int fdph_run_host(fdph_plan_t plan, int32_t steps, const double* D_host, double* T_host);

/* Self-test of the device-side timeout path (no counterpart in the paper): every wait of the
 * library's pipelines polls an mbarrier a bounded number of times and, if it gives up, records
 * the fact and lets the kernel finish, after which the host call returns FDPH_E_TIMEOUT and the
 * CUDA context stays usable.  This call runs one such wait, with `polls` in [1, 2^24], on a
 * barrier that nothing completes, on `device`.  Returns FDPH_E_TIMEOUT when the path works,
 * FDPH_E_ARG for an out-of-range `polls`, FDPH_E_CUDA on a CUDA error. */
int fdph_selftest_wait_timeout(int32_t device, int64_t polls);

/* Autotuner of the near-field work items (no counterpart in the paper): times `steps` replayed
 * steps (1..1024; plan's M >= steps + 2) at a steady-state step index for work items of 64, 32
 * and 16 kernel steps (divided by nrhs unless the tensor cores take them), keeps the fastest and
 * writes it to *chunk (may be NULL); then times the other form of the Eq. 32 FIR (source-major,
 * the default where the F blocks hold each source ~100 times or more, or sub-block-major; both
 * give the same bits) and keeps the faster.  The plan's state and step index are saved and
 * restored, so results continue as before (summation order within the near field may change:
 * rounding-level differences).  Cached step graphs are dropped.
 * Errors: FDPH_E_ARG, FDPH_E_STATE (profiling on), FDPH_E_OOM, FDPH_E_CUDA. */
int fdph_autotune(fdph_plan_t plan, int32_t steps, int32_t* chunk);

/* Return the plan to step 0 with zero history (rings, accumulators). */
int fdph_reset(fdph_plan_t plan);

/* Current step index (number of steps taken since plan or reset). */
int fdph_current_step(fdph_plan_t plan, int32_t* n);

/* The cudaStream_t the plan runs on (params.cuda_stream, or the non-blocking stream the plan
 * created when that was NULL; it lives as long as the plan).  Callers that order their own work
 * with a plan's steps, or build plans on several threads at once, should use this stream rather
 * than one shared with other work: a stream being captured into a step graph takes in whatever
 * any thread submits to it.  Errors: FDPH_E_ARG (null pointer). */
int fdph_plan_stream(fdph_plan_t plan, void** stream);

/* Wait for all work queued on the plan's stream. */
int fdph_synchronize(fdph_plan_t plan);

/* Copy the plan's statistics. */
int fdph_get_stats(fdph_plan_t plan, fdph_stats* stats);

/* Save / restore the time-stepping state (rings, accumulators, histories, step index; with a
 * friction law attached, the accumulated slip too) to / from a host buffer.  fdph_save_state with buf == NULL sets *len to the size needed.  Restoring into a
 * plan built from the same inputs reproduces the continuation bit for bit. */
int fdph_save_state(fdph_plan_t plan, void* buf, size_t* len);
int fdph_load_state(fdph_plan_t plan, const void* buf, size_t len);

/* Release the plan and its device memory.  NULL is ignored. */
void fdph_destroy(fdph_plan_t plan);

/* Per-kernel timing with CUDA events on the plan's stream (off by default).  Kernel ids:
 * 0 push, 1 fir (Eq. 32), 2 scatter (Eq. 42), 3 transient convolution (App. B.3),
 * 4 near field (App. E), 5 gather (Eq. 39).  fdph_kernel_times synchronises the stream and
 * returns, per id, the summed milliseconds and the launch count since profiling was enabled
 * (arrays of length FDPH_NUM_KERNELS).  Enabling resets the counters. */
#define FDPH_NUM_KERNELS 6
int fdph_set_profiling(fdph_plan_t plan, int enable);
int fdph_kernel_times(fdph_plan_t plan, double* ms, int64_t* launches);

/* Host-only inspection of the block-cluster tree and ART integers (Secs. 2.3, 4.2.2, 4.3,
 * App. C.3), no device needed.  Writes an int32 stream to buf (capacity cap entries; *len
 * receives the length needed, call with buf == NULL to size it):
 *   N, perm[N]                      (perm[p] = geometry index of internal position p)
 *   n_leaves, then per leaf:
 *     kind (1 admissible, 0 inadmissible), r0, nr, s0, ns   (internal positions)
 *     if admissible: dm[nr], mbar[ns], Dm[ns]
 * Errors: FDPH_E_ARG; FDPH_E_CAUSALITY if an admissible leaf violates causality. */
int fdph_tree_export(const fdph_geometry* geometry, const fdph_material* material, double dt,
                     const fdph_params* params, int32_t* buf, int64_t cap, int64_t* len);

/* Host-only inspection of the plan's low-rank approximation of one block (Sec. 2.3, Eq. 13),
 * no device needed: A (m x n, row-major) ~ F G^T with the smallest rank meeting
 * |A - F G^T|_F < eps |A|_F (the truncated SVD), or the block kept exact when that rank would
 * store at least m n numbers (Sec. 6.2 fallback: F = I, G = A^T when m <= n, else F = A, G = I).
 * F (m x rank) and G (n x rank) are written row-major into buffers of m * min(m, n) and
 * n * min(m, n) doubles; *rank and *exact (0 / 1) receive the result.  eps <= 0 keeps the block
 * exact.  Errors: FDPH_E_ARG (null pointer, m or n < 1), FDPH_E_NAN (non-finite entry). */
int fdph_low_rank(const double* A, int32_t m, int32_t n, double eps, double* F, double* G, int32_t* rank,
                  int32_t* exact);

/* Host-only inspection of the cross approximation the plan takes for large admissible blocks
 * (fdph_params.aca_min; Sec. 4 names ACA as the H-matrix construction): A (m x n, row-major) is read
 * one row or column at a time, as the plan evaluates the kernel on demand.  ACA with partial
 * pivoting and reference row / column (ACA+) runs to a relative update size of 1e-3 eps, then the
 * cross is recompressed (QR of both factors, truncated SVD of the small core) to the smallest rank
 * with |A_aca - F G^T|_F < eps |A_aca|_F.  *converged = 0 when the cross did not converge (more than
 * min(m, n, 96) crosses, or a reference row / column still large at the end): the plan then factorises
 * the dense block, and F, G are not written.  F and G are written row-major into buffers of
 * m * min(m, n, 96) and n * min(m, n, 96) doubles; *evaluated receives the number of entries read.
 * Errors: FDPH_E_ARG (null pointer, m or n < 1, eps <= 0), FDPH_E_NAN (non-finite entry). */
int fdph_low_rank_aca(const double* A, int32_t m, int32_t n, double eps, double* F, double* G, int32_t* rank,
                      int32_t* converged, int64_t* evaluated);

/* Host-only inspection of the quantization rule (App. A.1.1) the plan applies to the transient's
 * taps when eps_q > 0, no device needed: partitions of K (n values) into q ranges [b[r], b[r+1])
 * with b[0] = 0, b[q] = n, grown while |K_m - K_b| / 2 <= eps_q |(K_b + K_m) / 2|, and the range
 * values khat[r] = (K_b[r] + K_b[r+1]-1) / 2.  b: n + 1 entries of room, khat: n; *q receives the
 * count.  Errors: FDPH_E_ARG (null pointer, n < 1, eps_q <= 0), FDPH_E_NAN (non-finite value). */
int fdph_quantize(const double* K, int32_t n, double eps_q, int32_t* b, double* khat, int32_t* q);

/* Host-only evaluation of the discrete kernel's Domain-S remainder (App. B.3, App. H) for one
 * receiver point p = (x, y) and source element seg = (x0, y0, tx, ty, length) (first end point, unit
 * tangent, length): out[0], out[1] = the global stress components of K(t1, t1 + dt) - Kstat dt,
 * the ramp-response jump over [t1, t1 + dt] less the static stress per unit slip times dt;
 * out[2] = the bound the plan's threshold scans use (m_S of App. H for the near pairs, the
 * transient's taps), an upper bound on |out[0]|, |out[1]| and on any unit projection of them once
 * both end points' S fronts have passed (+inf before), falling with t1.  No device needed.
 * Errors: FDPH_E_ARG (null pointer, dt, mu, cs or length <= 0, t1 < 0). */
int fdph_kernel_tail(const double* p, const double* seg, double t1, double dt, double mu, double cs, double* out);

/* Allocation-free plain step.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory (code running inside another runtime's memory pool or
 * allocator budget, or where a cudaMalloc would synchronise the device at a bad moment).
 *
 * Computes one step of Eq. 4 from buffers the caller owns:
 *     T[i] = sum_{k=0}^{min(step, W-1)} sum_j K[(k * n + j) * n + i] * D_hist[((step - k) mod hist_len) * n + j]
 * K: device, W * n * n doubles (kernel step k, source j, receiver i); D_hist: device ring of
 * hist_len >= min(step + 1, W) slip-rate rows of n doubles, row s mod hist_len holding step s;
 * T: device, n doubles (written); stream: cudaStream_t or NULL.  Asynchronous on the stream.
 *
 * Its split-k partial sums live in one file-scope device array of FDPH_NOALLOC_MAX_PARTIALS
 * doubles (512 KiB), held by every GPU that loads the library until the process exits; the
 * call allocates nothing.  Sizes with ceil(n / 32) * ceil(min(step + 1, W) / 64) * 32 above
 * that maximum are rejected with FDPH_E_ARG (message in fdph_last_error).  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share the array, which
 * keeps the last call's contents (each call overwrites every slot it reads): calls that overlap
 * on the GPU race and must be ordered by the caller (one stream, or events).
 * Errors: FDPH_E_ARG, FDPH_E_CUDA. */
#define FDPH_NOALLOC_MAX_PARTIALS 65536
int fdph_plain_step_noalloc(const double* K, int32_t n, int32_t W, const double* D_hist, int32_t hist_len,
                            int32_t step, double* T, void* stream);

/* Message for a status code (static string). */
const char* fdph_strerror(int status);

/* Detail of the last error raised in the calling thread (static thread-local string). */
const char* fdph_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FDPH_H */
