"""Continuous-batching serving loop for independent rupture scenarios on one GPU.

Requests (fault geometry, size N, CFL, friction heterogeneity) arrive over time.  A request is
admitted as soon as its device footprint (plan operator + time-stepping state + outputs) fits
the HBM budget and a slot is free; admitted scenarios stay resident and all of them advance
together, each iteration moving every live scenario forward by `chunk` time steps: the
scenarios with a full chunk ahead as one batch (fdph_batch_rupture_run: every kernel of a step
is one launch over all of them), the others (a last, shorter chunk) with their own step graphs
on their own CUDA streams.  A finished scenario releases its memory at once and the next
waiting request takes its place.  Per request the loop records queueing, plan and run times and
the time to solution (arrival to last step on the device).

All arithmetic runs in libfdph (fdph_plan, fdph_rupture_init, fdph_batch_rupture_run,
fdph_rupture_run: captured step graphs replayed per chunk); this module only schedules, and
builds plans on background threads so that planning overlaps the stepping of the live
scenarios.  Plans are independent, so a scenario's result is bit-identical alone and in the mix
(tests/test_gpu_serving.py).
"""
import os
import time

import numpy as np

from . import fdph, inputs


class Request:
    def __init__(self, rid, arrival, N, cfl, seed, M=None, eta=0.5, eps=1e-4, eps_st=1e-4, soe_terms=16,
                 leaf=32, precision=fdph.FP32, geometry="curved", amp_window=1, aca_min=4096):
        self.rid, self.arrival, self.N, self.cfl, self.seed = rid, arrival, N, cfl, seed
        self.amp_window = amp_window   # Domain-F amplitude over each pair's own window (Eq. 28)
        self.aca_min = aca_min         # admissible blocks of >= aca_min entries by cross approximation
        self.M = M if M is not None else int(round(N / cfl))
        self.eta, self.eps, self.eps_st, self.soe_terms = eta, eps, eps_st, soe_terms
        self.leaf, self.precision, self.geometry = leaf, precision, geometry
        # filled by the server
        self.t_admit = self.t_planned = self.t_done = None
        self.plan_stats = None
        self.slip = None
        self.last_D = self.last_T = None

    def inputs(self):
        """Fault trace and prestress for linear slip weakening (0.45 + 5 % Gaussian heterogeneity,
        an overstressed nucleation patch of 64 elements at 0.61; mu_s 0.6, mu_d 0.3, Dc = 6.4);
        drawn once per request."""
        if getattr(self, "_inputs", None) is None:
            self._inputs = self._draw_inputs()
        return self._inputs

    def _draw_inputs(self):
        if self.geometry == "curved":
            xy = inputs.curved_fault(self.N, inputs.seed_for(self.seed, inputs.GEOMETRY))
        else:
            xy = inputs.straight_fault(self.N)
        rng = np.random.default_rng(inputs.seed_for(self.seed, inputs.FRICTION))
        tau0 = 0.45 * (1.0 + 0.05 * rng.standard_normal(self.N))
        c = self.N // 2
        w = min(32, self.N // 8)
        tau0[c - w:c + w] = 0.61
        return xy, tau0


def poisson_requests(count, rate, seed, n_min=512, n_max=16384, cfls=(0.25, 0.5), m_scale=1.0, **kw):
    """`count` requests with Poisson arrivals at `rate` per second, N log-uniform in
    [n_min, n_max], CFL uniform over `cfls`, M = N / CFL scaled by m_scale."""
    rng = np.random.default_rng(inputs.seed_for(seed, inputs.ARRIVALS))
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    out = []
    for k in range(count):
        N = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        cfl = float(rng.choice(cfls))
        M = max(64, int(round(m_scale * N / cfl)))
        out.append(Request(k, float(t[k]), N, cfl, seed * 1000 + k, M=M, **kw))
    return out


class Server:
    """Continuous batching on one GPU.  Plans are built by `planners` background threads (the
    library call releases the interpreter), so live scenarios keep stepping while new requests
    are planned; a request is admitted when a slot is free and the HBM estimate of its plan fits
    the budget (the estimate is replaced by the plan's real footprint once it exists)."""

    def __init__(self, hbm_budget=64 << 30, max_live=16, chunk=64, device=0, time_scale=1.0, planners=1,
                 precision=None, batch=True):
        import torch
        self.torch = torch
        self.budget, self.max_live, self.chunk, self.device = hbm_budget, max_live, chunk, device
        self.time_scale = time_scale
        self.planners = planners
        self.precision = precision
        # batch=True: live scenarios with a full chunk ahead step together, one near-field launch
        # per step for all of them (fdph_batch_rupture_run); otherwise each on its own stream
        self.batch = batch
        self._batch, self._batch_key = None, None
        # each planner builds with its share of the host cores (the builds run at the same time)
        self.host_threads = max(1, (os.cpu_count() or 16) // max(1, planners))
        self.used = 0

    @staticmethod
    def estimate(req):
        """Device footprint of the request's plan before it exists (footprint_model), bytes; computed
        once per request (admission asks again while the request waits for room)."""
        if getattr(req, "_estimate", None) is None:
            xy, _ = req.inputs()
            req._estimate = footprint_model(xy, req.cfl, req.M, eta=req.eta, leaf=req.leaf,
                                            precision=req.precision, soe_terms=req.soe_terms, eps_st=req.eps_st)
        return req._estimate

    def _admit(self, req):
        torch = self.torch
        torch.cuda.set_device(self.device)
        xy, tau0 = req.inputs()
        dt = req.cfl  # dx = cs = 1
        prec = self.precision if self.precision is not None else req.precision
        # each plan on a stream of its own, created by the library: torch's pooled streams repeat,
        # and a plan being built on a planner thread must not submit work to a stream that the
        # loop is capturing into another plan's step graph
        plan = fdph.Plan(xy, dt, req.M, req.eps, eta=req.eta, eps_st=req.eps_st, leaf_size=req.leaf,
                         precision=prec, soe_terms=req.soe_terms, device=self.device,
                         host_threads=self.host_threads, amp_window=req.amp_window, aca_min=req.aca_min)
        stream = torch.cuda.ExternalStream(plan.stream, device=self.device)
        st = plan.stats()
        foot = st["arena_bytes"] + st["state_bytes"] + 3 * req.N * 8 * (self.chunk + 2)
        with torch.cuda.stream(stream):
            t0 = torch.from_numpy(tau0).to(f"cuda:{self.device}")
            D = torch.zeros((self.chunk, req.N), dtype=torch.float64, device=f"cuda:{self.device}")
            T = torch.zeros_like(D)
        plan.rupture_init(t0, 1.0, 0.6, 0.3, 6.4)
        req.plan_stats = st
        return dict(req=req, plan=plan, stream=stream, tau0=t0, D=D, T=T, n=0, foot=foot)

    def _finish(self, s):
        torch = self.torch
        req = s["req"]
        with torch.cuda.stream(s["stream"]):
            slip = torch.empty(req.N, dtype=torch.float64, device=f"cuda:{self.device}")
            s["plan"].rupture_slip(slip)
        s["plan"].synchronize()
        req.slip = slip.cpu().numpy()
        k = (req.M - 1) % self.chunk
        req.last_D = s["D"][k].cpu().numpy()
        req.last_T = s["T"][k].cpu().numpy()
        s["plan"].close()
        self.used -= s["foot"]

    def _drop_batch(self):
        if self._batch is not None:
            self._batch.close()
        self._batch, self._batch_key = None, None

    def _advance(self, live):
        """One chunk for every live scenario; returns the element-steps done."""
        done = 0
        together = []
        if self.batch:
            groups = {}
            for s in live:
                if s["req"].M - s["n"] >= self.chunk:
                    groups.setdefault(s["plan"].precision, []).append(s)
            together = max(groups.values(), key=len) if groups else []
            if len(together) < 2:
                together = []
        if together:
            key = tuple(id(s) for s in together)
            if key != self._batch_key:
                self._drop_batch()
                self._batch = fdph.Batch([s["plan"] for s in together])
                self._batch_key = key
            self._batch.rupture_run(self.chunk, [s["D"] for s in together], [s["T"] for s in together])
            for s in together:
                s["n"] += self.chunk
                done += self.chunk * s["req"].N
        ids = set(id(s) for s in together)
        for s in live:
            if id(s) in ids:
                continue
            req = s["req"]
            k = min(self.chunk, req.M - s["n"])
            s["plan"].rupture_run(k, s["D"], s["T"])
            s["n"] += k
            done += k * req.N
        return done

    def serve(self, requests, realtime=True):
        """Run all requests; returns summary metrics.  With realtime=False arrivals are ignored
        (everything waits at t = 0), which gives the closed-batch throughput."""
        from concurrent.futures import ThreadPoolExecutor
        pending = sorted(requests, key=lambda r: r.arrival)
        live, planning = [], {}
        pool = ThreadPoolExecutor(max_workers=self.planners)
        t0 = time.perf_counter()
        steps_done = 0
        try:
            while pending or live or planning:
                now = (time.perf_counter() - t0) * self.time_scale
                # admission: a free slot, an arrived request and room in the HBM budget
                while (pending and len(live) + len(planning) < self.max_live
                       and (not realtime or pending[0].arrival <= now)):
                    est = self.estimate(pending[0])
                    if (live or planning) and self.used + est > self.budget:
                        break
                    req = pending.pop(0)
                    req.t_admit = time.perf_counter() - t0
                    self.used += est
                    planning[pool.submit(self._admit, req)] = (req, est)
                # plans that are ready join the live set
                for fut in [f for f in planning if f.done()]:
                    req, est = planning.pop(fut)
                    s = fut.result()
                    req.t_planned = time.perf_counter() - t0
                    self.used += s["foot"] - est
                    live.append(s)
                if not live:
                    time.sleep(0.001)
                    continue
                # every live scenario advances by one chunk of steps
                steps_done += self._advance(live)
                still = []
                if any(s["n"] >= s["req"].M for s in live):
                    self._drop_batch()
                for s in live:
                    if s["n"] >= s["req"].M:
                        s["plan"].synchronize()
                        s["req"].t_done = time.perf_counter() - t0
                        self._finish(s)
                    else:
                        still.append(s)
                live = still
        finally:
            self._drop_batch()
            pool.shutdown(wait=True)
        wall = time.perf_counter() - t0
        lat = np.array([r.t_done - (r.arrival / self.time_scale if realtime else 0.0) for r in requests])
        plan_s = np.array([r.t_planned - r.t_admit for r in requests])
        wait_s = np.array([r.t_admit - (r.arrival / self.time_scale if realtime else 0.0) for r in requests])
        return {"element_steps_per_s": steps_done / wall, "wall_s": wall, "requests": len(requests),
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "element_steps": steps_done, "plan_s_p50": float(np.percentile(plan_s, 50)),
                "plan_s_max": float(plan_s.max()), "admission_wait_s_p50": float(np.percentile(wait_s, 50))}


def footprint_model(xy, dt, M, eta=0.5, leaf=32, precision=fdph.FP32, soe_terms=16, rank=8, chunk=64, cs=1.0,
                    eps_st=1e-4):
    """Device bytes of a plan, from its block tree alone (fdph_tree_export, host only, milliseconds):
    the near-field windows dominate -- per inadmissible leaf W slices of ceil(ns / v) v nr stored
    coefficients (v = 16 bytes / element), W = the leaf's longest wave passage (farthest end point
    over c dt) + n_c with exponential tails (the whole march M when too little is left to fit a
    tail), or + the steps the remainder takes to decay to eps_st without them (the paper's cut),
    + the static and tail slices; the admissible blocks add their factors and rings
    (5 low-rank operators per leaf at `rank`, ring slots up to the largest delay); the state adds the
    slip-rate rings, and the serving loop its chunk buffers."""
    tx = fdph.tree_export(xy, dt, eta=eta, leaf_size=leaf, extra_steps=-1)
    perm = tx["perm"]
    N = xy.shape[0]
    ax, ay, bx, by = xy[:, 0], xy[:, 1], xy[:, 2], xy[:, 3]
    mx, my = 0.5 * (ax + bx), 0.5 * (ay + by)
    nc = int(np.ceil(10.0 * np.hypot(bx - ax, by - ay).max() / (cs * dt) - 1e-9))
    sw = {fdph.FP64: 8, fdph.FP32: 4, fdph.FP16: 2}[precision]      # window coefficient bytes
    sa = 8 if precision == fdph.FP64 else 4                           # aux / factor bytes
    near = far = 0.0
    wmax = 1
    for lf in tx["leaves"]:
        I = perm[lf["r0"]:lf["r0"] + lf["nr"]]
        J = perm[lf["s0"]:lf["s0"] + lf["ns"]]
        if lf["kind"] == 0:
            d = np.maximum(np.hypot(mx[I][:, None] - ax[J][None, :], my[I][:, None] - ay[J][None, :]),
                           np.hypot(mx[I][:, None] - bx[J][None, :], my[I][:, None] - by[J][None, :]))
            if soe_terms:
                W = int(np.ceil(d.max() / (cs * dt))) + nc
                if M - W < max(512, 2 * W):
                    W = M
            else:
                # the paper's cut: the exact kernel until its remainder falls below eps_st mu / (2 cs),
                # a remainder of about (dx / (pi cs dt)) / m^2 in those units m steps after the front
                W = min(M, int(np.ceil(d.max() / (cs * dt) + np.sqrt(1.0 / (np.pi * cs * dt * eps_st)))) + 2)
            wmax = max(wmax, W)
            v = 16 // sw
            near += W * (-(-lf["ns"] // v) * v) * lf["nr"] * sw + (1 + soe_terms) * (-(-lf["ns"] // 4) * 4) * lf["nr"] * sa
        else:
            L = int(np.max(lf["mbar"]) + np.max(lf["Dm"]) + np.max(lf["dm"]) - np.min(lf["dm"])) + 2
            far += 5 * rank * ((lf["nr"] + lf["ns"]) * sa + 8 * L) + 4 * (lf["nr"] + 2 * lf["ns"])
    state = (wmax + 1) * N * (8 + 4) + 2 * (wmax + 1) * N * 8 + 16 * N * 8
    return int(near + far + state + 3 * N * 8 * (chunk + 2))


def run_alone(req, chunk=64, device=0, precision=None):
    """The same request served on its own (reference for the mix)."""
    srv = Server(max_live=1, chunk=chunk, device=device, precision=precision)
    srv.serve([req], realtime=False)
    return req
