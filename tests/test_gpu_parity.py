"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances (relative L2 over all receivers and steps):
* FP64 path: 1e-10 against the oracle (plain march and compressed operator alike).  The two
  sides differ only by rounding order of O(1e5) products per output and by the two
  independent SVDs of each block (agreeing to ~1e-14 of the block norm).
* FP32 storage: 5e-6 (FP32 rounding 6e-8 per coefficient, summed over <= 2048 products in
  FP32 per near-field work item, then FP64).
"""
import numpy as np
import pytest

from oracle import dense
from oracle import fdph as ofd
from oracle import kernel as kn
from paper_1903_02118_gb300 import fdph, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL64 = 1e-10
TOL32 = 5e-6


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build
    build.build()


def _run(plan, D):
    Dd = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Td = torch.empty_like(Dd)
    plan.run(D.shape[0], Dd, Td)
    plan.synchronize()
    return Td.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _geom(name, N):
    return {"straight": inputs.straight_fault(N), "curved": inputs.curved_fault(N, inputs.seed_for(1, 0)),
            "kinked": inputs.kinked_fault(N)}[name]


@pytest.mark.parametrize("geom,N,M", [("straight", 256, 256), ("kinked", 203, 150)])
def test_plain_st_biem_fp64(geom, N, M):
    """The plain straight-fault workload (N = 256, M = 256, CFL 1/2, Gaussian-filtered slip rate)
    and a ragged kinked case."""
    _need_gpu()
    xy = _geom(geom, N)
    D = inputs.gaussian_filtered_history(N, M, inputs.seed_for(0, inputs.SLIP))
    plan = fdph.Plan(xy, 0.5, M, 0.0, eta=0.0, eps_st=0.0, leaf_size=32)
    T = _run(plan, D)
    el = kn.element_table(xy)
    K = kn.discrete_kernel(el, 0.5, M, 1.0, 1.0)
    T0 = dense.march(K, D)
    assert _rel(T, T0) < TOL64
    st = plan.stats()
    assert st["n_admissible"] == 0 and st["max_window"] == M


def _oracle_fdph(xy, M, eps, leaf, D, eps_st=1e-6, soe_terms=0, eta=0.5, art_interp=False, eta_scheme=0, lmin=0.0,
                 amp_window=0):
    el = kn.element_table(xy)
    p = ofd.Params(eta=eta, leaf=leaf, eps=eps, eps_st=eps_st, M=M, soe_terms=soe_terms, art_interp=art_interp,
                   eta_scheme=eta_scheme, lmin=lmin, amp_window=amp_window)
    plan = ofd.build_plan(el, p)
    Kc = ofd.operator_rows(el, plan, np.arange(xy.shape[0]))
    return dense.march(Kc, D), plan


@pytest.mark.parametrize("geom,N,leaf,amp", [("straight", 256, 16, 0), ("curved", 256, 16, 0), ("kinked", 233, 13, 0),
                                             ("curved", 256, 16, 1), ("kinked", 233, 13, 1)])
def test_fdph_fp64_equals_compressed_operator(geom, N, leaf, amp):
    """amp = 1: the Domain-F amplitude over the pair's own window of Eq. 28 (amp_window 1)."""
    _need_gpu()
    M, eps = 320, 1e-5
    xy = _geom(geom, N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    T0, oplan = _oracle_fdph(xy, M, eps, leaf, D, amp_window=amp)
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=1e-6, leaf_size=leaf, amp_window=amp)
    T = _run(plan, D)
    st = plan.stats()
    assert st["n_admissible"] == len(oplan["adm"]) and st["n_near"] == len(oplan["near"])
    assert _rel(T, T0) < TOL64


@pytest.mark.parametrize("geom,N,leaf,eta,interp,amp", [("curved", 160, 16, 0.5, False, 0),
                                                        ("straight", 150, 12, 0.25, False, 0),
                                                        ("curved", 170, 16, 0.5, True, 0),
                                                        ("curved", 160, 16, 0.5, False, 1)])
def test_fdph_exponential_tails_fp64_equals_compressed_operator(geom, N, leaf, eta, interp, amp):
    _need_gpu()
    M, eps = 900, 1e-5      # long enough that the exponential tails are used (fit range >= 512)
    xy = _geom(geom, N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    T0, oplan = _oracle_fdph(xy, M, eps, leaf, D, eps_st=1e-4, soe_terms=16, eta=eta, art_interp=interp,
                             amp_window=amp)
    plan = fdph.Plan(xy, 0.5, M, eps, eta=eta, eps_st=1e-4, leaf_size=leaf, soe_terms=16, art_interp=interp,
                     amp_window=amp)
    T = _run(plan, D)
    assert plan.stats()["max_window"] == max(d["W"] for d in oplan["near"]) < M
    assert _rel(T, T0) < TOL64


@pytest.mark.parametrize("geom,N,M,soe", [("curved", 300, 320, 0), ("kinked", 240, 900, 16)])
def test_fdph_eta2dist_fp64_equals_compressed_operator(geom, N, M, soe):
    """Constant eta^2 dist admissibility (Eq. 25, eta0 = 0.5, lmin = 6): same leaves and same
    compressed operator as the oracle, with and without exponential tails."""
    _need_gpu()
    eps, leaf, lmin = 1e-5, 16, 6.0
    eps_st = 1e-4 if soe else 1e-6
    xy = _geom(geom, N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    T0, oplan = _oracle_fdph(xy, M, eps, leaf, D, eps_st=eps_st, soe_terms=soe, eta_scheme=1, lmin=lmin)
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=eps_st, leaf_size=leaf, soe_terms=soe, eta_scheme=1, lmin=lmin)
    T = _run(plan, D)
    st = plan.stats()
    assert st["n_admissible"] == len(oplan["adm"]) > 0 and st["n_near"] == len(oplan["near"])
    assert _rel(T, T0) < TOL64


def test_fdph_fp32_storage():
    _need_gpu()
    N, M, eps, leaf = 256, 320, 1e-5, 16
    xy = _geom("curved", N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    T0, _ = _oracle_fdph(xy, M, eps, leaf, D)
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=1e-6, leaf_size=leaf, precision=fdph.FP32)
    T = _run(plan, D)
    assert _rel(T, T0) < TOL32


def test_step_run_host_reset_and_state_are_consistent():
    _need_gpu()
    N, M = 150, 120
    xy = _geom("curved", N)
    D = inputs.gaussian_filtered_history(N, M, 3)
    plan = fdph.Plan(xy, 0.5, M, 1e-4, eta=0.5, eps_st=1e-6, leaf_size=8)
    T_run = _run(plan, D)
    plan.reset()
    Dd = torch.from_numpy(D).cuda()
    Td = torch.empty_like(Dd)
    for n in range(60):
        plan.step(Dd[n], Td[n])
    saved = plan.save_state()
    for n in range(60, M):
        plan.step(Dd[n], Td[n])
    plan.synchronize()
    assert np.array_equal(Td.cpu().numpy(), T_run)            # bit for bit
    plan.load_state(saved)
    assert plan.current_step() == 60
    T_host = np.stack([plan.step_host(D[n]) for n in range(60, M)])
    assert np.array_equal(T_host, T_run[60:])
    plan.load_state(saved)
    assert np.array_equal(plan.run_host(D[60:]), T_run[60:])   # pipelined host-buffer steps
    plan.load_state(saved)
    assert np.array_equal(plan.run_host(D[60:65]), T_run[60:65])   # fewer steps than staging slots
    assert np.array_equal(plan.run_host(D[65:]), T_run[65:])
    with pytest.raises(fdph.FdphError):
        plan.step(Dd[0], Td[0])                                 # past M


def test_config2_full_size_sampled_receivers():
    """The curved-fault workload at full size (N = 4096, M = 4096, eps = 1e-4, leaf 32, eta = 1/2), in the
    launch configuration the benchmark times, against the oracle's compressed operator on sampled
    receivers (all steps)."""
    _need_gpu()
    N, M, eps = 4096, 4096, 1e-4
    xy = _geom("curved", N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=1e-6, leaf_size=32)
    T = _run(plan, D)
    rows = np.array([7, 2049])
    el = kn.element_table(xy)
    p = ofd.Params(eta=0.5, leaf=32, eps=eps, eps_st=1e-6, M=M)
    oplan = ofd.build_plan(el, p, receivers=rows)
    Kc = ofd.operator_rows(el, oplan, rows)
    T0 = dense.march_rows_fft(Kc, D)
    assert _rel(T[:, rows], T0) < 1e-9


@pytest.mark.parametrize("mode,law", [("plain", "linear"), ("fdph", "linear"), ("plain", "exponential"),
                                      ("fdph", "exponential")])
def test_rupture_matches_oracle(mode, law):
    """Dynamic rupture (Sec. 6.2, linear or the paper's exponential slip weakening): slip rate and
    traction of every element and step against the oracle's rupture march on the same operator."""
    _need_gpu()
    N, M, dt = 200, 240, 0.5
    xy = _geom("straight", N)
    rng = np.random.default_rng(inputs.seed_for(2, inputs.FRICTION))
    tau0 = 0.45 * (1.0 + 0.05 * rng.standard_normal(N))
    tau0[N // 2 - 8:N // 2 + 8] = 0.61
    el = kn.element_table(xy)
    if mode == "plain":
        Kop = kn.discrete_kernel(el, dt, M, 1.0, 1.0)
        plan = fdph.Plan(xy, dt, M, 0.0, eta=0.0, eps_st=0.0, leaf_size=32)
    else:
        p = ofd.Params(eta=0.5, leaf=16, eps=1e-6, eps_st=1e-4, M=M, soe_terms=16)
        oplan = ofd.build_plan(el, p)
        Kop = ofd.operator_rows(el, oplan, np.arange(N))
        plan = fdph.Plan(xy, dt, M, 1e-6, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16)
    D0, T0 = dense.rupture_march(Kop, tau0, 1.0, 0.6, 0.3, 2.0, dt, M, law=law)
    t0 = torch.from_numpy(tau0).cuda()
    plan.rupture_init(t0, 1.0, 0.6, 0.3, 2.0, law=0 if law == "linear" else 1)
    Dd = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    Td = torch.zeros_like(Dd)
    plan.rupture_run(M, Dd, Td)
    plan.synchronize()
    D, T = Dd.cpu().numpy(), Td.cpu().numpy()
    assert (D0 > 0).sum() > 0.3 * D0.size          # the rupture spreads over the fault
    assert _rel(D, D0) < 1e-9 and _rel(T, T0) < 1e-10


def test_cached_step_graphs_replay_bit_for_bit():
    """fdph_run keeps its step graph per (D, T) buffers: a second run on the same buffers, runs
    split at any step, and chunked runs through one staging buffer give the same T bit for bit."""
    _need_gpu()
    N, M = 150, 96
    xy = _geom("curved", N)
    D = inputs.gaussian_filtered_history(N, M, 5)
    plan = fdph.Plan(xy, 0.5, M, 1e-4, eta=0.5, eps_st=1e-4, leaf_size=8, soe_terms=16)
    Dd = torch.from_numpy(D).cuda()
    Td = torch.empty_like(Dd)
    torch.cuda.synchronize()
    plan.run(M, Dd, Td)
    plan.synchronize()                        # the plan has its own stream
    T1 = Td.cpu().numpy()
    plan.reset()
    plan.run(M, Dd, Td)                       # cached graph
    plan.synchronize()
    assert np.array_equal(Td.cpu().numpy(), T1)
    plan.reset()
    plan.run(40, Dd, Td)
    plan.run(M - 40, Dd[40:], Td[40:])
    plan.synchronize()
    assert np.array_equal(Td.cpu().numpy(), T1)
    plan.reset()
    Dc = torch.empty((16, N), dtype=torch.float64, device="cuda")
    Tc = torch.empty_like(Dc)
    out = np.empty_like(T1)
    for c in range(0, M, 16):
        Dc.copy_(Dd[c:c + 16])
        torch.cuda.synchronize()
        plan.run(16, Dc, Tc)                  # same buffers every call: rows restart at 0
        plan.synchronize()
        out[c:c + 16] = Tc.cpu().numpy()
    assert np.array_equal(out, T1)


def test_rupture_graph_equals_stepwise_rupture():
    """fdph_rupture_run (one replayed step graph, also in chunks through one buffer pair) equals
    fdph_rupture_step called step by step, bit for bit."""
    _need_gpu()
    N, M, dt = 140, 96, 0.5
    xy = _geom("kinked", N)
    tau0 = np.full(N, 0.45)
    tau0[N // 2 - 6:N // 2 + 6] = 0.61
    t0 = torch.from_numpy(tau0).cuda()
    outs = []
    for mode in ("graph", "steps", "chunks"):
        plan = fdph.Plan(xy, dt, M, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16)
        plan.rupture_init(t0, 1.0, 0.6, 0.3, 2.0)
        Dd = torch.zeros((M, N), dtype=torch.float64, device="cuda")
        Td = torch.zeros_like(Dd)
        torch.cuda.synchronize()
        if mode == "graph":
            plan.rupture_run(M, Dd, Td)
        elif mode == "steps":
            for n in range(M):
                plan.rupture_step(Dd[n], Td[n])
        else:
            Dc = torch.zeros((32, N), dtype=torch.float64, device="cuda")
            Tc = torch.zeros_like(Dc)
            torch.cuda.synchronize()
            for c in range(0, M, 32):
                plan.rupture_run(32, Dc, Tc)
                plan.synchronize()                # the plan has its own stream
                Dd[c:c + 32].copy_(Dc)
                Td[c:c + 32].copy_(Tc)
                torch.cuda.synchronize()
        plan.synchronize()
        outs.append((Dd.cpu().numpy(), Td.cpu().numpy()))
        plan.close()
    assert (outs[0][0] > 0).any()
    for D_, T_ in outs[1:]:
        assert np.array_equal(D_, outs[0][0]) and np.array_equal(T_, outs[0][1])


def test_fdph_fp16_near_window_within_rounding_bound():
    """FP16 storage of the near-field window: every output is within the rounding bound of its
    stored coefficients, |dT_i,n| <= 2^-11 sum |K_ijk| |D_j,n-k| + 2^-25 sum |D_j,n-k| over the
    window entries (FP16 unit roundoff; subnormal spacing), plus the FP32 slack of the other
    parts, against the oracle's compressed operator (FP64)."""
    _need_gpu()
    N, M, eps, leaf = 160, 900, 1e-5, 16
    xy = _geom("curved", N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    T0, oplan = _oracle_fdph(xy, M, eps, leaf, D, eps_st=1e-4, soe_terms=16)
    Kabs = np.zeros((M, N, N))
    Kone = np.zeros((M, N, N))
    for d in oplan["near"]:
        I, J, W = d["I"], d["J"], d["W"]
        Kabs[:W][:, I[:, None], J[None, :]] = np.abs(d["K"][:W])
        Kone[:W][:, I[:, None], J[None, :]] = 1.0
    B = dense.march(Kabs, np.abs(D)) * 2.0 ** -11 + dense.march(Kone, np.abs(D)) * 2.0 ** -25
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=1e-4, leaf_size=leaf, soe_terms=16, precision=fdph.FP16)
    T = _run(plan, D)
    slack = 5e-6 * np.abs(T0).max()
    assert np.all(np.abs(T - T0) <= B + slack)
    assert _rel(T, T0) > 1e-7          # the rounding is there (not an FP32 path)


def test_autotune_keeps_state_and_results():
    """fdph_autotune changes only the grouping of the near-field sums: a tuned plan continues from
    its saved state and matches an untuned plan to rounding (FP64).  M is long enough for the
    exponential tails (their states must keep their places when the items are rebuilt)."""
    _need_gpu()
    N, M = 180, 900
    xy = _geom("curved", N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    ref = fdph.Plan(xy, 0.5, M, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16)
    T_ref = _run(ref, D)
    plan = fdph.Plan(xy, 0.5, M, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16)
    Dd = torch.from_numpy(D).cuda()
    Td = torch.empty_like(Dd)
    torch.cuda.synchronize()
    plan.run(50, Dd, Td)
    plan.synchronize()
    assert plan.stats()["max_window"] < M        # tails present
    chunk = plan.autotune(steps=8)
    assert chunk in (16, 32, 64)
    assert plan.current_step() == 50
    plan.run(M - 50, Dd[50:], Td[50:])
    plan.synchronize()
    assert _rel(Td.cpu().numpy(), T_ref) < 1e-13


def test_predict_commit_split_equals_step_and_rupture():
    """fdph_predict + local solve + fdph_commit: with the prescribed slip rate it reproduces
    fdph_run (T_n = T_pred + K_{ii,0} D_n); with a friction law solved by the caller it reproduces
    fdph_rupture_run; K_{ii,0} equals the oracle's instantaneous self term; misuse is refused."""
    _need_gpu()
    N, M, dt = 180, 120, 0.5
    xy = _geom("straight", N)
    el = kn.element_table(xy)
    K0 = kn.discrete_kernel(el, dt, 1, 1.0, 1.0)[0]
    plan = fdph.Plan(xy, dt, M, 1e-6, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16)
    k0 = plan.self_coefficients()
    assert np.abs(k0 - np.diag(K0)).max() < 1e-13
    D = inputs.gaussian_filtered_history(N, M, 11)
    Dd = torch.from_numpy(D).cuda()
    Td = torch.empty_like(Dd)
    plan.run(M, Dd, Td)
    plan.synchronize()
    T_run = Td.cpu().numpy()
    plan.reset()
    k0d = torch.from_numpy(k0).cuda()
    Tp = torch.empty((M, N), dtype=torch.float64, device="cuda")
    for n in range(M):
        plan.predict(Tp[n])
        if n == 3:
            with pytest.raises(fdph.FdphError):
                plan.predict(Tp[n])               # one predict per step
            with pytest.raises(fdph.FdphError):
                plan.step(Dd[n], Td[n])           # the pending step blocks other stepping
        plan.commit(Dd[n])
    with pytest.raises(fdph.FdphError):
        plan.commit(Dd[0])                        # no predict pending
    plan.synchronize()
    T_split = (Tp + k0d[None, :] * Dd).cpu().numpy()
    assert _rel(T_split, T_run) < 1e-13

    # exponential slip weakening solved in the caller's code between predict and commit
    rng = np.random.default_rng(inputs.seed_for(3, inputs.FRICTION))
    tau0 = 0.45 * (1.0 + 0.05 * rng.standard_normal(N))
    tau0[N // 2 - 8:N // 2 + 8] = 0.61
    t0 = torch.from_numpy(tau0).cuda()
    plan.reset()
    plan.rupture_init(t0, 1.0, 0.6, 0.3, 2.0, law=1)
    Dr = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    Tr = torch.zeros_like(Dr)
    plan.rupture_run(M, Dr, Tr)
    plan.synchronize()
    plan.reset()
    slip = torch.zeros(N, dtype=torch.float64, device="cuda")
    Du = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    Tu = torch.zeros_like(Du)
    for n in range(M):
        plan.predict(Tu[n])
        plan.synchronize()
        tau = t0 + Tu[n]
        strength = 0.3 * torch.exp(-slip / 2.0) + 0.3
        v = torch.where(tau > strength, (tau - strength) / (-k0d), torch.zeros_like(tau))
        Du[n] = v
        Tu[n] = tau + k0d * v
        slip += v * dt
        torch.cuda.synchronize()
        plan.commit(Du[n])
    plan.synchronize()
    assert (Dr > 0).sum().item() > 0.2 * Dr.numel()
    assert _rel(Du.cpu().numpy(), Dr.cpu().numpy()) < 1e-10 and _rel(Tu.cpu().numpy(), Tr.cpu().numpy()) < 1e-10


@pytest.mark.parametrize("prec,R", [(fdph.FP64, 4), (fdph.FP32, 8), (fdph.FP16, 2)])
def test_multiple_right_hand_sides_equal_single_rhs_plans(prec, R):
    """nrhs = R slip-rate histories on one operator, read once per step for all of them: every
    RHS matches the single-RHS plan on that history (work items are shorter with R > 1, so the
    summation grouping differs: 1e-13 in FP64, 1e-6 with FP32 products), a permutation of the
    histories permutes the results bit for bit, and graph replay, plain steps, host buffers and a
    saved state agree bit for bit."""
    _need_gpu()
    N, M = 170, 100
    xy = _geom("curved", N)
    kw = dict(eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16, precision=prec)
    Ds = [inputs.gaussian_filtered_history(N, M, 30 + r) for r in range(R)]
    single = fdph.Plan(xy, 0.5, M, 1e-5, **kw)
    ref = []
    for D in Ds:
        single.reset()
        ref.append(_run(single, D))
    ref = np.stack(ref, 1)                                  # (M, R, N)
    plan = fdph.Plan(xy, 0.5, M, 1e-5, nrhs=R, **kw)
    Dm = np.ascontiguousarray(np.stack(Ds, 1))
    Dd = torch.from_numpy(Dm).cuda()
    Td = torch.empty_like(Dd)
    torch.cuda.synchronize()
    plan.run(M, Dd, Td)                                     # graph replay
    plan.synchronize()
    T_graph = Td.cpu().numpy()
    tol = 1e-13 if prec == fdph.FP64 else 1e-6
    for r in range(R):
        assert _rel(T_graph[:, r], ref[:, r]) < tol, r
    perm = np.roll(np.arange(R), 1)
    plan.reset()
    Dp = torch.from_numpy(np.ascontiguousarray(Dm[:, perm])).cuda()
    Tp = torch.empty_like(Dp)
    torch.cuda.synchronize()
    plan.run(M, Dp, Tp)
    plan.synchronize()
    assert np.array_equal(Tp.cpu().numpy(), T_graph[:, perm])
    plan.reset()
    Td.zero_()
    torch.cuda.synchronize()
    for n in range(6):                                      # plain launches
        plan.step(Dd[n], Td[n])
    plan.synchronize()
    buf = plan.save_state()
    plan.run(M - 6, Dd[6:], Td[6:])
    plan.synchronize()
    assert np.array_equal(Td.cpu().numpy(), T_graph)
    plan.load_state(buf)                                    # continue again from step 6
    T2 = plan.run_host(Dm[6:])
    assert np.array_equal(T2, T_graph[6:])
    c = plan.autotune(4)                                    # item lengths of R right-hand sides
    assert c <= (64 if prec == fdph.FP64 else 128) // R
    with pytest.raises(fdph.FdphError):
        plan.predict(Td[0])                                 # single-RHS calls refuse nrhs > 1


@pytest.mark.parametrize("geom,N,M,soe,prec", [("curved", 256, 320, 0, fdph.FP64), ("kinked", 200, 900, 16, fdph.FP64),
                                               ("curved", 180, 300, 16, fdph.FP32)])
def test_delayed_history_gather_equals_scatter(geom, N, M, soe, prec):
    """Eq. 42 in the delayed-history gather form of Sec. 5.3 (far_mode 1) gives the scatter form's
    traction (summation order aside) and, in FP64, the oracle's compressed operator; also with
    rupture steps and after a state save / restore."""
    _need_gpu()
    eps, leaf = 1e-5, 16
    eps_st = 1e-4 if soe else 1e-6
    xy = _geom(geom, N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    kw = dict(eta=0.5, eps_st=eps_st, leaf_size=leaf, soe_terms=soe, precision=prec)
    T = [_run(fdph.Plan(xy, 0.5, M, eps, far_mode=f, **kw), D) for f in (0, 1)]
    assert _rel(T[1], T[0]) < (1e-13 if prec == fdph.FP64 else 1e-6)
    if prec == fdph.FP64 and soe == 0:
        T0, _ = _oracle_fdph(xy, M, eps, leaf, D)
        assert _rel(T[1], T0) < TOL64
    # a restored state continues bit for bit (the histories are part of the state)
    plan = fdph.Plan(xy, 0.5, M, eps, far_mode=1, **kw)
    Dd = torch.from_numpy(D).cuda()
    Td = torch.empty_like(Dd)
    torch.cuda.synchronize()
    plan.run(M // 2, Dd, Td)
    plan.synchronize()
    buf = plan.save_state()
    plan.run(M - M // 2, Dd[M // 2:], Td[M // 2:])
    plan.synchronize()
    T_cont = Td.cpu().numpy()
    plan.load_state(buf)
    plan.run(M - M // 2, Dd[M // 2:], Td[M // 2:])
    plan.synchronize()
    assert np.array_equal(Td.cpu().numpy(), T_cont)
    # rupture steps (predict, friction, commit) through the history form
    rng = np.random.default_rng(inputs.seed_for(7, inputs.FRICTION))
    tau0 = 0.45 * (1.0 + 0.05 * rng.standard_normal(N))
    tau0[N // 2 - 8:N // 2 + 8] = 0.61
    t0 = torch.from_numpy(tau0).cuda()
    out = []
    for f in (0, 1):
        plan = fdph.Plan(xy, 0.5, M, eps, far_mode=f, **kw)
        plan.rupture_init(t0, 1.0, 0.6, 0.3, 2.0)
        Dr = torch.zeros((M, N), dtype=torch.float64, device="cuda")
        Tr = torch.zeros_like(Dr)
        torch.cuda.synchronize()
        plan.rupture_run(M // 2, Dr, Tr)
        plan.synchronize()
        buf = plan.save_state()                # includes the friction law's accumulated slip
        plan.rupture_run(M - M // 2, Dr[M // 2:], Tr[M // 2:])
        plan.synchronize()
        out.append((Dr.cpu().numpy(), Tr.cpu().numpy()))
        plan.load_state(buf)                   # the continuation repeats bit for bit
        Tr.zero_()
        torch.cuda.synchronize()
        plan.rupture_run(M - M // 2, Dr[M // 2:], Tr[M // 2:])
        plan.synchronize()
        assert np.array_equal(Tr[M // 2:].cpu().numpy(), out[-1][1][M // 2:])
    assert (out[0][0] > 0).mean() > 0.1
    tol = 1e-10 if prec == fdph.FP64 else 1e-5
    assert _rel(out[1][0], out[0][0]) < tol and _rel(out[1][1], out[0][1]) < tol


@pytest.mark.parametrize("geom,N,M,soe", [("curved", 200, 320, 0), ("kinked", 190, 900, 16)])
def test_quantized_transient_fp64_equals_compressed_operator(geom, N, M, soe):
    """eps_q > 0: the Domain-S transient's taps as App. A staircases evaluated by running window
    sums on the device; the oracle's compressed operator holds the same staircases (its partition
    rule, oracle/quantization.py), so the FP64 march matches it like the exact taps do."""
    _need_gpu()
    eps, leaf, eps_q = 1e-5, 16, 0.05
    eps_st = 1e-4 if soe else 1e-6
    xy = _geom(geom, N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    el = kn.element_table(xy)
    p = ofd.Params(eta=0.5, leaf=leaf, eps=eps, eps_st=eps_st, M=M, soe_terms=soe, amp_window=1, eps_q=eps_q)
    oplan = ofd.build_plan(el, p)
    # (a component whose remainder vanishes on the whole leaf has no transient, hence no staircase)
    assert any(d["TR"][c].get("qh") is not None and len(d["TR"][c]["qh"]) < d["TR"][c]["Dm"]
               for d in oplan["adm"] for c in "xy")
    T0 = dense.march_rows_fft(ofd.operator_rows(el, oplan, np.arange(N)), D)
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=eps_st, leaf_size=leaf, soe_terms=soe, amp_window=1, eps_q=eps_q)
    T = _run(plan, D)
    assert _rel(T, T0) < TOL64
    plan.reset()                                  # the running sums restart from zero
    assert _rel(_run(plan, D), T0) < TOL64


@pytest.mark.parametrize("geom,N,leaf,amp,soe", [("curved", 256, 16, 1, 0), ("kinked", 233, 13, 0, 16)])
def test_cross_approximation_plan_within_eps_of_compressed_operator(geom, N, leaf, amp, soe):
    """aca_min > 0: the admissible blocks from ACA+ (Sec. 4) instead of the truncated SVD, here every
    block of at least 12 x 12 entries.  Both sides meet |K_b - F G^T|_F < eps |K_b|_F per block, so
    their operators differ by at most 2 eps per block; the transient's spatial pivot may land on
    another pair of similar size, which moves the transient term within its own error (~eps_st).
    The outputs stay within 10 eps of the oracle's compressed operator, while the dense plan meets
    the FP64 bound; the plan statistics show the cross approximation ran (on these low-rank blocks
    the recompressed crosses often reproduce the truncated SVD to rounding)."""
    _need_gpu()
    M, eps = 320, 1e-5
    xy = _geom(geom, N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    T0, _ = _oracle_fdph(xy, M, eps, leaf, D, soe_terms=soe, amp_window=amp)
    kw = dict(eta=0.5, eps_st=1e-6, leaf_size=leaf, amp_window=amp, soe_terms=soe)
    dense = fdph.Plan(xy, 0.5, M, eps, **kw)
    Td = _run(dense, D)
    aca = fdph.Plan(xy, 0.5, M, eps, aca_min=144, **kw)
    T = _run(aca, D)
    assert dense.stats()["n_aca"] == 0 and aca.stats()["n_aca"] > 0
    assert _rel(Td, T0) < TOL64
    assert _rel(T, T0) < 10 * eps


@pytest.mark.parametrize("geom,N,leaf", [("curved", 200, 16), ("kinked", 190, 13)])
def test_bounded_threshold_scans_equal_the_full_scans(geom, N, leaf):
    """eps_st = 1e-4 over M = 900 steps: the near pairs' m_S (App. H) and the transient's taps
    (App. B.3) end well inside M, where the plan's scans stop at the falling tail bound; the
    operator still equals the oracle's, whose scans run over all M steps."""
    _need_gpu()
    M, eps = 900, 1e-5
    xy = _geom(geom, N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    T0, _ = _oracle_fdph(xy, M, eps, leaf, D, eps_st=1e-4)
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=1e-4, leaf_size=leaf)
    T = _run(plan, D)
    assert plan.stats()["max_window"] < M // 2
    assert _rel(T, T0) < TOL64
