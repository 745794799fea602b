"""Pins of the oracle's FDP=H plan and compressed operator (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import dense, fdph
from oracle import kernel as kn
from paper_1903_02118_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _setup(geom, N, **kw):
    xy = {"straight": inputs.straight_fault(N), "curved": inputs.curved_fault(N, inputs.seed_for(1, 0)),
          "kinked": inputs.kinked_fault(N)}[geom]
    el = kn.element_table(xy)
    p = fdph.Params(**kw)
    return el, p


@pytest.mark.parametrize("geom", ["straight", "curved", "kinked"])
def test_leaves_partition_the_index_square(geom):
    el, p = _setup(geom, 300, eta=0.5, leaf=16)
    leaves = fdph.block_tree(el, p)
    cover = np.zeros((300, 300), dtype=np.int64)
    for lf in leaves:
        cover[np.ix_(lf["tau"].idx, lf["sig"].idx)] += 1
        if lf["kind"] == "adm":
            assert lf["diam"] < p.eta * lf["dist"]                  # Eq. 8
        else:
            assert lf["tau"].idx.size <= p.leaf and lf["sig"].idx.size <= p.leaf
    assert np.all(cover == 1)


def test_boxes_of_one_level_share_shape():
    el, p = _setup("curved", 500, eta=0.5, leaf=8)
    root = fdph.root_cluster(el)
    level = [root]
    for _ in range(6):
        shapes = {(round(c.hi[0] - c.lo[0], 9), round(c.hi[1] - c.lo[1], 9)) for c in level}
        assert len(shapes) == 1
        level = [k for c in level for k in c.children(el)]


@pytest.mark.parametrize("geom", ["straight", "curved"])
def test_discretised_causality_and_integers(geom):
    el, p = _setup(geom, 400, eta=0.5, leaf=16, M=64)
    plan = fdph.build_plan(el, p)
    assert plan["nc"] == 20                                      # 10 dx / cs at CFL 1/2
    for lf in plan["leaves"]:
        if lf["kind"] != "adm":
            continue
        d = fdph.admissible_leaf(el, lf, p, plan["nc"], need_operator=False)
        assert d["causal"] >= 1                                  # Sec. 5.2
        # App. C.3: the discrete window brackets [r - dx/2, r + dx/2] / (c dt) at i*
        ist = lf["tau"].centre()
        r = np.hypot(el["mx"][d["J"]] - ist[0], el["my"][d["J"]] - ist[1])
        assert np.all(d["mbar"] * p.dt <= (r - 0.5 * el["len"][d["J"]]) / p.cs + 1e-12)
        assert np.all((d["mbar"] + d["Dm"] - plan["nc"]) * p.dt >= (r + 0.5 * el["len"][d["J"]]) / p.cs - 1e-12)


def test_art_is_exact_on_a_straight_line():
    # Sec. 4.2.2: with all sources and receivers on the degenerating ray path the travel time
    # separates exactly, t_ij = dt_i + tbar_j (continuous forms, Eqs. 18-19).
    el, p = _setup("straight", 512, eta=0.5, leaf=16)
    for lf in fdph.block_tree(el, p):
        if lf["kind"] != "adm":
            continue
        ist, jst = lf["tau"].centre(), lf["sig"].centre()
        I, J = lf["tau"].idx, lf["sig"].idx
        r_ij = np.abs(el["mx"][I][:, None] - el["mx"][J][None, :])
        dti = np.abs(el["mx"][I] - jst[0]) - abs(ist[0] - jst[0])
        tbj = np.abs(ist[0] - el["mx"][J])
        assert np.abs(dti[:, None] + tbj[None, :] - r_ij).max() < 1e-9


def test_effective_wave_speed_bound_eq24():
    # Eq. 24 on elements scattered in a square (the D_b = 2 setting of Sec. 6.1).
    rng = np.random.default_rng(5)
    n = 700
    c = rng.uniform(0, 160, (n, 2))
    ang = rng.uniform(0, 2 * np.pi, n)
    xy = np.stack([c[:, 0] - 0.5 * np.cos(ang), c[:, 1] - 0.5 * np.sin(ang),
                   c[:, 0] + 0.5 * np.cos(ang), c[:, 1] + 0.5 * np.sin(ang)], 1)
    el = kn.element_table(xy)
    coef = GOLD["wave_speed_bound_coefficient"]["value"]
    for eta in (0.25, 0.5, 1.0):
        p = fdph.Params(eta=eta, leaf=8)
        x = 1.0 / (1.0 + 1.0 / eta)
        worst = 0.0
        for lf in fdph.block_tree(el, p):
            if lf["kind"] != "adm":
                continue
            ist, jst = lf["tau"].centre(), lf["sig"].centre()
            I, J = lf["tau"].idx, lf["sig"].idx
            rij = np.hypot(el["mx"][I][:, None] - el["mx"][J][None], el["my"][I][:, None] - el["my"][J][None])
            dti = np.hypot(el["mx"][I] - jst[0], el["my"][I] - jst[1]) - lf["rbar"]
            tbj = np.hypot(ist[0] - el["mx"][J], ist[1] - el["my"][J])
            ceff = rij / (dti[:, None] + tbj[None, :])               # Eq. 23, c = 1
            worst = max(worst, np.abs(ceff - 1.0).max())
        assert worst < coef * x * x + x ** 3, (eta, worst)          # Eq. 24 incl. its O(x^3) term
        if eta == 1.0:
            assert worst < GOLD["wave_speed_error_at_eta_1_percent"]["value"] / 100 + x ** 3


@pytest.fixture(scope="module")
def curved_plan():
    el, p = _setup("curved", 256, eta=0.5, leaf=16, eps=1e-5, eps_st=1e-6, M=320)
    plan = fdph.build_plan(el, p)
    return el, p, plan


def test_waveform_normalisation(curved_plan):
    el, p, plan = curved_plan
    for d in plan["adm"]:
        for c in ("x", "y"):
            h = d["F"][c]["h"]
            assert np.allclose(h.sum(axis=1), 1.0, atol=1e-10)      # int h^F = 1 (Eq. 14)


def test_lra_criterion_and_minimal_rank(curved_plan):
    el, p, plan = curved_plan
    n_checked = 0
    for d in plan["adm"][:40]:
        I, J = d["I"], d["J"]
        Ks = kn.static_kernel(el, p.mu, I, J)
        S = d["S"]
        if S["exact"]:
            assert np.abs(S["op"] - Ks).max() == 0.0
            continue
        err = np.linalg.norm(S["op"] - Ks)
        assert err < p.eps * np.linalg.norm(Ks)                      # Sec. 2.3 criterion
        s = np.linalg.svd(Ks, compute_uv=False)
        r = S["rank"]
        assert np.sqrt((s[r - 1:] ** 2).sum()) >= p.eps * np.linalg.norm(Ks)   # r - 1 fails
        n_checked += 1
    assert n_checked > 10


def test_compressed_operator_sum_rules(curved_plan):
    # Amplitude (Eq. 28) and waveform (Eq. 29) sum rule: without truncation the compressed
    # operator integrates, over each pair's discrete Domain-F window, to the exact kernel.
    el, p0, _ = curved_plan
    p = fdph.Params(eta=0.5, leaf=16, eps=1e-15, eps_st=1e-6, M=320)
    plan = fdph.build_plan(el, p, receivers=[5, 130])
    rows = np.array([5, 130])
    Kc = fdph.operator_rows(el, plan, rows)
    K = kn.discrete_kernel(el, p.dt, p.M, p.mu, p.cs, rows)
    checked = 0
    for d in plan["adm"]:
        for il, i in enumerate(d["I"]):
            if i not in rows:
                continue
            r = int(np.nonzero(rows == i)[0][0])
            for jl, j in enumerate(d["J"]):
                a, kS = d["a"][il, jl], d["kS"][il, jl]
                if kS > p.M:
                    continue
                # static and transient parts only start at kS
                assert abs(Kc[a:kS, r, j].sum() - K[a:kS, r, j].sum()) < 1e-12
                assert np.all(Kc[:a, r, j] == 0.0)
                checked += 1
    assert checked > 100


def test_near_field_exact_then_static(curved_plan):
    el, p, plan = curved_plan
    thr = p.eps_st * p.mu / (2 * p.cs)
    for d in plan["near"][:30]:
        K = d["K"]
        tail = K - p.dt * d["Ks"][None]
        for il in range(d["I"].size):
            for jl in range(d["J"].size):
                mS = d["mS"][il, jl]
                assert np.all(np.abs(tail[mS:, il, jl]) < thr)
                if mS > 0:
                    assert abs(tail[mS - 1, il, jl]) >= thr


def test_plain_st_biem_is_the_all_near_special_case():
    # eta = 0 (nothing admissible) and eps_st = 0 (no static cut) give back Eq. 4 exactly.
    el, p = _setup("kinked", 48, eta=0.0, leaf=8, eps_st=0.0, M=60)
    plan = fdph.build_plan(el, p)
    assert not plan["adm"]
    Kc = fdph.operator_rows(el, plan, np.arange(48))
    K = kn.discrete_kernel(el, p.dt, p.M, p.mu, p.cs)
    assert np.abs(Kc - K).max() == 0.0


@pytest.mark.parametrize("geom,bound", [("straight", 2e-3), ("curved", 4e-3)])
def test_fdph_march_close_to_plain_march(geom, bound):
    # Sec. 6.3.2 / Sec. 7.1: FDP=H stays within a few 1e-3 of the original ST-BIEM at eta = 1/2.
    N, M = 256, 384
    el, p = _setup(geom, N, eta=0.5, leaf=16, eps=1e-6, eps_st=1e-6, M=M)
    plan = fdph.build_plan(el, p)
    Kc = fdph.operator_rows(el, plan, np.arange(N))
    K = kn.discrete_kernel(el, p.dt, M, p.mu, p.cs)
    D = inputs.gaussian_pulse(N, M, p.dt, 5)
    T0 = dense.march(K, D)
    T1 = dense.march(Kc, D)
    err = np.linalg.norm(T1 - T0) / np.linalg.norm(T0)
    assert err < bound
    assert err < GOLD["solution_error_eta_half"]["value"]


def test_exponential_tail_reproduces_the_kernel_beyond_the_window():
    # Extension (not the paper's): inadmissible pairs keep the exact kernel up to the leaf window
    # and the fitted exponential tail beyond it.  Pinned against the plain kernel itself.
    N, M = 200, 900
    el, p = _setup("curved", N, eta=0.5, leaf=16, eps=1e-6, eps_st=1e-4, M=M, soe_terms=16)
    plan = fdph.build_plan(el, p, receivers=[3, 100])
    K = None
    for d in plan["near"]:
        Kx = kn.discrete_kernel(el, p.dt, M, p.mu, p.cs, d["I"], d["J"])
        W = d["W"]
        assert W >= 2 * 10                                   # covers the wave passage
        op = np.concatenate([d["K"][:W], d["Ks"][None] * p.dt + d["fit"]], axis=0)
        assert np.abs(op - Kx).max() < 5e-9                  # |K_ijk - operator| for every k < M


def test_exponential_tail_removes_the_static_cut_bias():
    # App. H: cutting at eps_st leaves the slowly decaying remainder K - Kstat dt out; its sum
    # over the rest of the run is the systematic static-approximation error.  With the exponential
    # tails that accumulated error vanishes, and the march is as accurate as keeping every step.
    N, M = 256, 700
    el, _ = _setup("curved", N)
    rows = np.array([5, 128, 200])
    D = inputs.gaussian_pulse(N, M, 0.5, 5)
    K = kn.discrete_kernel(el, 0.5, M, 1.0, 1.0, rows)
    T0 = dense.march_rows_fft(K, D)

    def run(**kw):
        p = fdph.Params(eta=0.5, leaf=16, eps=1e-6, M=M, **kw)
        plan = fdph.build_plan(el, p, receivers=rows)
        Kc = fdph.operator_rows(el, plan, rows)
        near = [(np.nonzero(rows == i)[0][0], j) for d in plan["near"] for i in d["I"] if i in rows for j in d["J"]]
        r, j = np.array(near).T
        acc = np.abs(np.cumsum(Kc[:, r, j] - K[:, r, j], axis=0)).max()   # accumulated step-response error
        T = dense.march_rows_fft(Kc, D)
        return acc, np.linalg.norm(T - T0) / np.linalg.norm(T0)

    acc_cut, _ = run(eps_st=1e-6)
    acc_full, e_full = run(eps_st=0.0)
    acc_soe, e_soe = run(eps_st=1e-4, soe_terms=16)
    assert acc_cut > 1e-5            # the dropped remainder accumulates (App. H bias)
    assert acc_full == 0.0
    assert acc_soe < 1e-8
    assert e_soe < 1.01 * e_full + 1e-9


def _worst_travel_time_error(el, p):
    worst = 0.0
    for lf in fdph.block_tree(el, p):
        if lf["kind"] != "adm":
            continue
        ist, jst = lf["tau"].centre(), lf["sig"].centre()
        I, J = lf["tau"].idx, lf["sig"].idx
        rij = np.hypot(el["mx"][I][:, None] - el["mx"][J][None], el["my"][I][:, None] - el["my"][J][None])
        dti = np.hypot(el["mx"][I] - jst[0], el["my"][I] - jst[1]) - lf["rbar"]
        tbj = np.hypot(ist[0] - el["mx"][J], ist[1] - el["my"][J])
        worst = max(worst, np.abs(dti[:, None] + tbj[None, :] - rij).max() / p.cs)
    return worst


@pytest.mark.parametrize("geom,N", [("curved", 1024), ("kinked", 600), ("square", 700)])
def test_eta2dist_travel_time_bound_eq26(geom, N):
    # Constant eta^2 dist scheme (Eq. 25): the plane-wave travel-time error of every admissible
    # leaf stays under eta0 lmin / (4 c) whatever the distance (Eq. 26), while the constant eta
    # scheme with the same eta0 exceeds it on a bent fault (its error grows with dist, Eq. 17).
    if geom == "square":
        rng = np.random.default_rng(5)
        c = rng.uniform(0, 160, (N, 2))
        ang = rng.uniform(0, 2 * np.pi, N)
        xy = np.stack([c[:, 0] - 0.5 * np.cos(ang), c[:, 1] - 0.5 * np.sin(ang),
                       c[:, 0] + 0.5 * np.cos(ang), c[:, 1] + 0.5 * np.sin(ang)], 1)
        el = kn.element_table(xy)
    else:
        el, _ = _setup(geom, N)
    eta0 = 0.5
    for lmin in (8.0, 16.0):
        p = fdph.Params(eta=eta0, leaf=8 if geom == "square" else 32, eta_scheme=1, lmin=lmin)
        assert _worst_travel_time_error(el, p) < 0.25 * eta0 * lmin / p.cs, (geom, lmin)
        # eta = sqrt(eta0 lmin / dist) is at most eta0 on leaves with diam >= lmin
        for lf in fdph.block_tree(el, p):
            if lf["kind"] == "adm" and lf["diam"] >= lmin:
                assert lf["diam"] < eta0 * lf["dist"]
    if geom != "square":
        p0 = fdph.Params(eta=eta0, leaf=32, lmin=0.0)
        assert _worst_travel_time_error(el, p0) > 0.25 * eta0 * 16.0


def test_eta2dist_needs_lmin():
    el, _ = _setup("straight", 64)
    with pytest.raises(ValueError):
        fdph.block_tree(el, fdph.Params(eta=0.5, eta_scheme=1, lmin=0.0))
