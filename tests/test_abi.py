"""CPU tests of the C-ABI library: exports, argument checks, bit-exact tree and integers."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import fdph as ofd
from oracle import kernel as kn
from paper_1903_02118_gb300 import build, fdph, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return fdph.lib()


def test_library_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "fdph.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(fdph_[a-z_]+)\s*\(", hdr))
    assert len(declared) >= 17
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(fdph.EXPORTS)


def test_timeout_selftest_rejects_bad_poll_counts_without_a_device(L):
    assert L.fdph_selftest_wait_timeout(0, 0) == fdph.E_ARG
    assert L.fdph_selftest_wait_timeout(0, (1 << 24) + 1) == fdph.E_ARG


def test_invalid_arguments_are_rejected_without_a_device(L):
    g = fdph.Geometry(0, None)
    m = fdph.Material(1.0, 1.0)
    h = ctypes.c_void_p()
    assert L.fdph_plan(ctypes.byref(g), ctypes.byref(m), 0.5, 10, 1e-4, None, ctypes.byref(h)) == fdph.E_ARG
    xy = np.ascontiguousarray(inputs.straight_fault(8))
    g = fdph.Geometry(8, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert L.fdph_plan(ctypes.byref(g), ctypes.byref(m), -1.0, 10, 1e-4, None, ctypes.byref(h)) == fdph.E_ARG
    p = fdph.make_params(leaf_size=64)
    assert L.fdph_plan(ctypes.byref(g), ctypes.byref(m), 0.5, 10, 1e-4, ctypes.byref(p), ctypes.byref(h)) == fdph.E_ARG
    p = fdph.make_params(nrhs=3)
    assert L.fdph_plan(ctypes.byref(g), ctypes.byref(m), 0.5, 10, 1e-4, ctypes.byref(p), ctypes.byref(h)) == fdph.E_ARG
    p = fdph.make_params(far_mode=2)
    assert L.fdph_plan(ctypes.byref(g), ctypes.byref(m), 0.5, 10, 1e-4, ctypes.byref(p), ctypes.byref(h)) == fdph.E_ARG
    bad = xy.copy()
    bad[3, 2] = np.nan
    gb = fdph.Geometry(8, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert L.fdph_plan(ctypes.byref(gb), ctypes.byref(m), 0.5, 10, 1e-4, None, ctypes.byref(h)) == fdph.E_NAN
    assert not h.value
    assert L.fdph_step(None, None, None) == fdph.E_ARG
    assert L.fdph_predict(None, None) == fdph.E_ARG
    assert L.fdph_commit(None, None) == fdph.E_ARG
    assert L.fdph_self(None, None) == fdph.E_ARG
    out = ctypes.c_void_p()
    assert L.fdph_batch_create(None, 0, ctypes.byref(out)) == fdph.E_ARG
    arr = (ctypes.c_void_p * 1)(None)
    assert L.fdph_batch_create(arr, 1, ctypes.byref(out)) == fdph.E_ARG and not out.value
    assert L.fdph_batch_run(None, 1, None, None) == fdph.E_ARG
    assert L.fdph_batch_rupture_run(None, 1, None, None) == fdph.E_ARG
    assert L.fdph_batch_synchronize(None) == fdph.E_ARG
    L.fdph_batch_destroy(None)
    assert L.fdph_strerror(fdph.E_CAUSALITY)


def test_plan_refuses_a_causality_violation_before_any_device_work():
    """Sec. 5.2 / App. D: a time step so coarse that an admissible leaf's nearest pair has
    dm_i + mbar_j < 1 (cs dt = 4 dx, eta = 1/2, clusters down to one element) must be refused with
    FDPH_E_CAUSALITY and no plan; the check runs on the host before the device is touched, so it
    answers the same with or without a GPU.  A step half as long passes.  The oracle agrees."""
    L = fdph.lib()
    xy = inputs.straight_fault(64)
    g, keep = fdph._geometry(xy)
    mat = fdph.Material(1.0, 1.0)
    p = fdph.make_params(eta=0.5, leaf_size=1)
    h = ctypes.c_void_p()
    rc = L.fdph_plan(ctypes.byref(g), ctypes.byref(mat), 4.0, 64, 1e-4, ctypes.byref(p), ctypes.byref(h))
    assert rc == fdph.E_CAUSALITY and not h.value
    assert b"causality" in L.fdph_last_error()
    with pytest.raises(fdph.FdphError) as e:
        fdph.tree_export(xy, 4.0, eta=0.5, leaf_size=1)
    assert e.value.status == fdph.E_CAUSALITY
    fdph.tree_export(xy, 2.0, eta=0.5, leaf_size=1)        # causal
    el = kn.element_table(xy)
    with pytest.raises(ValueError, match="causality"):
        ofd.build_plan(el, ofd.Params(eta=0.5, leaf=1, dt=4.0, M=64))


def _compare_tree(xy, eta, leaf, eta_scheme=0, lmin=0.0):
    tr = fdph.tree_export(xy, 0.5, eta=eta, leaf_size=leaf, eta_scheme=eta_scheme, lmin=lmin)
    perm = tr["perm"]
    el = kn.element_table(xy)
    p = ofd.Params(eta=eta, leaf=leaf, eta_scheme=eta_scheme, lmin=lmin)
    leaves = ofd.block_tree(el, p)
    key = lambda a, b: (tuple(sorted(a)), tuple(sorted(b)))
    mine = {}
    for lf in tr["leaves"]:
        R = perm[lf["r0"]:lf["r0"] + lf["nr"]].tolist()
        S = perm[lf["s0"]:lf["s0"] + lf["ns"]].tolist()
        mine[key(R, S)] = (lf, R, S)
    assert len(mine) == len(leaves)
    nc = ofd.default_extra_steps(el, p)
    for ol in leaves:
        k = key(ol["tau"].idx.tolist(), ol["sig"].idx.tolist())
        assert k in mine
        lf, R, S = mine[k]
        assert lf["kind"] == (1 if ol["kind"] == "adm" else 0)
        if lf["kind"] == 1:
            d = ofd.admissible_leaf(el, ol, p, nc, need_operator=False)
            dm = dict(zip(ol["tau"].idx.tolist(), d["dm"].tolist()))
            mb = dict(zip(ol["sig"].idx.tolist(), d["mbar"].tolist()))
            Dm = dict(zip(ol["sig"].idx.tolist(), d["Dm"].tolist()))
            assert [dm[e] for e in R] == lf["dm"].tolist()
            assert [mb[e] for e in S] == lf["mbar"].tolist()
            assert [Dm[e] for e in S] == lf["Dm"].tolist()
    # every cluster is a contiguous range of the permutation
    assert sorted(perm.tolist()) == list(range(xy.shape[0]))


@pytest.mark.parametrize("geom,N,eta,leaf", [("straight", 300, 0.5, 16), ("curved", 700, 0.5, 32),
                                             ("kinked", 400, 1.0, 8), ("curved", 4096, 0.5, 32),
                                             ("scatter", 500, 0.25, 8)])
def test_tree_and_art_integers_bit_exact(L, geom, N, eta, leaf):
    if geom == "scatter":
        rng = np.random.default_rng(2)
        c = rng.uniform(0, 120, (N, 2))
        a = rng.uniform(0, 2 * np.pi, N)
        xy = np.stack([c[:, 0], c[:, 1], c[:, 0] + np.cos(a), c[:, 1] + np.sin(a)], 1)
    else:
        xy = {"straight": inputs.straight_fault(N), "curved": inputs.curved_fault(N, inputs.seed_for(1, 0)),
              "kinked": inputs.kinked_fault(N)}[geom]
    _compare_tree(xy, eta, leaf)


@pytest.mark.parametrize("geom,N,lmin", [("curved", 1500, 8.0), ("kinked", 600, 12.0), ("straight", 400, 6.0)])
def test_eta2dist_tree_bit_exact(L, geom, N, lmin):
    """Constant eta^2 dist admissibility (Eq. 25): the library's tree and ART integers equal the
    oracle's."""
    xy = {"straight": inputs.straight_fault(N), "curved": inputs.curved_fault(N, inputs.seed_for(1, 0)),
          "kinked": inputs.kinked_fault(N)}[geom]
    _compare_tree(xy, 0.5, 32, eta_scheme=1, lmin=lmin)


def test_eta2dist_needs_lmin(L):
    xy = np.ascontiguousarray(inputs.straight_fault(64))
    with pytest.raises(fdph.FdphError):
        fdph.tree_export(xy, 0.5, eta=0.5, eta_scheme=1, lmin=0.0)


def _svd_truncation(A, eps):
    """The definition the plan's LRA follows (Sec. 2.3): the truncated SVD of minimal rank with
    |A - A_r|_F < eps |A|_F."""
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    tail = np.sqrt(np.append(np.cumsum((s * s)[::-1])[::-1], 0.0))
    r = int(np.argmax(tail < eps * np.linalg.norm(A)))
    return r, (U[:, :r] * s[:r]) @ Vt[:r]


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
@pytest.mark.parametrize("r0,nr,s0,ns", [(0, 48, 200, 64), (300, 100, 40, 30), (10, 20, 560, 120)])
def test_low_rank_is_the_truncated_svd(L, eps, r0, nr, s0, ns):
    """The host LRA of the plan (QR with column pivoting + Jacobi SVD) gives the minimal rank of
    the truncated SVD and its product to 1e-11 of the block, on static-kernel blocks of the
    curved fault (the oracle's closed form), with the exact fallback of Sec. 6.2."""
    el = kn.element_table(inputs.curved_fault(700, inputs.seed_for(1, 0)))
    A = kn.static_kernel(el, 1.0, receivers=np.arange(r0, r0 + nr), sources=np.arange(s0, s0 + ns))
    F, G, exact = fdph.low_rank(A, eps)
    r, Ar = _svd_truncation(A, eps)
    if r * (nr + ns) >= nr * ns:
        assert exact and np.array_equal(F @ G.T, A)
        return
    assert not exact and F.shape[1] == r
    assert np.linalg.norm(F @ G.T - Ar) < 1e-11 * np.linalg.norm(A)
    assert np.linalg.norm(F @ G.T - A) < eps * np.linalg.norm(A)


def test_low_rank_fallback_zero_and_nan(L):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((12, 9))                  # full rank: kept exact
    F, G, exact = fdph.low_rank(A, 1e-4)
    assert exact and np.array_equal(F @ G.T, A)
    F, G, exact = fdph.low_rank(np.zeros((5, 7)), 1e-4)
    assert F.shape == (5, 0) and G.shape == (7, 0) and not exact
    A[2, 3] = np.nan
    with pytest.raises(fdph.FdphError):
        fdph.low_rank(A, 1e-4)


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
@pytest.mark.parametrize("r0,nr,s0,ns", [(0, 256, 700, 300), (1100, 400, 60, 320)])
def test_cross_approximation_of_a_large_block(L, eps, r0, nr, s0, ns):
    """The cross approximation the plan takes for large admissible blocks (Sec. 4): on static-kernel
    blocks of the curved fault (the oracle's closed form) its product is within eps |A|_F of the
    block, with at most one rank more than the truncated SVD needs, from a small share of the
    block's entries."""
    el = kn.element_table(inputs.curved_fault(1600, inputs.seed_for(1, 0)))
    A = kn.static_kernel(el, 1.0, receivers=np.arange(r0, r0 + nr), sources=np.arange(s0, s0 + ns))
    F, G, evaluated = fdph.low_rank_aca(A, eps)
    assert F is not None
    r, _ = _svd_truncation(A, eps)
    assert F.shape[1] <= r + 1
    assert np.linalg.norm(F @ G.T - A) < eps * np.linalg.norm(A)
    assert evaluated < 0.5 * nr * ns


def test_cross_approximation_exact_rank_and_refusal(L):
    """A block of exact rank 5 is recovered to rounding with rank 5; a full-rank random block makes
    the cross approximation give up (the plan then factorises the dense block)."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((300, 5)) @ rng.standard_normal((5, 240))
    F, G, _ = fdph.low_rank_aca(A, 1e-8)
    assert F.shape[1] == 5
    assert np.linalg.norm(F @ G.T - A) < 1e-10 * np.linalg.norm(A)
    F, G, evaluated = fdph.low_rank_aca(rng.standard_normal((200, 150)), 1e-4)
    assert F is None and G is None and evaluated > 0
    with pytest.raises(fdph.FdphError):
        fdph.low_rank_aca(np.zeros((4, 4)), 0.0)
