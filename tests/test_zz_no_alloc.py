"""The allocation-free plain step, through the C ABI, against the plan-based step.

Callers that cannot allocate device memory use fdph_plain_step_noalloc with buffers they own;
its partial sums live in the library's static device array.  This file is collected last so
that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from oracle import kernel as kn
from paper_1903_02118_gb300 import fdph, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL64 = 1e-10   # same FP64 tolerance as the other parity tests


def test_noalloc_step_matches_plan_step_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build
    build.build()
    N, M = 97, 90
    xy = inputs.kinked_fault(N)
    D = inputs.gaussian_filtered_history(N, M, inputs.seed_for(0, inputs.SLIP))
    # existing entry point: a plain (all-exact) plan stepped by fdph_run
    plan = fdph.Plan(xy, 0.5, M, 0.0, eta=0.0, eps_st=0.0, leaf_size=32)
    Dd = torch.from_numpy(D).cuda()
    Td = torch.empty_like(Dd)
    plan.run(M, Dd, Td)
    plan.synchronize()
    T_plan = Td.cpu().numpy()
    # caller-held buffers for the allocation-free entry point: kernel tensor [k][j][i], history ring
    el = kn.element_table(xy)
    K = kn.discrete_kernel(el, 0.5, M, 1.0, 1.0)                    # [m, i, j]
    Kd = torch.from_numpy(np.ascontiguousarray(K.transpose(0, 2, 1))).cuda()
    hist = torch.from_numpy(D).cuda()                                 # hist_len = M, row s = step s
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    for step in (57, 58):                                             # two calls in a row
        fdph.plain_step_noalloc(Kd, N, M, hist, M, step, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = T_plan[step]
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL64
    # sizes beyond the static array are rejected by the library itself, before any launch
    import ctypes
    L = fdph.lib()
    rc = L.fdph_plain_step_noalloc(ctypes.c_void_p(Kd.data_ptr()), 100000, 10000, ctypes.c_void_p(hist.data_ptr()),
                                   10000, 9999, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == fdph.E_ARG
    assert b"FDPH_NOALLOC_MAX_PARTIALS" in L.fdph_last_error()
    # and the binding refuses buffers shorter than the sizes it is given
    with pytest.raises(fdph.FdphError):
        fdph.plain_step_noalloc(Kd, N, M + 1, hist, M, step, out)


def test_noalloc_ring_wrap_and_split_k_match_the_oracle():
    """A kernel window W shorter than the history (W < step + 1), a slip-rate ring of hist_len <
    step + 1 rows holding step s in row s mod hist_len, and enough kernel steps that the
    partial sums of several chunks (ceil(W / 64) = 4) are reduced: compared on two calls in a
    row with the oracle's truncated sum T_n = sum_{k < W} K_k D_{n-k}."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import dense
    from paper_1903_02118_gb300 import build
    build.build()
    N, M, W, hist_len = 97, 300, 200, 210
    xy = inputs.curved_fault(N, inputs.seed_for(1, inputs.GEOMETRY))
    D = inputs.gaussian_filtered_history(N, M, inputs.seed_for(1, inputs.SLIP))
    el = kn.element_table(xy)
    K = kn.discrete_kernel(el, 0.5, W, 1.0, 1.0)                    # [k < W, i, j]
    T_or = dense.march(K, D)                                          # sum over k <= min(n, W - 1)
    Kd = torch.from_numpy(np.ascontiguousarray(K.transpose(0, 2, 1))).cuda()
    ring = np.zeros((hist_len, N))
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    for step in (250, 251):
        for s in range(step - hist_len + 1, step + 1):
            ring[s % hist_len] = D[s]
        hist = torch.from_numpy(ring).cuda()
        fdph.plain_step_noalloc(Kd, N, W, hist, hist_len, step, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.linalg.norm(got - T_or[step]) / np.linalg.norm(T_or[step]) < TOL64
