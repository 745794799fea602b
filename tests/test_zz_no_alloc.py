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
    # sizes beyond the static array are rejected with a clear error
    with pytest.raises(fdph.FdphError):
        fdph.plain_step_noalloc(Kd, 100000, 10000, hist, 10000, 9999, out)
