"""Failure detection without a GPU fault: a bounded device wait that runs out (on a barrier that
nothing completes) is reported as FDPH_E_TIMEOUT and the context keeps working."""
import numpy as np
import pytest

from oracle import dense
from oracle import kernel as kn
from paper_1903_02118_gb300 import fdph, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_times_out_and_the_context_stays_usable():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build
    build.build()
    assert fdph.selftest_wait_timeout(0, 1000) == fdph.E_TIMEOUT
    assert "gave up" in fdph.lib().fdph_last_error().decode()
    assert fdph.selftest_wait_timeout(0, 1) == fdph.E_TIMEOUT
    # the same device then runs a plan normally
    N, M = 96, 80
    xy = inputs.kinked_fault(N)
    D = inputs.gaussian_filtered_history(N, M, inputs.seed_for(0, inputs.SLIP))
    plan = fdph.Plan(xy, 0.5, M, 0.0, eta=0.0, eps_st=0.0, leaf_size=32)
    Dd = torch.from_numpy(D).cuda()
    Td = torch.empty_like(Dd)
    torch.cuda.synchronize()
    plan.run(M, Dd, Td)
    plan.synchronize()
    T0 = dense.march(kn.discrete_kernel(kn.element_table(xy), 0.5, M, 1.0, 1.0), D)
    assert np.linalg.norm(Td.cpu().numpy() - T0) / np.linalg.norm(T0) < 1e-10
