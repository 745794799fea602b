"""Serving: continuous batching of independent rupture scenarios gives each scenario the same
result as serving it alone (bit for bit), and reports latency percentiles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_mix_equals_alone_and_reports_latency():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build, serving
    build.build()
    reqs = serving.poisson_requests(6, rate=50.0, seed=7, n_min=256, n_max=1024, m_scale=0.25)
    srv = serving.Server(max_live=4, chunk=32)
    summary = srv.serve(reqs, realtime=True)
    assert summary["requests"] == 6 and summary["p99_latency_s"] >= summary["p50_latency_s"] > 0
    for r in reqs[:3]:
        alone = serving.Request(r.rid, 0.0, r.N, r.cfl, r.seed, M=r.M)
        serving.run_alone(alone, chunk=32)
        assert np.array_equal(alone.slip, r.slip)
        assert np.array_equal(alone.last_T, r.last_T)
        assert (r.slip > 0).any()


def test_footprint_model_bounds_the_real_plan():
    """The admission estimate (footprint_model: block tree only, no device) against the device
    bytes of the plan once built (operator + state), on curved faults of several sizes: within a
    factor of two either way, so that admission neither starves nor overfills the HBM budget; with
    exponential tails and with the paper's cut (soe_terms 0)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build, fdph, inputs, serving
    build.build()
    for N, cfl, soe in ((512, 0.5, 16), (1500, 0.25, 16), (3000, 0.5, 16), (1500, 0.25, 0), (3000, 0.5, 0)):
        xy = inputs.curved_fault(N, inputs.seed_for(3, inputs.GEOMETRY))
        M = int(round(N / cfl))
        est = serving.footprint_model(xy, cfl, M, soe_terms=soe)
        plan = fdph.Plan(xy, cfl, M, 1e-4, eta=0.5, eps_st=1e-4, leaf_size=32, soe_terms=soe, precision=fdph.FP32)
        st = plan.stats()
        plan.close()
        real = st["arena_bytes"] + st["state_bytes"]
        assert 0.5 * real <= est <= 2.0 * real, (N, soe, est, real)
