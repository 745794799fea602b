"""The seeded input generators (inputs.py): the synthetic workloads' shapes hold as stated.

These generators feed the oracle and the product alike, so they carry no arithmetic of the
method; what is checked is the geometry and slip-rate recipe the workloads are defined by."""
import numpy as np
import pytest

from paper_1903_02118_gb300 import inputs, serving


@pytest.mark.parametrize("n,seed", [(256, 1), (4096, 7), (16384, 3)])
def test_curved_trace_is_a_chain_of_unit_chords(n, seed):
    """n chords of length dx = 1 (Newton's method to rounding), each starting where the previous
    one ends, marching in x, with slope at most 0.2 and curvature at most 0.1 / dx."""
    xy = inputs.curved_fault(n, inputs.seed_for(seed, inputs.GEOMETRY))
    assert xy.shape == (n, 4)
    length = np.hypot(xy[:, 2] - xy[:, 0], xy[:, 3] - xy[:, 1])
    assert np.abs(length - 1.0).max() < 1e-11 * max(1.0, n / 1024)
    assert np.array_equal(xy[1:, :2], xy[:-1, 2:])
    assert (np.diff(xy[:, 0]) > 0).all() and (xy[:, 2] > xy[:, 0]).all()
    slope = np.abs((xy[:, 3] - xy[:, 1]) / (xy[:, 2] - xy[:, 0]))
    assert slope.max() <= 0.2 * (1 + 1e-3)
    # discrete curvature: turning angle between consecutive chords per unit length
    ang = np.arctan2(xy[:, 3] - xy[:, 1], xy[:, 2] - xy[:, 0])
    assert np.abs(np.diff(ang)).max() <= 0.1 * (1 + 1e-2)


def test_generators_are_seeded():
    a = inputs.curved_fault(512, inputs.seed_for(2, inputs.GEOMETRY))
    b = inputs.curved_fault(512, inputs.seed_for(2, inputs.GEOMETRY))
    c = inputs.curved_fault(512, inputs.seed_for(3, inputs.GEOMETRY))
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    p = inputs.gaussian_pulse(512, 1024, 0.5, inputs.seed_for(1, inputs.SLIP))
    q = inputs.gaussian_pulse(512, 2048, 0.5, inputs.seed_for(1, inputs.SLIP))
    # from M = 1024 on the pulse does not depend on M: a march of the first 1024 steps is the
    # beginning of the longer one (the large workload steps only those)
    assert np.array_equal(p, q[:1024])


def test_serving_requests_draw_their_inputs_once():
    """A request's trace, prestress and admission estimate are computed once and reused (the
    admission test asks for the estimate again while the request waits for room)."""
    from paper_1903_02118_gb300 import build
    build.build()   # the estimate reads the block tree (fdph_tree_export, host only)
    req = serving.poisson_requests(3, rate=8.0, seed=4, n_min=512, n_max=2048)[2]
    xy0, tau0 = req.inputs()
    xy1, tau1 = req.inputs()
    assert xy0 is xy1 and tau0 is tau1
    e0 = serving.Server.estimate(req)
    assert serving.Server.estimate(req) == e0 and e0 > 0
    w = min(32, req.N // 8)
    c = req.N // 2
    assert np.all(tau0[c - w:c + w] == 0.61)
