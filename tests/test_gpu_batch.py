"""Batches of plans (fdph_batch_*): one near-field launch per step for several plans gives every
plan the results it gets alone, bit for bit."""
import numpy as np
import pytest
import torch

from oracle import dense
from oracle import fdph as ofd
from oracle import kernel as kn
from paper_1903_02118_gb300 import build, fdph, inputs

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


SHAPES = [("curved", 180), ("kinked", 150), ("straight", 220)]


def _xy(geom, N):
    return {"straight": inputs.straight_fault(N), "curved": inputs.curved_fault(N, inputs.seed_for(1, 0)),
            "kinked": inputs.kinked_fault(N)}[geom]


def _plans(prec, M):
    return [fdph.Plan(_xy(g, N), 0.5, M, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16, precision=prec)
            for g, N in SHAPES]


@pytest.mark.parametrize("prec", [fdph.FP64, fdph.FP32, fdph.FP16])
def test_batch_run_equals_each_plan_alone(prec):
    _need_gpu()
    M = 120
    plans = _plans(prec, M)
    Ds = [torch.from_numpy(inputs.gaussian_filtered_history(p.n, M, 20 + k)).cuda() for k, p in enumerate(plans)]
    torch.cuda.synchronize()
    alone = []
    for p, D in zip(plans, Ds):
        T = torch.empty_like(D)
        torch.cuda.synchronize()
        p.run(M, D, T)
        p.synchronize()
        alone.append(T.cpu().numpy())
        p.reset()
    Ts = [torch.zeros_like(D) for D in Ds]
    torch.cuda.synchronize()
    batch = fdph.Batch(plans)
    batch.run(50, Ds, Ts)                                   # two calls: graph per buffer set,
    batch.run(M - 50, [D[50:] for D in Ds], [T[50:] for T in Ts])   # step index carried on
    batch.synchronize()
    for k, (T, Ta) in enumerate(zip(Ts, alone)):
        assert np.array_equal(T.cpu().numpy(), Ta), k
    # the plans step on alone afterwards from where the batch left them
    for p in plans:
        p.reset()
    batch.run(40, Ds, Ts)
    batch.synchronize()
    for k, (p, D, T) in enumerate(zip(plans, Ds, Ts)):
        p.run(M - 40, D[40:], T[40:])
        p.synchronize()
        assert np.array_equal(T.cpu().numpy(), alone[k]), k
    batch.close()
    # and the first plan's FP64 result is the oracle's compressed operator applied to D
    if prec == fdph.FP64:
        g, N = SHAPES[0]
        el = kn.element_table(_xy(g, N))
        op = ofd.build_plan(el, ofd.Params(eta=0.5, leaf=16, eps=1e-5, eps_st=1e-4, M=M, soe_terms=16))
        T0 = dense.march(ofd.operator_rows(el, op, np.arange(N)), Ds[0].cpu().numpy())
        assert np.linalg.norm(alone[0] - T0) / np.linalg.norm(T0) < 1e-10


def test_batch_rupture_equals_each_plan_alone():
    _need_gpu()
    M = 110
    plans = _plans(fdph.FP32, M)
    taus = []
    for k, p in enumerate(plans):
        rng = np.random.default_rng(inputs.seed_for(5 + k, inputs.FRICTION))
        tau0 = 0.45 * (1.0 + 0.05 * rng.standard_normal(p.n))
        tau0[p.n // 2 - 8:p.n // 2 + 8] = 0.61
        taus.append(torch.from_numpy(tau0).cuda())
    alone = []
    for k, (p, t0) in enumerate(zip(plans, taus)):
        p.rupture_init(t0, 1.0, 0.6, 0.3, 2.0, law=k % 2)
        D = torch.zeros((M, p.n), dtype=torch.float64, device="cuda")
        T = torch.zeros_like(D)
        torch.cuda.synchronize()
        p.rupture_run(M, D, T)
        p.synchronize()
        alone.append((D.cpu().numpy(), T.cpu().numpy()))
    for k, (p, t0) in enumerate(zip(plans, taus)):
        p.reset()
        p.rupture_init(t0, 1.0, 0.6, 0.3, 2.0, law=k % 2)
    Ds = [torch.zeros((M, p.n), dtype=torch.float64, device="cuda") for p in plans]
    Ts = [torch.zeros_like(D) for D in Ds]
    torch.cuda.synchronize()
    batch = fdph.Batch(plans)
    batch.rupture_run(M, Ds, Ts)
    batch.synchronize()
    for k in range(len(plans)):
        assert np.array_equal(Ds[k].cpu().numpy(), alone[k][0]), k
        assert np.array_equal(Ts[k].cpu().numpy(), alone[k][1]), k
    assert (alone[0][0] > 0).mean() > 0.2
    batch.close()


def test_batch_refuses_mixed_precision_and_stale_schedules():
    _need_gpu()
    M = 80
    a = fdph.Plan(_xy("curved", 120), 0.5, M, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16,
                  precision=fdph.FP32)
    b = fdph.Plan(_xy("kinked", 100), 0.5, M, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16,
                  precision=fdph.FP64)
    with pytest.raises(fdph.FdphError):
        fdph.Batch([a, b])
    with pytest.raises(fdph.FdphError):
        fdph.Batch([a, a])
    c = fdph.Plan(_xy("kinked", 100), 0.5, M, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=16, soe_terms=16,
                  precision=fdph.FP32)
    batch = fdph.Batch([a, c])
    a.autotune(4)
    D = [torch.zeros((8, p.n), dtype=torch.float64, device="cuda") for p in (a, c)]
    T = [torch.zeros_like(x) for x in D]
    torch.cuda.synchronize()
    with pytest.raises(fdph.FdphError):
        batch.run(8, D, T)
    batch.close()
