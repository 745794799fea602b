"""Parity of exactly the setting the benchmark times, against the oracle.

The benchmark's line is the curved fault (N = 4096, M = 4096, eps = 1e-4, eta = 1/2, leaf 32) with
FP32 storage, 16 exponential-tail terms, eps_st = 1e-4 and the near-field work-item length that
fdph_autotune picks.  Here the same plan, tuned the same way, marches all M steps and is compared
with the oracle's compressed operator (FP64) at sampled receivers, element by element:

    |T_gpu - T_oracle| <= 64 u sum |K_ijk| |D_j,n-k|  +  1e-6 max |T_oracle|,   u = 2^-24,

the FP32 rounding of the stored coefficients and slip-rate rows (2u) and of FP32 sums of at most
~32 terms per lane before they are added in FP64 (reasoned bound of ~34u, taken as 64u), plus a
slack for the far-field factors (FP32 f, g, h whose products may cancel).  A smaller case
(N = 256, leaves of 8, FP32 + tails) runs the near kernel's lane-group path (several receiver
groups per warp) against the oracle the same way.
"""
import numpy as np
import pytest

import oracle_workers
from paper_1903_02118_gb300 import fdph

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build
    build.build()


def _march(plan, D):
    Dd = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Td = torch.empty_like(Dd)
    plan.run(D.shape[0], Dd, Td)
    plan.synchronize()
    return Td.cpu().numpy()


def _check_fp32(T, T0, B):
    bound = 64.0 * U32 * B + 1e-6 * np.abs(T0).max()
    err = np.abs(T - T0)
    worst = float((err / bound).max())
    assert worst <= 1.0, "worst error / bound = %.3f" % worst
    assert np.linalg.norm(T - T0) / np.linalg.norm(T0) < 5e-6
    assert np.linalg.norm(T - T0) / np.linalg.norm(T0) > 1e-10      # FP32 rounding is there


def test_benchmarked_configuration_matches_the_oracle():
    _need_gpu()
    desc = dict(geometry="curved", N=4096, M=4096)
    xy, D = oracle_workers.workload(desc)
    plan = fdph.Plan(xy, 0.5, 4096, 1e-4, eta=0.5, eps_st=1e-4, leaf_size=32, soe_terms=16, precision=fdph.FP32)
    chunk = plan.autotune(16)
    assert chunk in (16, 32, 64) and plan.current_step() == 0
    T = _march(plan, D)
    st = plan.stats()
    plan.close()
    assert st["max_window"] < 4096                      # exponential tails in use
    rows = ((np.arange(8) + 0.5) * 4096 / 8).astype(int)
    params = dict(eta=0.5, leaf=32, eps=1e-4, eps_st=1e-4, M=4096, soe_terms=16)
    T0, B = oracle_workers.operator_march_rows(desc, params, rows)
    _check_fp32(T[:, rows], T0, B)


def test_fp32_tails_lane_groups_match_the_oracle():
    _need_gpu()
    desc = dict(geometry="curved", N=256, M=1024)
    xy, D = oracle_workers.workload(desc)
    plan = fdph.Plan(xy, 0.5, 1024, 1e-5, eta=0.5, eps_st=1e-4, leaf_size=8, soe_terms=16, precision=fdph.FP32)
    T = _march(plan, D)
    st = plan.stats()
    plan.close()
    assert st["max_window"] < 1024 and st["n_near"] > 0
    rows = np.arange(256)
    params = dict(eta=0.5, leaf=8, eps=1e-5, eps_st=1e-4, M=1024, soe_terms=16)
    T0, B = oracle_workers.operator_march_rows(desc, params, rows, per=32)
    _check_fp32(T, T0, B)
