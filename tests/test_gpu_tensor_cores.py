"""Several right-hand sides with the FP16 near-field window on the tensor cores.

With FP16 storage and nrhs = 2, 4 or 8 the near kernel multiplies each 32 x 32 window slice with
the slip rates of all right-hand sides as warp-level MMAs (FP16 inputs, FP32 accumulation), the
slip rates split into two FP16 parts under a per-row power-of-two scale.  Every output of every
right-hand side must stay within the rounding bound of the stored coefficients, as for the FP16
path on the CUDA cores:

    |dT_i,n| <= 2^-11 sum_window |K_ijk| |D_j,n-k|        (FP16 coefficients)
              + 2^-20 sum |Kc_ijk| |D_j,n-k|               (FP32 slip-rate rows, hi/lo split,
                                                            FP32 sums)
              + 5e-6 max |T|                               (FP32 far field, as in the FP16 test)

against the oracle's compressed operator (FP64), on a curved fault with full 32 x 32 leaves and
on a kinked fault whose leaves have ragged receiver and source counts (13).
"""
import numpy as np
import pytest

from oracle import dense
from oracle import fdph as ofd
from oracle import kernel as kn
from paper_1903_02118_gb300 import fdph, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02118_gb300 import build
    build.build()


@pytest.mark.parametrize("geom,N,leaf", [("curved", 192, 32), ("kinked", 181, 13)])
@pytest.mark.parametrize("R", [2, 4, 8])
def test_fp16_tensor_core_rhs_within_rounding_bound(geom, N, leaf, R):
    _need_gpu()
    M, eps = 800, 1e-5
    xy = inputs.curved_fault(N, inputs.seed_for(1, 0)) if geom == "curved" else inputs.kinked_fault(N)
    Ds = [inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1 + 100 * r, inputs.SLIP)) for r in range(R)]
    el = kn.element_table(xy)
    p = ofd.Params(eta=0.5, leaf=leaf, eps=eps, eps_st=1e-4, M=M, soe_terms=16, amp_window=1)
    oplan = ofd.build_plan(el, p)
    Kc = ofd.operator_rows(el, oplan, np.arange(N))
    Kw = np.zeros_like(Kc)                       # |K| over the FP16 windows of the near leaves
    for d in oplan["near"]:
        I, J, W = d["I"], d["J"], d["W"]
        Kw[:W][:, I[:, None], J[None, :]] = np.abs(d["K"][:W])
    plan = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=1e-4, leaf_size=leaf, soe_terms=16, amp_window=1,
                     precision=fdph.FP16, nrhs=R)
    st = plan.stats()
    assert st["max_window"] < M and st["n_near"] > 0
    Dd = torch.from_numpy(np.ascontiguousarray(np.stack(Ds, 1))).cuda()
    Td = torch.empty_like(Dd)
    plan.run(M, Dd, Td)
    plan.synchronize()
    T = Td.cpu().numpy()
    plan.close()
    single = fdph.Plan(xy, 0.5, M, eps, eta=0.5, eps_st=1e-4, leaf_size=leaf, soe_terms=16, amp_window=1,
                       precision=fdph.FP16)
    for r in range(R):
        T0 = dense.march_rows_fft(Kc, Ds[r])
        B = (2.0 ** -11 * dense.march_rows_fft(Kw, np.abs(Ds[r])) + 2.0 ** -20 * dense.march_rows_fft(np.abs(Kc), np.abs(Ds[r]))
             + 5e-6 * np.abs(T0).max())
        err = np.abs(T[:, r] - T0)
        assert np.all(err <= B), (r, float((err / B).max()))
        assert np.linalg.norm(T[:, r] - T0) / np.linalg.norm(T0) > 1e-7      # FP16 rounding is there
        # the single-RHS FP16 plan (CUDA-core products) agrees to FP32 rounding, not bit for bit
        single.reset()
        D1 = torch.from_numpy(Ds[r]).cuda()
        T1 = torch.empty_like(D1)
        single.run(M, D1, T1)
        single.synchronize()
        T1 = T1.cpu().numpy()
        assert np.linalg.norm(T[:, r] - T1) / np.linalg.norm(T1) < 1e-6
    single.close()
