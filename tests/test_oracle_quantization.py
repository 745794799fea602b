"""Pins of the oracle's quantization method (App. A): CPU only."""
import numpy as np
import pytest

from oracle import kernel as kn
from oracle import quantization as qz
from paper_1903_02118_gb300 import inputs


def _fibre(M=1200):
    # the kernel of one element on a neighbour two elements away, from the wave's passage on
    # (the smooth decaying part the method quantizes)
    el = kn.element_table(inputs.straight_fault(8))
    K = kn.discrete_kernel(el, 0.5, M, 1.0, 1.0, receivers=np.array([5]), sources=np.array([2]))[:, 0, 0]
    return K[12:]


@pytest.mark.parametrize("eps_q", [0.2, 0.05, 0.01])
def test_running_window_sums_equal_the_staircase_convolution(eps_q):
    # Eq. A.2 with the running update of Eq. A.4 is the convolution with the staircase kernel
    K = _fibre()
    b, kh = qz.partitions(K, eps_q)
    rng = np.random.default_rng(4)
    D = rng.standard_normal((700, 3))
    T = qz.convolve_running(b, kh, D)
    Ks = qz.staircase(b, kh, K.shape[0])
    brute = np.stack([np.convolve(Ks, D[:, c])[:D.shape[0]] for c in range(3)], 1)
    assert np.abs(T - brute).max() < 1e-12 * np.abs(brute).max()
    assert b[0] == 0 and b[-1] == K.shape[0] and np.all(np.diff(b) > 0)


@pytest.mark.parametrize("eps_q", [0.2, 0.05, 0.01])
def test_every_range_meets_the_error_condition(eps_q):
    # App. A.1.1: for a positive kernel every value of a range lies in [x (1-e)/(1+e), x (1+e)/(1-e)]
    # around its first value x; so the average of the end values keeps |K_m - Khat_q| within
    # eps_Q |Khat_q| where K is monotone over the range, and within (2 e (1+e)/(1-e) + e) |Khat_q|
    # (about 3 eps_Q) where it turns inside the range
    e = eps_q
    cases = ((_fibre(), 0), (np.arange(1, 3001) ** -1.5, 0), (np.cos(np.arange(400) / 40.0) + 1.5, 3))
    for K, turns in cases:   # cos(m / 40) turns at pi, 2 pi, 3 pi; the others are monotone
        b, kh = qz.partitions(K, eps_q)
        turned = 0
        for q in range(len(kh)):
            seg = K[b[q]:b[q + 1]]
            err = np.abs(seg - kh[q]).max()
            mono = np.all(np.diff(seg) >= 0) or np.all(np.diff(seg) <= 0)
            turned += not mono
            bound = e if mono else 2 * e * (1 + e) / (1 - e) + e
            assert err <= bound * abs(kh[q]) * (1 + 1e-12)
        assert turned <= turns


def test_partitions_grow_like_log_of_the_length_for_a_power_law():
    # App. A.1.2: O((a / eps_Q) log(M_fin - M_init)) partitions for K_m ~ m^a
    K = np.arange(1, 100001, dtype=np.float64) ** -1.5
    Q = [len(qz.partitions(K[:M], 0.05)[1]) for M in (1000, 10000, 100000)]
    d1, d2 = Q[1] - Q[0], Q[2] - Q[1]
    assert 0.8 < d2 / d1 < 1.25 and Q[2] < 0.01 * 100000


def test_special_cases():
    b, kh = qz.partitions(np.full(50, 2.5), 0.01)            # constant: one range, exact
    assert list(b) == [0, 50] and kh[0] == 2.5
    K = np.linspace(1.0, 2.0, 101)                             # the absolute bound takes over
    b_rel, _ = qz.partitions(K, 0.1)
    b_abs, kh = qz.partitions(K, 0.1, eps_abs=1e-3)
    assert len(b_abs) > len(b_rel)
    assert np.abs(qz.staircase(b_abs, kh, 101) - K).max() <= 1e-3 + 1e-15


def test_library_partitions_equal_the_oracle_bit_for_bit():
    """The plan's quantization of the transient taps (fdph_quantize, host only) takes the same
    ranges and values as the oracle's partition rule: on kernel fibres, a power law and a
    turning sequence, at several eps_Q."""
    fdph = pytest.importorskip("paper_1903_02118_gb300.fdph")
    try:
        fdph.lib()
    except ImportError:
        pytest.skip("libfdph.so not built")
    seqs = [_fibre(), _fibre(600)[40:] / _fibre(600)[40], np.arange(1, 2001) ** -1.5,
            np.cos(np.arange(400) / 40.0) + 1.5]
    for K in seqs:
        for eps_q in (0.2, 0.05, 0.01, 1e-3):
            b, kh = qz.partitions(K, eps_q)
            b2, kh2 = fdph.quantize(K, eps_q)
            assert np.array_equal(b, b2) and np.array_equal(kh, kh2)


def test_quantized_transient_keeps_the_accuracy():
    """App. A.3: inside FDP=H the solution accuracy is unchanged for eps_Q from 1e-1 to 1e-3.  The
    oracle's march with the transient's taps quantized (eps_Q = 0.05, 0.01) against the plain march
    stays within 1 % of the error with exact taps, with far fewer ranges than taps."""
    from oracle import dense
    from oracle import fdph as ofd
    N, M = 200, 400
    xy = inputs.kinked_fault(N)
    D = inputs.gaussian_pulse(N, M, 0.5, inputs.seed_for(1, inputs.SLIP))
    el = kn.element_table(xy)
    rows = np.arange(0, N, 5)
    T0 = dense.march_rows_fft(kn.discrete_kernel(el, 0.5, M, 1.0, 1.0, receivers=rows), D)
    errs, ratio = [], []
    for eq in (0.0, 0.05, 0.01):
        plan = ofd.build_plan(el, ofd.Params(eta=0.5, leaf=16, eps=1e-4, eps_st=1e-6, M=M, amp_window=1, eps_q=eq),
                              receivers=rows)
        T1 = dense.march_rows_fft(ofd.operator_rows(el, plan, rows), D)
        errs.append(np.linalg.norm(T1 - T0) / np.linalg.norm(T0))
        if eq:
            trs = [d["TR"][c] for d in plan["adm"] for c in "xy" if d["TR"][c]["rank"] and d["TR"][c]["Dm"] > 8]
            ratio.append(np.mean([len(t["qh"]) / t["Dm"] for t in trs]))
    assert abs(errs[1] - errs[0]) < 0.01 * errs[0] and abs(errs[2] - errs[0]) < 0.01 * errs[0], errs
    assert ratio[0] < 0.3 and ratio[1] < 0.6, ratio
