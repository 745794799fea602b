"""The oracle on several host cores for the large parity cases.  TEST INFRASTRUCTURE ONLY.

Worker processes are spawned (not forked: the test process holds a CUDA context), run one
BLAS / OpenMP thread each, and rebuild the seeded inputs themselves from a small description
instead of receiving large arrays.  Each task evaluates, for a few receivers, the oracle's FDP=H
compressed operator (plan restricted to the leaves of those receivers) and its plain FP64 march,
together with the march of the absolute values (the scale of rounding bounds).
"""
import multiprocessing as mp
import os

import numpy as np


def workload(desc):
    from paper_1903_02118_gb300 import inputs
    N, M = desc["N"], desc["M"]
    if desc["geometry"] == "curved":
        xy = inputs.curved_fault(N, inputs.seed_for(1, inputs.GEOMETRY))
    elif desc["geometry"] == "kinked":
        xy = inputs.kinked_fault(N)
    else:
        xy = inputs.straight_fault(N)
    D = inputs.gaussian_pulse(N, M, desc.get("dt", 0.5), inputs.seed_for(1, inputs.SLIP))
    return xy, D


def _operator_task(job):
    desc, params, rows = job
    from oracle import dense
    from oracle import fdph as ofd
    from oracle import kernel as kn
    xy, D = workload(desc)
    el = kn.element_table(xy)
    rows = np.asarray(rows)
    plan = ofd.build_plan(el, ofd.Params(**params), receivers=rows)
    Kc = ofd.operator_rows(el, plan, rows)
    return dense.march_rows_fft(Kc, D), dense.march_rows_fft(np.abs(Kc), np.abs(D))


def operator_march_rows(desc, params, rows, per=1, workers=None):
    """(T, B): the compressed operator's march T[n, r] and the march of |K|, |D| at the receivers."""
    chunks = [list(map(int, rows[c:c + per])) for c in range(0, len(rows), per)]
    n = workers or min(len(chunks), os.cpu_count() or 1)
    names = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {v: os.environ.get(v) for v in names}
    for v in names:
        os.environ[v] = "1"          # inherited by the workers spawned now, not kept by this process
    try:
        pool = mp.get_context("spawn").Pool(n)
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
    with pool:
        out = pool.map(_operator_task, [(desc, params, c) for c in chunks])
    return np.concatenate([o[0] for o in out], axis=1), np.concatenate([o[1] for o in out], axis=1)
