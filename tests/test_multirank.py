"""Several ranks on CPU (gloo, world size 2): the timing protocol of a multi-GPU run (replicas)
and the receiver-sharded rupture step with one allgather of D_n per step, which must reproduce
the single-process march."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from oracle import fdph as ofd
    from oracle import kernel as kn
    from paper_1903_02118_gb300 import fdph, inputs, replicas, sharding
    w, r, _ = replicas.init()
    replicas.barrier(w)
    mx = replicas.max_over_ranks(1.5 + r, w)
    tot = replicas.sum_over_ranks(r + 1, w)
    # receiver-sharded dynamic rupture on the compressed operator (Sec. 6.2 law, as the oracle's
    # rupture_march): each rank predicts and solves its own receivers, then D_n is gathered
    N, M, dt = 120, 90, 0.5
    xy = inputs.kinked_fault(N)
    perm = fdph.tree_export(xy, dt, eta=0.5, leaf_size=16)["perm"]
    owners = sharding.receiver_ranges(perm, w)
    rows = owners[r]
    el = kn.element_table(xy)
    p = ofd.Params(eta=0.5, leaf=16, eps=1e-6, eps_st=1e-4, M=M, soe_terms=16)
    Krows = ofd.operator_rows(el, ofd.build_plan(el, p, receivers=rows), rows)   # [M, len(rows), N]
    tau0 = np.full(N, 0.45)
    tau0[55:65] = 0.61
    k0 = Krows[0, np.arange(len(rows)), rows]
    D = np.zeros((M, N))
    slip = np.zeros(len(rows))
    for n in range(M):
        mm = min(n + 1, M)
        pred = np.einsum("mij,mj->i", Krows[1:mm], D[n - 1::-1][:mm - 1]) if n > 0 else np.zeros(len(rows))
        tau = tau0[rows] + pred
        strength = 1.0 * (0.6 - 0.3 * np.minimum(slip / 2.0, 1.0))
        v = np.where(tau > strength, (tau - strength) / (-k0), 0.0)
        slip = slip + v * dt
        D[n] = sharding.allgather_rows(v, owners, N)
    np.save(os.path.join(out_dir, "rank%d.npy" % r), D)
    np.save(os.path.join(out_dir, "stats%d.npy" % r), np.array([mx, tot]))
    dist.destroy_process_group()


def test_two_cpu_ranks_replica_timing_and_sharded_rupture(tmp_path):
    import torch.multiprocessing as mp
    from oracle import dense
    from oracle import fdph as ofd
    from oracle import kernel as kn
    from paper_1903_02118_gb300 import build, inputs
    build.build()   # the tree export is a host call of libfdph
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    Ds = [np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world)]
    for r in range(world):
        mx, tot = np.load(tmp_path / ("stats%d.npy" % r))
        assert mx == 2.5 and tot == 3.0
    assert np.array_equal(Ds[0], Ds[1])
    N, M, dt = 120, 90, 0.5
    xy = inputs.kinked_fault(N)
    el = kn.element_table(xy)
    p = ofd.Params(eta=0.5, leaf=16, eps=1e-6, eps_st=1e-4, M=M, soe_terms=16)
    Kop = ofd.operator_rows(el, ofd.build_plan(el, p), np.arange(N))
    tau0 = np.full(N, 0.45)
    tau0[55:65] = 0.61
    D0, _ = dense.rupture_march(Kop, tau0, 1.0, 0.6, 0.3, 2.0, dt, M)
    assert (D0 > 0).sum() > 0.1 * D0.size
    assert np.abs(Ds[0] - D0).max() <= 1e-12 * np.abs(D0).max()
