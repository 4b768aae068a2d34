"""Replica runs over two gloo processes on CPU: sharding and the FP64
combination of per-replica fluxes (the oracle solve stands in for each
replica's transport_solve)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _load_replicas():
    # the package __init__ needs libgmc.so; this module does not
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location(
        "gmc_replicas", os.path.join(root, "paper_2512_13965_gb300", "replicas.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_shard_covers_all_histories():
    R = _load_replicas()
    for n in (0, 1, 7, 1000, 10 ** 7 + 3):
        for w in (1, 2, 3, 8):
            parts = [R.shard(n, w, r) for r in range(w)]
            assert sum(parts) == n and max(parts) - min(parts) <= 1
    assert R.seed_for(5, 0) == 5 and R.seed_for(5, 1) != R.seed_for(5, 2)
    with pytest.raises(ValueError):
        R.shard(10, 2, 2)


def _worker(rank, world, port, n, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import transport as T
    R = _load_replicas()
    tau, c, src = synth.grid_problem(n=8, seed=3, tau_range=(0.1, 4.0), block=4, source=2)
    nl = R.shard(n, world, rank)
    f, _ = T.solve_analog(tau, c, src, nl, R.seed_for(11, rank))
    comb = R.combine(f, nl)
    q.put((rank, nl, f, comb))
    dist.destroy_process_group()


def test_two_replicas_combine_to_weighted_mean():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n = 3001
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, n0, f0, c0), (_, n1, f1, c1) = res
    assert n0 + n1 == n
    expect = (n0 * f0 + n1 * f1) / n
    np.testing.assert_allclose(c0, expect, rtol=1e-14, atol=0)
    np.testing.assert_array_equal(c0, c1)
    # rank 0's share with seed_for(11, 0) = 11 is the first shard of a plain solve
    from oracle import transport as T
    tau, c, src = synth.grid_problem(n=8, seed=3, tau_range=(0.1, 4.0), block=4, source=2)
    single, _ = T.solve_analog(tau, c, src, n0, 11)
    np.testing.assert_array_equal(f0, single)
