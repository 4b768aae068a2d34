"""Replica runs over gloo processes on CPU: sharding, the FP64 combination
of per-replica fluxes (the oracle solve stands in for each replica's
transport_solve), and failure detection before the combination (a replica
that reports a failure, or leaves without reporting, is named on the others,
which never enter the collective)."""
import os
import socket
import time

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


def _worker_failure(rank, world, port, mode, q):
    # rank 1 fails (reports it) or leaves silently; the others must learn of
    # it on the host and never enter the collective
    import datetime
    import torch.distributed as dist
    R = _load_replicas()
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0,
                          timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    if rank == 1:
        if mode == "raise":
            try:
                raise RuntimeError("solver error")
            except RuntimeError as ex:
                R.report(store, rank, 0, ok=False, message=str(ex))
            q.put((rank, "reported", 0.0))
            return
        q.put((rank, "left", 0.0))
        q.close()
        q.join_thread()  # deliver the message before the abrupt exit
        os._exit(3)
    from oracle import transport as T
    tau, c, src = synth.grid_problem(n=4, seed=3, tau_range=(0.1, 2.0), block=2, source=2)
    f, _ = T.solve_analog(tau, c, src, 100, R.seed_for(11, rank))
    R.report(store, rank, 0)
    # the healthy ranks start their bounded wait together, so the time one of
    # them takes to start up (imports under load) is not read as a silence
    store.set("test_ready_%d" % rank, "1")
    store.wait(["test_ready_%d" % r for r in range(world) if r != 1], datetime.timedelta(seconds=60))
    t0 = time.monotonic()
    try:
        R.await_replicas(store, world, 0, 5.0)
        R.combine(f, 100)
        q.put((rank, "combined", time.monotonic() - t0))
    except R.ReplicaFailure as ex:
        q.put((rank, "detected: " + str(ex), time.monotonic() - t0))


@pytest.mark.parametrize("mode", ["raise", "leave"])
def test_replica_failure_is_detected_before_the_combination(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_worker_failure, args=(r, world, port, mode, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = {r: (msg, dt) for r, msg, dt in [q.get(timeout=120) for _ in procs]}
    for p in procs:
        p.join(timeout=60)
    assert procs[0].exitcode == 0 and procs[2].exitcode == 0
    for r in (0, 2):
        msg, dt = res[r]
        if mode == "raise":
            assert msg == "detected: replica 1 failed: solver error", msg
            assert dt < 5.0
        else:
            assert msg == "detected: replica 1 did not report", msg
            assert 4.0 < dt < 30.0


def test_all_replicas_reporting_pass_the_check():
    import datetime
    import torch.distributed as dist
    R = _load_replicas()
    port = _free_port()
    store = dist.TCPStore("127.0.0.1", port, 1, True, timeout=datetime.timedelta(seconds=10))
    for r in range(3):
        R.report(store, r, 7)
    R.await_replicas(store, 3, 7, 1.0)
    R.report(store, 1, 7, ok=False, message="x")
    with pytest.raises(R.ReplicaFailure) as e:
        R.await_replicas(store, 3, 7, 1.0)
    assert e.value.failed == [(1, "x")] and e.value.missing == []
    # the outcomes of solve 7 say nothing about solve 8
    R.report(store, 0, 8)
    with pytest.raises(R.ReplicaFailure) as e:
        R.await_replicas(store, 3, 8, 0.5)
    assert e.value.failed == [] and e.value.missing == [1, 2]
    R.forget(store, 3, 7)
    assert not store.check(["gmc_replica/7/0"]) and store.check(["gmc_replica/8/0"])


def _worker_second_solve(rank, world, port, q):
    # two solves in a row on one process group: every replica completes the
    # first; in the second, rank 1 leaves without reporting. Its "ok" from the
    # first solve must not satisfy the check of the second.
    import datetime
    import torch.distributed as dist
    R = _load_replicas()
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0,
                          timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    from oracle import transport as T
    tau, c, src = synth.grid_problem(n=4, seed=3, tau_range=(0.1, 2.0), block=2, source=2)
    out = []
    for solve_id in (0, 1):
        if rank == 1 and solve_id == 1:
            q.put((rank, ["left"], 0.0))
            q.close()
            q.join_thread()
            os._exit(3)
        f, _ = T.solve_analog(tau, c, src, 50, R.seed_for(11 + solve_id, rank))
        R.report(store, rank, solve_id)
        t0 = time.monotonic()
        try:
            R.await_replicas(store, world, solve_id, 4.0)
            R.combine(f, 50)
            out.append("combined")
        except R.ReplicaFailure as ex:
            out.append("detected: " + str(ex))
            q.put((rank, out, time.monotonic() - t0))
            return
    q.put((rank, out, 0.0))


def test_stale_outcome_of_an_earlier_solve_does_not_hide_a_failure():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_worker_second_solve, args=(r, world, port, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = {r: (out, dt) for r, out, dt in [q.get(timeout=120) for _ in procs]}
    for p in procs:
        p.join(timeout=60)
    assert procs[0].exitcode == 0 and procs[2].exitcode == 0
    for r in (0, 2):
        out, dt = res[r]
        assert out == ["combined", "detected: replica 1 did not report"], out
        assert 3.0 < dt < 30.0
