"""Replica (data-parallel) runs of a transport solve over several processes.

Histories are independent, so a solve of N histories splits into W replicas
with no exchange during the run: replica r simulates its share of the
histories with its own Philox seed (seed_for(seed, r)), and the per-source-
particle fluxes combine as the history-weighted mean
    phi = sum_r n_r phi_r / sum_r n_r.
The one collective is that final FP64 sum (torch.distributed all_reduce on
whatever backend the process group uses). Nothing here computes a step of
the method; the per-replica solve is transport_solve.

Failure detection happens on the host, before the collective: every replica
publishes its outcome in the process group's key-value store (report), and
await_replicas waits, with a bound, until every replica has reported. A
replica that failed, or that left without reporting, raises ReplicaFailure
on the others instead of leaving them blocked in the all_reduce. Outcomes
are keyed by a solve id that every replica of one solve passes alike (a
counter of the solves the group has run, say), so an outcome left in the
store by an earlier solve never stands in for the current one; `forget`
removes one solve's keys once it is combined.
"""
import datetime
import time

import numpy as np


class ReplicaFailure(RuntimeError):
    """One or more replicas failed or did not report before the combination."""

    def __init__(self, failed, missing):
        parts = ["replica %d failed: %s" % (r, m) for r, m in failed]
        parts += ["replica %d did not report" % r for r in missing]
        super().__init__("; ".join(parts))
        self.failed = failed
        self.missing = missing


def _key(solve_id, rank):
    return "gmc_replica/%s/%d" % (solve_id, rank)


def report(store, rank, solve_id, ok=True, message=""):
    """Publishes replica `rank`'s outcome of solve `solve_id` (a
    torch.distributed Store)."""
    store.set(_key(solve_id, rank), "ok" if ok else "fail:" + str(message))


def await_replicas(store, world, solve_id, timeout_s):
    """Waits until all `world` replicas have reported their outcome of solve
    `solve_id`, at most timeout_s seconds in total; raises ReplicaFailure
    naming the replicas that reported a failure or did not report in time."""
    deadline = time.monotonic() + float(timeout_s)
    failed, missing = [], []
    for r in range(world):
        left = max(deadline - time.monotonic(), 0.001)
        try:
            store.wait([_key(solve_id, r)], datetime.timedelta(seconds=left))
        except Exception:  # the store's timeout error
            missing.append(r)
            continue
        v = store.get(_key(solve_id, r)).decode()
        if v != "ok":
            failed.append((r, v[len("fail:"):]))
    if failed or missing:
        raise ReplicaFailure(failed, missing)


def forget(store, world, solve_id):
    """Deletes the outcomes of solve `solve_id` (one replica calls it after
    the combination; keys that are absent are skipped)."""
    for r in range(world):
        try:
            store.delete_key(_key(solve_id, r))
        except Exception:  # a store without delete_key keeps them: ids never repeat
            pass


def shard(n_histories, world, rank):
    """Histories of replica `rank` out of `world` (the first n % world get one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(int(n_histories), world)
    return base + (1 if rank < extra else 0)


def seed_for(seed, rank):
    """Philox key of replica `rank`: distinct per replica, equal to `seed` for rank 0."""
    return (int(seed) + 0x9E3779B97F4A7C15 * int(rank)) & 0xFFFFFFFFFFFFFFFF


def combine(flux, n_local, group=None):
    """History-weighted mean of the replicas' flux arrays (FP64 all_reduce).

    flux: numpy array (this replica's flux per source particle),
    n_local: this replica's history count. Returns the combined flux.
    """
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(flux, dtype=np.float64) * float(n_local)).reshape(-1)
    t = torch.cat([t, torch.tensor([float(n_local)], dtype=torch.float64)])
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    total = t[-1].item()
    return (t[:-1] / total).numpy().reshape(np.shape(flux))
