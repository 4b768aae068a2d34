"""Oracle solves in a pool of spawned processes, for the per-cell statistical
comparisons of the GPU transport solve (test infrastructure; every solve
here is the FP64 oracle's event loop, one seed per task).

A task names its sampler by a plain description (the closures of
oracle.transport do not cross process boundaries):
    {"grid": (tau, c, src), "n": histories, "seed": s, "wall": strengths or None,
     "sampler": ("mlp", weights_path, steps, integrator)
              | ("mlp_e4m3", weights_path, steps, integrator)
              | ("hybrid", weights_path, steps, min_tau)
              | ("equivalent", weights_path, steps, integrator, box)
              | ("walk_global",)
              | ("mlp_xy", weights_path, steps, integrator) | ("walk_global_xy",)
              | ("equivalent_xy", weights_path, steps, integrator, box),
     "geometry": "flat" (default) | "xy" (x-y solves: the *_xy samplers),
     "cell": None | (dx, dy): rectangular cells (solve_gmc_rect; tau holds sigma;
             samplers ("mlp_rect", weights_path, steps, integrator) | ("walk_global_rect",)),
     "internal": None | ("mlp", weights_path, steps, integrator)
               | ("mlp_xy", weights_path, steps, integrator)  (x-y internal model)
               | ("equivalent", weights_path, steps, integrator, box)}
"equivalent" is the network at each cell's scattering-equivalent condition in
the training box ((tau_lo, tau_hi), (c_lo, c_hi)), the walk in the cell's own
frame where there is none.
The pool is started with the spawn method (a process forked after the
parent has touched the GPU can hang), each worker with one BLAS thread.
"""
import multiprocessing as mp
import os

import numpy as np


def _net(path, e4m3=False):
    from oracle import mlp
    net = mlp.read_weights(path)
    return mlp.quantized_e4m3(net) if e4m3 else net


def _hybrid(net, steps, seed, min_tau):
    # the network in cells at least min_tau thick, the walk in the cell's own
    # frame (what the GPU's random-walk kernel draws) in thinner ones
    from oracle import transport as OT
    mlp_s = OT.mlp_sampler(net, steps, "euler", seed)
    walk = OT.walk_sampler_global(seed)

    def f(xi, cx, cy, t, cc, ids, events, rot=None):
        thin = np.asarray(t) < min_tau
        out = [np.zeros(len(ids)) for _ in range(5)] + [np.zeros(len(ids), np.uint32)]
        for sel, fn in ((thin, walk), (~thin, mlp_s)):
            if sel.any():
                res = fn(np.asarray(xi)[sel], np.asarray(cx)[sel], np.asarray(cy)[sel],
                         np.asarray(t)[sel], np.asarray(cc)[sel], np.asarray(ids)[sel],
                         np.asarray(events)[sel], rot=np.asarray(rot)[sel])
                for a, v in zip(out, res):
                    a[sel] = v
        return out[0].astype(np.int64), out[1], out[2], out[3], out[4], out[5]
    return f


def _sampler(spec, seed):
    from oracle import transport as OT
    kind = spec[0]
    if kind == "mlp":
        return OT.mlp_sampler(_net(spec[1]), spec[2], spec[3], seed)
    if kind == "mlp_e4m3":
        return OT.mlp_sampler(_net(spec[1], e4m3=True), spec[2], spec[3], seed)
    if kind == "hybrid":
        return _hybrid(_net(spec[1]), spec[2], seed, spec[3])
    if kind == "walk_global":
        return OT.walk_sampler_global(seed)
    if kind == "equivalent":
        return OT.equivalent_sampler(OT.mlp_sampler(_net(spec[1]), spec[2], spec[3], seed),
                                     OT.walk_sampler_global(seed), *spec[4])
    if kind == "mlp_rect":
        return OT.mlp_sampler_rect(_net(spec[1]), spec[2], spec[3], seed)
    if kind == "walk_global_rect":
        return OT.walk_sampler_global_rect(seed)
    if kind == "equivalent_rect":
        return OT.equivalent_sampler_rect(OT.mlp_sampler_rect(_net(spec[1]), spec[2], spec[3], seed),
                                          OT.walk_sampler_global_rect(seed), *spec[4])
    if kind == "mlp_xy":
        return OT.mlp_sampler_xy(_net(spec[1]), spec[2], spec[3], seed)
    if kind == "walk_global_xy":
        return OT.walk_sampler_global_xy(seed)
    if kind == "equivalent_xy":
        return OT.equivalent_sampler(OT.mlp_sampler_xy(_net(spec[1]), spec[2], spec[3], seed),
                                     OT.walk_sampler_global_xy(seed), *spec[4])
    raise ValueError(kind)


def solve_task(task):
    """One oracle solve; returns (flux [ny, nx], stats dict)."""
    from oracle import transport as OT
    tau, c, src = task["grid"]
    seed = task["seed"]
    internal = None
    if task.get("internal"):
        spec = task["internal"]
        if spec[0] == "mlp_xy":
            internal = OT.mlp_internal_sampler_xy(_net(spec[1]), spec[2], spec[3], seed)
        else:
            internal = OT.mlp_internal_sampler(_net(spec[1]), spec[2], spec[3], seed)
        if spec[0] == "equivalent":
            internal = OT.equivalent_internal_sampler(internal, OT.walk_internal_sampler(seed),
                                                      *spec[4])
    if task.get("cell"):  # rectangular cells: (dx, dy), tau holds sigma
        dx, dy = task["cell"]
        return OT.solve_gmc_rect(tau, c, src, dx, dy, task["n"], seed, _sampler(task["sampler"], seed))
    return OT.solve_gmc(tau, c, src, task["n"], seed, _sampler(task["sampler"], seed),
                        internal=internal, wall=task.get("wall"),
                        geometry=task.get("geometry", "flat"))


def _init():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)


def solve_many(tasks, processes=None):
    """Runs the tasks in a spawned pool; results in task order."""
    processes = processes or max(1, min(len(tasks), (os.cpu_count() or 2) - 1))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(processes, initializer=_init) as pool:
            return pool.map(solve_task, tasks, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def per_cell_z(gpu_runs, oracle_runs):
    """Two-sample z statistic per cell from independent runs on each side:
    (mean_gpu - mean_oracle) / sqrt(var_gpu / K_gpu + var_oracle / K_oracle),
    variances from the run-to-run (seed) spread. Cells with no spread on
    either side (never reached) get z = 0 if both means agree exactly, inf
    otherwise."""
    a = np.asarray(gpu_runs, dtype=np.float64).reshape(len(gpu_runs), -1)
    b = np.asarray(oracle_runs, dtype=np.float64).reshape(len(oracle_runs), -1)
    se = np.sqrt(a.var(0, ddof=1) / a.shape[0] + b.var(0, ddof=1) / b.shape[0])
    d = a.mean(0) - b.mean(0)
    z = np.where(se > 0, d / np.where(se > 0, se, 1.0), np.where(d == 0, 0.0, np.inf))
    return z


def assert_per_cell(gpu_runs, oracle_runs, z_cell=4.0, frac=0.99, z_max=6.0):
    """|z| <= z_cell in at least frac of the cells, and |z| <= z_max in all."""
    z = np.abs(per_cell_z(gpu_runs, oracle_runs))
    ok = np.mean(z <= z_cell)
    assert ok >= frac, ("cells within %.1f sigma: %.4f" % (z_cell, ok), np.sort(z)[-5:])
    assert z.max() <= z_max, ("largest |z|", z.max(), int(np.argmax(z)))
    return z
