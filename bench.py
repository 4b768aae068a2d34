"""Benchmark: GMC cell transmissions per second on GB300.

Workload (one step = one pass of the sampler hot path over one batch):
  velocity MLP 25 -> 256 x4 (SiLU) -> 4, Kaiming-normal weights (seed 1),
  16 explicit Euler steps, batch 2^20 particles, tau log-uniform in
  [0.1, 1000], c uniform in [0.5, 0.999], entry xi ~ U[0,1], cosine-weighted
  entry direction; Philox noise, BF16 tensor-core sampler, decoded exits.
  Inputs are resident in HBM before the timed region; L2 is flushed (256 MiB
  write) between steps, outside the per-step CUDA-event pairs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmc|reference]

Multi-GPU: one process per GPU under torchrun; every rank samples its own
batch (distinct Philox ids), no collective on the data path ("weak").
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BATCH = 1 << 20
ODE_STEPS = 16
HIDDEN = 256
# algorithmic FLOPs per transmission (Eq. 8 with the 25-256x4-4 network):
# per ODE step 2 (4*256 + 3*256^2 + 256*4); the condition part of layer 1
# (2*5*256) once; the time embedding is shared by all particles.
FLOPS_PER_STEP = 2 * (4 * HIDDEN + 3 * HIDDEN * HIDDEN + HIDDEN * 4)
FLOPS_COND = 2 * 5 * HIDDEN
METRIC = "cell transmissions/s GMC vs analog MC at flux err <=1%; p99 latency"
# networks trained by the package's own trainer (commands in the weights folder)
TRAINED_BOUNDARY = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_boundary.bin")
TRAINED_INTERNAL = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_internal.bin")
# networks trained on tau log-uniform in [0.01, 1000] (the paper's thin
# benchmark cells map inside their box), with that box
WIDE_BOUNDARY = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_boundary_wide.bin")
WIDE_INTERNAL = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_internal_wide.bin")
WIDE_BOX = [0.01, 1000.0, 0.5, 0.999]
TRAINED_XY = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_xy.bin")
TRAINED_INTERNAL_XY = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_internal_xy.bin")
# the architecture comparison: the residual-modulated boundary network and an
# MLP control, both trained with the FP32 path on the same data and schedule
ARCH_RM = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_boundary_rm.bin")
ARCH_MLP = os.path.join(ROOT, "paper_2512_13965_gb300", "weights", "gmc_boundary_mlp_fp32.bin")
SAMPLER_FLOP_PER_EVAL = 2 * (4 * 256 + 3 * 256 * 256 + 256 * 4)
SAMPLER_FLOP_PER_TRANSMISSION = 2 * 5 * 256
# stated GMC-vs-analog relative L2 flux error at 1e7 histories, per precision
# of the network (the metric's condition is the BF16 one, 1 %)
FLUX_ERR_BOUND = {"bf16": 0.01, "fp8": 0.02}
WORKLOAD = ("GMC sampler inference: 25-256x4-4 SiLU velocity MLP, Kaiming-normal seed 1, "
            "16 Euler steps, batch 2^20, tau logU[0.1,1000], c U[0.5,0.999]")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"bf16": p["bf16_tflops"], "hbm": p["hbm_gbs"], "src": "measured"}
    except Exception:
        return {"bf16": 1900.0, "hbm": 6800.0, "src": "fallback"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _oracle_timing(rows, steps, warmup):
    """Runs the FP64 oracle sampler (numpy) in a fresh process on all host
    cores: `warmup` untimed and `steps` timed passes over `rows` particles."""
    code = r"""
import json, os, sys, time, tempfile
sys.path.insert(0, %r)
import numpy as np
import oracle, synth
n, steps, warmup = %d, %d, %d
with tempfile.TemporaryDirectory() as d:
    p = os.path.join(d, "w.bin")
    synth.write_weights(p, synth.kaiming_weights(1))
    net = oracle.mlp.read_weights(p)
cond, _, _ = synth.sampler_conditions(n, 1)
z = synth.gaussian_noise(n, 3)
times = []
for i in range(warmup + steps):
    t0 = time.perf_counter()
    y = oracle.mlp.sample(net, cond, z, %d, "euler")
    oracle.mlp.decode(net, y)
    if i >= warmup:
        times.append(time.perf_counter() - t0)
print(json.dumps({"times": times, "n": n}))
""" % (ROOT, rows, steps, warmup, ODE_STEPS)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=900)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return r["times"], r["n"], cores


def cpu_baseline(rows=1 << 17):
    times, n, cores = _oracle_timing(rows, 1, 0)
    return {"value": n / times[0], "unit": "cell transmissions/s", "cores": cores,
            "kind": "oracle",
            "sample": "%d transmissions of the benchmark workload (16 Euler steps, FP64 numpy "
                      "oracle incl. decode, BLAS on all cores), %.1f s" % (n, times[0])}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    rows = 4096
    times, n, cores = _oracle_timing(rows, args.steps, args.warmup)
    total = sum(times)
    value = n * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell transmissions/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded sample: 4096 transmissions per step)",
                       "batch": rows, "ode_steps": ODE_STEPS},
            "cpu_baseline": {"value": value, "unit": "cell transmissions/s", "cores": cores,
                             "kind": "oracle",
                             "sample": "%d steps of %d transmissions" % (len(times), n)},
            "e2e": {"value": value, "unit": "cell transmissions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gmc", choices=["gmc", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp8", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--workload", default="sampler",
                    choices=["sampler", "solve", "hohlraum", "serve", "sweep", "heldout", "sigma",
                             "walks", "paper", "train", "arch", "xy"])
    ap.add_argument("--weights", default=None,
                    help="GMCW file of the boundary model for the solve, serve, sigma, sweep and "
                         "heldout workloads (default: the package's trained network; 'kaiming': "
                         "untrained Kaiming-normal seed 1)")
    ap.add_argument("--internal-weights", default=None,
                    help="GMCW file of the internal-source model (solve/serve: births sampled by "
                         "it; default: the package's trained network; 'none': births walked)")
    ap.add_argument("--serve-leg-requests", type=int, default=40,
                    help="requests of the short serving leg in the default line")
    ap.add_argument("--model", default="boundary", choices=["boundary", "xy"],
                    help="heldout: the square-cell boundary model or the x-y geometry model")
    ap.add_argument("--capacity-sample", type=int, default=None,
                    help="serve: estimate the server's capacity from the first N requests "
                         "(default: the whole stream)")
    ap.add_argument("--histories", type=float, default=1e6)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--hist-range", type=float, nargs=2, default=(1e3, 1e5),
                    help="serve: histories per request, log-uniform in [lo, hi]")
    ap.add_argument("--train-batch", type=int, default=16384, help="train: batch rows per step")
    ap.add_argument("--geometry", default="flat", choices=["flat", "xy"],
                    help="paper: flat (directions on the circle) or xy (3-D directions)")
    ap.add_argument("--sampler-weights", default=None,
                    help="sampler: time this GMCW network instead of the Kaiming-normal MLP")
    ap.add_argument("--net-box", type=float, nargs=4, default=None,
                    metavar=("TAU_LO", "TAU_HI", "C_LO", "C_HI"),
                    help="solve/paper: the (tau, c) box the networks were trained on (default: "
                         "the library's, [0.1, 1000] x [0.5, 0.999])")
    ap.add_argument("--solve-variants", default=None,
                    help="comma list for --workload solve, e.g. analog,gmc_bf16_rk412 (default: all)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("solve", "hohlraum"):
        return run_solve(args)
    if args.workload == "sigma":
        return run_sigma(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "heldout":
        return run_heldout(args)
    if args.workload == "walks":
        return run_walks(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "train":
        return run_train(args)
    if args.workload == "arch":
        return run_arch(args)
    if args.workload == "xy":
        return run_xy(args)

    import numpy as np
    import torch

    import synth
    import paper_2512_13965_gb300 as g

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = {"bf16": g.GMC_BF16, "fp8": g.GMC_FP8, "fp32": g.GMC_FP32}[args.precision]

    ctx = g.Context(local)
    # one explicit stream for the library and for the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    g.gmc_set_stream(ctx, stream)
    workload = WORKLOAD
    if args.sampler_weights:
        # the same workload on another network (e.g. the residual-modulated one)
        g.gmc_load_weights(ctx, args.sampler_weights)
        workload = WORKLOAD.replace("25-256x4-4 SiLU velocity MLP, Kaiming-normal seed 1",
                                    "velocity network " + os.path.relpath(args.sampler_weights, ROOT))
    else:
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "w.bin")
            synth.write_weights(path, synth.kaiming_weights(1))
            g.gmc_load_weights(ctx, path)
    cond_h, _, _ = synth.sampler_conditions(BATCH, 1 + rank)
    cond = torch.from_numpy(cond_h).cuda()
    exit_d = torch.empty(4, BATCH, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    id0 = rank * BATCH

    def step(i):
        g.gmc_transmit(ctx, BATCH, cond, None, 12345, id0 + 0 * i, ODE_STEPS, g.GMC_EULER, prec,
                       None, exit_d)

    for i in range(args.warmup):
        step(i)
        flush.zero_()
    g.gmc_synchronize(ctx)

    clocks = Clocks(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        starts[i].record(stream)
        step(i)
        ends[i].record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    g.gmc_synchronize(ctx)
    per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(per_step)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * BATCH * args.steps / (total_ms * 1e-3)

    # end to end through the C ABI with pinned host buffers (copies timed)
    cond_pin = torch.from_numpy(cond_h).pin_memory()
    exit_pin = torch.empty(4, BATCH, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 10))
    g.gmc_transmit(ctx, BATCH, cond_pin.numpy(), None, 7, id0, ODE_STEPS, g.GMC_EULER, prec,
                   None, exit_pin.numpy())
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        g.gmc_transmit(ctx, BATCH, cond_pin.numpy(), None, 7, id0, ODE_STEPS, g.GMC_EULER, prec,
                       None, exit_pin.numpy())
    e2e_s = time.perf_counter() - t0
    e2e_val = torch.tensor([e2e_s], device="cuda")
    if world > 1:
        torch.distributed.all_reduce(e2e_val, op=torch.distributed.ReduceOp.MAX)
    e2e = {"value": world * BATCH * e2e_steps / float(e2e_val.item()), "unit": "cell transmissions/s",
           "h2d_bytes_per_step": int(cond_pin.numel() * 4), "d2h_bytes_per_step": int(exit_pin.numel() * 4)}

    pk = peaks()
    avg_s = (sum(per_step) / len(per_step)) * 1e-3
    flops = BATCH * (FLOPS_PER_STEP * ODE_STEPS + FLOPS_COND)
    achieved = flops / avg_s / 1e12
    if prec == g.GMC_BF16:
        # DRAM read + write bytes of one launch of this kernel (BF16, Euler, 2^20 rows x
        # 16 steps), from ncu dram__bytes_read.sum + dram__bytes_write.sum of the
        # current kernel (one CTA per SM, no clusters): the Kaiming MLP, and the
        # committed residual-modulated network
        traffic = None
        if ODE_STEPS == 16 and BATCH == 1 << 20:
            if not args.sampler_weights:
                traffic = 21712555
            elif os.path.abspath(args.sampler_weights) == ARCH_RM:
                traffic = 21508608 + 2048
        roof = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16"], "unit": "TFLOP/s",
                "frac": achieved / pk["bf16"], "traffic": traffic, "traffic_unit": "bytes per launch",
                "peak_source": pk["src"] + " bf16 burst", "kernel": "sampler_tc_kernel"}
    elif prec == g.GMC_FP8:
        # 97% of the flops run in E4M3: the FP8 dense rate is twice BF16's
        fp8 = 2.0 * pk["bf16"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": fp8, "unit": "TFLOP/s",
                "frac": achieved / fp8, "traffic": None,
                "peak_source": pk["src"] + " bf16 burst x 2 (nominal fp8/bf16 ratio)",
                "kernel": "sampler_tc_kernel<fp8>"}
    else:
        # FP32 SIMT: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
        alu = 152 * 128 * 2 * 2.07e9 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu, "unit": "TFLOP/s",
                "frac": achieved / alu, "traffic": None, "peak_source": "derived FP32 FMA peak",
                "kernel": "sampler_f32_kernel"}

    extras = {}
    if not args.no_extras:
        extras = analog_extras(g, ctx, torch)
        if world == 1:
            extras.update(headline_extras(args))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "cell transmissions/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {g.GMC_BF16: "bf16", g.GMC_FP8: "e4m3+bf16", g.GMC_FP32: "f32"}[prec],
                "data": "synthetic",
                "config": {"workload": workload, "batch": BATCH, "ode_steps": ODE_STEPS,
                           "integrator": "euler", "precision": args.precision,
                           "l2": "flushed between steps (256 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roof, "e2e": e2e, "gpu_launches": 2 * args.steps,
                "clocks": clk, "per_step_ms": {"min": min(per_step), "p50": statistics.median(per_step),
                                               "max": max(per_step)}}
        line.update(extras)
        if not args.no_cpu_baseline:
            try:
                line["cpu_baseline"] = cpu_baseline()
            except Exception as ex:  # reported, not fatal
                line["cpu_baseline"] = {"error": str(ex)[:200]}
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def analog_extras(g, ctx, torch):
    """GPU analog random walk at tau = 100 (the baseline GMC replaces), same batch."""
    import synth
    out = {}
    n = 1 << 20
    e = synth.cell_entries(n, 9)
    xi, cs, sn = (torch.from_numpy(e[k]).cuda() for k in ("xi", "cos", "sin"))
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for c in (0.9, 0.999):
        tau = torch.full((n,), 100.0, device="cuda")
        cc = torch.full((n,), c, device="cuda")
        g.analog_transmit(ctx, n, xi, cs, sn, tau, cc, g.GMC_ABSORB_ANALOG, 1, 0, 0, st, ex, nc)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        g.analog_transmit(ctx, n, xi, cs, sn, tau, cc, g.GMC_ABSORB_ANALOG, 2, 0, 0, st, ex, nc)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        flights = float(nc.double().mean().item())
        out["analog_tau100_c%s" % c] = {"value": n / (ms * 1e-3), "unit": "cell transmissions/s",
                                        "mean_collisions": flights, "mode": "analog survival",
                                        "position_precision": "fp64 (tau > 64)"}
    return out


def _weights(args):
    """(boundary, internal) weight files of a solve-level workload: the
    package's trained networks unless the flags say otherwise."""
    b = TRAINED_BOUNDARY if args.weights is None else args.weights
    i = getattr(args, "internal_weights", None)
    i = TRAINED_INTERNAL if i is None else (None if i == "none" else i)
    return b, i


def _context(args):
    import torch
    import synth
    import paper_2512_13965_gb300 as g
    torch.cuda.set_device(0)
    ctx = g.Context(0)
    bw, iw = _weights(args)
    args.weights, args.internal_weights = bw, iw
    if iw:
        g.gmc_load_internal_weights(ctx, iw)
    if bw != "kaiming":
        g.gmc_load_weights(ctx, bw)
    else:
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "w.bin")
            synth.write_weights(path, synth.kaiming_weights(1))
            g.gmc_load_weights(ctx, path)
    box = getattr(args, "net_box", None)
    if box:
        cfg = g.gmc_get_config(ctx)
        cfg.net_tau_lo, cfg.net_tau_hi, cfg.net_c_lo, cfg.net_c_hi = box
        g.gmc_set_config(ctx, cfg)
    return g, ctx


def _rel(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solve_cfg4(g, ctx, n_hist, variants):
    """The 128x128 transport solve (tau logU[0.1,500], c {0.5,0.999} per 16x16
    block, seed 2; central 8x8 source; vacuum boundaries): the GPU random walk
    as two independent runs of n/2 histories (averaged: the reference flux;
    their difference / sqrt(2): the statistical floor of an n-history run),
    then each GMC variant (precision, integrator, steps) with n histories.
    Device time per solve from CUDA events around the whole solve."""
    import numpy as np
    import synth
    N = 128
    tau, c, src = synth.grid_problem(n=N, seed=2)
    tau, c, src = (np.ascontiguousarray(a.ravel()) for a in (tau, c, src))

    def solve(method, seed, n, prec=None, integ=0, steps=16):
        cfg = g.gmc_get_config(ctx)
        cfg.steps, cfg.integrator = steps, integ
        cfg.precision = g.GMC_BF16 if prec is None else prec
        cfg.gmc_min_tau = 0.0
        g.gmc_set_config(ctx, cfg)
        f = np.zeros(N * N)
        st = g.transport_solve(ctx, N, N, tau, c, src, n, method, seed, f)
        return f, st

    half = n_hist // 2
    f_a, st_a = solve(g.GMC_METHOD_ANALOG, 1, half)
    f_b, st_b = solve(g.GMC_METHOD_ANALOG, 2, n_hist - half)
    f_mc = 0.5 * (f_a + f_b)
    secs = st_a.seconds + st_b.seconds
    trans = st_a.transmissions + st_b.transmissions
    out = {"analog": {"seconds": secs, "transmissions": trans, "transmissions_per_s": trans / secs,
                      "collisions": st_a.collisions + st_b.collisions,
                      "flux_floor_at_n": _rel(f_a, f_b) / np.sqrt(2.0)}}
    names = {g.GMC_EULER: "euler", g.GMC_MIDPOINT: "midpoint", g.GMC_RK4: "rk4"}
    for prec, integ, steps in variants:
        pname = "bf16" if prec == g.GMC_BF16 else "fp8"
        key = "gmc_%s_%s%d" % (pname, names[integ], steps)
        f, st = solve(g.GMC_METHOD_GMC, 3, n_hist, prec, integ, steps)
        err = _rel(f, f_mc)
        out[key] = {"seconds": st.seconds, "transmissions": st.transmissions,
                    "transmissions_per_s": st.transmissions / st.seconds,
                    "flux_rel_err_vs_analog": err, "flux_err_bound": FLUX_ERR_BOUND[pname],
                    "within_bound": err <= FLUX_ERR_BOUND[pname],
                    "solve_speedup_vs_analog": secs / st.seconds,
                    "transmission_rate_vs_analog": (st.transmissions / st.seconds) / (trans / secs)}
    return out


def serve_stream(g, ctx, reqs, method, prec, integ, steps, rng, load=0.7, min_tau=0.0,
                 capacity_sample=None):
    """One serving run: the capacity of the server (the whole stream, or its
    first `capacity_sample` requests, submitted at once), then the requests
    arriving as a Poisson stream at `load` of that capacity; latency =
    completion - submission per request."""
    import numpy as np
    cfg = g.gmc_get_config(ctx)
    cfg.steps, cfg.integrator, cfg.precision, cfg.gmc_min_tau = steps, integ, prec, min_tau
    cfg.bank_capacity = 1 << 20
    g.gmc_set_config(ctx, cfg)
    g.gmc_serve_start(ctx, method, 4 << 30)
    try:
        cap_reqs = reqs if not capacity_sample else reqs[:capacity_sample]
        t0 = time.perf_counter()
        tks = [g.gmc_submit(ctx, n, n, tau, c, src, h, 7 + i) for i, (n, tau, c, src, h) in enumerate(cap_reqs)]
        for tk, r in zip(tks, cap_reqs):
            g.gmc_wait(ctx, tk, 1800.0, np.zeros(r[0] * r[0]))
        cap = len(cap_reqs) / (time.perf_counter() - t0)
        gaps = rng.exponential(1.0 / (load * cap), len(reqs))
        t0 = time.perf_counter()
        tks = []
        t_next = t0
        for i, (n, tau, c, src, h) in enumerate(reqs):
            t_next += gaps[i]
            while time.perf_counter() < t_next:
                time.sleep(0.0002)
            tks.append(g.gmc_submit(ctx, n, n, tau, c, src, h, 100000 + i))
        lat, trans = [], 0
        for tk, r in zip(tks, reqs):
            st = g.gmc_wait(ctx, tk, 1800.0, np.zeros(r[0] * r[0]))
            lat.append(st.latency)
            trans += st.transmissions
        wall = time.perf_counter() - t0
    finally:
        g.gmc_serve_stop(ctx)
    return {"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(reqs) / wall, "capacity_solves_per_s": cap,
            "capacity_from_requests": len(cap_reqs), "offered_load": load,
            "transmissions_per_s": trans / wall, "histories": int(sum(r[4] for r in reqs))}


def serve_requests(n_req, hist_range, seed=4):
    """Serving stream requests: grids n x n with n ~ U{16..256}, tau
    logU[0.1,1000], c {0.5,0.999} per 16x16 block, a central source of n/16
    cells a side, histories log-uniform in hist_range."""
    import numpy as np
    import synth
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        n = int(rng.integers(16, 257))
        tau, c, src = synth.grid_problem(n=n, seed=1000 + k, tau_range=(0.1, 1000.0),
                                         block=16, source=max(2, n // 16))
        hist = int(np.exp(rng.uniform(np.log(hist_range[0]), np.log(hist_range[1]))))
        reqs.append((n, np.ascontiguousarray(tau.ravel()), np.ascontiguousarray(c.ravel()),
                     np.ascontiguousarray(src.ravel()), hist))
    return reqs, rng


def headline_extras(args):
    """The solve-level headline on the trained networks: the 128x128 solve at
    1e7 histories (analog vs GMC BF16 midpoint 8, FP8 midpoint 8 and BF16 RK4
    12) and a short Poisson serving leg (GMC FP8 midpoint 8 vs analog)."""
    import numpy as np
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, TRAINED_BOUNDARY)
        g.gmc_load_internal_weights(ctx, TRAINED_INTERNAL)
        n = int(1e7)
        solve = solve_cfg4(g, ctx, n, ((g.GMC_BF16, g.GMC_MIDPOINT, 8), (g.GMC_FP8, g.GMC_MIDPOINT, 8),
                                       (g.GMC_BF16, g.GMC_RK4, 12)))
        out = {"solve_cfg4": {"workload": "transport solve 128x128, tau logU[0.1,500], c {0.5,0.999} "
                              "16x16 blocks (seed 2), central 8x8 source, vacuum, %d histories" % n,
                              "networks": "trained (package weights folder): boundary and internal "
                              "models, births sampled by the internal model",
                              "results": solve}}
        reqs, rng = serve_requests(args.serve_leg_requests, (1e4, 1e6))
        leg = {}
        for name, method, prec in (("gmc_fp8_midpoint8", g.GMC_METHOD_GMC, g.GMC_FP8),
                                   ("analog", g.GMC_METHOD_ANALOG, g.GMC_BF16)):
            leg[name] = serve_stream(g, ctx, reqs, method, prec, g.GMC_MIDPOINT, 8, rng)
        out["serve_leg"] = {"workload": "%d Poisson-arriving solves, n~U{16..256}, tau logU[0.1,1000], "
                            "histories logU[1e4,1e6], offered load 0.7 of measured capacity"
                            % len(reqs), "results": leg}
    finally:
        ctx.close()
    return out


def run_solve(args):
    """Full transport solve, GMC (BF16 and FP8; Euler, midpoint and RK4; hybrid)
    against the GPU random walk. --workload solve: 128x128 cells, tau
    logU[0.1,500], c in {0.5, 0.999} per 16x16 block (seed 2), unit source on
    the central 8x8 cells, vacuum boundaries. --workload hohlraum: the
    hohlraum-like boundary-source problem (64x64 cells, five materials, the
    entrance hole driven from the left boundary)."""
    import numpy as np
    import synth
    g, ctx = _context(args)
    hohl = args.workload == "hohlraum"
    if hohl:
        N = 64
        tau, c, wall = synth.hohlraum_problem(N)
        tau, c = (np.ascontiguousarray(a.ravel()) for a in (tau, c))
        src = np.ascontiguousarray(wall)
        desc = ("hohlraum-like boundary source 64x64: gas (tau 0.2, c 1), wall (200, 0.6), window "
                "(0.5, 1), ablator (20, 0.9), fuel (2, 0.99); entrance rows 16-47 driven from x = 0")
    else:
        N = 128
        tau, c, src = synth.grid_problem(n=N, seed=2)
        tau, c, src = (np.ascontiguousarray(a.ravel()) for a in (tau, c, src))
        desc = ("transport solve 128x128, tau logU[0.1,500], c {0.5,0.999} 16x16 blocks, central "
                "8x8 source")
    solve_fn = g.transport_solve_wall if hohl else g.transport_solve
    n = int(args.histories)
    out = {}

    def solve(method, seed, steps=16, integ=0, prec=None, n_hist=None, min_tau=0.0):
        cfg = g.gmc_get_config(ctx)
        cfg.steps = steps
        cfg.integrator = integ
        cfg.precision = g.GMC_BF16 if prec is None else prec
        cfg.gmc_min_tau = min_tau
        g.gmc_set_config(ctx, cfg)
        f = np.zeros(N * N)
        st = solve_fn(ctx, N, N, tau, c, src, n if n_hist is None else n_hist, method, seed, f)
        return f, st

    # the analog reference: two independent runs of n/2 histories, averaged
    # (= one run of n); their difference gives the statistical floor, which
    # for two independent n-history runs is sqrt(1/2) of theirs
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    want = None if args.solve_variants is None else set(args.solve_variants.split(","))
    f_mc = None
    if want is None or "analog" in want:
        n_half = n // 2
        f_a, st_a = solve(g.GMC_METHOD_ANALOG, 1, n_hist=n_half)
        f_b, st_b = solve(g.GMC_METHOD_ANALOG, 2, n_hist=n - n_half)
        f_mc = 0.5 * (f_a + f_b)
        secs = st_a.seconds + st_b.seconds
        trans = st_a.transmissions + st_b.transmissions
        out["analog"] = {"seconds": secs, "transmissions": trans, "transmissions_per_s": trans / secs,
                         "collisions": st_a.collisions + st_b.collisions,
                         "waves": st_a.waves + st_b.waves,
                         "floor_rel_err_half_vs_half": rel(f_a, f_b),
                         "floor_rel_err_at_n": rel(f_a, f_b) / np.sqrt(2.0)}
    names = {g.GMC_EULER: "euler", g.GMC_MIDPOINT: "midpoint", g.GMC_RK4: "rk4"}
    for prec, integ, steps in ((g.GMC_BF16, g.GMC_EULER, 16), (g.GMC_BF16, g.GMC_EULER, 8),
                               (g.GMC_BF16, g.GMC_MIDPOINT, 8), (g.GMC_BF16, g.GMC_MIDPOINT, 12),
                               (g.GMC_BF16, g.GMC_RK4, 4), (g.GMC_BF16, g.GMC_RK4, 6),
                               (g.GMC_BF16, g.GMC_RK4, 12), (g.GMC_FP8, g.GMC_EULER, 16),
                               (g.GMC_FP8, g.GMC_EULER, 8), (g.GMC_FP8, g.GMC_MIDPOINT, 8),
                               (g.GMC_FP8, g.GMC_RK4, 12)):
        pname = "bf16" if prec == g.GMC_BF16 else "fp8"
        key = "gmc_%s_%s%d" % (pname, names[integ], steps)
        if want is not None and key not in want:
            continue
        f, st = solve(g.GMC_METHOD_GMC, 3, steps, integ, prec)
        out[key] = {"seconds": st.seconds, "transmissions": st.transmissions,
                    "transmissions_per_s": st.transmissions / st.seconds, "waves": st.waves,
                    "flux_rel_err_vs_analog": None if f_mc is None else rel(f, f_mc)}
    # GMC only in cells thicker than tau = 64 (where the walk switches to FP64
    # positions and one transmission costs more than the network); thinner
    # cells and their births by the random walk
    for integ, steps in ((g.GMC_MIDPOINT, 8), (g.GMC_RK4, 12)):
        key = "hybrid64_bf16_%s%d" % (names[integ], steps)
        if want is not None and key not in want:
            continue
        f, st = solve(g.GMC_METHOD_GMC, 3, steps, integ, g.GMC_BF16, min_tau=64.0)
        out[key] = {"seconds": st.seconds, "transmissions": st.transmissions,
                    "transmissions_per_s": st.transmissions / st.seconds, "waves": st.waves,
                    "collisions": st.collisions,
                    "flux_rel_err_vs_analog": None if f_mc is None else rel(f, f_mc)}
    line = {"metric": METRIC, "workload": "%s, %d histories" % (desc, n),
            "weights": args.weights,
            "births": "on the left boundary (no birth walk)" if hohl else (
                ("internal model " + args.internal_weights) if args.internal_weights else "random walk"),
            "results": out, "unit": "cell transmissions/s"}
    print(json.dumps(line))
    ctx.close()


def run_sigma(args):
    """Statistical convergence of the 128x128 solve (the solve workload's grid):
    the cell-averaged run-to-run standard deviation of the flux over K = 5
    independent runs, sigma_bar(N) = mean over cells of the sample standard
    deviation (Eq. 12), at N = 1e5, 1e6, 1e7 histories, for the random walk,
    GMC (BF16, midpoint 8) and the hybrid; the log-log slope should be -1/2."""
    import numpy as np
    import synth
    g, ctx = _context(args)
    tau, c, src = synth.grid_problem(n=128, seed=2)
    tau, c, src = (np.ascontiguousarray(a.ravel()) for a in (tau, c, src))
    Ns = [int(1e5), int(1e6), int(1e7)]
    K = 5
    methods = {"analog": (g.GMC_METHOD_ANALOG, 0.0), "gmc_bf16_midpoint8": (g.GMC_METHOD_GMC, 0.0),
               "hybrid64_bf16_midpoint8": (g.GMC_METHOD_GMC, 64.0)}
    out = {}
    for name, (method, min_tau) in methods.items():
        cfg = g.gmc_get_config(ctx)
        cfg.steps, cfg.integrator, cfg.precision, cfg.gmc_min_tau = 8, g.GMC_MIDPOINT, g.GMC_BF16, min_tau
        g.gmc_set_config(ctx, cfg)
        rows = []
        for n in Ns:
            runs, secs = [], 0.0
            for k in range(K):
                f = np.zeros(128 * 128)
                st = g.transport_solve(ctx, 128, 128, tau, c, src, n, method, 1000 + 17 * k, f)
                runs.append(f)
                secs += st.seconds
            runs = np.asarray(runs)
            sd = np.sqrt(((runs - runs.mean(0)) ** 2).sum(0) / (K - 1))
            rows.append({"histories": n, "sigma_bar": float(sd.mean()), "seconds_per_run": secs / K})
        x = np.log([r["histories"] for r in rows])
        y = np.log([r["sigma_bar"] for r in rows])
        out[name] = {"runs": rows, "slope": float(np.polyfit(x, y, 1)[0])}
    print(json.dumps({"metric": "sigma_bar(N), Eq. 12, K = %d runs" % K,
                      "workload": "transport solve 128x128 (solve workload grid)",
                      "weights": args.weights,
                      "births": ("internal model " + args.internal_weights) if args.internal_weights
                      else "random walk", "results": out}))
    ctx.close()


def run_paper(args):
    """Solves of the paper's two benchmark problems with their printed cross
    sections (stand-in layouts): the lattice (112 x 112 cells, central
    volumetric source) and the linearized hohlraum (112 x 112 cells, surface
    source on the left boundary). Every cell is thin (tau <= 1.16) and most
    leave the networks' training box (c = 1 scatterers, c = 0.05 absorbers):
    GMC samples them at their scattering-equivalent condition and walks the
    cells that have none. --histories per solve: the random walk with two
    seeds (its run-to-run difference is the statistical floor), then GMC
    (trained networks, BF16, midpoint 8 and RK4 12); solve time,
    transmissions/s and the flux error against the walk. Default networks:
    the pair trained on tau log-uniform in [0.01, 1000], with that box.
    --geometry xy: both problems in x-y geometry (3-D directions;
    transport_solve_xy / transport_solve_wall_xy), the walk on the sphere
    against GMC with the package's x-y networks (boundary and internal
    models, --weights and --internal-weights; 'none' walks the births) and
    their box [0.1, 1000] x [0.5, 0.999]."""
    import numpy as np
    import synth
    xy = getattr(args, "geometry", "flat") == "xy"
    if args.weights is None and args.internal_weights is None and args.net_box is None:
        args.weights, args.internal_weights, args.net_box = WIDE_BOUNDARY, WIDE_INTERNAL, list(WIDE_BOX)
        if xy:
            args.weights, args.internal_weights, args.net_box = TRAINED_XY, TRAINED_INTERNAL_XY, None
    if xy:
        # the square-cell slots are unused by x-y solves
        xy_weights, xy_internal = args.weights, args.internal_weights
        args.weights, args.internal_weights = "kaiming", "none"
    g, ctx = _context(args)
    if xy:
        g.gmc_load_xy_weights(ctx, xy_weights)
        if xy_internal and xy_internal != "none":
            g.gmc_load_internal_xy_weights(ctx, xy_internal)
        args.weights, args.internal_weights = xy_weights, xy_internal
        problems = {"lattice": (synth.paper_lattice_problem(112), g.transport_solve_xy),
                    "hohlraum": (synth.paper_hohlraum_problem(112), g.transport_solve_wall_xy)}
    else:
        problems = {"lattice": (synth.paper_lattice_problem(112), g.transport_solve),
                    "hohlraum": (synth.paper_hohlraum_problem(112), g.transport_solve_wall)}
    n_hist = int(args.histories)
    out = {}
    box = ((0.1, 1000.0), (0.5, 0.999)) if not args.net_box else (tuple(args.net_box[:2]), tuple(args.net_box[2:]))
    for name, ((tau, c, src), solve) in problems.items():
        n_equiv, n_walk, n_inside = _equivalent_summary(tau, c, box)
        tau, c, src = (np.ascontiguousarray(a.ravel()) for a in (tau, c, src))

        def run(method, seed, prec=g.GMC_BF16, integ=g.GMC_MIDPOINT, steps=8):
            cfg = g.gmc_get_config(ctx)
            cfg.precision, cfg.integrator, cfg.steps, cfg.gmc_min_tau = prec, integ, steps, 0.0
            g.gmc_set_config(ctx, cfg)
            f = np.zeros(112 * 112)
            st = solve(ctx, 112, 112, tau, c, src, n_hist, method, seed, f)
            return f, st

        fl, secs, trans = [], [], []
        for seed in (11, 12):
            f, st = run(g.GMC_METHOD_ANALOG, seed)
            fl.append(f)
            secs.append(st.seconds)
            trans.append(st.transmissions)
        f_mc = 0.5 * (fl[0] + fl[1])
        res = {"analog": {"histories": n_hist, "seconds": secs, "transmissions": trans,
                          "transmissions_per_s": float(np.mean(trans) / np.mean(secs)),
                          "flux_floor_at_n": _rel(fl[0], fl[1]) / np.sqrt(2.0)},
               "cells": {"outside_box_sampled_at_equivalent": n_equiv, "walked_no_equivalent": n_walk,
                         "inside_box": n_inside}}
        for key, integ, steps in (("gmc_bf16_midpoint8", g.GMC_MIDPOINT, 8),
                                  ("gmc_bf16_rk412", g.GMC_RK4, 12)):
            f, st = run(g.GMC_METHOD_GMC, 13, integ=integ, steps=steps)
            res[key] = {"seconds": st.seconds, "transmissions": st.transmissions,
                        "transmissions_per_s": st.transmissions / st.seconds,
                        "collisions_of_walked_cells": st.collisions,
                        "flux_rel_err_vs_analog": _rel(f, f_mc),
                        "solve_speedup_vs_analog": float(np.mean(secs)) / st.seconds}
        out[name] = res
    print(json.dumps({"metric": "solves of the paper's benchmark problems, GMC vs the random walk",
                      "workload": "lattice and linearized hohlraum, 112x112 cells, printed cross "
                                  "sections, stand-in layouts, %d histories%s"
                                  % (n_hist, ", x-y geometry" if xy else ""),
                      "weights": args.weights, "internal_weights": args.internal_weights,
                      "net_box": [list(box[0]), list(box[1])], "results": out}))
    ctx.close()


def _equivalent_summary(tau, c, box=((0.1, 1000.0), (0.5, 0.999))):
    """Cell counts: outside the training box with an equivalent condition,
    without one (walked), inside (host arithmetic of the same reading as the
    solve)."""
    import numpy as np
    tau = np.asarray(tau, np.float64)
    c = np.asarray(c, np.float64)
    (t_lo, t_hi), (c_lo, c_hi) = box
    inside = (tau >= t_lo) & (tau <= t_hi) & (c >= c_lo) & (c <= c_hi)
    w = c * tau
    ok = inside | ((w > 0) & (np.maximum(c_lo, w / t_hi) <= np.minimum(c_hi, w / t_lo)))
    return int((ok & ~inside).sum()), int((~ok).sum()), int(inside.sum())


def run_arch(args):
    """The paper's architecture (residual blocks with adaptive modulation)
    against the MLP at equal flux error: both boundary networks trained with
    the FP32 path on the same data, batch, steps and schedule; the 128x128
    solve (tau logU[0.1,500], c {0.5,0.999} per 16x16 block, central 8x8
    source, the package's internal model for births) at --histories, GMC BF16
    with midpoint K in {2, 4, 8} and Euler 16, flux error against the walk
    (two half runs: the reference flux and the statistical floor); then the
    BF16 sampler kernel of each network on 2^20 transmissions x 16 Euler steps
    (CUDA events, median of 7 after 3 warm-up launches; algorithmic FLOPs as
    the sampler workload's) against the measured BF16 peak."""
    import numpy as np
    import torch
    import synth
    args.weights = args.weights or ARCH_MLP
    g, ctx = _context(args)
    stream = torch.cuda.Stream()
    g.gmc_set_stream(ctx, stream)
    torch.cuda.set_stream(stream)
    N = 128
    tau, c, src = synth.grid_problem(n=N, seed=2)
    tau, c, src = (np.ascontiguousarray(a.ravel()) for a in (tau, c, src))
    n_hist = int(args.histories)

    def solve(method, seed, n, integ=0, steps=16):
        cfg = g.gmc_get_config(ctx)
        cfg.steps, cfg.integrator, cfg.precision, cfg.gmc_min_tau = steps, integ, g.GMC_BF16, 0.0
        g.gmc_set_config(ctx, cfg)
        f = np.zeros(N * N)
        st = g.transport_solve(ctx, N, N, tau, c, src, n, method, seed, f)
        return f, st

    half = n_hist // 2
    f_a, st_a = solve(g.GMC_METHOD_ANALOG, 1, half)
    f_b, st_b = solve(g.GMC_METHOD_ANALOG, 2, n_hist - half)
    f_mc = 0.5 * (f_a + f_b)
    out = {"analog": {"seconds": st_a.seconds + st_b.seconds,
                      "flux_floor_at_n": _rel(f_a, f_b) / np.sqrt(2.0)}}
    pk = peaks()
    n = 1 << 20
    cond, _, _ = synth.sampler_conditions(n, 3)
    z = synth.gaussian_noise(n, 4)
    dc, dz = torch.from_numpy(cond).cuda(), torch.from_numpy(z).cuda()
    yb = torch.empty(4, n, device="cuda")
    flop = n * (SAMPLER_FLOP_PER_EVAL * 16 + SAMPLER_FLOP_PER_TRANSMISSION)
    for arch, path in (("mlp", args.weights), ("rm", ARCH_RM)):
        g.gmc_load_weights(ctx, path)
        res = {"weights": os.path.relpath(path, ROOT)}
        for name, integ, steps in (("midpoint2", g.GMC_MIDPOINT, 2), ("midpoint4", g.GMC_MIDPOINT, 4),
                                   ("midpoint8", g.GMC_MIDPOINT, 8), ("euler16", g.GMC_EULER, 16)):
            f, st = solve(g.GMC_METHOD_GMC, 3, n_hist, integ, steps)
            res[name] = {"seconds": st.seconds, "transmissions_per_s": st.transmissions / st.seconds,
                         "flux_rel_err_vs_analog": _rel(f, f_mc)}
        for _ in range(3):
            g.gmc_transmit(ctx, n, dc, dz, 0, 0, 16, g.GMC_EULER, g.GMC_BF16, yb, None)
        torch.cuda.synchronize()
        ts = []
        for _ in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.gmc_transmit(ctx, n, dc, dz, 0, 0, 16, g.GMC_EULER, g.GMC_BF16, yb, None)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        tf = flop / (ms * 1e-3) / 1e12
        res["sampler_2e20_euler16_bf16"] = {"ms": ms, "transmissions_per_s": n / (ms * 1e-3),
                                            "tflops": tf, "frac_of_%s_bf16_peak" % pk["src"]: tf / pk["bf16"]}
        out[arch] = res
    print(json.dumps({"metric": "flux error and speed of the residual-modulated network vs the MLP",
                      "workload": "transport solve 128x128, %d histories; sampler 2^20 x 16 Euler" % n_hist,
                      "results": out}))
    ctx.close()


def run_xy(args):
    """The 128x128 solve of the solve workload (tau logU[0.1,500], c
    {0.5,0.999} per 16x16 block, seed 2, central 8x8 source, vacuum) in x-y
    geometry (transport_solve_xy: prism cells, 3-D directions): the x-y
    random walk as two half runs (reference flux and statistical floor),
    then GMC with the committed x-y network (BF16, midpoint 8 and Euler 16;
    births walked), and midpoint 8 again with the committed x-y internal
    model sampling the births, at --histories; device seconds per solve,
    cell transmissions/s and the flux error against the walk."""
    import numpy as np
    import synth
    import paper_2512_13965_gb300 as g
    import torch
    torch.cuda.set_device(0)
    ctx = g.Context(0)
    g.gmc_load_xy_weights(ctx, args.weights or TRAINED_XY)
    N = 128
    tau, c, src = synth.grid_problem(n=N, seed=2)
    tau, c, src = (np.ascontiguousarray(a.ravel()) for a in (tau, c, src))
    n_hist = int(args.histories)

    def solve(method, seed, n, integ=0, steps=16):
        cfg = g.gmc_get_config(ctx)
        cfg.steps, cfg.integrator, cfg.precision, cfg.gmc_min_tau = steps, integ, g.GMC_BF16, 0.0
        g.gmc_set_config(ctx, cfg)
        f = np.zeros(N * N)
        st = g.transport_solve_xy(ctx, N, N, tau, c, src, n, method, seed, f)
        return f, st

    half = n_hist // 2
    f_a, st_a = solve(g.GMC_METHOD_ANALOG, 1, half)
    f_b, st_b = solve(g.GMC_METHOD_ANALOG, 2, n_hist - half)
    f_mc = 0.5 * (f_a + f_b)
    secs = st_a.seconds + st_b.seconds
    trans = st_a.transmissions + st_b.transmissions
    out = {"analog_xy": {"seconds": secs, "transmissions_per_s": trans / secs,
                         "collisions": st_a.collisions + st_b.collisions,
                         "flux_floor_at_n": _rel(f_a, f_b) / np.sqrt(2.0)}}
    for name, integ, steps in (("gmc_xy_bf16_midpoint8", g.GMC_MIDPOINT, 8),
                               ("gmc_xy_bf16_euler16", g.GMC_EULER, 16)):
        f, st = solve(g.GMC_METHOD_GMC, 3, n_hist, integ, steps)
        out[name] = {"seconds": st.seconds, "transmissions_per_s": st.transmissions / st.seconds,
                     "collisions_of_walked_births": st.collisions,
                     "flux_rel_err_vs_analog": _rel(f, f_mc), "solve_speedup_vs_analog": secs / st.seconds}
    g.gmc_load_internal_xy_weights(ctx, TRAINED_INTERNAL_XY)
    f, st = solve(g.GMC_METHOD_GMC, 3, n_hist, g.GMC_MIDPOINT, 8)
    out["gmc_xy_bf16_midpoint8_internal_births"] = {
        "seconds": st.seconds, "transmissions_per_s": st.transmissions / st.seconds,
        "collisions": st.collisions, "flux_rel_err_vs_analog": _rel(f, f_mc),
        "solve_speedup_vs_analog": secs / st.seconds}
    print(json.dumps({"metric": "x-y geometry solve, GMC vs the random walk",
                      "workload": "transport solve 128x128 in x-y geometry, %d histories" % n_hist,
                      "weights": os.path.relpath(args.weights or TRAINED_XY, ROOT), "results": out}))
    ctx.close()


def run_walks(args):
    """The random walk in its three cell geometries on one batch: 2^22 entries
    with the sampler workload's (tau, c) law (tau logU[0.1, 1000], c U[0.5,
    0.999]), implicit capture; square cells (analog_transmit), rectangles of
    sides (tau, tau / 2) (analog_transmit_rect) and x-y geometry with 3-D
    directions in square prisms (analog_transmit_xy, 3-D cosine-law entries).
    Cell transmissions/s and flights/s, median of --steps timed launches after
    --warmup, L2 flushed (256 MiB write) before each."""
    import numpy as np
    import torch
    import synth
    g, ctx = _context(args)
    n = 1 << 22
    tau, c = synth.materials(n, 21)
    e2 = synth.cell_entries(n, 22)
    e3 = synth.cell_entries_xy(n, 23)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    tau_d, half_d, c_d = d(tau), d(tau * 0.5), d(c)
    xi2, cs2, sn2 = d(e2["xi"]), d(e2["cos"]), d(e2["sin"])
    xi3, ux3, uy3 = d(e3["xi"]), d(e3["ux"]), d(e3["uy"])
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    imp = g.GMC_ABSORB_IMPLICIT
    calls = {
        "square": lambda s: g.analog_transmit(ctx, n, xi2, cs2, sn2, tau_d, c_d, imp, s, 0, 0, st,
                                              ex, nc),
        "rect_2to1": lambda s: g.analog_transmit_rect(ctx, n, xi2, cs2, sn2, tau_d, half_d, c_d,
                                                      imp, s, 0, 0, st, ex, nc),
        "xy_3d_square_prism": lambda s: g.analog_transmit_xy(ctx, n, xi3, ux3, uy3, tau_d, tau_d,
                                                             c_d, imp, s, 0, 0, st, ex, nc),
    }
    stream = torch.cuda.current_stream()
    out = {}
    for name, call in calls.items():
        times = []
        for k in range(args.warmup + args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            call(100 + k)
            t1.record(stream)
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append(t0.elapsed_time(t1))
        ms = statistics.median(times)
        flights = float(nc.double().sum().item())
        out[name] = {"ms": ms, "transmissions_per_s": n / (ms * 1e-3),
                     "flights_per_s": flights / (ms * 1e-3), "mean_flights": flights / n,
                     "mean_s": float(ex[3].double().mean().item())}
    print(json.dumps({"metric": "cell transmissions/s of the random walk", "unit": "cell transmissions/s",
                      "workload": "2^22 entries, tau logU[0.1,1000], c U[0.5,0.999], implicit capture",
                      "steps": args.steps, "warmup": args.warmup, "l2": "flushed (256 MiB write)",
                      "results": out}))
    ctx.close()


# FLOP per batch row of one training step: forward 2 (32*256 + 3*256^2 +
# 256*4) (layer 1 at its 32 padded inputs) and twice that for the input and
# weight gradients
TRAIN_FLOP_PER_ROW = 3 * 2 * (32 * 256 + 3 * 256 * 256 + 256 * 4)


def run_train(args):
    """The BF16 training step of Eq. 9 (gmc_train_steps, precision BF16):
    batch rows drawn from 2^20 GPU-walk training samples, forward, loss,
    backward and AdamW, at --train-batch rows. Whole steps timed with CUDA
    events on the context's stream: --warmup steps, then --steps steps, median
    of 5 such runs (at least 2000 steps each). The working set is the step's own (about 100 MB of
    operand images per 16384 rows), not flushed: consecutive steps of a
    training run meet the same cache state."""
    import numpy as np
    import torch
    g, ctx = _context(argparse.Namespace(**{**vars(args), "weights": "kaiming", "internal_weights": "none"}))
    stream = torch.cuda.Stream()
    g.gmc_set_stream(ctx, stream)
    n = 1 << 20
    cond = torch.empty(5, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data(ctx, n, 3, 0.1, 1000.0, 0.5, 0.999, cond, y)
    B = args.train_batch
    cfg = g.gmc_train_config(batch=B, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01,
                             seed=7, precision=g.GMC_BF16)
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    steps = max(args.steps, 2000)  # long enough for the clock samples
    clk = Clocks(0)
    clk.start()
    runs = []
    for _ in range(5):
        g.gmc_train_steps(ctx, max(args.warmup, 3))
        g.gmc_synchronize(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.gmc_train_steps(ctx, steps)
        e1.record(stream)
        g.gmc_synchronize(ctx)
        runs.append(e0.elapsed_time(e1) / steps)
    clocks = clk.stop()
    losses = np.zeros(8, np.float32)
    g.gmc_train_steps(ctx, 8, losses)
    ms = statistics.median(runs)
    pk = peaks()
    tflops = TRAIN_FLOP_PER_ROW * B / (ms * 1e-3) / 1e12
    print(json.dumps({
        "metric": "training rows/s (BF16 tensor-core step, Eq. 9)", "unit": "rows/s",
        "value": B / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "warmup": max(args.warmup, 3),
        "workload": "CFM training step, batch %d, 2^20 GPU-walk samples (tau logU[0.1,1000], "
                    "c U[0.5,0.999]), untrained Kaiming-normal start" % B,
        "flop_per_step": TRAIN_FLOP_PER_ROW * B, "loss_last": float(losses[-1]),
        "runs_ms": runs, "gpu_launches_per_step": 4,
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": pk["bf16"], "unit": "TFLOP/s",
                     "frac": tflops / pk["bf16"], "peak_src": pk["src"] + " bf16 burst"},
        "clocks": clocks}))
    ctx.close()


def run_sweep(args):
    """Cost per cell transmission against optical thickness (the paper's
    computational-scaling study): the GPU random walk in a purely scattering
    cell (implicit capture, c = 1) for tau from 0.1 to 1000, against the
    GMC sampler (BF16, 16 and 8 Euler steps), 2^20 transmissions each."""
    import numpy as np
    import torch
    import synth
    g, ctx = _context(args)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    g.gmc_set_stream(ctx, stream)
    n = 1 << 20
    e = synth.cell_entries(n, 9)
    xi, cs, sn = (torch.from_numpy(e[k]).cuda() for k in ("xi", "cos", "sin"))
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / reps * 1e-3

    rows = []
    for tau in (0.1, 0.3, 1, 3, 10, 30, 100, 300, 1000):
        tt = torch.full((n,), float(tau), device="cuda")
        cc = torch.ones(n, device="cuda")
        sec = timed(lambda: g.analog_transmit(ctx, n, xi, cs, sn, tt, cc, g.GMC_ABSORB_IMPLICIT, 3, 0, 0,
                                              st, ex, nc), reps=1 if tau >= 300 else 3)
        rows.append({"tau": tau, "analog_transmissions_per_s": n / sec,
                     "mean_collisions": float(nc.double().mean().item())})
    cond_h, _, _ = synth.sampler_conditions(n, 1)
    cond = torch.from_numpy(cond_h).cuda()
    gmc = {}
    for k in (16, 8):
        sec = timed(lambda: g.gmc_transmit(ctx, n, cond, None, 5, 0, k, g.GMC_EULER, g.GMC_BF16, None, ex))
        gmc["bf16_k%d" % k] = n / sec
    cross = None
    for r in rows:
        if r["analog_transmissions_per_s"] < gmc["bf16_k16"]:
            cross = r["tau"]
            break
    line = {"metric": METRIC, "workload": "tau sweep, pure scattering cell, 2^20 transmissions per point",
            "analog": rows, "gmc": gmc, "crossover_tau_k16": cross,
            "note": "analog positions in FP64 above tau = 64"}
    print(json.dumps(line))
    ctx.close()


def run_heldout(args):
    """Distributional error of the sampler at 20 held-out (tau, c) pairs:
    tau in {0.3, 3, 30, 300, 900} x c in {0.55, 0.75, 0.9, 0.99}, 1e5 entries
    each (xi uniform, cosine-weighted inward direction). Per output (p, cos,
    sin, ln s): the 1-D Wasserstein distance and the mean and variance of GMC
    with the given weights and with the untrained (Kaiming seed 1) network,
    against the GPU implicit-capture walk (the law the network learns), and
    the distance between two independent walks (the statistical floor)."""
    import numpy as np
    import torch
    import synth
    if args.weights == "kaiming":
        raise SystemExit("--workload heldout compares a trained network with the untrained one")
    xy = args.model == "xy"
    if xy and args.weights is None:
        args.weights = TRAINED_XY
    g, ctx = _context(args)
    args_u = argparse.Namespace(**vars(args))
    args_u.weights = "kaiming"
    args_u.internal_weights = "none"
    _, ctx_u = _context(args_u)
    if xy:
        # the x-y network (and the untrained one) in the x-y slot: exits
        # decoded into the unit disk
        g.gmc_load_xy_weights(ctx, args.weights)
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "w.bin")
            synth.write_weights(path, synth.kaiming_weights(1))
            g.gmc_load_xy_weights(ctx_u, path)
    # one stream for torch and the library: inputs made by torch, outputs read
    # by torch, in stream order (a null stream would select the context's own)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    for cx in (ctx, ctx_u):
        g.gmc_set_stream(cx, stream)
    n = 100000
    if xy:
        e = synth.cell_entries_xy(n, 2024)
        xi, cs, sn = (torch.from_numpy(e[k].astype(np.float32)).cuda() for k in ("xi", "ux", "uy"))
        names = ("p", "ux", "uy", "ln_s")
    else:
        e = synth.cell_entries(n, 2024)
        xi, cs, sn = (torch.from_numpy(e[k]).cuda() for k in ("xi", "cos", "sin"))
        names = ("p", "cos", "sin", "ln_s")
    walk = (lambda *a: g.analog_transmit_xy(a[0], a[1], a[2], a[3], a[4], a[5], a[5], *a[6:])) if xy \
        else g.analog_transmit
    transmit = g.gmc_transmit_xy if xy else g.gmc_transmit

    def outputs(ex):
        a = ex.cpu().numpy().astype(np.float64)
        a[3] = np.log(a[3])
        return a

    def w1(a, b):
        return float(np.mean(np.abs(np.sort(a) - np.sort(b))))

    rows = []
    samplers = (("gmc_rk4_12", ctx, g.GMC_RK4, 12), ("gmc_euler16", ctx, g.GMC_EULER, 16),
                ("untrained_euler16", ctx_u, g.GMC_EULER, 16))
    for tau in (0.3, 3.0, 30.0, 300.0, 900.0):
        for c in (0.55, 0.75, 0.9, 0.99):
            tt = torch.full((n,), tau, device="cuda")
            cc = torch.full((n,), c, device="cuda")
            st = torch.empty(n, dtype=torch.int32, device="cuda")
            ref = []
            for seed in (11, 12):
                ex = torch.empty(4, n, device="cuda")
                walk(ctx, n, xi, cs, sn, tt, cc, g.GMC_ABSORB_IMPLICIT, seed, 0, 1, st, ex)
                ref.append(outputs(ex))
            cond = torch.stack([xi, cs, sn, torch.log(tt), cc])
            row = {"tau": tau, "c": c}
            row["floor_w1"] = [w1(ref[1][k], ref[0][k]) for k in range(4)]
            row["analog_mean"] = [float(ref[0][k].mean()) for k in range(4)]
            row["analog_var"] = [float(ref[0][k].var()) for k in range(4)]
            for name, cx, integ, steps in samplers:
                ex = torch.empty(4, n, device="cuda")
                transmit(cx, n, cond, None, 31, 0, steps, integ, g.GMC_BF16, None, ex)
                o = outputs(ex)
                row[name + "_w1"] = [w1(o[k], ref[0][k]) for k in range(4)]
                row[name + "_mean"] = [float(o[k].mean()) for k in range(4)]
                row[name + "_var"] = [float(o[k].var()) for k in range(4)]
            rows.append(row)
    summ = {}
    for name, _, _, _ in samplers:
        r = np.array([[row[name + "_w1"][k] / max(row["floor_w1"][k], 1e-12) for k in range(4)]
                      for row in rows])
        summ[name] = {"median_w1_over_floor": dict(zip(names, np.median(r, axis=0).tolist())),
                      "max_w1_over_floor": dict(zip(names, r.max(axis=0).tolist()))}
    won = sum(all(row["gmc_rk4_12_w1"][k] < row["untrained_euler16_w1"][k] for k in range(4))
              for row in rows)
    line = {"metric": "1-D Wasserstein distance to the implicit-capture walk at 20 held-out (tau, c) pairs",
            "workload": "held-out evaluation%s, 1e5 entries per pair, outputs " % (
                " in x-y geometry (3-D directions on the unit disk)" if xy else "") + ", ".join(names),
            "weights": args.weights, "precision": "bf16", "summary": summ,
            "pairs_trained_beats_untrained_on_all_outputs": won, "rows": rows}
    print(json.dumps(line))
    ctx_u.close()
    ctx.close()


def run_serve(args):
    """Serving: Poisson stream of solves (serve_requests: grids n x n with
    n ~ U{16..256}, tau logU[0.1,1000], c {0.5,0.999} blocks, histories
    log-uniform in --hist-range); p50/p99 latency and solves/s for GMC FP8
    and BF16 (midpoint, 8 steps) and the analog walk."""
    g, ctx = _context(args)
    reqs, rng = serve_requests(args.requests, args.hist_range)
    out = {}
    want = None if args.solve_variants is None else set(args.solve_variants.split(","))
    for name, method, prec in (("gmc_fp8_midpoint8", g.GMC_METHOD_GMC, g.GMC_FP8),
                               ("gmc_bf16_midpoint8", g.GMC_METHOD_GMC, g.GMC_BF16),
                               ("analog", g.GMC_METHOD_ANALOG, g.GMC_BF16)):
        if want is not None and name not in want:
            continue
        out[name] = serve_stream(g, ctx, reqs, method, prec, g.GMC_MIDPOINT, 8, rng,
                                 capacity_sample=args.capacity_sample)
    line = {"metric": METRIC, "workload": "serving: %d Poisson-arriving solves, n~U{16..256}, "
            "tau logU[0.1,1000], histories logU[%g,%g]" % (len(reqs), args.hist_range[0],
                                                          args.hist_range[1]), "results": out,
            "births": ("internal model " + args.internal_weights) if args.internal_weights else "random walk",
            "weights": args.weights}
    print(json.dumps(line))
    ctx.close()


if __name__ == "__main__":
    main()
