"""Train the GMC velocity network on the GPU and write a GMCW weight file.

    python -m paper_2512_13965_gb300.train --out weights.bin \\
        [--samples 16777216] [--steps 20000] [--batch 8192] [--lr 1e-3] \\
        [--lr-min 1e-5] [--warmup 500]

Data: `gmc_train_data` (implicit-capture random walks from the left face,
tau log-uniform in [0.1, 1000], c uniform in [0.5, 0.999]), with
--model internal `gmc_train_data_internal` (walks from a uniform point inside
the cell, for the internal-source model), with --model xy
`gmc_train_data_xy` (walks in x-y geometry: 3-D directions, the cell the
cross-section of a prism), with --model internal_xy
`gmc_train_data_internal_xy` (births inside a prism cell), with --model rect
`gmc_train_data_rect` (rectangular cells, aspect log-uniform in --aspect; the
network gets the aspect as a sixth condition and trains at --precision
fp32); objective: conditional flow
matching (Eq. 9) with AdamW, learning rate warmed up linearly and then
decayed along a cosine to --lr-min; everything runs in libgmc.so, the GEMMs
on tensor cores with BF16 operands and FP32 accumulation and master weights
(--precision fp32 selects the FP32 SIMT GEMMs). The network
starts from Kaiming-normal weights drawn by `synth` (seed --init-seed).
--arch rm trains the residual-modulated network (residual blocks whose
pre-activations are shifted by the condition and scaled channel-wise by the
cell's ln tau and c; shifts and scales start at zero) on the FP32 path.
Prints one JSON line per report interval (loss, samples/s).
"""
import argparse
import json
import os
import sys
import tempfile
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--samples", type=int, default=1 << 24)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-min", type=float, default=1e-5)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--chunk", type=int, default=100, help="steps per learning-rate update")
    ap.add_argument("--weight-decay", type=float, default=0.01)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--init-seed", type=int, default=1)
    ap.add_argument("--tau", type=float, nargs=2, default=(0.1, 1000.0))
    ap.add_argument("--c", type=float, nargs=2, default=(0.5, 0.999))
    ap.add_argument("--report", type=int, default=1000)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--model", default="boundary",
                    choices=["boundary", "internal", "xy", "internal_xy", "rect"],
                    help="boundary: cell transmissions from the left face; internal: births "
                         "inside a cell (volumetric source); xy: transmissions in x-y geometry "
                         "(3-D directions projected on the unit disk); internal_xy: births in x-y "
                         "geometry; rect: transmissions of rectangular cells")
    ap.add_argument("--aspect", type=float, nargs=2, default=(0.25, 4.0),
                    help="rect: range of tau_y / tau_x (log-uniform)")
    ap.add_argument("--precision", default=None, choices=["bf16", "fp32"],
                    help="GEMM operands: bf16 (tensor cores; the MLP's default) or fp32 (SIMT; "
                         "the only choice for --arch rm)")
    ap.add_argument("--arch", default="mlp", choices=["mlp", "rm"],
                    help="mlp: 4 x 256 SiLU MLP; rm: residual-modulated blocks")
    args = ap.parse_args(argv)
    if args.precision is None:
        args.precision = "fp32" if (args.arch == "rm" or args.model == "rect") else "bf16"
    if (args.arch == "rm" or args.model == "rect") and args.precision != "fp32":
        ap.error("--arch rm and --model rect train at --precision fp32")
    if args.arch == "rm" and args.model == "rect":
        ap.error("--arch rm has no rectangular-cell variant")

    import numpy as np
    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth
    from . import _abi as g

    torch.cuda.set_device(args.device)
    ctx = g.Context(args.device)
    stream = torch.cuda.Stream()
    g.gmc_set_stream(ctx, stream)
    with tempfile.TemporaryDirectory() as d:
        init = os.path.join(d, "init.bin")
        w0 = (synth.kaiming_weights_rect if args.model == "rect" else synth.kaiming_weights)(args.init_seed)
        if args.arch == "rm":
            w0 = synth.rm_weights(args.init_seed, base=w0)
        synth.write_weights(init, w0)
        g.gmc_load_weights(ctx, init)
    n = args.samples
    with torch.cuda.stream(stream):
        cond = torch.empty(6 if args.model == "rect" else 5, n, device="cuda")
        y = torch.empty(4, n, device="cuda")
    t0 = time.perf_counter()
    if args.model == "rect":
        g.gmc_train_data_rect(ctx, n, args.seed, args.tau[0], args.tau[1], args.aspect[0],
                              args.aspect[1], args.c[0], args.c[1], cond, y)
    else:
        data = {"boundary": g.gmc_train_data, "internal": g.gmc_train_data_internal,
                "xy": g.gmc_train_data_xy, "internal_xy": g.gmc_train_data_internal_xy}[args.model]
        data(ctx, n, args.seed, args.tau[0], args.tau[1], args.c[0], args.c[1], cond, y)
    g.gmc_synchronize(ctx)
    t_data = time.perf_counter() - t0
    print(json.dumps({"phase": "data", "samples": n, "seconds": t_data}), flush=True)
    cfg = g.gmc_train_config(batch=args.batch, lr=args.lr, beta1=0.9, beta2=0.999, eps=1e-8,
                             weight_decay=args.weight_decay, seed=args.seed + 1000,
                             precision=g.GMC_BF16 if args.precision == "bf16" else g.GMC_FP32)
    g.gmc_train_begin(ctx, n, cond, y, cfg)
    import math

    def lr_at(step):
        if step < args.warmup:
            return args.lr * (step + 1) / args.warmup
        f = (step - args.warmup) / max(1, args.steps - args.warmup)
        return args.lr_min + 0.5 * (args.lr - args.lr_min) * (1 + math.cos(math.pi * min(f, 1.0)))

    done = 0
    recent = []
    t1 = time.perf_counter()
    while done < args.steps:
        k = min(args.chunk, args.steps - done)
        g.gmc_train_set_lr(ctx, lr_at(done))
        losses = np.zeros(k, np.float32)
        g.gmc_train_steps(ctx, k, losses)
        recent.extend(losses.tolist())
        done += k
        if done % args.report == 0 or done == args.steps:
            dt = time.perf_counter() - t1
            print(json.dumps({"phase": "train", "step": done, "lr": lr_at(done - 1),
                              "loss": float(np.mean(recent[-100:])),
                              "rows_per_s": len(recent) * args.batch / dt}), flush=True)
            recent = []
            t1 = time.perf_counter()
    g.gmc_train_commit(ctx, args.out)
    print(json.dumps({"phase": "done", "out": args.out, "steps": done}), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
