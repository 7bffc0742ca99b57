"""Throughput of the early-stop network's tensor-core kernels.

    python -m paper_1302_2669_gb300.cnn_bench [--L 17] [--batch 1024] [--steps 50]

Training steps (forward, backward, Adam) on a fixed batch of synthetic
syndromes (the library's generator, p = 0.12) with soft targets, and the
inference forward on a larger batch, timed with CUDA events on the launching
stream after warm-up.  Prints one JSON line with samples/s and the
algorithmic tensor FLOP/s (2 x multiply-adds of the convolutions on the
L x L maps: forward = conv1..conv4, a training step = forward + input
gradients of conv2..conv4 + weight gradients of conv1..conv4; the last layer,
evaluated and differentiated on the 2L middle-line outputs only, and the
readout run on the CUDA cores and are not counted) against the measured bf16
peak.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

CIN = [2, 64, 64, 64, 64]
COUT = [64, 64, 64, 64, 2]


def flops_per_position():
    fwd = [2 * 9 * ci * co for ci, co in zip(CIN, COUT)][:4]   # tensor-core convs conv1..conv4
    dgrad = sum(fwd[1:4])           # tensor-core input gradients of conv2..conv4
    wgrad = sum(fwd[0:4])           # tensor-core weight gradients of conv1..conv4
    return sum(fwd), sum(fwd) + dgrad + wgrad


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=17)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--infer", type=int, default=16384)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    args = ap.parse_args(argv)

    import torch
    import paper_1302_2669_gb300 as P
    from paper_1302_2669_gb300 import build as b
    b.build()
    L = args.L
    ctx = P.Context(0)
    like = torch.zeros(1, device="cuda")
    syn, _ = ctx.gen_syndromes(6100, 0, args.batch, L, 0.12, like=like)
    rng = np.random.default_rng(6101)
    q = torch.from_numpy(rng.dirichlet(np.ones(4), size=args.batch).astype(np.float32)).cuda()
    net = P.Network(ctx, L, max_batch=args.batch)
    p0 = rng.normal(0, 0.05, size=P.Network.n_params()).astype(np.float32)
    net.set_params(p0)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        net.train_step(syn, q, 1e-4, loss_out=loss)
    net.status()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        net.train_step(syn, q, 1e-4, loss_out=loss)
    e.record()
    torch.cuda.synchronize()
    net.status()
    t_step = a.elapsed_time(e) / 1000.0 / args.steps

    inf = P.Network(ctx, L, max_batch=min(args.infer, 8192))
    inf.set_params(p0)
    isyn, _ = ctx.gen_syndromes(6200, 0, args.infer, L, 0.12, like=like)
    out = torch.empty((args.infer, 4), dtype=torch.float32, device="cuda")
    for _ in range(2):
        inf.forward(isyn, out=out)
    torch.cuda.synchronize()
    a.record()
    reps = 5
    for _ in range(reps):
        inf.forward(isyn, out=out)
    e.record()
    torch.cuda.synchronize()
    t_fwd = a.elapsed_time(e) / 1000.0 / reps

    f_fwd, f_train = flops_per_position()
    pos_train = args.batch * L * L
    pos_inf = args.infer * L * L
    peaks = {}
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        peaks = json.load(open(path))
    peak = peaks.get("bf16_tflops", 1900.0)
    train_tf = pos_train * f_train / t_step / 1e12
    fwd_tf = pos_inf * f_fwd / t_fwd / 1e12
    line = {"metric": "network tensor-core throughput", "L": L,
            "train": {"batch": args.batch, "ms_per_step": t_step * 1e3, "samples_per_s": args.batch / t_step,
                      "tflops": train_tf, "frac_of_bf16_peak": train_tf / peak},
            "forward": {"batch": args.infer, "ms": t_fwd * 1e3, "samples_per_s": args.infer / t_fwd,
                        "tflops": fwd_tf, "frac_of_bf16_peak": fwd_tf / peak},
            "bf16_peak_tflops": peak, "peak_source": "MEASURED_PEAKS.json burst" if peaks else "fallback",
            "loss_last": float(loss[0])}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
