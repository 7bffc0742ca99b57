"""Learned early stop for the MCMC decoder: data, training, calibration and
the timed comparison against plain long chains.

    python -m paper_1302_2669_gb300.early_stop [--L 17] [--train 1048576] ...

Steps (all arithmetic in the library's kernels; this module only moves
buffers and keeps counts):
1. Data: syndromes of a size-L code from the library's generator at error
   rates stratified over [p_lo, p_hi] (n_p equal strata, one seed, distinct
   ids); labels from the library's decoder (K = 4 classes x R chains,
   label_sweeps sweeps, the first quarter annealed in 16 stages from
   0.1 beta_bar): soft targets = softmax
   of its class log-ratios -beta_bar (<n>_k - min <n>).
2. Training: Adam on mini-batches, the tensor-core forward/backward kernels.
3. Calibration, per evaluated error rate p, on a validation set at p: one
   chunked run of the long-chain decoder gives its decision at every
   checkpoint; for each candidate tau the early-stop rule is replayed on those
   decisions, and the smallest tau whose error rate does not exceed the
   long-chain rate is kept (the test set then has to stay within one sigma).
4. Test at p: the long-chain decoder and the early-stop decoder on a fresh
   test set (one call each), both timed on the device; error rates against
   the true classes.  With --reorder, also the early stop with budget
   reordering (the chains of the network's two least likely classes become
   replicas of its two most likely ones at the first checkpoint) at the same
   tau.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def strata(p_lo, p_hi, n_p):
    return [p_lo + (p_hi - p_lo) * (j + 0.5) / n_p for j in range(n_p)]


def make_set(ctx, L, n, seed, p_lo, p_hi, n_p, label_opts=None, id_base=0):
    """Returns dict(syn [n][2L(L-1)] u8 CUDA, cls [n] (true class, CUDA),
    p [n] numpy, targets [n][4] f32 CUDA or None)."""
    import torch
    import paper_1302_2669_gb300 as P
    like = torch.zeros(1, device="cuda")
    ps = strata(p_lo, p_hi, n_p)
    syn = torch.empty((n, P.n_stabs(L)), dtype=torch.uint8, device="cuda")
    tc = torch.empty(n, dtype=torch.int32, device="cuda")
    tg = torch.empty((n, 4), dtype=torch.float32, device="cuda") if label_opts else None
    pv = np.empty(n)
    bounds = [n * j // n_p for j in range(n_p + 1)]
    for j, p in enumerate(ps):
        a, b = bounds[j], bounds[j + 1]
        if a == b:
            continue
        ctx.gen_syndromes(seed, id_base + a, b - a, L, p, syndromes=syn[a:b], true_class=tc[a:b])
        pv[a:b] = p
        if label_opts:
            _, _, lr = ctx.decode(syn[a:b], L, p, label_opts, seed=seed + 100, id0=id_base + a)
            P.Network.soft_targets(lr, out=tg[a:b])
    return {"syn": syn, "cls": tc, "p": pv, "targets": tg, "bounds": bounds, "ps": ps, "id_base": id_base}


def label_opts(L, R=4, sweeps=None):
    import paper_1302_2669_gb300 as P
    sweeps = sweeps or L * L
    burn = sweeps // 4
    return P.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, anneal_stages=min(16, burn),
                  anneal_beta0=0.1)


def train(net, data, epochs, batch, lr, seed=0, lr_final=None, log=None):
    """Adam over shuffled mini-batches; returns the mean loss of each epoch."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    syn, tg = data["syn"], data["targets"]
    n = syn.shape[0]
    steps = epochs * (n // batch)
    losses, k = [], 0
    loss_dev = torch.zeros(1, dtype=torch.float32, device="cuda")
    for ep in range(epochs):
        order = torch.randperm(n, generator=g).cuda()
        acc = torch.zeros((), dtype=torch.float64, device="cuda")
        for b in range(n // batch):
            idx = order[b * batch:(b + 1) * batch]
            xs = syn.index_select(0, idx).contiguous()
            qs = tg.index_select(0, idx).contiguous()
            rate = lr if lr_final is None else lr * (lr_final / lr) ** (k / max(1, steps - 1))
            net.train_step(xs, qs, rate, loss_out=loss_dev)
            acc += loss_dev[0].double()
            k += 1
        net.status()
        losses.append(float(acc) / (n // batch))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4f}")
    return losses


def checkpoint_marks(opts, chunk):
    marks = list(range(opts.burn_in + chunk, opts.n_sweeps, chunk))
    return marks + [opts.n_sweeps]


def chunked_decisions(ctx, data, L, opts, chunk, seed):
    """Decision of the long-chain decoder at every checkpoint: [n][n_marks]
    (resumed runs, so the cost is one full run)."""
    import torch
    import paper_1302_2669_gb300 as P
    marks = checkpoint_marks(opts, chunk)
    n = data["syn"].shape[0]
    out = np.empty((n, len(marks)), np.int32)
    for j, p in enumerate(data["ps"]):
        a, b = data["bounds"][j], data["bounds"][j + 1]
        if a == b:
            continue
        frames = sums = None
        t = 0
        for k, tk in enumerate(marks):
            o = P.Opts(**{**opts.__dict__, "n_sweeps": tk})
            r = ctx.decode_ex(data["syn"][a:b], L, p, o, seed=seed, id0=data["id_base"] + a, sweep_begin=t,
                              init_frames=frames, init_chain_sum=sums, chain_n=False)
            out[a:b, k] = r["cls"].cpu().numpy()
            frames, sums, t = r["chain_frames"], r["chain_sum"], tk
    return marks, out


def replay(logprob, dec, marks, tau):
    """Early-stop decisions and sweeps for threshold tau from the per-checkpoint
    decisions (same rule as the library's decode_early)."""
    lp = logprob.astype(np.float32)
    am = lp.argmax(1)
    top = lp[np.arange(len(lp)), am]
    masked = lp.copy()
    masked[np.arange(len(lp)), am] = -np.inf
    margin = top - masked.max(1)
    n, m = dec.shape
    stop = np.full(n, m - 1)
    ok = (margin > np.float32(tau))[:, None] & (dec[:, :m - 1] == am[:, None])
    has = ok.any(1)
    stop[has] = ok[has].argmax(1)
    cls = dec[np.arange(n), stop]
    return cls, np.asarray(marks)[stop]


def calibrate(logprob, dec, marks, true_cls, taus, margin_sigma=0.0):
    """Smallest tau whose validation error rate exceeds the long chains' by
    at most margin_sigma binomial sigmas.  The default, no excess at all,
    leaves room for the noise of a fresh test set, on which the early stop
    has to stay within one sigma of the long chains."""
    n = len(true_cls)
    ler_long = float((dec[:, -1] != true_cls).mean())
    sigma = math.sqrt(max(ler_long * (1 - ler_long), 1.0 / n) / n)
    rows = []
    best = None
    for tau in sorted(taus):
        cls, sw = replay(logprob, dec, marks, tau)
        ler = float((cls != true_cls).mean())
        rows.append({"tau": tau, "ler": ler, "mean_sweeps": float(sw.mean())})
        if best is None and ler <= ler_long + margin_sigma * sigma:
            best = tau
    return best, ler_long, sigma, rows


def timed(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        r = fn()
    b.record()
    torch.cuda.synchronize()
    return r, a.elapsed_time(b) / reps / 1000.0


def evaluate_p(ctx, fwd_net, L, p, long_opts, chunk, n_val, n_test, seed, log=None, reorder=False):
    """Calibrate tau on a validation set at error rate p, then time the
    long-chain and early-stop decoders on a test set at p (one call each);
    with reorder, also the early stop with budget reordering at the same
    tau."""
    import torch
    va = make_set(ctx, L, n_val, seed + 1, p, p, 1)
    lp_va = fwd_net.forward(va["syn"]).cpu().numpy()
    marks, dec_va = chunked_decisions(ctx, va, L, long_opts, chunk, seed + 101)
    taus = [float(x) for x in np.linspace(0.0, 12.0, 49)] + [float("inf")]
    tau, ler_long_va, sig_va, rows = calibrate(lp_va, dec_va, marks, va["cls"].cpu().numpy(), taus)
    del va
    te = make_set(ctx, L, n_test, seed + 2, p, p, 1)
    true = te["cls"].cpu().numpy()
    out_long = torch.empty(n_test, dtype=torch.int32, device="cuda")
    run_long = lambda: ctx.decode(te["syn"], L, p, long_opts, seed=seed + 102, out_class=out_long, want_sums=False)
    run_early = lambda: ctx.decode_early(fwd_net, te["syn"], L, p, long_opts, chunk_sweeps=chunk, tau=tau,
                                         seed=seed + 102)
    run_long()  # warm-ups: scratch sizing, kernel attributes
    run_early()
    _, t_long = timed(run_long)
    (cls_early, _, sw), t_early = timed(run_early)
    extra = {}
    if reorder:
        run_re = lambda: ctx.decode_early(fwd_net, te["syn"], L, p, long_opts, chunk_sweeps=chunk, tau=tau,
                                          seed=seed + 102, reorder=True)
        run_re()
        (cls_re, _, sw_re), t_re = timed(run_re)
        cls_re = cls_re.cpu().numpy()
        sw_re = sw_re.view(torch.int32).cpu().numpy()
        extra = {"ler_reorder": float((cls_re != true).mean()), "mean_sweeps_reorder": float(sw_re.mean()),
                 "syn_per_s_reorder": n_test / t_re, "gain_reorder": t_long / t_re}
    cls_long = out_long.cpu().numpy()
    cls_early = cls_early.cpu().numpy()
    sw = sw.view(torch.int32).cpu().numpy()
    ler_long = float((cls_long != true).mean())
    ler_early = float((cls_early != true).mean())
    sigma = math.sqrt(max(ler_long * (1 - ler_long), 1.0 / n_test) / n_test)
    row = {"p": p, "tau": tau, "ler_long": ler_long, "ler_early": ler_early, "sigma": sigma,
           "within_1sigma": ler_early <= ler_long + sigma, "mean_sweeps_early": float(sw.mean()),
           "stopped_at_first_checkpoint": float((sw == marks[0]).mean()),
           "syn_per_s_long": n_test / t_long, "syn_per_s_early": n_test / t_early, "gain": t_long / t_early,
           "val_ler_long": ler_long_va, "calibration": rows, **extra}
    if log:
        log(f"p={p:.3f}: tau {tau} LER long {ler_long:.5f} early {ler_early:.5f} (sigma {sigma:.5f}) "
            f"sweeps {row['mean_sweeps_early']:.1f}/{long_opts.n_sweeps} gain {row['gain']:.2f}"
            + (f" | reorder LER {extra['ler_reorder']:.5f} gain {extra['gain_reorder']:.2f}" if extra else ""))
    return row


def run(args, log=print):
    import torch
    import paper_1302_2669_gb300 as P
    from paper_1302_2669_gb300 import build as bld
    bld.build()
    L = args.L
    ctx = P.Context(0)
    lo = label_opts(L, args.label_R, args.label_sweeps)
    t0 = time.time()
    tr, t_lab = timed(lambda: make_set(ctx, L, args.train, args.seed, args.p_lo, args.p_hi, args.n_p, lo))
    log(f"train set {args.train}: labels {t_lab:.2f} s")
    net = P.Network(ctx, L, max_batch=args.batch)
    net.set_params(_he_init(np.random.default_rng(args.seed)))
    losses, t_train = timed(lambda: train(net, tr, args.epochs, args.batch, args.lr, seed=args.seed,
                                          lr_final=args.lr_final, log=log))
    del tr
    long_opts = P.Opts(chains_per_class=args.R, n_sweeps=args.sweeps, burn_in=args.burn_in,
                       anneal_stages=getattr(args, "anneal_stages", 4), anneal_beta0=getattr(args, "anneal_beta0", 0.3))
    fwd_net = P.Network(ctx, L, max_batch=8192)
    fwd_net.set_params(net.get_params())
    net.close()
    rows = [evaluate_p(ctx, fwd_net, L, p, long_opts, args.chunk, args.val, args.test, args.seed + 10 * i, log=log,
                       reorder=getattr(args, "reorder", False))
            for i, p in enumerate(args.eval_ps)]
    te = make_set(ctx, L, args.test, args.seed + 7, args.p_lo, args.p_hi, args.n_p)
    _, t_fwd = timed(lambda: fwd_net.forward(te["syn"]), reps=3)
    # tensor-core work of the forward: conv1..conv4 on the L x L maps (the
    # last layer runs on the CUDA cores at the middle-line outputs only)
    flops = 2.0 * L * L * sum(ci * 9 * co for ci, co in zip([2, 64, 64, 64], [64, 64, 64, 64]))
    res = {
        "metric": "early-stop decoding throughput at matched logical error rate",
        "L": L, "train_p_range": [args.p_lo, args.p_hi], "strata": args.n_p,
        "train": args.train, "epochs": args.epochs, "batch": args.batch, "losses": losses,
        "label_chains": f"4 x {args.label_R} x {lo.n_sweeps} sweeps",
        "label_seconds": t_lab, "train_seconds": t_train,
        "train_samples_per_s": args.train * args.epochs / t_train,
        "long_chain": {"sweeps": args.sweeps, "burn_in": args.burn_in, "chains": f"4 x {args.R}",
                       "anneal": f"{long_opts.anneal_stages} stages from {long_opts.anneal_beta0}"},
        "chunk": args.chunk, "val": args.val, "test": args.test, "per_p": rows,
        "cnn_forward_syn_per_s": args.test / t_fwd, "cnn_forward_tflops": args.test * flops / t_fwd / 1e12,
        "wall_seconds": time.time() - t0,
    }
    ctx.close()
    return res


def _he_init(rng):
    """He-normal weights, zero biases but -4 on the last layer (flips start
    unlikely, so the parity products start near 1), in the flat layout."""
    parts = []
    for ci, co in zip([2, 64, 64, 64, 64], [64, 64, 64, 64, 2]):
        parts.append(rng.normal(0, math.sqrt(2.0 / (9 * ci)), size=co * 9 * ci))
        parts.append(np.full(co, -4.0 if co == 2 else 0.0))
    return np.concatenate(parts).astype(np.float32)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=17)
    ap.add_argument("--train", type=int, default=1 << 20)
    ap.add_argument("--val", type=int, default=65536)
    ap.add_argument("--test", type=int, default=65536)
    ap.add_argument("--p-lo", type=float, default=0.08)
    ap.add_argument("--p-hi", type=float, default=0.18)
    ap.add_argument("--n-p", type=int, default=32)
    ap.add_argument("--label-R", type=int, default=4)
    ap.add_argument("--label-sweeps", type=int, default=4000)
    ap.add_argument("--epochs", type=int, default=16)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--R", type=int, default=4)
    ap.add_argument("--sweeps", type=int, default=20000)
    ap.add_argument("--burn-in", type=int, default=4000)
    ap.add_argument("--anneal-stages", type=int, default=16)
    ap.add_argument("--anneal-beta0", type=float, default=0.1)
    ap.add_argument("--chunk", type=int, default=500,
                    help="sweeps between checkpoints after the burn-in (500 measured 5-9 %% faster than 1000 "
                         "at p = 0.08-0.14, and 250 no better)")
    ap.add_argument("--seed", type=int, default=4001)
    ap.add_argument("--eval-ps", default="0.08,0.10,0.12,0.14,0.16")
    ap.add_argument("--out", default=None)
    ap.add_argument("--reorder", action="store_true",
                    help="also decode each test set with budget reordering at the calibrated tau")
    args = ap.parse_args(argv)
    args.eval_ps = [float(x) for x in args.eval_ps.split(",")]
    res = run(args, log=lambda m: print(m, flush=True))
    line = json.dumps(res)
    print(line, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
