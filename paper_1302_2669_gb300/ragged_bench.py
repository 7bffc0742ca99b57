"""Throughput of ragged batches: syndromes of mixed code sizes in one call.

    python -m paper_1302_2669_gb300.ragged_bench [--n 65536] [--reps 3]

Workload: p = 0.14, L drawn uniformly from {5, 9, 13, 17, 25} (numpy seed
3001), sweeps = L^2 per item, 4 classes x 4 chains; syndromes from the
library's generator (seed 3001, item i at id i).  Timed with CUDA events on
the launching stream after a warm-up, all buffers on the device:

  ragged  one surfmcmc_decode_ragged call (every size in the same persistent
          sweep launches, largest work first)
  plan    the same batch captured once as a CUDA graph (surfmcmc_ragged_plan)
          and replayed
  per_L   five surfmcmc_decode calls, one per size, on that size's items

With --autotune (the default) the launch shape of every size is tuned
first (surfmcmc_autotune: lanes per bundle x resident blocks per
multiprocessor, timed on that size's own items) and the three timings use
the tuned shapes; the ragged call is also timed on a fresh context with the
fixed rule-based shape for comparison.  Prints one JSON line: syndromes/s
and stabilizer updates/s of each, the tuned shapes, and whether the plan's
and the fixed-shape call's classes and sums equal the ragged call's.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

LS = (5, 9, 13, 17, 25)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--p", type=float, default=0.14)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args(argv)

    import torch
    import paper_1302_2669_gb300 as P
    from paper_1302_2669_gb300 import build as b
    b.build()
    n, p, R = args.n, args.p, 4
    rng = np.random.default_rng(3001)
    Ls = rng.choice(LS, size=n).astype(np.int32)
    ctx = P.Context(0)
    like = torch.zeros(1, device="cuda")
    rows = [None] * n
    per_size = {}
    for L in LS:
        g, _ = ctx.gen_syndromes(3001, 0, n, L, p, like=like)
        idx = np.nonzero(Ls == L)[0]
        per_size[L] = g[torch.from_numpy(idx).cuda()].contiguous()
        gh = g.cpu().numpy()
        for i in idx:
            rows[i] = gh[i]
    cat = torch.from_numpy(np.concatenate(rows)).cuda()
    dLs = torch.from_numpy(Ls).cuda()
    sw = torch.from_numpy((Ls.astype(np.int64) ** 2).astype(np.uint32)).cuda()
    opts = P.Opts(chains_per_class=R, n_sweeps=int(max(LS)) ** 2)
    updates = float(sum(4 * R * int(L) ** 2 * 2 * int(L) * (int(L) - 1) for L in Ls))
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        return a.elapsed_time(e) / 1000.0 / args.reps

    out = {}
    tuned = {}
    if not args.no_autotune:
        for L in LS:
            lam, bps, grid = ctx.autotune(int(L), R, p, n_probe=max(1, int((Ls == L).sum())),
                                          sweeps=min(int(L) * int(L), 64))
            tuned[int(L)] = {"lanes_per_bundle": lam, "blocks_per_sm": bps,
                             "ms": {f"{a}x{b}": v for (a, b), v in grid.items() if v == v}}
        fixed_ctx = P.Context(0)
        t_fixed = timed(lambda: out.__setitem__("f", fixed_ctx.decode_ragged(cat, dLs, p, opts, n_sweeps=sw,
                                                                               seed=3101)))
    t_ragged = timed(lambda: out.__setitem__("r", ctx.decode_ragged(cat, dLs, p, opts, n_sweeps=sw, seed=3101)))
    if not args.no_autotune:
        same_fixed = bool((out["f"][0].cpu() == out["r"][0].cpu()).all()) and \
            bool((out["f"][1].cpu() == out["r"][1].cpu()).all())
        fixed_ctx.close()
    cls = torch.empty(n, dtype=torch.int32, device="cuda")
    csum = torch.empty((n, 4), dtype=torch.uint64, device="cuda")
    plan = P.RaggedPlan(ctx, dLs, p, cat, cls, csum, opts=opts, n_sweeps=sw, seed=3101)
    t_plan = timed(plan.launch)
    same = bool((cls.cpu() == out["r"][0].cpu()).all()) and bool((csum.cpu() == out["r"][1].cpu()).all())
    plan.close()

    def per_l():
        for L in LS:
            ctx.decode(per_size[L], L, p, P.Opts(chains_per_class=R, n_sweeps=L * L), seed=3101)

    t_perl = timed(per_l)
    counts = {int(L): int((Ls == L).sum()) for L in LS}
    line = {"metric": "ragged decoding throughput", "n": n, "p": p, "sizes": counts, "chains": "4 x 4",
            "sweeps": "L^2", "updates_per_batch": updates,
            "ragged": {"ms": t_ragged * 1e3, "syndromes_per_s": n / t_ragged, "updates_per_s": updates / t_ragged},
            "plan": {"ms": t_plan * 1e3, "syndromes_per_s": n / t_plan, "updates_per_s": updates / t_plan,
                     "equals_ragged": same},
            "per_L": {"ms": t_perl * 1e3, "syndromes_per_s": n / t_perl, "updates_per_s": updates / t_perl}}
    if tuned:
        line["tuned"] = tuned
        line["ragged_fixed_shape"] = {"ms": t_fixed * 1e3, "syndromes_per_s": n / t_fixed,
                                      "updates_per_s": updates / t_fixed, "equals_tuned": same_fixed}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
