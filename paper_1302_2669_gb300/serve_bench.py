"""Serving benchmark: Poisson arrivals of single syndromes through the
library's continuous-batching server.

    python -m paper_1302_2669_gb300.serve_bench [--rate 20000] [--seconds 5]

Requests: L uniform over {9, 13, 17, 25}, depolarizing p = 0.12, sweeps = L^2
(the first quarter annealed from 0.3 beta_bar in 4 stages, not sampled),
4 classes x 4 chains.  Syndromes are seeded synthetic inputs made by the
library's generator before the run.  The same arrivals are served without a
memory budget and then under each of --memory-budgets (bytes of device
scratch; default 2 MiB, 512 KiB and 256 KiB), so that admission has to
shrink batches and, under the tighter budgets, wait for memory.  Prints one
JSON line with, per run, the offered and achieved rates, p50/p99/max
latency, batches and memory stalls.
"""
from __future__ import annotations

import argparse
import json
import threading
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=20000.0, help="offered requests per second")
    ap.add_argument("--seconds", type=float, default=5.0)
    ap.add_argument("--sizes", default="9,13,17,25")
    ap.add_argument("--p", type=float, default=0.12)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=1024)
    ap.add_argument("--max-wait-us", type=float, default=500.0)
    ap.add_argument("--memory-budgets", default="2097152,524288,262144",
                    help="comma-separated budgets of the runs after the unbudgeted one (empty: none)")
    ap.add_argument("--seed", type=int, default=5001)
    args = ap.parse_args(argv)

    import torch
    import paper_1302_2669_gb300 as pkg
    from paper_1302_2669_gb300 import build as b
    b.build()
    sizes = [int(x) for x in args.sizes.split(",")]
    n_req = int(args.rate * args.seconds)
    rng = np.random.default_rng(args.seed)
    Ls = rng.choice(sizes, size=n_req)
    gaps = rng.exponential(1.0 / args.rate, size=n_req)
    ctx = pkg.Context(0)
    like = torch.zeros(1, device="cuda")
    rows = {}
    for L in sizes:
        syn, _ = ctx.gen_syndromes(args.seed, 0, n_req, L, args.p, like=like)
        rows[L] = syn.cpu().numpy()
    ctx.close()
    opts = pkg.Opts(chains_per_class=4, n_sweeps=100, burn_in=25, anneal_stages=4, anneal_beta0=0.3)

    def serve(budget):
        srv = pkg.Server(0, args.p, opts, seed=args.seed + 100, max_batch=args.max_batch, slots=args.slots,
                         max_L=max(sizes), memory_budget=budget, max_wait_us=args.max_wait_us)
        lat = []
        done = threading.Event()

        def collect():
            got = 0
            while got < n_req:
                ids, cls, sums, l = srv.poll(max_results=8192, wait_us=20000)
                lat.extend(l.tolist())
                got += len(ids)
            done.set()

        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        t_next = t0
        for i in range(n_req):
            t_next += gaps[i]
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                if t_next - now > 2e-4:
                    time.sleep(t_next - now - 1e-4)
            L = int(Ls[i])
            srv.submit(i, L, L * L, rows[L][i])
        t_sub = time.perf_counter() - t0
        done.wait()
        t_all = time.perf_counter() - t0
        th.join()
        st = srv.stats()
        srv.close()
        lat_ms = np.array(lat) / 1000.0
        return {"memory_budget": budget, "submitted_rps": n_req / t_sub, "completed_rps": n_req / t_all,
                "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "max_ms": float(lat_ms.max()), "batches": st["batches"], "memory_stalls": st["memory_stalls"]}

    budgets = [int(x) for x in args.memory_budgets.split(",") if x.strip()]
    runs = [serve(0)] + [serve(b) for b in budgets if b > 0]
    line = {"metric": "serving latency and throughput", "offered_rps": args.rate, "requests": n_req,
            **{k: v for k, v in runs[0].items() if k != "memory_budget"},
            "runs": runs,
            "config": {"sizes": sizes, "p": args.p, "sweeps": "L^2 (first quarter annealed, 4 stages from 0.3)",
                       "chains": "4 classes x 4", "slots": args.slots, "max_batch": args.max_batch,
                       "max_wait_us": args.max_wait_us},
            "updates_per_request_mean": float(np.mean([16 * L * L * 2 * L * (L - 1) for L in Ls]))}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
