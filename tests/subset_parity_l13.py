"""Bit-exact comparison of the benchmark workload's first syndromes with the
CPU oracle, at full length: the 256-syndrome subset per error rate.

    python tests/subset_parity_l13.py [--n-check 256] [--ps 0.10,0.13,0.16,0.18]

The benchmark's configuration: planar code L = 13, 16,384 syndromes per error
rate (syndrome seeds 2010/2013/2016/2018, decoder seed + 100), 4 classes x 16
chains, 20,000 sweeps, the first 4,000 annealed in 16 stages from
0.1 beta_bar.  The GPU decodes the whole batch in the benchmark's launch
configuration; the oracle decodes syndromes 0 .. n_check - 1 (one process per
syndrome on the host cores, about 18 core-seconds each), and every output is
compared: decided class, class sums, log-ratios, per-chain sums, final n and
final frames.  Prints one JSON line per error rate and exits non-zero on any
mismatch.  Too long for the test suite (about five minutes of 16 host cores
per error rate); run on its own.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SEEDS = {0.10: 2010, 0.13: 2013, 0.16: 2016, 0.18: 2018}
L, N, R, T, BURN, STAGES, BETA0 = 13, 16384, 16, 20000, 4000, 16, 0.1


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-check", type=int, default=256)
    ap.add_argument("--ps", default="0.10,0.13,0.16,0.18")
    args = ap.parse_args(argv)
    import numpy as np
    import torch

    import oracle as O
    import paper_1302_2669_gb300 as P
    from paper_1302_2669_gb300 import build as b
    b.build()
    ctx = P.Context(0)
    opts = P.Opts(chains_per_class=R, n_sweeps=T, burn_in=BURN, anneal_stages=STAGES, anneal_beta0=BETA0)
    bad_total = 0
    for p in [float(x) for x in args.ps.split(",")]:
        seed = SEEDS[round(p, 2)]
        syn, _ = O.gen_syndromes(seed, 0, N, L, p)
        t0 = time.perf_counter()
        out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=seed + 100, id0=0)
        torch.cuda.synchronize()
        t_gpu = time.perf_counter() - t0
        g = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
        idx = list(range(args.n_check))
        t0 = time.perf_counter()
        refs = O.decode_batch(L, p, 4, R, T, seed + 100, idx, syn[idx], burn_in=BURN, anneal_stages=STAGES,
                              anneal_beta0=BETA0)
        t_cpu = time.perf_counter() - t0
        bad = []
        for i, ref in zip(idx, refs):
            same = (int(g["cls"][i]) == ref["cls"] and (g["class_sum"][i] == ref["class_sum"]).all()
                    and (g["log_ratio"][i] == ref["log_ratio"]).all()
                    and (g["chain_sum"][i] == ref["chain_sum"]).all()
                    and (g["chain_n"][i] == ref["chain_n"]).all()
                    and (g["chain_frames"][i][:, 0, :] == O.pack_bits(ref["frames_x"])).all()
                    and (g["chain_frames"][i][:, 1, :] == O.pack_bits(ref["frames_z"])).all())
            if not same:
                bad.append(i)
        bad_total += len(bad)
        print(json.dumps({"p": p, "checked": len(idx), "mismatches": len(bad), "first_bad": bad[:8],
                          "compared": "class, class sums, log-ratios, per-chain sums, final n, final frames",
                          "gpu_seconds_for_the_batch": t_gpu, "oracle_seconds": t_cpu,
                          "oracle_processes": os.cpu_count()}), flush=True)
    ctx.close()
    return 1 if bad_total else 0


if __name__ == "__main__":
    raise SystemExit(main())
