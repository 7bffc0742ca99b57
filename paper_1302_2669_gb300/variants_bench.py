"""Throughput and logical error rate of the decoder's variants.

    python -m paper_1302_2669_gb300.variants_bench [--reps 2]

One seeded batch per variant, decoded by the library (CUDA events on the
launching stream, after a warm-up call, device buffers), against the true
classes of the sampled errors:

  sweeps      planar code, depolarizing, colour sweeps (the default path)
  scan        the same with random scan (Sec. IV as written)
  ti          thermodynamic integration over 21 temperatures (Eq. 6)
  flips       independent bit and phase flips, beta* = 0.85 beta_bar
  general     general Pauli channel, energies (eX, eY, eZ) = (2, 3, 1),
              random scan
  toric       toric code, 16 classes

All at L = 9 (toric: L = 8), 4 chains per class, 400 sweeps of which the
first 100 are annealed in 4 stages from 0.3 beta_bar; and the small parity
configuration itself (small: L = 5, p = 0.15, 200 syndromes of seed 1001,
decoder seed 1101, 4 x 4 chains, 2,000 sweeps, no burn-in).  Prints one JSON
line per variant: syndromes/s, stabilizer updates/s (proposals; x 21 for
TI) and the logical error rate with its binomial sigma.
"""
from __future__ import annotations

import argparse
import json
import math


def general_channel_probs(p, e):
    """(pX, pY, pZ) of the general channel with total error probability p and
    integer energies e = (eX, eY, eZ): p_P = (1 - p) r^e_P with r the root of
    (1 - p) sum_P r^e_P = p (bisection; an input recipe only)."""
    lo, hi = 0.0, 1.0
    for _ in range(100):
        r = 0.5 * (lo + hi)
        if (1.0 - p) * sum(r ** k for k in e) < p:
            lo = r
        else:
            hi = r
    r = 0.5 * (lo + hi)
    return tuple((1.0 - p) * r ** k for k in e)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)

    import torch
    import paper_1302_2669_gb300 as P
    from paper_1302_2669_gb300 import build as b
    b.build()
    ctx = P.Context(0)
    like = torch.zeros(1, device="cuda")
    R, T, burn = 4, 400, 100
    base = dict(chains_per_class=R, n_sweeps=T, burn_in=burn, anneal_stages=4, anneal_beta0=0.3)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(name, L, p, n, syn, tc, fn, K, n_stab, factor=1, T=T, R=R):
        out = fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.reps):
            out = fn()
        e.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(e) / 1000.0 / args.reps
        cls = out[0]
        ler = float((cls != tc).float().mean())
        upd = n * K * R * T * n_stab * factor
        print(json.dumps({"variant": name, "L": L, "p": p, "syndromes": n, "classes": K, "chains_per_class": R,
                          "sweeps": T, "ms": t * 1e3, "syndromes_per_s": n / t, "updates_per_s": upd / t,
                          "ler": ler, "sigma": math.sqrt(max(ler * (1 - ler), 1e-12) / n)}), flush=True)

    L, p = 9, 0.10
    ns = 2 * L * (L - 1)
    syn, tc = ctx.gen_syndromes(9001, 0, 16384, L, p, like=like)
    o = P.Opts(**base)
    run("sweeps", L, p, 16384, syn, tc, lambda: ctx.decode(syn, L, p, o, seed=9101), 4, ns)
    s4, t4 = syn[:4096].contiguous(), tc[:4096].contiguous()
    o = P.Opts(**base, scan=1)
    run("scan", L, p, 4096, s4, t4, lambda: ctx.decode(s4, L, p, o, seed=9101), 4, ns)
    o = P.Opts(**base)
    run("ti", L, p, 4096, s4, t4, lambda: ctx.decode_ti(s4, L, p, o, n_beta=21, seed=9101), 4, ns, factor=21)

    pf = 0.05
    syn, tc = ctx.gen_syndromes(9002, 0, 16384, L, pf, like=like, noise=1)
    o = P.Opts(**base, noise=1, beta_scale=0.85)
    run("flips", L, pf, 16384, syn, tc, lambda: ctx.decode(syn, L, pf, o, seed=9102), 4, ns)

    eg = (2, 3, 1)
    px, py, pz = general_channel_probs(p, eg)
    syn, tc = ctx.gen_syndromes_pauli(9003, 0, 4096, L, px, py, pz, like=like)
    o = P.Opts(**base, noise=2, scan=1, pauli_energy=eg)
    run("general", L, p, 4096, syn, tc, lambda: ctx.decode(syn, L, p, o, seed=9103), 4, ns)

    Ls, ps, Ts = 5, 0.15, 2000
    syn, tc = ctx.gen_syndromes(1001, 0, 200, Ls, ps, like=like)
    o = P.Opts(chains_per_class=4, n_sweeps=Ts)
    run("small", Ls, ps, 200, syn, tc, lambda: ctx.decode(syn, Ls, ps, o, seed=1101), 4, 2 * Ls * (Ls - 1), T=Ts)

    Lt, pt = 8, 0.08
    syn, tc = ctx.gen_syndromes_toric(9004, 0, 16384, Lt, pt, like=like)
    o = P.Opts(**base, n_classes=16)
    run("toric", Lt, pt, 16384, syn, tc, lambda: ctx.decode(syn, Lt, pt, o, seed=9104), 16, 2 * Lt * Lt)
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
