#!/usr/bin/env python3
"""Throughput of the single-temperature MCMC decoder (arXiv:1302.2669, Sec. IV.A).

Workload (one step = one decode call over one resident batch): planar code
L = 13 (313 qubits), depolarizing p cycling through 0.10, 0.13, 0.16, 0.18,
16,384 seeded synthetic syndromes per batch, 4 classes x 16 chains, 20,000
sweeps per chain (= 312 proposals each), of which the first 4,000 prepare
the start by annealing from 0.1 beta_bar to beta_bar in 16 stages and are
not sampled.  Metric: syndromes decoded per second
(and stabilizer updates per second = proposals, accepted or not), with the
logical error rate of the decoded batches beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain C, one process per syndrome on
the host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L = 13
PS = [0.10, 0.13, 0.16, 0.18]
SYN_SEEDS = [2010, 2013, 2016, 2018]
N_PER_STEP = 16384
K_CLASSES = 4
R_CHAINS = 16
SWEEPS = 20000
BURN_IN = 4000         # not sampled; annealed from ANNEAL_BETA0 beta_bar in ANNEAL_STAGES stages
ANNEAL_STAGES = 16
ANNEAL_BETA0 = 0.1
NQ = 2 * L * L - 2 * L + 1
NSTAB = 2 * L * (L - 1)
UPDATES_PER_SYNDROME = K_CLASSES * R_CHAINS * SWEEPS * NSTAB
WORKLOAD = (f"planar surface code L={L} ({NQ} qubits), depolarizing p cycling {PS}, {N_PER_STEP} syndromes "
            f"per step, {K_CLASSES} classes x {R_CHAINS} chains, {SWEEPS} sweeps (first {BURN_IN} annealed "
            f"from {ANNEAL_BETA0} beta_bar in {ANNEAL_STAGES} stages, not sampled)")
METRIC = "syndromes decoded/sec & stabilizer updates/sec at matched logical error rate"
SM_COUNT = 152
INT_LANES_PER_SM = 128


# DRAM bytes (read + write) of one sampled sweep launch per syndrome of the
# L = 13, 4 x 16-chain workload, from one ncu capture at 8,192 syndromes
# (41,110,784 B read + 3,584 B written: the bit-sliced chain state handed
# over from the last annealing launch, proportional to the syndromes).
SWEEP_DRAM_BYTES_PER_SYNDROME = (41110784 + 3584) / 8192


def ops_per_update() -> float:
    """Algorithmic integer operations per proposal of one chain in the
    bit-sliced formulation (32 chains per word): 28 bitwise ops to classify
    Delta n and apply the flip, 6 digit planes to decide the Metropolis test
    of a 32-chain word (10 ops of Philox4x32-10 per 32-bit plane + 6 compare
    ops), and the carry-save recount of n after each colour phase (3 ops per
    qubit, spread over the phase's n_stab/4 proposals)."""
    per_word = 28 + 6 * (10 + 6) + 3.0 * NQ / (NSTAB / 4)
    return per_word / 32.0


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples (the bench line carries their summary); directory
        # from SURFMCMC_CLOCKS_DIR, else the system's temporary directory
        self.path = os.path.join(os.environ.get("SURFMCMC_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def parity_ids(n: int, per_p: int = 4):
    """Syndrome indices of the batch checked against the oracle: spread over
    the batch, first and last included."""
    if n <= per_p:
        return list(range(n))
    return sorted({(j * (n - 1)) // (per_p - 1) for j in range(per_p)})


def cpu_baseline(ids_per_p, sweeps=SWEEPS, id0=0):
    """The oracle as it stands, one process per syndrome on the host cores,
    on the syndromes `ids_per_p[i]` (batch indices) of p = PS[i], at full
    length.  Returns the timing record and the oracle's decodes per p."""
    import multiprocessing as mp

    import oracle as O
    cores = os.cpu_count() or 1
    jobs, where = [], []
    for i, (p, s) in enumerate(zip(PS, SYN_SEEDS)):
        for j in ids_per_p[i]:
            syn, _ = O.gen_syndromes(s, id0 + j, 1, L, p)
            jobs.append((p, s, id0 + j, syn[0]))
            where.append((i, j))
    burn = BURN_IN * sweeps // SWEEPS
    stages = ANNEAL_STAGES if burn >= ANNEAL_STAGES else 0
    burn = burn if stages else 0
    work = [(L, p, K_CLASSES, R_CHAINS, sweeps, s + 100, ident, syn, burn, 1.0, stages, ANNEAL_BETA0, 0, 0, None)
            for p, s, ident, syn in jobs]
    procs = min(cores, len(work))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(O._decode_worker, work, chunksize=1)
    dt = time.perf_counter() - t0
    n_syn = len(jobs)
    out = {i: {} for i in range(len(PS))}
    for (i, j), r in zip(where, res):
        out[i][j] = r
    rec = {"value": n_syn / dt, "unit": "syndromes/s", "cores": procs,
           "kind": "oracle",
           "sample": f"{n_syn} syndromes of the workload ({', '.join(str(len(x)) for x in ids_per_p)} at p = "
                     f"{', '.join(str(p) for p in PS)}; L={L}, {K_CLASSES}x{R_CHAINS} chains, {sweeps} sweeps), "
                     "one process per syndrome",
           "updates_per_s": n_syn * UPDATES_PER_SYNDROME * sweeps / SWEEPS / dt, "seconds": dt}
    return rec, out


def early_stop_leg():
    """The learned early stop (batched decoding with the network) against
    plain long chains, measured inside the run: L = 17, a network
    trained from seeds on 2^20 syndromes labelled by the library's own
    chains (p stratified over [0.08, 0.18]), tau calibrated per p on 65,536
    validation syndromes, then plain long chains (4 x 4 chains, 20,000
    sweeps, the first 4,000 annealed in 16 stages from 0.1 beta_bar) and
    the early-stopped decode (checkpoints every 500 sweeps after the
    burn-in) timed on 65,536 fresh test syndromes at p = 0.10 and 0.14
    (CUDA events, one call each after a warm-up call)."""
    import argparse
    from paper_1302_2669_gb300 import early_stop as E
    ns = argparse.Namespace(L=17, train=1 << 20, val=65536, test=65536, p_lo=0.08, p_hi=0.18, n_p=32, label_R=4,
                            label_sweeps=4000, epochs=16, batch=1024, lr=2e-3, lr_final=1e-4, R=4, sweeps=20000,
                            burn_in=4000, anneal_stages=16, anneal_beta0=0.1, chunk=500, seed=4001,
                            eval_ps=[0.10, 0.14], reorder=False)
    t0 = time.perf_counter()
    res = E.run(ns, log=lambda m: None)
    keys = ("p", "tau", "syn_per_s_long", "syn_per_s_early", "gain", "ler_long", "ler_early", "sigma",
            "within_1sigma", "mean_sweeps_early", "stopped_at_first_checkpoint")
    return {"L": ns.L, "train_syndromes": ns.train, "epochs": ns.epochs, "label_chains": res["label_chains"],
            "long_chain": res["long_chain"], "chunk_sweeps": ns.chunk, "val": ns.val, "test": ns.test,
            "final_loss": res["losses"][-1], "label_seconds": res["label_seconds"],
            "train_seconds": res["train_seconds"], "cnn_forward_syn_per_s": res["cnn_forward_syn_per_s"],
            "per_p": [{k: r[k] for k in keys} for r in res["per_p"]], "seconds": time.perf_counter() - t0}


def compare_parity(orc, last, ids_per_p):
    """Element-by-element comparison of the GPU's decisions and class sums
    with the oracle's on the sampled syndromes of every p."""
    checked, bad = 0, []
    for i, p in enumerate(PS):
        cls, sums = last[i][0].cpu().numpy(), last[i][1].cpu().numpy()
        for j in ids_per_p[i]:
            r = orc[i][j]
            checked += 1
            if int(cls[j]) != int(r["cls"]) or not (sums[j].astype("uint64") == r["class_sum"]).all():
                bad.append({"p": p, "index": j})
    return {"checked": checked, "mismatches": len(bad), "ps": PS, "indices": ids_per_p,
            "compared": "decided class and the 4 class sums, bit for bit", "bad": bad[:8]}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    times = []
    per_p = max(1, cores // len(PS))
    for step in range(args.warmup + args.steps):
        # a different sample of the batch every step: ids step*per_p ..
        ids = [list(range(step * per_p, (step + 1) * per_p)) for _ in PS]
        r, _ = cpu_baseline(ids)
        if step >= args.warmup:
            times.append(r["seconds"])
    cores = per_p * len(PS)
    total = sum(times)
    value = cores * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "updates_per_s": value * UPDATES_PER_SYNDROME,
            "config": {"workload": WORKLOAD, "sample_per_step": f"{cores} syndromes", "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": cores, "kind": "oracle",
                             "sample": f"{cores} syndromes per step, full length"},
            "e2e": {"value": value, "unit": "syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_PER_STEP, help="syndromes per step (default: the workload's)")
    ap.add_argument("--sweeps", type=int, default=SWEEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-early-stop", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    from paper_1302_2669_gb300 import shard
    if "WORLD_SIZE" not in os.environ:
        import torch
        have = torch.cuda.device_count()
        if have < args.gpus:
            print(f"bench.py: --gpus {args.gpus} needs {args.gpus} GPUs, this machine has {have}", file=sys.stderr)
            return 2
        if args.gpus > 1:
            # one process per GPU: this command again under torch.distributed.run
            return shard.spawn_ranks(args.gpus, os.path.abspath(__file__), sys.argv[1:])

    import torch
    import paper_1302_2669_gb300 as pkg
    from paper_1302_2669_gb300 import build as b

    rank, world, local = dist_env()
    if world != args.gpus:
        print(f"bench.py: WORLD_SIZE={world} but --gpus {args.gpus}", file=sys.stderr)
        return 2
    if world > 1:
        import torch.distributed as dist
        # NCCL's initialisation log (communicator size and ranks) on stderr
        os.environ.setdefault("NCCL_DEBUG", "INFO")
        os.environ.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        os.environ.setdefault("NCCL_DEBUG_FILE", "/dev/stderr")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        print(f"bench.py: rank {rank} of {dist.get_world_size()} on cuda:{local} ({dist.get_backend()})",
              file=sys.stderr, flush=True)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    b.build()
    ctx = pkg.Context(local)
    n, sweeps = args.n, args.sweeps
    burn = BURN_IN * sweeps // SWEEPS       # the same share of a reduced run
    if burn < ANNEAL_STAGES:
        burn = 0
    opts = pkg.Opts(n_classes=K_CLASSES, chains_per_class=R_CHAINS, n_sweeps=sweeps, burn_in=burn,
                    anneal_stages=ANNEAL_STAGES if burn >= ANNEAL_STAGES else 0, anneal_beta0=ANNEAL_BETA0)
    id0 = shard.weak_id0(rank, n)
    like = torch.zeros(1, device=dev)
    syn, tcls = [], []
    for p, s in zip(PS, SYN_SEEDS):
        a, t = ctx.gen_syndromes(s, id0, n, L, p, like=like)
        syn.append(a)
        tcls.append(t)
    out_cls = torch.empty(n, dtype=torch.int32, device=dev)
    out_sum = torch.empty((n, K_CLASSES), dtype=torch.uint64, device=dev)
    out_lr = torch.empty((n, K_CLASSES), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def step(j):
        i = j % 4
        ctx.decode(syn[i], L, PS[i], opts, seed=SYN_SEEDS[i] + 100, id0=id0, out_class=out_cls,
                   out_class_sum=out_sum, out_log_ratio=out_lr)
        return i

    # the decisions of the last decode of each p (copied after the step's
    # end event, outside the timed region)
    last = {}

    def keep(i):
        last[i] = (out_cls.clone(), out_sum.clone())

    for j in range(args.warmup):
        keep(step(j))
    torch.cuda.synchronize()

    fails = {p: [0, 0] for p in PS}
    ctx.set_timing(True)
    ctx.sweep_time()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    for j in range(args.warmup, args.warmup + args.steps):
        flush.fill_(j)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        i = step(j)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        fails[PS[i]][0] += int((out_cls != tcls[i]).sum())
        fails[PS[i]][1] += n
        keep(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    sweep_ms, sweep_launches = ctx.sweep_time()
    ctx.set_timing(False)
    total_ms = shard.max_value(sum(step_ms), device=dev)
    merged = shard.sum_counts([v for p in PS for v in fails[p]], device=dev)
    fails = {p: merged[2 * i:2 * i + 2] for i, p in enumerate(PS)}
    for i in range(len(PS)):   # a p that no step reached (fewer than four steps)
        if i not in last:
            keep(step(i))
    # all-gather of the per-syndrome decisions: the job's decisions in id
    # order on every rank, and their failures recounted from them
    gathered = {}
    for i, p in enumerate(PS):
        dec = shard.all_gather_rows(last[i][0], device=dev)
        tru = shard.all_gather_rows(tcls[i], device=dev)
        gathered[p] = {"syndromes": int(dec.numel()), "failures": int((dec != tru).sum())}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hsyn = [s.cpu().pin_memory() for s in syn]
        hcls = torch.empty(n, dtype=torch.int32).pin_memory()
        hsum = torch.empty((n, K_CLASSES), dtype=torch.uint64).pin_memory()
        hlr = torch.empty((n, K_CLASSES), dtype=torch.float64).pin_memory()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for j in range(args.warmup, args.warmup + args.steps):
            i = j % 4
            ctx.decode(hsyn[i], L, PS[i], opts, seed=SYN_SEEDS[i] + 100, id0=id0, out_class=hcls, out_class_sum=hsum,
                       out_log_ratio=hlr)
        e2e_s = shard.max_value(time.perf_counter() - t0, device=dev)
        e2e = {"value": world * n * args.steps / e2e_s, "unit": "syndromes/s", "h2d_bytes_per_step": n * NSTAB,
               "d2h_bytes_per_step": n * (4 + 8 * K_CLASSES + 8 * K_CLASSES)}

    if rank != 0:
        return 0
    value = world * n * args.steps / (total_ms / 1000.0)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = SM_COUNT * INT_LANES_PER_SM * sm_max * 1e6
    # the sweep kernel runs once per annealing stage and once for the sampled
    # sweeps; its achieved rate is the whole step's proposals over the summed
    # sweep-kernel time
    sweep_s_per_step = (sweep_ms / args.steps) / 1000.0
    updates_per_step = n * UPDATES_PER_SYNDROME * sweeps / SWEEPS
    achieved = updates_per_step * ops_per_update() / sweep_s_per_step
    line = {
        "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "updates_per_s": value * UPDATES_PER_SYNDROME * sweeps / SWEEPS,
        "config": {"workload": WORKLOAD if (n == N_PER_STEP and sweeps == SWEEPS) else
                   f"reduced: L={L}, {n} syndromes per step, {sweeps} sweeps",
                   "L": L, "p": PS, "syndromes_per_step": n, "classes": K_CLASSES, "chains_per_class": R_CHAINS,
                   "sweeps": sweeps, "burn_in": burn, "anneal": {"stages": ANNEAL_STAGES, "beta0": ANNEAL_BETA0},
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"shard{world}" if world > 1 else "single GPU"},
        "ler": {f"{p:.2f}": {"ler": f / max(m, 1), "sigma": math.sqrt(max(f / max(m, 1) * (1 - f / max(m, 1)), 0)
                                                                     / max(m, 1)), "syndromes": m}
                for p, (f, m) in fails.items() if m},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "frac": achieved / peak_ops,
                     "traffic": SWEEP_DRAM_BYTES_PER_SYNDROME * n,
                     "traffic_unit": "bytes per sampled sweep launch",
                     "kernel": "sweep_kernel", "ops_per_update": ops_per_update(),
                     "kernel_ms_per_step": sweep_s_per_step * 1000.0, "kernel_launches": sweep_launches,
                     "peak_basis": f"{SM_COUNT} SMs x {INT_LANES_PER_SM} int32 lanes x {sm_max:.0f} MHz "
                                   "(max SM clock of measured peaks)"},
        "gpu_launches": (2 + sweep_launches // args.steps) * args.steps,
        "clocks": clk,
        "e2e": e2e,
    }
    line["decisions"] = {"gathered_over_ranks": world, "per_p": {f"{p:.2f}": v for p, v in gathered.items()}}
    if not args.no_early_stop:
        ctx.close()
        line["early_stop"] = early_stop_leg()
    ids = [parity_ids(n) for _ in PS]
    if (world == 1 and not args.no_cpu_baseline) or not args.no_parity:
        rec, orc = cpu_baseline(ids, sweeps=sweeps, id0=id0)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = rec
        if not args.no_parity:
            line["parity"] = compare_parity(orc, last, ids)
    print(json.dumps(line), flush=True)
    if args.no_early_stop:
        ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
