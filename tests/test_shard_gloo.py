"""Sharding of syndromes over two CPU ranks (gloo): the merged failure counts
of the sharded run equal those of one process decoding every syndrome.  Each
rank decodes its share with the oracle, keyed by global syndrome id."""
import json
import os
import socket
import subprocess
import sys

import pytest

from paper_1302_2669_gb300 import shard

L, P, K, R, SWEEPS, BURN, N = 5, 0.15, 4, 4, 60, 12, 14
SYN_SEED, DEC_SEED = 1001, 1101


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, cnt = shard.id_range(rank, world, N)
    syn, tc = O.gen_syndromes(SYN_SEED, start, cnt, L, P)
    fails = 0
    for i in range(cnt):
        d = O.decode_one(L, P, K, R, SWEEPS, DEC_SEED, start + i, syn[i], burn_in=BURN, anneal_stages=4,
                         anneal_beta0=0.3)
        fails += int(d["cls"] != tc[i])
    tot = shard.sum_counts([fails, cnt])
    tmax = shard.max_value(float(rank + 1))
    if rank == 0:
        with open(out_path, "w") as f:
            f.write(f"{tot[0]} {tot[1]} {tmax}")
    dist.barrier()
    dist.destroy_process_group()


def test_id_ranges_partition():
    for n in (0, 1, 7, 14, 100):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                s, c = shard.id_range(r, world, n)
                got += list(range(s, s + c))
            assert got == list(range(n))
    assert shard.weak_id0(3, 16384) == 3 * 16384
    with pytest.raises(ValueError):
        shard.id_range(2, 2, 5)


def test_two_rank_gloo_matches_single_process(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle as O
    out = tmp_path / "res.txt"
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    fails, cnt, tmax = out.read_text().split()
    syn, tc = O.gen_syndromes(SYN_SEED, 0, N, L, P)
    ref = sum(int(O.decode_one(L, P, K, R, SWEEPS, DEC_SEED, i, syn[i], burn_in=BURN, anneal_stages=4,
                               anneal_beta0=0.3)["cls"] != tc[i]) for i in range(N))
    assert int(cnt) == N and int(fails) == ref and float(tmax) == 2.0


def test_spawned_ranks_gather_the_decisions_of_one_process(tmp_path):
    """The rank-spawning path of bench.py (shard.spawn_ranks: two ranks under
    torch.distributed.run, gloo on CPU): the all-gathered decisions equal one
    process's decisions for the same ids, and the summed failures match."""
    pytest.importorskip("torch")
    import numpy as np

    import oracle as O
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, here)
    import gloo_rank_worker as W
    out = tmp_path / "gathered.json"
    env = dict(os.environ, PYTHONPATH=os.path.dirname(here), OMP_NUM_THREADS="1")
    rc = shard.spawn_ranks(2, os.path.join(here, "gloo_rank_worker.py"), [str(out)], env=env)
    assert rc == 0
    got = json.loads(out.read_text())
    n = 2 * W.N_PER_RANK
    syn, tc = O.gen_syndromes(W.SYN_SEED, 0, n, W.L, W.P)
    ref = [O.decode_one(W.L, W.P, W.K, W.R, W.SWEEPS, W.DEC_SEED, i, syn[i], burn_in=W.BURN, anneal_stages=4,
                        anneal_beta0=0.3)["cls"] for i in range(n)]
    assert got["world"] == 2 and got["syndromes"] == n
    assert got["decisions"] == ref
    assert got["failures"] == int((np.array(ref) != tc).sum())


def test_bench_refuses_more_gpus_than_present():
    """bench.py --gpus N on a machine with fewer than N GPUs exits with a
    clear error instead of printing a one-rank line."""
    torch = pytest.importorskip("torch")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    n = torch.cuda.device_count() + 1
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", str(n), "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 2
    assert f"--gpus {n} needs {n} GPUs" in r.stderr
    assert not r.stdout.strip()
