"""Sharding of syndromes over two CPU ranks (gloo): the merged failure counts
of the sharded run equal those of one process decoding every syndrome.  Each
rank decodes its share with the oracle, keyed by global syndrome id."""
import os
import socket

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
