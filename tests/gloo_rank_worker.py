"""One rank of the sharded decode, started by shard.spawn_ranks under
torch.distributed.run with the gloo backend (CPU).  Each rank decodes
N_PER_RANK syndromes with the oracle (ids rank * N_PER_RANK ..), the ranks
all-gather their decisions and sum their failure counts, and rank 0 writes
both to the file named on the command line.  Not collected by pytest; run by
tests/test_shard_gloo.py."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L, P, K, R, SWEEPS, BURN, N_PER_RANK = 5, 0.15, 4, 4, 60, 12, 7
SYN_SEED, DEC_SEED = 1001, 1101


def main(out_path):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_1302_2669_gb300 import shard
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    assert world == int(os.environ["WORLD_SIZE"])
    id0 = shard.weak_id0(rank, N_PER_RANK)
    syn, tc = O.gen_syndromes(SYN_SEED, id0, N_PER_RANK, L, P)
    dec = [O.decode_one(L, P, K, R, SWEEPS, DEC_SEED, id0 + i, syn[i], burn_in=BURN, anneal_stages=4,
                        anneal_beta0=0.3)["cls"] for i in range(N_PER_RANK)]
    dec = torch.tensor(dec, dtype=torch.int32)
    fails = int((dec != torch.from_numpy(tc)).sum())
    allp = shard.all_gather_rows(dec)
    tot = shard.sum_counts([fails, N_PER_RANK])
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"world": world, "decisions": allp.tolist(), "failures": tot[0], "syndromes": tot[1]}, f)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1])
