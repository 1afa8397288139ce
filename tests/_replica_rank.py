"""One gloo rank of tests/test_replicas_cpu.py (run as a subprocess)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

ws, rank, _ = bench.dist_init()
assert dist.get_backend() == "gloo"
probs, _ = bench.make_batch_problems(3, rank)
goals = [p.muN[:2].tolist() for p in probs]
t = bench.max_over_ranks(ws, 1.5 + rank)
bench.barrier(ws)
gathered = [None] * ws
dist.all_gather_object(gathered, goals)
if rank == 0:
    print(json.dumps({"t": t, "goals": gathered}), flush=True)
dist.destroy_process_group()
