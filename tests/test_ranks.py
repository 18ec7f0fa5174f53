"""Host-side multi-rank logic (CPU only): the split of independent instances over ranks, and the
end-of-run reductions run as two gloo processes."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

from paper_1707_04333_gb300 import ranks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lpt_shards_cover_every_instance_once_and_balance():
    rng = np.random.default_rng(3)
    costs = rng.lognormal(10, 1.2, 64)
    for world in (1, 2, 3, 4, 8):
        parts = ranks.shard_instances(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [costs[p].sum() for p in map(np.array, parts)]
        assert max(loads) <= costs.sum() / world + costs.max() + 1e-6
        assert parts == ranks.shard_instances(list(costs), world)      # deterministic


def test_lpt_on_equal_costs_is_round_robin():
    assert ranks.shard_instances([1.0] * 6, 3) == [[0, 3], [1, 4], [2, 5]]


def test_reductions_without_a_process_group_return_the_value():
    assert ranks.max_over_ranks(2.5) == 2.5
    assert ranks.sum_over_ranks(7) == 7.0
    assert ranks.aggregate_rate(8e6, 100, 200.0) == 8e6 * 100 / 0.2


WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
from paper_1707_04333_gb300 import inputs, ranks
dist.init_process_group("gloo")
r, w = dist.get_rank(), dist.get_world_size()
ws = inputs.batched_pair_plasmas(n_inst=64, seed=5, scale=float(sys.argv[2]))
costs = [ranks.instance_cost(x.n_particles, len(x.mesh.triangles)) for x in ws]
mine = ranks.shard_instances(costs, w)[r]
n_mine = sum(ws[i].n_particles for i in mine)
ms = 100.0 + 50.0 * r                      # this rank's time
out = {"rank": r, "mine": mine, "n_mine": n_mine, "n_all": ranks.sum_over_ranks(n_mine),
       "ms_max": ranks.max_over_ranks(ms), "n_total": sum(x.n_particles for x in ws)}
dist.barrier()
print(json.dumps(out))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_split_the_batch_and_reduce():
    """World size 2 over gloo: the two ranks take disjoint shares of the 64-instance batch that
    together cover it, the summed particle count is the batch's, and both ranks see the slower
    rank's time."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT, "0.05"], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    a, b = sorted(outs, key=lambda x: x["rank"])
    assert set(a["mine"]).isdisjoint(b["mine"]) and sorted(a["mine"] + b["mine"]) == list(range(64))
    assert a["n_all"] == b["n_all"] == a["n_mine"] + b["n_mine"] == a["n_total"]
    assert a["ms_max"] == b["ms_max"] == 150.0
