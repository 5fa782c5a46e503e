"""One problem over several ranks, on CPU with gloo (world size 2): the work-balanced
`a`-range partition that bench.py uses for N GPUs (cc_ladder_partition, host-only) gives
disjoint ranges covering [0, v) with balanced issued flops, and the ranks' shares of the pair
energy -- the terms with min(a, b) in each rank's range, computed by the oracle -- add up
under an all-reduce to the oracle's full energy."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2310_04559_gb300 import binding as B  # noqa: E402
from paper_2310_04559_gb300 import build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("o,v,n,parts", [(40, 400, 2000, 2), (40, 400, 2000, 8), (20, 200, 1000, 3),
                                         (60, 600, 3000, 4)])
def test_partition_balances_issued_flops(o, v, n, parts):
    b = B.partition(o, v, n, parts, mode="ozaki_bf16", symmetric=True)
    assert b[0] == 0 and b[-1] == v and all(b[g] < b[g + 1] for g in range(parts))
    fl = [B.plan(o, v, n, mode="ozaki_bf16", symmetric=True, a_range=(b[g], b[g + 1]))["flops_issued"]
          for g in range(parts)]
    full = B.plan(o, v, n, mode="ozaki_bf16", symmetric=True)["flops_issued"]
    assert abs(sum(fl) / full - 1) < 0.01  # the shards redo no work
    assert max(fl) / min(fl) < 1.05, fl


def test_partition_equal_counts_without_pair_symmetry():
    assert B.partition(4, 24, 60, 4, mode="fp64") == [0, 6, 12, 18, 24]
    assert B.partition(4, 5, 60, 5, mode="fp64") == [0, 1, 2, 3, 4, 5]
    from paper_2310_04559_gb300 import _lib
    with pytest.raises(_lib.LadderError):
        B.partition(4, 5, 60, 6, mode="fp64")  # more parts than `a` values


_WORKER = r'''
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import torch
import torch.distributed as dist
from oracle import oracle as O
from paper_2310_04559_gb300 import binding as B, synth
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
o, v, n = 3, 11, 17
L, t2 = synth.ladder_inputs(o, v, n, seed=5)
b = B.partition(o, v, n, world, mode="ozaki_bf16", symmetric=True)
R = O.ladder(L, t2)
e = torch.tensor([O.energy_range(R, t2, b[rank], b[rank + 1])], dtype=torch.float64)
dist.all_reduce(e)
print("RESULT", json.dumps({"rank": rank, "bounds": b, "e_sum": float(e[0]), "e_full": O.energy(R, t2)}),
      flush=True)
dist.destroy_process_group()
'''


def test_two_rank_shard_energies_sum_to_oracle_energy():
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT="29547", CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=180)[0] for p in procs]
    res = [json.loads(l.split(" ", 1)[1]) for o in outs for l in o.splitlines() if l.startswith("RESULT")]
    assert len(res) == 2, outs
    assert res[0]["bounds"] == res[1]["bounds"]
    b = res[0]["bounds"]
    assert b[0] == 0 and b[-1] == 11 and b[0] < b[1] < b[2]
    for r in res:
        assert abs(r["e_sum"] - r["e_full"]) <= 1e-13 * abs(r["e_full"]), r
