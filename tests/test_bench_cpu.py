"""CPU checks of bench.py's host logic: the reference arm's JSON line, the
multi-rank timing reduction over gloo ranks (world size 2), and the clock
summary parser."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_json(capsys):
    bench.main(["--impl", "reference", "--workload", "o4_v24_n60", "--steps", "2", "--warmup", "3"])
    line = capsys.readouterr().out.strip().splitlines()[-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["unit"] == "TFLOP/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_warmup_floor():
    with pytest.raises(SystemExit):
        bench.main(["--impl", "reference", "--warmup", "2"])


def test_clock_summary_parser():
    c = bench.Clocks()
    c.lines = ["0, 1800, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active",
               "0, 1900, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 1900 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]


_WORKER = r'''
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank, local, world = bench.dist_init()
t = 1.0 + rank          # rank 1 is the slow one
m = bench.dist_max(t, world)
bench.dist_barrier(world)
print("RESULT", rank, world, m, flush=True)
dist.destroy_process_group()
'''


def test_two_rank_max_reduction(tmp_path):
    """torchrun-style env, gloo backend: every rank sees the max time."""
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT="29533", CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    res = sorted(l.split() for o in outs for l in o.splitlines() if l.startswith("RESULT"))
    assert [r[1:] for r in res] == [["0", "2", "2.0"], ["1", "2", "2.0"]], outs
