"""Autotuner: timed trials of both contraction orders, the recorded choice used by
order="auto", and the on-disk record (CC_LADDER_CACHE) read back by a new process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2310_04559_gb300 import binding as B
from paper_2310_04559_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_picks_the_faster_order_and_is_used(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    # o=4, v=96, n=480: the Cholesky-first order needs 3x fewer flops
    o, v, n = 4, 96, 480
    L, t2 = synth.ladder_inputs(o, v, n, seed=21)
    Lg, tg = torch.from_numpy(L).to(dev), torch.from_numpy(t2).to(dev)
    res = B.autotune(Lg, tg, mode="ozaki_bf16", symmetric=True, budget=8 << 30)
    t_if, t_cf = res["ms_integral_first"], res["ms_cholesky_first"]
    assert t_if > 0 and t_cf > 0
    assert res["order"] == ("cholesky_first" if t_cf < t_if else "integral_first")
    # order="auto" now follows the recorded decision, and the result is right
    assert B.plan(o, v, n, mode="ozaki_bf16", symmetric=True, budget=8 << 30)["order"] == res["order"]
    R = B.ladder_forward(Lg, tg, mode="ozaki_bf16", symmetric=True, budget=8 << 30).cpu().numpy()
    R_ref = oracle.ladder(L, t2)
    assert np.linalg.norm(R - R_ref) / np.linalg.norm(R_ref) < 1e-10


def test_autotune_record_persists(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = str(tmp_path / "ladder_tune.txt")
    env = dict(os.environ, CC_LADDER_CACHE=cache, PYTHONPATH=ROOT)
    tune = ("import torch, json\n"
            "from paper_2310_04559_gb300 import binding as B, synth\n"
            "L, t = synth.ladder_inputs(3, 40, 90, seed=2)\n"
            "r = B.autotune(torch.from_numpy(L).cuda(), torch.from_numpy(t).cuda(), mode='fp64', budget=1<<30)\n"
            "print(json.dumps(r))\n")
    out = subprocess.run([sys.executable, "-c", tune], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    chosen = json.loads(out.stdout.strip().splitlines()[-1])["order"]
    fields = open(cache).read().split()
    assert fields[:5] == ["3", "40", "90", "0", "0"] and fields[5] in ("1", "2")
    # a fresh process reads the record back (plan queries need no GPU work)
    query = ("from paper_2310_04559_gb300 import binding as B\n"
             "print(B.plan(3, 40, 90, mode='fp64', budget=1<<30)['order'])\n")
    out = subprocess.run([sys.executable, "-c", query], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip().splitlines()[-1] == chosen
