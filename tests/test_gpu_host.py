"""Host-resident amplitudes (CC_FLAG_HOST_T2R): t2 and R stay in page-locked host memory and are
read / written by the kernels over the host link, the device holding one block of pairs at a time
(for problems whose o^2 v^2 exceeds device memory).  Parity against the FP64 CPU oracle with
budgets small enough to force many pair blocks and integral blocks."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2310_04559_gb300 import _lib
from paper_2310_04559_gb300 import binding as B
from paper_2310_04559_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki_bf16": 1e-10, "tf32": 1e-2, "bf16": 5e-2}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def pinned(x):
    return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()


@pytest.mark.parametrize("mode,budget,pblocks", [("ozaki_bf16", 0, 1), ("ozaki_bf16", 2700 << 10, 15),
                                                ("fp64", 0, 1), ("fp64", 4100 << 10, 8), ("tf32", 3500 << 10, 23)])
def test_host_resident_parity(dev, oracle, mode, budget, pblocks):
    o, v, n = 9, 40, 70
    plan = B.plan(o, v, n, mode=mode, symmetric=True, budget=budget, host_t2r=True)
    assert plan["pair_blocks"] == pblocks  # the budget forces this many blocks of pairs
    rng = np.random.default_rng(21)
    L = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=True, rng=rng)
    R_ref = oracle.ladder(L, t2)
    Lg = torch.from_numpy(L).to(dev)
    R = B.ladder_forward(Lg, pinned(t2), mode=mode, symmetric=True, host_t2r=True, budget=budget)
    torch.cuda.synchronize()
    assert R.device.type == "cpu" and R.is_pinned()
    assert rel(R.numpy(), R_ref) < TOL[mode], (mode, budget, rel(R.numpy(), R_ref))


def test_host_resident_accumulate_energy(dev, oracle):
    o, v, n = 6, 33, 50
    L, t2 = synth.ladder_inputs(o, v, n, seed=22)
    R_ref = oracle.ladder(L, t2)
    E_ref = oracle.energy(R_ref, t2)
    Lg = torch.from_numpy(L).to(dev)
    R0 = np.random.default_rng(23).standard_normal(t2.shape)
    R = pinned(R0)
    B.ladder_forward(Lg, pinned(t2), R=R, mode="ozaki_bf16", symmetric=True, accumulate=True, host_t2r=True,
                     budget=4 << 20)
    torch.cuda.synchronize()
    assert rel(R.numpy() - R0, R_ref) < 1e-9
    R, E = B.ladder_forward(Lg, pinned(t2), mode="ozaki_bf16", symmetric=True, host_t2r=True, energy=True)
    torch.cuda.synchronize()
    assert abs(float(E.cpu()) - E_ref) / abs(E_ref) < 1e-10
    # the same call with device tensors gives the same R
    Rd = B.ladder_forward(Lg, torch.from_numpy(t2).to(dev), mode="ozaki_bf16", symmetric=True).cpu().numpy()
    assert rel(R.numpy(), Rd) < 1e-13


def test_host_flag_rejects_device_pointers(dev):
    """The library checks the pointers itself: device t2 / R with the host flag is CC_ERR_ARG,
    and the host flag without pair symmetry is CC_ERR_UNSUPPORTED."""
    lib = _lib.load()
    o, v, n = 3, 16, 20
    L, t2 = synth.ladder_inputs(o, v, n, seed=24)
    Lg, tg = torch.from_numpy(L).to(dev), torch.from_numpy(t2).to(dev)
    R = torch.empty_like(tg)
    a = B.make_args(o, v, n, "ozaki_bf16", "auto", True, host_t2r=True)
    ws = ctypes.c_size_t()
    assert lib.cc_ladder_workspace_size_ex(ctypes.byref(a), ctypes.byref(ws)) == 0
    w = B.alloc_workspace(ws.value, dev)
    a.L, a.t2, a.R = B._ptr(Lg), B._ptr(tg), B._ptr(R)
    a.workspace, a.ws_bytes, a.stream = B._ptr(w), w.numel(), B._stream(dev)
    assert lib.cc_ladder_fwd_ex(ctypes.byref(a)) == -9  # CC_ERR_ARG
    b = B.make_args(o, v, n, "ozaki_bf16", "auto", False, host_t2r=True)
    assert lib.cc_ladder_workspace_size_ex(ctypes.byref(b), ctypes.byref(ws)) == -6  # CC_ERR_UNSUPPORTED
