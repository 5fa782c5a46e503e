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


# ------------------------------------------------------ streamed L (CC_FLAG_HOST_L)
@pytest.mark.parametrize("mode,chunk,a_block", [("ozaki_bf16", 40, 0), ("ozaki_bf16", 64, 7), ("ozaki_bf16", 150, 0),
                                                ("fp64", 33, 5), ("tf32", 50, 0), ("bf16", 29, 11)])
def test_streamed_L_parity(dev, oracle, mode, chunk, a_block):
    """L in page-locked host memory, copied to the device in chunks of `chunk` Cholesky vectors
    (ragged last chunk) on a second stream, the integrals of every block summed over the chunks."""
    o, v, n = 5, 37, 150
    rng = np.random.default_rng(25)
    L = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=True, rng=rng)
    R_ref = oracle.ladder(L, t2)
    E_ref = oracle.energy(R_ref, t2)
    R, E = B.ladder_forward(pinned(L), torch.from_numpy(t2).to(dev), mode=mode, symmetric=True, host_L=True,
                            chol_chunk=chunk, a_block=a_block, energy=True)
    assert R.device.type == "cuda"
    assert rel(R.cpu().numpy(), R_ref) < TOL[mode], (mode, chunk, rel(R.cpu().numpy(), R_ref))
    assert abs(float(E) - E_ref) < TOL[mode] * abs(E_ref)
    # the same as the device-resident call up to rounding: the chunks split the integral build's
    # contraction, so the emulated mode rounds each chunk's low levels to the fixed-point grid once more
    if mode in ("ozaki_bf16", "fp64"):
        Rd = B.ladder_forward(torch.from_numpy(L).to(dev), torch.from_numpy(t2).to(dev), mode=mode, symmetric=True,
                              a_block=a_block)
        assert rel(R.cpu().numpy(), Rd.cpu().numpy()) < (2e-11 if mode == "ozaki_bf16" else 1e-13)


def test_streamed_L_with_host_amplitudes_and_budget(dev, oracle):
    """Everything on the host: L streamed, t2 and R read and written over the host link, with a
    budget small enough to force chunks of L, blocks of pairs and blocks of `a`."""
    o, v, n = 7, 40, 300
    rng = np.random.default_rng(26)
    L = synth.cholesky_vectors(n, v, symmetric=True, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=True, rng=rng)
    R_ref = oracle.ladder(L, t2)
    budget = 6 << 20
    plan = B.plan(o, v, n, mode="ozaki_bf16", symmetric=True, budget=budget, host_t2r=True, host_L=True)
    assert plan["n_blocks"] > 1 and plan["pair_blocks"] > 1
    R = B.ladder_forward(pinned(L), pinned(t2), mode="ozaki_bf16", symmetric=True, host_t2r=True, host_L=True,
                         budget=budget, device=dev)
    torch.cuda.synchronize()
    assert R.device.type == "cpu"
    assert rel(R.numpy(), R_ref) < TOL["ozaki_bf16"]


def test_streamed_L_rejects_device_L_and_unpacked(dev):
    lib = _lib.load()
    o, v, n = 3, 16, 20
    L, t2 = synth.ladder_inputs(o, v, n, seed=27)
    Lg, tg = torch.from_numpy(L).to(dev), torch.from_numpy(t2).to(dev)
    R = torch.empty_like(tg)
    a = B.make_args(o, v, n, "ozaki_bf16", "auto", True, host_L=True)
    ws = ctypes.c_size_t()
    assert lib.cc_ladder_workspace_size_ex(ctypes.byref(a), ctypes.byref(ws)) == 0
    w = B.alloc_workspace(ws.value, dev)
    a.L, a.t2, a.R = B._ptr(Lg), B._ptr(tg), B._ptr(R)
    a.workspace, a.ws_bytes, a.stream = B._ptr(w), w.numel(), B._stream(dev)
    assert lib.cc_ladder_fwd_ex(ctypes.byref(a)) == -9  # device L with the host flag: CC_ERR_ARG
    b = B.make_args(o, v, n, "ozaki_bf16", "auto", False, host_L=True)
    assert lib.cc_ladder_workspace_size_ex(ctypes.byref(b), ctypes.byref(ws)) == -6  # CC_ERR_UNSUPPORTED
