"""cc_ladder_energy_noalloc: the pair energy for callers that cannot allocate
device memory (no workspace argument; its partial sums live in a fixed array
inside the library).  Checked through the C ABI against cc_ladder_energy, which
takes a caller workspace, on two calls in a row, and against the FP64 CPU oracle's
energy of the same R.  This file sorts last so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2310_04559_gb300 import _lib

pytestmark = pytest.mark.gpu


def _p(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else None


@pytest.mark.parametrize("o,v", [(4, 24), (7, 53), (40, 400), (300, 8)])
def test_noalloc_energy_matches_workspace_entry_point(oracle, o, v):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(o * 1000 + v)
    R = torch.randn((o, o, v, v), generator=g, dtype=torch.float64).to(dev)
    t2 = torch.randn((o, o, v, v), generator=g, dtype=torch.float64).to(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    # reference: the workspace entry point
    nbytes = ctypes.c_size_t()
    assert lib.cc_ladder_energy_workspace_size(o, v, ctypes.byref(nbytes)) == 0
    ws = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
    E_ref = torch.empty((), dtype=torch.float64, device=dev)
    ep_ref = torch.empty((o, o), dtype=torch.float64, device=dev)
    assert lib.cc_ladder_energy(o, v, _p(R), _p(t2), _p(E_ref), _p(ep_ref), _p(ws), ws.numel(), stream) == 0
    for _ in range(2):  # two calls in a row share the library's array
        E = torch.full((), float("nan"), dtype=torch.float64, device=dev)
        ep = torch.full((o, o), float("nan"), dtype=torch.float64, device=dev)
        assert lib.cc_ladder_energy_noalloc(o, v, _p(R), _p(t2), _p(E), _p(ep), stream) == 0
        E2 = torch.full((), float("nan"), dtype=torch.float64, device=dev)
        assert lib.cc_ladder_energy_noalloc(o, v, _p(R), _p(t2), _p(E2), None, stream) == 0
        torch.cuda.synchronize(dev)
        e, e_ref = float(E), float(E_ref)
        assert abs(e - e_ref) <= 1e-12 * abs(e_ref)
        assert abs(float(E2) - e_ref) <= 1e-12 * abs(e_ref)
        assert np.allclose(ep.cpu().numpy(), ep_ref.cpu().numpy(), rtol=1e-12, atol=0)
    # and the oracle's energy (Neumaier sums over the same R, in FP64 on the host)
    e_or, ep_or = oracle.energy(R.cpu().numpy(), t2.cpu().numpy(), pair=True)
    assert abs(float(E) - e_or) <= 1e-12 * np.abs(ep_or).sum()
    assert np.allclose(ep.cpu().numpy(), ep_or, rtol=1e-11, atol=1e-12 * np.abs(ep_or).max())


def test_noalloc_rejects_sizes_beyond_its_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    x = torch.zeros(16, dtype=torch.float64, device=dev)
    # o = 100, v = 700: 22^2 * 100^2 partials > 2^21 -> rejected before any launch
    assert lib.cc_ladder_energy_noalloc(100, 700, _p(x), _p(x), _p(x), None, None) == -10
    # o = 1448, v = 32: 1448^2 partials fit only when e_pair is given (no room for the o^2 pair sums)
    assert lib.cc_ladder_energy_noalloc(1448, 32, _p(x), _p(x), _p(x), None, None) == -10
    assert lib.cc_ladder_energy_noalloc(0, 7, _p(x), _p(x), _p(x), None, None) == -1
