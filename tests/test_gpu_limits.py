"""GPU checks at the edges of the argument space, through the C ABI against the FP64 CPU oracle:

* many occupied orbitals with few virtuals (o = 300: o^2 = 90 000 pairs, beyond the 65 535 limit
  of one grid dimension), forward with the pair energy and the pair-symmetric adjoint;
* the allocation-free energy at o = 300 and o = 1000 against the oracle's energy;
* non-finite inputs: the emulated mode reports CC_ERR_NONFINITE (its integer slices cannot carry
  NaN / Inf), the FP64 mode propagates them into R like IEEE arithmetic.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2310_04559_gb300 import _lib
from paper_2310_04559_gb300 import binding as B
from paper_2310_04559_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki_bf16": 1e-10}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cu(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


@pytest.fixture(scope="module")
def big_o(oracle):
    o, v, n = 300, 8, 20
    L, t2 = synth.ladder_inputs(o, v, n, seed=31)
    R = oracle.ladder(L, t2)
    return L, t2, R, oracle.energy(R, t2)


@pytest.mark.parametrize("mode", ["fp64", "ozaki_bf16"])
@pytest.mark.parametrize("symmetric", [True, False])
def test_forward_with_energy_o300(dev, big_o, mode, symmetric):
    L, t2, R_ref, E_ref = big_o
    R, E = B.ladder_forward(cu(L, dev), cu(t2, dev), mode=mode, symmetric=symmetric, energy=True)
    assert rel(R.cpu().numpy(), R_ref) < TOL[mode]
    assert abs(float(E) - E_ref) <= TOL[mode] * abs(E_ref)


@pytest.mark.parametrize("mode", ["fp64", "ozaki_bf16"])
def test_pair_symmetric_adjoint_o300(dev, oracle, big_o, mode):
    L, t2, _, _ = big_o
    W = synth.cotangent(300, 8, seed=32)
    dL_ref, dt2_ref = oracle.ladder_grad(L, t2, W)
    dL, dt2 = B.ladder_backward(cu(L, dev), cu(t2, dev), cu(W, dev), mode=mode, symmetric=True)
    assert rel(dt2.cpu().numpy(), dt2_ref) < TOL[mode]
    assert rel(dL.cpu().numpy(), dL_ref) < TOL[mode]


def _noalloc(lib, R, t2, e_pair=None):
    o, v = t2.shape[0], t2.shape[2]
    E = torch.full((), float("nan"), dtype=torch.float64, device=R.device)
    st = lib.cc_ladder_energy_noalloc(o, v, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(t2.data_ptr()),
                                      ctypes.c_void_p(E.data_ptr()),
                                      ctypes.c_void_p(e_pair.data_ptr()) if e_pair is not None else None,
                                      ctypes.c_void_p(torch.cuda.current_stream(R.device).cuda_stream))
    return st, E


def test_noalloc_energy_large_o_against_oracle(dev, oracle, big_o):
    lib = _lib.load()
    L, t2, R_ref, E_ref = big_o
    st, E = _noalloc(lib, cu(R_ref, dev), cu(t2, dev))
    assert st == 0
    assert abs(float(E) - E_ref) <= 1e-12 * abs(E_ref)
    # o = 1000, v = 8: 10^6 partial sums (half the library's array) with e_pair given
    rng = np.random.default_rng(33)
    R = rng.standard_normal((1000, 1000, 8, 8))
    t = rng.standard_normal((1000, 1000, 8, 8))
    ep = torch.empty((1000, 1000), dtype=torch.float64, device=dev)
    st, E = _noalloc(lib, cu(R, dev), cu(t, dev), ep)
    assert st == 0
    e_ref, ep_ref = oracle.energy(R, t, pair=True)
    assert abs(float(E) - e_ref) <= 1e-12 * abs(e_ref) + 1e-9
    assert np.allclose(ep.cpu().numpy(), ep_ref, rtol=1e-12, atol=1e-12)


def test_nonfinite_inputs(dev):
    o, v, n = 3, 20, 30
    L, t2 = synth.ladder_inputs(o, v, n, seed=34)
    t_nan = t2.copy()
    t_nan[1, 2, 3, 4] = np.nan
    t_nan[2, 1, 4, 3] = np.nan  # keep the pair symmetry
    L_inf = L.copy()
    L_inf[5, 2, 7] = np.inf
    for Lx, tx in ((L, t_nan), (L_inf, t2)):
        for sym in (True, False):
            with pytest.raises(_lib.LadderError) as e:
                B.ladder_forward(cu(Lx, dev), cu(tx, dev), mode="ozaki_bf16", symmetric=sym)
            assert e.value.status == -11
            # FP64 propagates: some entries of R are NaN / Inf, the call succeeds
            R = B.ladder_forward(cu(Lx, dev), cu(tx, dev), mode="fp64", symmetric=sym).cpu().numpy()
            assert not np.isfinite(R).all()
    # the GEMM building block and the adjoint report it too
    A = np.ones((10, 40))
    A[3, 5] = np.inf
    with pytest.raises(_lib.LadderError) as e:
        B.gemm(cu(A, dev), cu(np.ones((9, 40)), dev), mode="ozaki_bf16")
    assert e.value.status == -11
    W = synth.cotangent(o, v, seed=35)
    W[0, 0, 1, 1] = np.nan
    with pytest.raises(_lib.LadderError) as e:
        B.ladder_backward(cu(L, dev), cu(t2, dev), cu(W, dev), mode="ozaki_bf16", symmetric=True)
    assert e.value.status == -11
    # finite inputs afterwards: the status word starts clean on every call
    R = B.ladder_forward(cu(L, dev), cu(t2, dev), mode="ozaki_bf16", symmetric=True)
    assert torch.isfinite(R).all()
