"""GPU parity of the two further Cholesky terms (Eq. 8: tt_ijkl, Eq. 9: tt_ijbk) against the
FP64 CPU oracle, through the C ABI.  Same tolerances as the ladder (relative Frobenius error):
fp64 1e-12, ozaki_bf16 1e-10, tf32 1e-2, bf16 5e-2."""
import numpy as np
import pytest
import torch

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


def cu(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _inputs(o, v, n, seed):
    rng = np.random.default_rng(seed)
    Lvv = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    Lov = synth.cholesky_ov(n, o, v, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=False, rng=rng)
    return Lov, Lvv, t2


@pytest.mark.parametrize("mode", list(TOL))
@pytest.mark.parametrize("o,v,n", [(3, 37, 50), (7, 20, 130), (10, 64, 200)])
def test_terms_vs_oracle(dev, oracle, mode, o, v, n):
    Lov, Lvv, t2 = _inputs(o, v, n, o * 1000 + v)
    T1 = B.tijkl(cu(Lov, dev), cu(t2, dev), mode=mode).cpu().numpy()
    assert rel(T1, oracle.tijkl(Lov, t2)) < TOL[mode], (mode, "ijkl")
    T2 = B.tijbk(cu(Lov, dev), cu(Lvv, dev), cu(t2, dev), mode=mode).cpu().numpy()
    assert rel(T2, oracle.tijbk(Lov, Lvv, t2)) < TOL[mode], (mode, "ijbk")


@pytest.mark.parametrize("mode", ["fp64", "ozaki_bf16"])
def test_terms_blocked_and_degenerate(dev, oracle, mode):
    """A small budget forces blocks of a few k (ragged last block); o = 1 and v = 1 shapes."""
    Lov, Lvv, t2 = _inputs(9, 30, 70, 7)
    ref1, ref2 = oracle.tijkl(Lov, t2), oracle.tijbk(Lov, Lvv, t2)
    g = lambda x: cu(x, dev)
    budget = 3 << 20
    T1 = B.tijkl(g(Lov), g(t2), mode=mode, budget=budget).cpu().numpy()
    T2 = B.tijbk(g(Lov), g(Lvv), g(t2), mode=mode, budget=budget).cpu().numpy()
    assert rel(T1, ref1) < TOL[mode] and rel(T2, ref2) < TOL[mode]
    for o, v, n in [(1, 12, 5), (4, 1, 3), (1, 1, 1)]:
        Lov, Lvv, t2 = _inputs(o, v, n, 11)
        assert rel(B.tijkl(g(Lov), g(t2), mode=mode).cpu().numpy(), oracle.tijkl(Lov, t2)) < TOL[mode]
        assert rel(B.tijbk(g(Lov), g(Lvv), g(t2), mode=mode).cpu().numpy(), oracle.tijbk(Lov, Lvv, t2)) < TOL[mode]


def test_terms_reduce_to_ladder_on_device(dev):
    """With Lov = the first o rows of Lvv, the device terms equal the device ladder's blocks."""
    o, v, n = 6, 40, 90
    L, t2 = synth.ladder_inputs(o, v, n, seed=5)
    Lg, tg = cu(L, dev), cu(t2, dev)
    R = B.ladder_forward(Lg, tg, mode="ozaki_bf16").cpu().numpy()
    Lov = Lg[:, :o, :].contiguous()
    T1 = B.tijkl(Lov, tg, mode="ozaki_bf16").cpu().numpy()
    T2 = B.tijbk(Lov, Lg, tg, mode="ozaki_bf16").cpu().numpy()
    assert rel(T1, R[:, :, :o, :o]) < 1e-10
    assert rel(T2, R[:, :, :o, :].transpose(0, 1, 3, 2)) < 1e-10


@pytest.mark.parametrize("mode", list(TOL))
def test_golden_cases_on_device(dev, oracle, mode):
    """The hand-computed o = 1, v = 2, n = 2 cases (ladder, energy, exchange, Eq. 8, Eq. 9) through
    the C ABI: small integers, so every mode should reproduce them to its tolerance or better."""
    import json
    import os
    gdir = os.path.join(os.path.dirname(__file__), "golden")
    g1 = json.load(open(os.path.join(gdir, "ladder_o1_v2_n2.json")))
    g2 = json.load(open(os.path.join(gdir, "terms_o1_v2_n2.json")))
    L, t2, Lov = (np.array(g2[k], dtype=float) for k in ("L", "t2", "Lov"))
    R, E = B.ladder_forward(cu(L, dev), cu(t2, dev), mode=mode, energy=True)
    assert rel(R.cpu().numpy(), np.array(g1["R"], dtype=float)) < TOL[mode]
    assert abs(float(E) - g1["E"]) <= TOL[mode] * abs(g1["E"])
    X = B.ladder_forward(cu(L, dev), cu(t2, dev), mode=mode, exchange=True).cpu().numpy()
    assert rel(X, np.array(g2["X"], dtype=float)) < TOL[mode]
    T1 = B.tijkl(cu(Lov, dev), cu(t2, dev), mode=mode).cpu().numpy()
    assert rel(T1, np.array(g2["tijkl"], dtype=float)) < TOL[mode]
    T2 = B.tijbk(cu(Lov, dev), cu(L, dev), cu(t2, dev), mode=mode).cpu().numpy()
    assert rel(T2, np.array(g2["tijbk"], dtype=float)) < TOL[mode]
