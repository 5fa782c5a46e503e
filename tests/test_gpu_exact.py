"""Exactness of the emulated-FP64 mode for inputs whose slice products add with one sign.

The Ozaki slices are balanced base-2^7 digits; every product of two digits is at most 2^12 in
magnitude.  For sign-mixed data the FP32 level sums on the tensor cores grow like a random walk,
but for sign-aligned data (all-positive amplitudes and Cholesky vectors, constant matrices,
the diagonal of a Gram matrix) they grow linearly in the contraction length and would pass
2^24 -- the end of exact FP32 integers -- after a few thousand terms.  The slice GEMM therefore
drains every level to exact int64 at most every 4096 / (products per level) elements.  These
tests take contraction lengths well beyond that bound through the C ABI and hold the result to
the emulated mode's 1e-10 against FP64 references (the oracle, or numpy's FP64 product, whose own
error is below K 2^-53 relative for positive data)."""
import numpy as np
import pytest
import torch

from paper_2310_04559_gb300 import binding as B
from paper_2310_04559_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def positive_inputs(o, v, n, seed):
    """All-positive, symmetric Cholesky vectors and pair-symmetric amplitudes."""
    rng = np.random.default_rng(seed)
    L = rng.uniform(0.5, 1.0, (n, v, v))
    L = 0.5 * (L + L.transpose(0, 2, 1))
    t = rng.uniform(0.5, 1.0, (o, o, v, v)) * 1e-2
    t = 0.5 * (t + t.transpose(1, 0, 3, 2))
    return np.ascontiguousarray(L), np.ascontiguousarray(t)


@pytest.mark.parametrize("symmetric", [True, False])
def test_positive_ladder_long_contraction(dev, oracle, symmetric):
    # v = 100: the packed ladder GEMM contracts over v(v+1)/2 = 5050 > 4096 pairs (c <= d), the
    # unpacked one over v^2 = 10 000; the integral build over n = 5000
    o, v, n = 3, 100, 5000
    L, t2 = positive_inputs(o, v, n, seed=41)
    R_ref = oracle.ladder(L, t2)
    R = B.ladder_forward(cu(L, dev), cu(t2, dev), mode="ozaki_bf16", symmetric=symmetric,
                         order="integral_first").cpu().numpy()
    assert rel(R, R_ref) < TOL, rel(R, R_ref)
    # the Cholesky-first order contracts over n v = 500 000 in its second GEMM
    Rc = B.ladder_forward(cu(L, dev), cu(t2, dev), mode="ozaki_bf16", symmetric=symmetric,
                          order="cholesky_first").cpu().numpy()
    assert rel(Rc, R_ref) < TOL, rel(Rc, R_ref)


@pytest.mark.parametrize("kind", ["positive", "constant", "gram"])
def test_gemm_aligned_k20000(dev, kind):
    rng = np.random.default_rng(42)
    M, N, K = 300, 260, 20000
    if kind == "positive":
        A = rng.uniform(0.5, 1.0, (M, K))
        Bm = rng.uniform(0.5, 1.0, (N, K))
    elif kind == "constant":
        # every digit of every element is the same, so every level sums one value K times
        A = np.full((M, K), 0.7777777777777777)
        Bm = np.full((N, K), -0.3333333333333333)
    else:
        A = rng.standard_normal((M, K))
        Bm = A[:N].copy()  # C[i, i] = sum_k A_ik^2: squares of every digit add with one sign
    ref = A @ Bm.T
    C = B.gemm(cu(A, dev), cu(Bm, dev), mode="ozaki_bf16").cpu().numpy()
    assert rel(C, ref) < TOL, (kind, rel(C, ref))
    if kind == "gram":
        d = np.arange(N)
        assert rel(C[d, d], ref[d, d]) < TOL
    if kind == "constant":
        assert np.max(np.abs(C - ref) / np.abs(ref)) < TOL


def test_positive_adjoint(dev, oracle):
    o, v, n = 2, 70, 3000
    L, t2 = positive_inputs(o, v, n, seed=43)
    W = np.random.default_rng(44).uniform(0.5, 1.0, (o, o, v, v))
    dL_ref, dt2_ref = oracle.ladder_grad(L, t2, W)
    dL, dt2 = B.ladder_backward(cu(L, dev), cu(t2, dev), cu(W, dev), mode="ozaki_bf16", symmetric=True)
    assert rel(dt2.cpu().numpy(), dt2_ref) < TOL
    assert rel(dL.cpu().numpy(), dL_ref) < TOL
