"""Failure detection without a GPU fault: every mbarrier wait in the tensor-core
kernel is bounded.  With the bound set to 1 ns the waits run out, the kernel
raises its status word, drains its in-flight copies and MMAs, frees TMEM and
returns; the call reports CC_ERR_DEVICE_TIMEOUT and the device stays usable."""
import numpy as np
import pytest
import torch

from paper_2310_04559_gb300 import _lib
from paper_2310_04559_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_bounded_wait_expiry_reports_and_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    lib = _lib.load()
    rng = np.random.default_rng(3)
    A = torch.from_numpy(rng.standard_normal((300, 700))).to(dev)
    Bm = torch.from_numpy(rng.standard_normal((520, 700))).to(dev)
    ref = (A @ Bm.T).cpu().numpy()
    try:
        lib.cc_ladder_set_wait_limit_ns(1)
        with pytest.raises(_lib.LadderError) as ei:
            B.gemm(A, Bm, mode="ozaki_bf16")
        assert ei.value.status == -8
    finally:
        lib.cc_ladder_set_wait_limit_ns(0)  # back to the default bound
    C = B.gemm(A, Bm, mode="ozaki_bf16").cpu().numpy()
    assert np.linalg.norm(C - ref) / np.linalg.norm(ref) < 1e-10
    torch.cuda.synchronize(dev)
