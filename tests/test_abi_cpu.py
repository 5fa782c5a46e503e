"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every function include/cc_ladder.h declares, and rejects bad arguments
before it enqueues anything."""
import ctypes
import os
import re

import pytest

from paper_2310_04559_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "cc_ladder.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_ladder_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SYMBOLS)


def test_version_and_strerror(lib):
    assert b"sm_103a" in lib.cc_ladder_version()
    for code in range(-11, 1):
        assert lib.cc_ladder_strerror(code) != b"unknown status"
    assert lib.cc_ladder_strerror(-99) == b"unknown status"


def _args(**kw):
    from paper_2310_04559_gb300.binding import make_args
    base = dict(o=4, v=24, n=60, mode="fp64")
    base.update(kw)
    return make_args(base.pop("o"), base.pop("v"), base.pop("n"), **base)


def _fake(addr):
    return ctypes.c_void_p(addr)


def test_argument_errors(lib):
    a = _args()
    assert lib.cc_ladder_fwd_ex(ctypes.byref(a)) == -2  # NULL pointers
    a.L = a.t2 = a.R = _fake(0x10000)
    a.workspace = _fake(0x20000)
    a.ws_bytes = 1 << 30
    a.t2 = _fake(0x10008)  # 8-byte aligned only
    assert lib.cc_ladder_fwd_ex(ctypes.byref(a)) == -3
    a.t2 = _fake(0x10000)
    a.workspace = _fake(0x20080)  # not 256-aligned
    assert lib.cc_ladder_fwd_ex(ctypes.byref(a)) == -3
    a.workspace = _fake(0x20000)
    a.ws_bytes = 1024  # too small for any plan
    assert lib.cc_ladder_fwd_ex(ctypes.byref(a)) == -4
    for bad, code in [(dict(o=0), -1), (dict(v=-3), -1), (dict(n=0), -1), (dict(mode="ozaki_int8"), -6)]:
        b = _args(**bad)
        b.L = b.t2 = b.R = _fake(0x10000)
        b.workspace, b.ws_bytes = _fake(0x20000), 1 << 40
        assert lib.cc_ladder_fwd_ex(ctypes.byref(b)) == code, bad
    b = _args()
    b.mode = 17
    assert lib.cc_ladder_fwd_ex(ctypes.byref(b)) == -9
    b = _args()
    b.flags = 1 << 10
    assert lib.cc_ladder_fwd_ex(ctypes.byref(b)) == -9
    b = _args(mode="ozaki_bf16", slices=1)
    assert lib.cc_ladder_fwd_ex(ctypes.byref(b)) == -9
    # bwd / gemm / energy validation
    assert lib.cc_ladder_bwd(0, 4, 4, None, None, None, None, None, 0, None, 0, None) == -1
    assert lib.cc_ladder_bwd(2, 4, 4, None, None, None, None, None, 0, None, 0, None) == -2
    assert lib.cc_ladder_gemm(0, 4, 4, 0, None, 4, None, 4, None, 4, 0, 0, None, 0, None) == -1
    assert lib.cc_ladder_gemm(2, 4, 4, 4, None, 4, None, 4, None, 4, 0, 0, None, 0, None) == -6
    assert lib.cc_ladder_energy(2, 3, None, None, None, None, None, 0, None) == -2


def test_workspace_queries_monotone_in_budget(lib):
    from paper_2310_04559_gb300 import binding as Ld
    for mode in ["fp64", "ozaki_bf16", "tf32", "bf16"]:
        for order in ["integral_first", "cholesky_first"]:
            sizes = []
            for budget in [1 << 26, 1 << 28, 1 << 30, 1 << 34]:
                try:
                    sizes.append(Ld.workspace_size(20, 200, 1000, mode=mode, order=order, budget=budget))
                except _lib.LadderError as e:
                    assert e.status == -5
                    sizes.append(0)
            assert sizes == sorted(sizes)
            assert all(s <= b for s, b in zip(sizes, [1 << 26, 1 << 28, 1 << 30, 1 << 34]))
    # the plan the forward would run for exactly the queried bytes is the same block
    ws = Ld.workspace_size(40, 400, 2000, mode="ozaki_bf16", symmetric=True, budget=40 << 30)
    p = Ld.plan(40, 400, 2000, ws_bytes=ws, mode="ozaki_bf16", symmetric=True)
    # pair-symmetric tensor-core plans widen their blocks as the b >= a range shrinks
    assert p["ws_bytes"] == ws and 1 <= p["n_blocks"] <= -(-400 // p["a_block"])
    assert p["flops_algorithmic"] == 2.0 * (1600 + 2000) * 400 ** 4
    # ... and issue about (n + o^2/2) v^4 multiply-adds per slice product instead of 2 (n + o(o+1)/2) v^4
    unpacked = 21 * 2.0 * (820 + 2000) * 400 ** 4
    assert 0.45 < p["flops_issued"] / unpacked < 0.6
    # the FP64 (DMMA) mode runs the same packed plan; without pair symmetry blocks are uniform
    p = Ld.plan(40, 400, 2000, mode="fp64", symmetric=True, budget=40 << 30)
    assert 0.45 < p["flops_issued"] / (2.0 * (820 + 2000) * 400 ** 4) < 0.6
    ws = Ld.workspace_size(40, 400, 2000, mode="fp64", budget=40 << 30)
    p = Ld.plan(40, 400, 2000, ws_bytes=ws, mode="fp64")
    assert p["ws_bytes"] == ws and p["n_blocks"] * p["a_block"] >= 400


def test_planner_orders(lib):
    from paper_2310_04559_gb300 import binding as Ld
    # integral-first is cheaper for the o << v << n shapes, Cholesky-first when n o^2 << v
    assert Ld.plan(40, 400, 2000, mode="ozaki_bf16")["order"] == "integral_first"
    assert Ld.plan(4, 96, 480, mode="ozaki_bf16")["order"] == "cholesky_first"
    assert Ld.plan(4, 96, 480, mode="ozaki_bf16", order="integral_first")["order"] == "integral_first"
    p = Ld.plan(60, 600, 3000, mode="ozaki_bf16", symmetric=True, budget=150 << 30)
    assert p["ws_bytes"] < 150 << 30 and p["pairs"] == 60 * 61 // 2 and p["slices"] == 6


def test_host_resident_plans(lib):
    """CC_FLAG_HOST_T2R: only the pair-symmetric integral-first path; the planner splits the pairs
    into more blocks as the device budget shrinks, never below one `a` per integral block."""
    from paper_2310_04559_gb300 import binding as Ld
    with pytest.raises(_lib.LadderError) as e:
        Ld.plan(9, 40, 70, mode="ozaki_bf16", symmetric=False, host_t2r=True, budget=1 << 30)
    assert e.value.status == -6
    with pytest.raises(_lib.LadderError) as e:
        Ld.plan(9, 40, 70, mode="ozaki_bf16", symmetric=True, exchange=True, host_t2r=True, budget=1 << 30)
    assert e.value.status == -6
    last = 0
    for kb in (64 << 10, 8 << 10, 4100, 3500, 2700):
        p = Ld.plan(9, 40, 70, mode="ozaki_bf16", symmetric=True, host_t2r=True, budget=kb << 10)
        assert p["order"] == "integral_first" and p["ws_bytes"] <= kb << 10
        assert p["pair_blocks"] >= last and 1 <= p["a_block"] <= 40
        last = p["pair_blocks"]
    assert last > 1
    # the work is the same however the pairs are blocked
    full = Ld.plan(9, 40, 70, mode="ozaki_bf16", symmetric=True, budget=1 << 30)["flops_algorithmic"]
    assert p["flops_algorithmic"] == full


def test_term_workspace_queries(lib):
    """Eq. 8 / Eq. 9 workspace queries: monotone in the budget, CC_ERR_BUDGET below the smallest
    plan, CC_ERR_ARG for an unknown term."""
    sizes = []
    for b in (1 << 22, 1 << 26, 1 << 30):
        out = ctypes.c_size_t()
        st = lib.cc_ladder_term_workspace_size(2, 10, 64, 200, 1, 0, b, ctypes.byref(out))
        sizes.append(out.value if st == 0 else 0)
        assert st in (0, -5)
    assert sizes == sorted(sizes) and sizes[-1] > 0
    out = ctypes.c_size_t()
    assert lib.cc_ladder_term_workspace_size(2, 10, 64, 200, 1, 0, 1 << 12, ctypes.byref(out)) == -5
    assert lib.cc_ladder_term_workspace_size(3, 10, 64, 200, 1, 0, 1 << 30, ctypes.byref(out)) == -9
    assert lib.cc_ladder_term(1, 2, 4, 4, None, None, None, None, 1, 0, 0, None, 0, None) == -2


def test_binding_refuses_cpu_tensors(lib):
    """The product path has no CPU fallback: CPU tensors, wrong dtypes, shapes and layouts are
    refused before anything reaches the library."""
    import torch

    from paper_2310_04559_gb300 import binding as Ld
    o, v, n = 2, 5, 3
    L = torch.zeros((n, v, v), dtype=torch.float64)
    t2 = torch.zeros((o, o, v, v), dtype=torch.float64)
    calls = [lambda: Ld.ladder_forward(L, t2), lambda: Ld.ladder_backward(L, t2, t2),
             lambda: Ld.pair_energy(t2, t2), lambda: Ld.gemm(L[0], L[0]),
             lambda: Ld.tijkl(torch.zeros((n, o, v), dtype=torch.float64), t2),
             lambda: Ld.ladder(L, t2)]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()
    with pytest.raises(ValueError, match="page-locked"):
        Ld._check_host_tensor(t2, "t2", (o, o, v, v))  # host_t2r=True wants pinned t2 and R
    with pytest.raises(ValueError, match="unknown mode"):
        Ld.workspace_size(o, v, n, mode="fp16")
    with pytest.raises(ValueError, match="unknown order"):
        Ld.plan(o, v, n, order="sideways")


def test_probe_and_partition_argument_errors(lib):
    out = ctypes.c_double()
    assert lib.cc_ladder_peak_probe(0, 10, None, ctypes.byref(out)) == -9   # unknown probe
    assert lib.cc_ladder_peak_probe(6, 10, None, ctypes.byref(out)) == -9
    assert lib.cc_ladder_peak_probe(1, 0, None, ctypes.byref(out)) == -9    # no iterations
    assert lib.cc_ladder_peak_probe(1, 10, None, None) == -2
    bounds = (ctypes.c_int * 5)()
    a = _args()
    assert lib.cc_ladder_partition(ctypes.byref(a), 4, None) == -2
    assert lib.cc_ladder_partition(ctypes.byref(a), 0, bounds) == -9
    assert lib.cc_ladder_partition(ctypes.byref(a), 25, bounds) == -9      # more parts than v = 24
    assert lib.cc_ladder_partition(ctypes.byref(a), 4, bounds) == 0
    assert list(bounds) == [0, 6, 12, 18, 24]


def test_energy_shape_limits(lib):
    x = _fake(0x10000)
    # o beyond the library's pair-count limit is a shape error, before anything is enqueued
    assert lib.cc_ladder_energy(46341, 2, x, x, x, None, _fake(0x20000), 1 << 40, None) == -1
    assert lib.cc_ladder_energy_noalloc(46341, 2, x, x, x, None, None) == -1
    assert lib.cc_ladder_energy_noalloc(2, 0, x, x, x, None, None) == -1
