"""PyTorch-facing wrapper of the C ABI: workspace allocation, stream hand-off and
a torch.autograd.Function for the ladder term

    R[i,j,a,b] = sum_cd (sum_P L[P,a,c] L[P,b,d]) t2[i,j,c,d]      (Eq. 5 + Eq. 6)

PyTorch provides device memory and the current stream only; the computation
itself runs in libcc_ladder.so.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

_MODE_ALIASES = {"ozaki": "ozaki_bf16", "emulated_fp64": "ozaki_bf16"}


def _mode(m) -> int:
    if isinstance(m, int):
        return m
    m = _MODE_ALIASES.get(m, m)
    if m not in _lib.MODES:
        raise ValueError(f"unknown mode {m!r}; one of {sorted(_lib.MODES)}")
    return _lib.MODES[m]


def _order(o) -> int:
    if isinstance(o, int):
        return o
    if o not in _lib.ORDERS:
        raise ValueError(f"unknown order {o!r}; one of {sorted(_lib.ORDERS)}")
    return _lib.ORDERS[o]


def _flags(symmetric=False, exchange=False, accumulate=False, no_sync=False, host_t2r=False, host_L=False) -> int:
    return ((_lib.FLAG_SYMMETRIC_T if symmetric else 0) | (_lib.FLAG_EXCHANGE if exchange else 0)
            | (_lib.FLAG_ACCUMULATE if accumulate else 0) | (_lib.FLAG_NO_STATUS_SYNC if no_sync else 0)
            | (_lib.FLAG_HOST_T2R if host_t2r else 0) | (_lib.FLAG_HOST_L if host_L else 0))


def _check_tensor(x: torch.Tensor, name: str, shape):
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if x.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path exists)")
    if x.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {tuple(shape)}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _same_device(*xs):
    """All CUDA tensors of one call live on one device (the stream is that device's)."""
    devs = {x.device for x in xs if x is not None and x.device.type == "cuda"}
    if len(devs) > 1:
        raise ValueError(f"tensors on different devices: {sorted(str(d) for d in devs)}")


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else None


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _shapes(L, t2):
    n, v, _ = L.shape
    o = t2.shape[0]
    return o, v, n


def make_args(o, v, n, mode="fp64", order="auto", symmetric=False, exchange=False, accumulate=False,
              a_block=0, slices=0, budget=0, no_sync=False, a_range=None, host_t2r=False, host_L=False,
              chol_chunk=0) -> _lib.Args:
    a = _lib.Args()
    if a_range is not None:
        a.a_lo, a.a_hi = int(a_range[0]), int(a_range[1])
    a.chol_chunk = int(chol_chunk)
    a.o, a.v, a.n_chol = o, v, n
    a.mode, a.order = _mode(mode), _order(order)
    a.a_block, a.slices = int(a_block), int(slices)
    a.flags = _flags(symmetric, exchange, accumulate, no_sync, host_t2r, host_L)
    a.budget_bytes = int(budget)
    return a


def workspace_size(o, v, n, **kw) -> int:
    """Bytes of workspace the forward plan needs (keywords as in make_args)."""
    lib = _lib.load()
    a = make_args(o, v, n, **kw)
    out = ctypes.c_size_t()
    _lib.check(lib.cc_ladder_workspace_size_ex(ctypes.byref(a), ctypes.byref(out)), "cc_ladder_workspace_size_ex")
    return out.value


def plan(o, v, n, ws_bytes=0, **kw) -> dict:
    lib = _lib.load()
    a = make_args(o, v, n, **kw)
    a.ws_bytes = int(ws_bytes)
    p = _lib.Plan()
    _lib.check(lib.cc_ladder_plan_query(ctypes.byref(a), ctypes.byref(p)), "cc_ladder_plan_query")
    return {"order": {1: "integral_first", 2: "cholesky_first"}[p.order], "a_block": p.a_block,
            "n_blocks": p.n_blocks, "slices": p.slices, "pairs": p.pairs, "ws_bytes": p.ws_bytes,
            "flops_algorithmic": p.flops_algorithmic, "flops_issued": p.flops_issued, "pair_blocks": p.pair_blocks}


def partition(o, v, n, parts, **kw) -> list:
    """Work-balanced bounds [0 = b_0 < b_1 < ... < b_parts = v] of the `a` range of one problem
    over `parts` devices (keywords as in make_args): part g computes a_range=(b_g, b_g+1).
    Host-only; no device is touched."""
    lib = _lib.load()
    a = make_args(o, v, n, **kw)
    out = (ctypes.c_int * (parts + 1))()
    _lib.check(lib.cc_ladder_partition(ctypes.byref(a), int(parts), out), "cc_ladder_partition")
    return list(out)


def autotune(L, t2, R=None, mode="ozaki_bf16", symmetric=False, exchange=False, slices=0, budget=0,
             workspace=None) -> dict:
    """Time both contraction orders on this shape and record the faster one for
    order="auto"; returns the chosen plan and the per-order estimates (ms)."""
    lib = _lib.load()
    o, v, n = _shapes(L, t2)
    _check_tensor(L, "L", (n, v, v))
    _check_tensor(t2, "t2", (o, o, v, v))
    R = torch.empty_like(t2) if R is None else R
    a = make_args(o, v, n, mode, "auto", symmetric, exchange, False, 0, slices, budget)
    if workspace is None:
        # big enough for either order under the budget
        ws = max(workspace_size(o, v, n, mode=mode, order=od, symmetric=symmetric, exchange=exchange,
                                slices=slices, budget=budget) for od in ("integral_first", "cholesky_first"))
        workspace = alloc_workspace(ws, L.device)
    a.L, a.t2, a.R = _ptr(L), _ptr(t2), _ptr(R)
    a.workspace, a.ws_bytes = _ptr(workspace), workspace.numel()
    a.stream = _stream(L.device)
    p = _lib.Plan()
    t_if, t_cf = ctypes.c_double(), ctypes.c_double()
    _lib.check(lib.cc_ladder_autotune(ctypes.byref(a), ctypes.byref(p), ctypes.byref(t_if), ctypes.byref(t_cf)),
               "cc_ladder_autotune")
    return {"order": {1: "integral_first", 2: "cholesky_first"}[p.order], "a_block": p.a_block,
            "ms_integral_first": t_if.value, "ms_cholesky_first": t_cf.value}


def alloc_workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _check_host_tensor(x: torch.Tensor, name: str, shape):
    if not isinstance(x, torch.Tensor) or x.device.type != "cpu" or not x.is_pinned():
        raise ValueError(f"{name} must be a page-locked CPU tensor (tensor.pin_memory()) with host_t2r / host_L")
    if x.dtype != torch.float64 or tuple(x.shape) != tuple(shape) or not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous float64 of shape {tuple(shape)}")


def ladder_forward(L, t2, R=None, mode="ozaki_bf16", order="auto", symmetric=False, exchange=False,
                   accumulate=False, a_block=0, slices=0, energy=False, workspace=None, budget=0, no_sync=False,
                   a_range=None, host_t2r=False, host_L=False, chol_chunk=0, device=None):
    """R (new tensor unless given) and optionally the pair energy E (0-d tensor).
    a_range=(lo, hi) computes only the columns a in [lo, hi) (see cc_ladder_args).
    host_t2r=True: t2 and R are page-locked CPU tensors read and written over the host link
    (problems whose o^2 v^2 exceeds device memory); needs symmetric=True.
    host_L=True: L is a page-locked CPU tensor streamed to the device in chunks of chol_chunk
    Cholesky vectors (problems whose n_chol v^2 exceeds device memory); needs symmetric=True.
    device: the GPU when no argument lives there (host_L with host_t2r; default: the current one)."""
    lib = _lib.load()
    o, v, n = _shapes(L, t2)
    (_check_host_tensor if host_L else _check_tensor)(L, "L", (n, v, v))
    check = _check_host_tensor if host_t2r else _check_tensor
    check(t2, "t2", (o, o, v, v))
    if device is None:
        gpu = [x.device for x in (L, t2) if x.device.type == "cuda"]
        device = gpu[0] if gpu else torch.device("cuda", torch.cuda.current_device())
    if R is None:
        R = torch.empty_like(t2) if not accumulate else torch.zeros_like(t2)
        if host_t2r:
            R = R.pin_memory()
    check(R, "R", (o, o, v, v))
    a = make_args(o, v, n, mode, order, symmetric, exchange, accumulate, a_block, slices, budget, no_sync, a_range,
                  host_t2r, host_L, chol_chunk)
    if workspace is None:
        ws = ctypes.c_size_t()
        _lib.check(lib.cc_ladder_workspace_size_ex(ctypes.byref(a), ctypes.byref(ws)), "cc_ladder_workspace_size_ex")
        workspace = alloc_workspace(ws.value, device)
    _same_device(L, t2, R, workspace)
    E = torch.empty((), dtype=torch.float64, device=device) if energy else None
    a.L, a.t2, a.R, a.energy = _ptr(L), _ptr(t2), _ptr(R), _ptr(E)
    a.workspace, a.ws_bytes = _ptr(workspace), workspace.numel()
    a.stream = _stream(device)
    _lib.check(lib.cc_ladder_fwd_ex(ctypes.byref(a)), "cc_ladder_fwd_ex")
    return (R, E) if energy else R


def ladder_backward(L, t2, dR, mode="ozaki_bf16", symmetric=False, want_dL=True, want_dt2=True, slices=0,
                    budget=0, workspace=None):
    """Adjoint of the forward for loss = <dR, R>: returns (dL, dt2) (None where not wanted)."""
    lib = _lib.load()
    o, v, n = _shapes(L, t2)
    _check_tensor(L, "L", (n, v, v))
    _check_tensor(t2, "t2", (o, o, v, v))
    _check_tensor(dR, "dR", (o, o, v, v))
    _same_device(L, t2, dR, workspace)
    if workspace is None:
        ws = ctypes.c_size_t()
        _lib.check(lib.cc_ladder_bwd_workspace_size(o, v, n, _mode(mode), int(budget), ctypes.byref(ws)),
                   "cc_ladder_bwd_workspace_size")
        workspace = alloc_workspace(ws.value, L.device)
    dL = torch.empty_like(L) if want_dL else None
    dt2 = torch.empty_like(t2) if want_dt2 else None
    st = lib.cc_ladder_bwd_ex(o, v, n, _ptr(L), _ptr(t2), _ptr(dR), _ptr(dL), _ptr(dt2), _mode(mode),
                              _flags(symmetric), int(slices), _ptr(workspace), workspace.numel(), _stream(L.device))
    _lib.check(st, "cc_ladder_bwd_ex")
    return dL, dt2


def term(which, Lov, t2, Lvv=None, mode="ozaki_bf16", slices=0, budget=0, T=None, workspace=None, no_sync=False):
    """The two further Cholesky terms that share the ladder's contraction (Eq. 8, Eq. 9):
    which="ijkl": T[i,j,k,l] = sum_{P,c,d} Lov[P,k,c] Lov[P,l,d] t2[i,j,c,d]   (o x o x o x o)
    which="ijbk": T[i,j,b,k] = sum_{P,c,d} Lvv[P,b,d] Lov[P,k,c] t2[i,j,c,d]   (o x o x v x o)
    Lov is n x o x v, Lvv n x v x v."""
    lib = _lib.load()
    w = _lib.TERMS[which]
    n, o, v = Lov.shape
    _check_tensor(Lov, "Lov", (n, o, v))
    _check_tensor(t2, "t2", (o, o, v, v))
    if w == 2:
        _check_tensor(Lvv, "Lvv", (n, v, v))
    shape = (o, o, o, o) if w == 1 else (o, o, v, o)
    if T is None:
        T = torch.empty(shape, dtype=torch.float64, device=Lov.device)
    _check_tensor(T, "T", shape)
    _same_device(Lov, Lvv, t2, T, workspace)
    if workspace is None:
        ws = ctypes.c_size_t()
        _lib.check(lib.cc_ladder_term_workspace_size(w, o, v, n, _mode(mode), int(slices), int(budget),
                                                     ctypes.byref(ws)), "cc_ladder_term_workspace_size")
        workspace = alloc_workspace(ws.value, Lov.device)
    st = lib.cc_ladder_term(w, o, v, n, _ptr(Lov), _ptr(Lvv) if w == 2 else None, _ptr(t2), _ptr(T), _mode(mode),
                            _flags(no_sync=no_sync), int(slices), _ptr(workspace), workspace.numel(),
                            _stream(Lov.device))
    _lib.check(st, "cc_ladder_term")
    return T


def tijkl(Lov, t2, mode="ozaki_bf16", **kw):
    """Eq. 8 (see term)."""
    return term("ijkl", Lov, t2, mode=mode, **kw)


def tijbk(Lov, Lvv, t2, mode="ozaki_bf16", **kw):
    """Eq. 9 (see term)."""
    return term("ijbk", Lov, t2, Lvv=Lvv, mode=mode, **kw)


def pair_energy(R, t2, pairs=False):
    """E = sum_ijab (2 R_ijab - R_ijba) t2_ijab (and e_ij if pairs)."""
    lib = _lib.load()
    o, v = t2.shape[0], t2.shape[2]
    _check_tensor(R, "R", (o, o, v, v))
    _check_tensor(t2, "t2", (o, o, v, v))
    _same_device(R, t2)
    ws = ctypes.c_size_t()
    _lib.check(lib.cc_ladder_energy_workspace_size(o, v, ctypes.byref(ws)), "cc_ladder_energy_workspace_size")
    w = alloc_workspace(ws.value, R.device)
    E = torch.empty((), dtype=torch.float64, device=R.device)
    ep = torch.empty((o, o), dtype=torch.float64, device=R.device) if pairs else None
    _lib.check(lib.cc_ladder_energy(o, v, _ptr(R), _ptr(t2), _ptr(E), _ptr(ep), _ptr(w), w.numel(), _stream(R.device)),
               "cc_ladder_energy")
    return (E, ep) if pairs else E


def gemm(A, B, mode="ozaki_bf16", C=None, accumulate=False, slices=0):
    """C = A @ B.T (FP64 in and out) through the library's GEMM core in `mode`."""
    lib = _lib.load()
    M, K = A.shape
    N = B.shape[0]
    _check_tensor(A, "A", (M, K))
    _check_tensor(B, "B", (N, K))
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float64, device=A.device)
    _check_tensor(C, "C", (M, N))
    _same_device(A, B, C)
    ws = ctypes.c_size_t()
    _lib.check(lib.cc_ladder_gemm_workspace_size(_mode(mode), M, N, K, int(slices), ctypes.byref(ws)),
               "cc_ladder_gemm_workspace_size")
    w = alloc_workspace(ws.value, A.device)
    _lib.check(lib.cc_ladder_gemm(_mode(mode), M, N, K, _ptr(A), K, _ptr(B), K, _ptr(C), N, int(accumulate),
                                  int(slices), _ptr(w), w.numel(), _stream(A.device)), "cc_ladder_gemm")
    return C


def peak_probe(which, iters=0, device=None) -> float:
    """Measured peak rate (TFLOP/s of the whole GPU) of one arithmetic unit: "dmma", "dfma",
    "tc_bf16", "tc_tf32" or "imma" (TOP/s; see cc_ladder_peak_probe)."""
    lib = _lib.load()
    default_iters = {"dmma": 4096, "dfma": 16384, "tc_bf16": 20000, "tc_tf32": 10000, "imma": 4096}
    out = ctypes.c_double()
    _lib.check(lib.cc_ladder_peak_probe(_lib.PROBES[which], int(iters or default_iters[which]), _stream(device),
                                        ctypes.byref(out)), "cc_ladder_peak_probe")
    return out.value


def profile_enable(on=True):
    _lib.load().cc_ladder_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{phase: {"launches", "ms", "flops", "bytes"}} accumulated since profile_enable(True)."""
    lib = _lib.load()
    n = lib.cc_ladder_profile_read(None, 0)
    arr = (_lib.ProfileEntry * max(n, 1))()
    n = lib.cc_ladder_profile_read(arr, n)
    return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "flops": arr[i].flops,
                                   "bytes": arr[i].bytes} for i in range(n)}


def launch_count() -> int:
    return int(_lib.load().cc_ladder_launch_count())


class LadderFunction(torch.autograd.Function):
    """R = ladder(L, t2) with the hand-written adjoint (integral blocks recomputed)."""

    @staticmethod
    def forward(ctx, L, t2, mode, order, symmetric, slices):
        ctx.save_for_backward(L, t2)
        ctx.mode, ctx.symmetric, ctx.slices = mode, symmetric, slices
        return ladder_forward(L, t2, mode=mode, order=order, symmetric=symmetric, slices=slices)

    @staticmethod
    def backward(ctx, dR):
        L, t2 = ctx.saved_tensors
        dL, dt2 = ladder_backward(L, t2, dR.contiguous(), mode=ctx.mode, symmetric=ctx.symmetric,
                                  want_dL=ctx.needs_input_grad[0], want_dt2=ctx.needs_input_grad[1],
                                  slices=ctx.slices)
        return dL, dt2, None, None, None, None


def ladder(L, t2, mode="ozaki_bf16", order="auto", symmetric=False, slices=0):
    """Differentiable ladder term R[i,j,a,b] = sum_cd (ac|bd) t2[i,j,c,d]."""
    return LadderFunction.apply(L, t2, mode, order, symmetric, slices)
