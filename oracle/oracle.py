"""ctypes wrapper around the FP64 CPU oracle (ladder_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference leg are the only users.  The product path never imports
this module.  ``build()`` compiles the C source with gcc + OpenMP into
``oracle/_build/liboracle.so``.

Functions (each follows the passage cited in ladder_oracle.c):

* ``ladder(L, t2, a_list=None, compensated=False)`` -- Eq. 5 + Eq. 6 through the
  for-loop over ``a`` of Section 3.2.
* ``ladder_eri(L, t2)`` -- brute force through the dense integral tensor (Eq. 4/5).
* ``ladder_entries(L, t2, idx)`` -- selected entries of Eq. 6, one by one.
* ``energy(R, t2)`` -- E = sum (2 R_ijab - R_ijba) t_ijab.
* ``energy_range(R, t2, lo, hi)`` -- the terms of E with min(a, b) in [lo, hi).
* ``ladder_grad(L, t2, W)`` -- dt2, dL of loss = <W, R>.
* ``ladder_grad_entries(...)`` -- selected gradient entries.
* ``exchange(L, t2, a_list=None)`` -- Eq. 7.
* ``tijkl(Lov, t2)``, ``tijbk(Lov, Lvv, t2)`` -- Eq. 8 and Eq. 9 through
  ``general(A, B, t2)``, G[i,j,p,q] = sum_cd (sum_P A[P,p,c] B[P,q,d]) t2[i,j,c,d].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ladder_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2 -fopenmp); returns its path."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_ladder.argtypes = [ctypes.c_int] * 3 + [_dp, _dp, _dp, ctypes.POINTER(ctypes.c_int),
                                                           ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_ladder_eri.argtypes = [ctypes.c_int] * 3 + [_dp, _dp, _dp, _dp]
        lib.oracle_ladder_entries.argtypes = [ctypes.c_int] * 3 + [_dp, _dp, ctypes.POINTER(ctypes.c_longlong),
                                                                   ctypes.c_int, _dp, ctypes.c_int]
        lib.oracle_energy.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        lib.oracle_energy.restype = ctypes.c_double
        lib.oracle_energy_range.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_energy_range.restype = ctypes.c_double
        lib.oracle_ladder_grad.argtypes = [ctypes.c_int] * 3 + [_dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        _llp = ctypes.POINTER(ctypes.c_longlong)
        lib.oracle_ladder_grad_entries.argtypes = ([ctypes.c_int] * 3 + [_dp, _dp, _dp, _llp, ctypes.c_int, _dp,
                                                                         _llp, ctypes.c_int, _dp, ctypes.c_int])
        lib.oracle_exchange.argtypes = [ctypes.c_int] * 3 + [_dp, _dp, _dp, ctypes.POINTER(ctypes.c_int),
                                                             ctypes.c_int, ctypes.c_int]
        lib.oracle_general.argtypes = [ctypes.c_int] * 5 + [_dp, _dp, _dp, _dp, ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(x):
    return x.ctypes.data_as(_dp) if x is not None else None


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _shapes(L, t2):
    n, v, v2 = L.shape
    o, o2, v3, v4 = t2.shape
    assert v == v2 == v3 == v4 and o == o2, (L.shape, t2.shape)
    return o, v, n


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def ladder(L, t2, a_list=None, compensated=False, threads=0):
    """R[i, j, k, b] for a = a_list[k] (all a when a_list is None)."""
    lib = _load()
    L, t2 = _f64(L), _f64(t2)
    o, v, n = _shapes(L, t2)
    if a_list is None:
        R = np.empty((o, o, v, v))
        lib.oracle_ladder(o, v, n, _p(L), _p(t2), _p(R), None, 0, int(compensated), threads)
    else:
        al = np.ascontiguousarray(a_list, dtype=np.int32)
        assert al.size == 0 or (al.min() >= 0 and al.max() < v)
        R = np.empty((o, o, al.size, v))
        lib.oracle_ladder(o, v, n, _p(L), _p(t2), _p(R), al.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          al.size, int(compensated), threads)
    return R


def ladder_eri(L, t2):
    lib = _load()
    L, t2 = _f64(L), _f64(t2)
    o, v, n = _shapes(L, t2)
    R = np.empty((o, o, v, v))
    eri = np.empty((v, v, v, v))
    lib.oracle_ladder_eri(o, v, n, _p(L), _p(t2), _p(R), _p(eri))
    return R


def ladder_entries(L, t2, idx, threads=0):
    """R.ravel()[idx] for flat indices into o*o*v*v, each computed on its own."""
    lib = _load()
    L, t2 = _f64(L), _f64(t2)
    o, v, n = _shapes(L, t2)
    ii = np.ascontiguousarray(idx, dtype=np.int64)
    assert ii.size == 0 or (ii.min() >= 0 and ii.max() < o * o * v * v)
    out = np.empty(ii.size)
    lib.oracle_ladder_entries(o, v, n, _p(L), _p(t2), ii.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                              ii.size, _p(out), threads)
    return out


def energy(R, t2, pair=False):
    lib = _load()
    R, t2 = _f64(R), _f64(t2)
    o, v = t2.shape[0], t2.shape[2]
    assert R.shape == t2.shape
    ep = np.empty((o, o)) if pair else None
    e = lib.oracle_energy(o, v, _p(R), _p(t2), _p(ep))
    return (e, ep) if pair else e


def energy_range(R, t2, lo, hi):
    """Terms of the pair energy with min(a, b) in [lo, hi): one part's share under an
    `a`-range partition of the pair-symmetric path."""
    lib = _load()
    R, t2 = _f64(R), _f64(t2)
    o, v = t2.shape[0], t2.shape[2]
    assert R.shape == t2.shape
    return lib.oracle_energy_range(o, v, _p(R), _p(t2), int(lo), int(hi))


def ladder_grad(L, t2, W, want_dL=True, want_dt2=True, threads=0):
    lib = _load()
    L, t2, W = _f64(L), _f64(t2), _f64(W)
    o, v, n = _shapes(L, t2)
    dL = np.empty_like(L) if want_dL else None
    dt2 = np.empty_like(t2) if want_dt2 else None
    lib.oracle_ladder_grad(o, v, n, _p(L), _p(t2), _p(W), _p(dL), _p(dt2), threads)
    return dL, dt2


def ladder_grad_entries(L, t2, W, dt2_idx, dL_idx, threads=0):
    """Flat-index entries of dt2 (into o*o*v*v) and dL (into n*v*v)."""
    lib = _load()
    L, t2, W = _f64(L), _f64(t2), _f64(W)
    o, v, n = _shapes(L, t2)
    i1 = np.ascontiguousarray(dt2_idx, dtype=np.int64)
    i2 = np.ascontiguousarray(dL_idx, dtype=np.int64)
    o1 = np.empty(i1.size)
    o2 = np.empty(i2.size)
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib.oracle_ladder_grad_entries(o, v, n, _p(L), _p(t2), _p(W), i1.ctypes.data_as(llp), i1.size, _p(o1),
                                   i2.ctypes.data_as(llp), i2.size, _p(o2), threads)
    return o1, o2


def exchange(L, t2, a_list=None, threads=0):
    lib = _load()
    L, t2 = _f64(L), _f64(t2)
    o, v, n = _shapes(L, t2)
    if a_list is None:
        X = np.empty((o, o, v, v))
        lib.oracle_exchange(o, v, n, _p(L), _p(t2), _p(X), None, 0, threads)
    else:
        al = np.ascontiguousarray(a_list, dtype=np.int32)
        X = np.empty((o, o, al.size, v))
        lib.oracle_exchange(o, v, n, _p(L), _p(t2), _p(X), al.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            al.size, threads)
    return X


def general(A, B, t2, threads=0):
    """G[i,j,p,q] = sum_cd (sum_P A[P,p,c] B[P,q,d]) t2[i,j,c,d]; A is n x np x v, B is n x nq x v."""
    lib = _load()
    A, B, t2 = _f64(A), _f64(B), _f64(t2)
    n, np_, v = A.shape
    n2, nq, v2 = B.shape
    o, o2, v3, v4 = t2.shape
    assert n == n2 and v == v2 == v3 == v4 and o == o2, (A.shape, B.shape, t2.shape)
    G = np.empty((o, o, np_, nq))
    lib.oracle_general(o, v, n, np_, nq, _p(A), _p(B), _p(t2), _p(G), threads)
    return G


def tijkl(Lov, t2, threads=0):
    """Eq. 8: tt[i,j,k,l] = sum_{P,c,d} Lov[P,k,c] Lov[P,l,d] t2[i,j,c,d]."""
    return general(Lov, Lov, t2, threads)


def tijbk(Lov, Lvv, t2, threads=0):
    """Eq. 9: tt[i,j,b,k] = sum_{P,c,d} Lvv[P,b,d] Lov[P,k,c] t2[i,j,c,d]."""
    return np.ascontiguousarray(general(Lov, Lvv, t2, threads).transpose(0, 1, 3, 2))
