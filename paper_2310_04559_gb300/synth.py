"""Seeded synthetic inputs for the particle-particle ladder term.

This module only draws random numbers; it holds none of the ladder arithmetic, so
both the CUDA path and the CPU oracle can take their inputs from it.

The paper benchmarks on random Cholesky vectors (Section 6.1: "random arrays" of
size 5K^3, i.e. n_chol = 5K vectors of K x K) and random amplitudes; it states
no distribution.  The recipe used here:

* ``L[P, a, c]``: draw ``X[P, a, c] ~ N(0, 1)`` for ``a <= c``, mirror it so that
  ``L[P, a, c] = L[P, c, a]`` (real orbitals, 8-fold ERI symmetry, Eq. 5 and the
  remark after it), then scale vector ``P`` (0-based) by ``exp(-5 P / n_chol)``
  so the vectors decay like a pivoted Cholesky decomposition.
* ``t2[i, j, a, b]``: draw ``X ~ N(0, sigma^2)`` with ``sigma = 1e-2`` and
  symmetrise ``t = (X + X^swap) / 2`` with ``X^swap[i, j, a, b] = X[j, i, b, a]``
  (the pair symmetry of closed-shell doubles amplitudes).
* ``W[i, j, a, b] ~ N(0, 1)``: a cotangent for the adjoint (``loss = <W, R>``).

All arrays are float64, C-contiguous, row-major.
"""
from __future__ import annotations

import numpy as np

__all__ = ["cholesky_vectors", "amplitudes", "cholesky_ov", "cotangent", "ladder_inputs", "ladder_inputs_torch",
           "WORKLOADS"]

# Named workloads (o occupied, v virtual, n Cholesky vectors).  The paper's
# synthetic shapes (Section 6.2, Table 1) use n = 5K, v = int(3K/4), o = K - v;
# the workloads below follow the same o << v << n regime.
WORKLOADS = {
    "tiny_o4_v24_n60": (4, 24, 60),
    "o20_v200_n1000": (20, 200, 1000),
    "o40_v400_n2000": (40, 400, 2000),
    "adjoint_o16_v160_n800": (16, 160, 800),
    "large_o60_v600_n3000": (60, 600, 3000),
    "crossover_o4_v96_n480": (4, 96, 480),
}


def cholesky_vectors(n: int, v: int, seed: int = 0, symmetric: bool = True,
                     decay: float = 5.0, rng: np.random.Generator | None = None) -> np.ndarray:
    """Random Cholesky vectors ``L[P, a, c]`` (n x v x v, float64)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    x = rng.standard_normal((n, v, v))
    if symmetric:
        iu = np.triu_indices(v, 1)
        # keep the a <= c triangle as drawn, mirror it onto a > c
        x[:, iu[1], iu[0]] = x[:, iu[0], iu[1]]
    if decay:
        x *= np.exp(-decay * np.arange(n, dtype=np.float64) / max(n, 1))[:, None, None]
    return np.ascontiguousarray(x)


def amplitudes(o: int, v: int, seed: int = 1, sigma: float = 1e-2, symmetric: bool = True,
               rng: np.random.Generator | None = None) -> np.ndarray:
    """Random doubles amplitudes ``t2[i, j, a, b]`` (o x o x v x v, float64)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    x = sigma * rng.standard_normal((o, o, v, v))
    if symmetric:
        x = 0.5 * (x + x.transpose(1, 0, 3, 2))
    return np.ascontiguousarray(x)


def cholesky_ov(n: int, o: int, v: int, seed: int = 3, decay: float = 5.0,
                rng: np.random.Generator | None = None) -> np.ndarray:
    """Random occupied-virtual Cholesky block ``Lov[P, k, c]`` (n x o x v), vector P scaled by exp(-decay P / n)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    x = rng.standard_normal((n, o, v))
    x *= np.exp(-decay * np.arange(n, dtype=np.float64) / max(n, 1))[:, None, None]
    return np.ascontiguousarray(x)


def cotangent(o: int, v: int, seed: int = 2, rng: np.random.Generator | None = None) -> np.ndarray:
    """Random cotangent ``W[i, j, a, b] ~ N(0, 1)`` for ``loss = sum W * R``."""
    rng = np.random.default_rng(seed) if rng is None else rng
    return np.ascontiguousarray(rng.standard_normal((o, o, v, v)))


def ladder_inputs(o: int, v: int, n: int, seed: int = 0, symmetric: bool = True):
    """(L, t2) for one workload; one generator drives both so a seed fixes the pair."""
    rng = np.random.default_rng(seed)
    L = cholesky_vectors(n, v, symmetric=symmetric, rng=rng)
    t2 = amplitudes(o, v, symmetric=symmetric, rng=rng)
    return L, t2


def ladder_inputs_torch(o: int, v: int, n: int, seed: int = 0, device="cuda"):
    """(L, t2) by the same recipe, drawn with torch's generator on `device` (for workloads whose
    host-side generation would take minutes, e.g. o = 60, v = 600, n = 3000).  The numbers differ
    from ladder_inputs' for the same seed; the distributions and symmetries are the same."""
    import torch

    g = torch.Generator(device=device).manual_seed(seed)
    L = torch.randn((n, v, v), generator=g, dtype=torch.float64, device=device)
    iu = torch.triu_indices(v, v, 1, device=device)
    L[:, iu[1], iu[0]] = L[:, iu[0], iu[1]]
    L *= torch.exp(-5.0 * torch.arange(n, dtype=torch.float64, device=device) / max(n, 1))[:, None, None]
    x = torch.randn((o, o, v, v), generator=g, dtype=torch.float64, device=device).mul_(1e-2)
    t2 = x.permute(1, 0, 3, 2).contiguous().add_(x).mul_(0.5)
    del x
    return L.contiguous(), t2
