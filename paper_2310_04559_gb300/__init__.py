"""GB300 (sm_103a) particle-particle ladder term of Cholesky-decomposed CCSD
(arXiv:2310.04559): R[i,j,a,b] = sum_cd (sum_P L[P,a,c] L[P,b,d]) t2[i,j,c,d].

The computation lives in libcc_ladder.so (csrc/, C ABI in include/cc_ladder.h);
this package only builds it, marshals arguments and wraps it for PyTorch.
Importing the package does not load the library; the first call does, and it
raises if the library is missing.
"""
from .binding import (LadderFunction, alloc_workspace, gemm, ladder, ladder_backward, ladder_forward, make_args,
                     pair_energy, plan, workspace_size)

__all__ = ["ladder", "ladder_forward", "ladder_backward", "pair_energy", "plan", "workspace_size",
           "alloc_workspace", "make_args", "LadderFunction", "gemm"]
