"""GB300-native low-order-refined (LOR) preconditioning for high-order H1
diffusion on hexahedral meshes (arXiv 2210.12253).

The compute path is the C-ABI library ``liblor`` (hand-written CUDA for
sm_103a, declared in ``include/lor.h``); ``lor.py`` only marshals arguments
to it.  Importing the package does not load the library; creating an ``LOR``
context does, and raises if the library is missing (there is no CPU path).
"""
from .lor import (LOR, LORApply, LORError, LORSolve, load_library, solve, solve_with_adjoint,  # noqa: F401
                  LOR_F32, LOR_F64, LOR_PRECOND_CHEB, LOR_PRECOND_JACOBI, LOR_PRECOND_NONE)
