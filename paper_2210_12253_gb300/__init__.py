"""GB300-native low-order-refined (LOR) preconditioning for high-order H1
diffusion on hexahedral meshes (arXiv 2210.12253).

The compute path is the C-ABI library ``liblor`` (hand-written CUDA for
sm_103a, declared in ``include/lor.h``); this package only marshals
arguments to it.  Importing the package does not load the library; the first
call does, and it raises if the library is missing.
"""
