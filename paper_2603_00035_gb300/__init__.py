"""GB300-native differentiable Randers eikonal solver (arXiv 2603.00035).

The hot path -- feasibility projection, forward fast sweep with stencil
record, adjoint and parameter gradients -- runs in librf (CUDA, sm_103a,
C ABI in include/rf.h).  This package is its thin Python face:

* ``build``   -- compiles librf.so in-tree;
* ``api``     -- torch-tensor wrappers named after the C entry points;
* ``autograd`` -- ``RFSolve``, a torch.autograd.Function over the path.

Importing the package does not load the CUDA library; the first call does,
and raises if it is missing (there is no CPU fallback).
"""
__all__ = ["build", "api", "autograd"]
