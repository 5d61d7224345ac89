"""GB300-native dual-tree-traversal FMM for the 3-D Laplace kernel (arXiv:1209.3516).

The compute path is the C-ABI library built from ``csrc/`` (hand-written
sm_103a CUDA kernels); ``fmm`` is its thin ctypes binding.  Importing this
package loads nothing: the binding loads the library on first use and raises
if it is missing.
"""
__all__ = ["fmm", "inputs"]
