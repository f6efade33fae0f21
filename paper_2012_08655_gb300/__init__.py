"""GB300-native block-wise foveated Gaussian blur (arXiv 2012.08655).

The compute path is the C-ABI library ``libfovea.so`` (hand-written sm_103a
CUDA kernels) declared in ``include/fovea.h``; ``paper_2012_08655_gb300.fovea``
is its thin ctypes binding plus the ``torch.autograd.Function``. Importing this
package does not load the library; importing ``fovea`` does, and it raises if
the library was not built (there is no CPU fallback).
"""
