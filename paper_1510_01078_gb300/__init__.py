"""GB300-native NEDNER-NUFFT reconstruction for planar photoacoustic
tomography (Schmid et al., arXiv:1510.01078).

The compute path is the CUDA library built from ``csrc/`` (C-ABI declared in
``include/nedner.h``); ``nedner`` is its thin Python binding.  Importing this
package loads nothing: the library is opened on first use and the binding
raises if it is missing.
"""
__all__ = ["nedner", "inputs"]
