"""GB300-native TNMH proposal path (arXiv:2104.13264).

The compute lives in the C-ABI library ``libtnmc.so`` (CUDA, sm_103a) built
from ``csrc/``; ``binding`` marshals arguments to it.  Importing this package
loads nothing: the library is opened on first use by ``binding.lib()``, which
raises if it is missing.
"""
__all__ = ["binding", "instances"]
