"""GB300-native multigrid Monge-Ampere reconstruction (arXiv:1709.06350).

The compute path is ``librecon.so`` (hand-written sm_103a CUDA behind a C
ABI, declared in ``include/recon.h``); ``recon`` is its thin Python binding.
Importing the package does not load the library; the first call does, and
fails loudly when it has not been built.
"""
__all__ = ["recon", "synth", "analysis"]
