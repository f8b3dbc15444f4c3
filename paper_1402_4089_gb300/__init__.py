"""GB300-native HMC for Bayesian multinomial regression (Beam, Ghosh & Doyle,
arXiv 1402.4089).

The compute path is the C-ABI library ``libhmc.so`` built from ``csrc/``
(hand-written sm_103a CUDA); ``hmc`` is its thin Python binding and
``autograd`` the ``torch.autograd.Function`` over it.  Submodules are imported
lazily so that the seeded input generator (``synthetic``) can be used without
the library.
"""
__all__ = ["hmc", "autograd", "synthetic", "build"]
