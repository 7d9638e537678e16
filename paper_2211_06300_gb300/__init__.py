"""GB300-native time-domain extended-source inversion (ESI) hot path.

The compute path lives in the C-ABI library ``libesi.so`` (CUDA, sm_103a) built from
``csrc/``; ``esi`` is its thin Python binding.  ``synth`` generates seeded synthetic
inputs.  Importing the package does not load the library; ``esi.load()`` does, and it
raises if the library is missing or no CUDA device is present.
"""
__all__ = ["synth", "esi"]
