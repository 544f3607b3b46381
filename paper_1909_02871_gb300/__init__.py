"""GF(2^n) random linear network coding on NVIDIA GB300 (sm_103a).

The compute path lives in the CUDA library ``libgf_gb300.so`` built from
``csrc/`` and declared by ``include/gf.h``; :mod:`.gf` is its thin ctypes
binding (argument marshalling only).  :mod:`.synth` draws the seeded
synthetic inputs.  Importing the package does not load the library; the
first call through :mod:`.gf` does, and fails loudly if it is missing.
"""
__all__ = ["gf", "synth", "build"]
