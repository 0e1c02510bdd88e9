"""tvbx: GB300 (sm_103a) engine for the TVB-AdEx parameter sweep of
arXiv 2311.13337 — lock-step integration of many whole-brain AdEx mean-field
simulations and their reduction to functional connectivity.

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``)
behind the C-ABI in ``include/tvbx.h``; ``tvbx`` is its Python binding and
``synth`` makes the seeded synthetic connectomes. Nothing here falls back to
the CPU.
"""
__all__ = ["tvbx", "synth", "build"]
