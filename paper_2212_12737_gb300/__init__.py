"""GB300-native preconditioned CG solver for GDML force-field kernel systems.

The compute path lives in the CUDA library built from ``csrc/`` (C ABI,
declared in ``include/gdml.h``); ``paper_2212_12737_gb300.gdml`` is its thin
Python binding.  ``synth`` draws seeded synthetic workloads.
"""
