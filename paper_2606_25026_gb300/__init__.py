"""GB300-native split-step Schroedinger-Poisson solver (libspe) -- Python side.

Importing this package loads nothing: ``paper_2606_25026_gb300.spe`` is the ctypes binding of the
CUDA library, ``paper_2606_25026_gb300.inputs`` holds the seeded synthetic initial conditions,
and ``paper_2606_25026_gb300.build`` compiles libspe.so.
"""
