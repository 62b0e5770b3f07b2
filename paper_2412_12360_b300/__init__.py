"""B300-native time-reversible 3D FDTD (Yee leapfrog, CPML, soft sources, detectors, and the
time-reversal gradient dL/deps of arXiv 2412.12360, Sec. 2.1-2.2).

Importing the package loads nothing native; `paper_2412_12360_b300.fdtd` loads the CUDA library and
fails loudly if it is missing.
"""
