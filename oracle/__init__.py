"""FP64 CPU oracle for the Yee FDTD hot path (test infrastructure only; see oracle.py)."""
