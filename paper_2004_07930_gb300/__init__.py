"""GB300-native two-level ORAS-preconditioned GMRES for the 3D P3 Helmholtz system.

Kept import-light: the seeded input generators (`workloads`) load without the
CUDA library; the solver binding lives in `paper_2004_07930_gb300.hz`.
"""
