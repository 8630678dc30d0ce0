"""GB300-native Poisson-Fermi solver.

The solver of Chen, Chen and Liu ("A GPU Poisson-Fermi Solver for Ion Channel Simulations"):
Jacobi-preconditioned BiCGSTAB (Table 3) on the 7-point variable-dielectric operator with
SMIB/harmonic interface faces, inside the relaxed inexact-Newton PF iteration (Table 4) whose
pointwise step evaluates the Fermi-like concentrations and steric potential of Eq. (1), as
hand-written sm_103a CUDA kernels behind the C ABI of include/pf_gb300.h.

Importing the package loads nothing: `paper_1711_04060_gb300.api` loads libpf_gb300.so on first
use and fails loudly when it has not been built; `workloads` generates the seeded inputs.
"""
