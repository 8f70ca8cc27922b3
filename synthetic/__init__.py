"""Seeded synthetic inputs shared by the oracle and the GPU engine.

This package holds only input generation: geometries, basis-set exponent
tables, the pairing (electron-pair subspace) map, orbital coefficient
matrices and occupation angles.  It contains none of the method's
arithmetic (no integrals, no fitting, no transforms, no energies), so the
oracle and the CUDA path may both draw their inputs from it without
sharing any computation.
"""
from .systems import (  # noqa: F401
    ANGSTROM_TO_BOHR,
    System,
    Workload,
    make_system,
    make_workload,
    orthonormal_orbitals,
    workload_system,
    pairing_columns,
    random_orthogonal,
    draw_gamma,
    ring_workload,
    standard_gamma,
    with_near_duplicate_aux,
    without_basis_functions,
    WORKLOADS,
)
