"""Workloads for the tests: the seeded synthetic inputs with orbitals C = S^-1/2 Q,
the overlap S taken from the oracle's integrals (test infrastructure only)."""
from __future__ import annotations

from oracle import integrals
from synthetic import systems


def make_workload(name: str, seed: int | None = None) -> systems.Workload:
    """A named workload whose orbitals are orthonormal in the overlap metric."""
    return systems.make_workload(name, integrals.overlap, seed=seed)


def ring_workload(n_c: int, seed: int, jitter: float = 0.05) -> systems.Workload:
    return systems.ring_workload(n_c, seed, integrals.overlap, jitter=jitter)
