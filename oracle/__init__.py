"""FP64 CPU oracle for the RI Coulomb/exchange engine of PNOF7 (test infrastructure).

This package is test infrastructure only.  It is a plain, slow, obviously
correct restatement of what the paper (arXiv 2012.15662) computes, written in
numpy/scipy FP64 with library primitives (matmul, einsum, Cholesky,
triangular solve) as its only building blocks.  It shares no code with the
CUDA engine: only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import it.  The engine never calls it.

Modules
-------
integrals  closed-form s-type Gaussian integrals (overlap, kinetic, nuclear
           attraction, two-, three- and four-centre Coulomb) via Boys F0.
modchol    the paper's modified Cholesky of the metric (Bunch-Kaufman LDL^T,
           Cheng-Higham correction of D's blocks) and the fit it defines.
ri         metric factorisation, fitted three-index tensor, the half / full
           MO transforms, J_pq / K_pq and the per-orbital AO J^(p) / K^(p)
           (Eq. AOERI and the RI equations of Sec. 2, Tables 2 and 3).
pnof7      occupation map, PNOF7 coupling coefficients, energy (Eq. PNOF) and
           the orthonormality Lagrangian.
brute      four-index fitted ERIs and the explicit O(N^5) transform of
           Eqs. (Jpq)-(Kpq) / Table 1, used to pin the factored path.
rhf        closed-shell determinant energy from the AO density, the special
           case PNOF7 reduces to when every strong orbital is fully occupied;
           the closed-shell Hartree-Fock orbitals of the NO guess (Sec. 4), by
           Roothaan-Hall iterations in the overlap metric with DIIS.
onopt      the occupation (gamma) optimisation for fixed orbitals: dE/dn,
           dn/dgamma, dE/dgamma and an L-BFGS minimiser (Sec. 2, "Occupancy
           Optimization with RI"), and the standard starting guess.
mlp        the learned warm start: per-subspace features, BF16-weight MLP
           forward pass, loss gradients and the Adam update.

Parity unpinned: the absolute PNOF7 energies of the synthetic systems (no
printed value exists for them); they are pinned only through the invariants,
brute-force equivalences, special cases and finite differences in the tests.
"""
