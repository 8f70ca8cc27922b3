"""RI error against exact four-centre integrals and the RI -> exact restart of the
occupation optimisation, at fixed orbitals (the paper's Table 4 measures the RI
error of converged PNOF7 energies; Sec. 4 restarts exact PNOF7 from RI).

For each workload, with the engine's FP64 form on one context:
  1. RI: FULL transform, occupation optimisation from the standard guess, then
     the energy at the optimised angles (E_RI);
  2. exact: donof_ri_exact_jk at the same orbitals, the energy at the RI angles
     (E_exact(gamma_RI)), then the occupation optimisation restarted from the RI
     angles (iterations, E_exact) and, for comparison, from the standard guess.
Prints one JSON line per workload.  Host orchestration only: every number comes
from the engine's kernels.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as bd


def run(name: str, gtol: float = 1e-8) -> dict:
    from synthetic import standard_gamma
    eng, w = bd.engine_and_workload(name, bd.DONOF_RI_FP64)
    s = w.system
    m = s.n_omega
    g0 = standard_gamma(s.n_strong, s.n_weak_per)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J_ri, K_ri = eng.jk_mo()
    g_ri, E_ri, _, it_ri, _ = eng.optimize_occupations(g0, max_iter=20000, gtol=gtol, etol=1e-14)
    J = np.empty((m, m))
    K = np.empty((m, m))
    t0 = time.perf_counter()
    bd.donof_ri_exact_jk(eng.ctx, bd.Engine.colmajor(w.C), J, K)
    t_exact = time.perf_counter() - t0
    _, E_ex_at_ri, _, _, _ = eng.optimize_occupations(g_ri, max_iter=0)
    g_rs, E_rs, _, it_rs, _ = eng.optimize_occupations(g_ri, max_iter=20000, gtol=gtol, etol=1e-14)
    _, E_std, _, it_std, _ = eng.optimize_occupations(g0, max_iter=20000, gtol=gtol, etol=1e-14)
    eng.close()
    return dict(workload=name, nbf=s.nbf, naux=s.naux, n_omega=m,
                E_ri=E_ri, E_exact_at_ri_angles=E_ex_at_ri, E_exact=E_rs, ri_error=E_ri - E_rs,
                max_dJ=float(np.abs(J - J_ri).max()), max_dK=float(np.abs(K - K_ri).max()),
                on_iterations_ri=it_ri, on_iterations_restart=it_rs, on_iterations_exact_from_guess=it_std,
                E_exact_from_guess=E_std, exact_jk_seconds=t_exact)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["square4", "c6h12"])
    args = ap.parse_args()
    for name in args.workloads:
        print(json.dumps(run(name)), flush=True)


if __name__ == "__main__":
    main()
