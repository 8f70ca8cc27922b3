"""PNOF7 energy minimisation with the engine: outer and inner iterations.

Host orchestration only; every computation runs in the library's kernels.  The
scheme is the paper's (Sec. 2, Fig. "general scheme"): an outer iteration
optimises the occupations for fixed orbitals (J, K from one FULL transform,
donof_ri_optimize_occupations), and inner iterations optimise the orbitals for
fixed occupations (J^(q), K^(q) and the Lagrangian recomputed at every step).
Two inner steps: the plain rotation driver (donof_ri_rotate_orbitals: steepest
descent on dE/dkappa = 4 (lambda - lambda^T) with a trust radius that grows by
1.5 after an accepted step and halves after a rejected one), and the paper's
iterative diagonalisation of F^lambda (donof_ri_flambda_step,
flambda_iterations) with the same accept / reject control on its damping bound.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as bd


class _Inner:
    """Device state of the inner iterations of one engine."""

    def __init__(self, eng: "bd.Engine"):
        import torch
        self.eng = eng
        nb = eng.nbf
        self.dev = torch.device("cuda")
        self.C = torch.empty(nb * nb, dtype=torch.float64, device=self.dev)
        self.C_try = torch.empty_like(self.C)
        self.E = np.zeros(1)

    def evaluate(self, C_dev, gamma):
        """E at orbitals C_dev (also leaves lambda in the context for the next rotation)."""
        ctx = self.eng.ctx
        bd.donof_ri_transform(ctx, C_dev, bd.DONOF_RI_HALF)
        bd.donof_ri_jk_ao_batch(ctx)
        bd.donof_ri_energy_lagrangian(ctx, gamma, self.E, None)
        return float(self.E[0])


def orbital_iterations(eng, C_colmajor, gamma, max_iter=100, gtol=1e-4, etol=1e-10, radius=0.05, r_max=0.3,
                       state=None):
    """Inner iterations from C (column-major numpy or device tensor) at fixed gamma.
    Returns dict(C (column-major numpy), E, gmax, iterations, evaluations, ms_per_iteration, radius)."""
    import torch
    st = state or _Inner(eng)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    st.C.copy_(torch.as_tensor(np.ascontiguousarray(C_colmajor).reshape(-1)) if isinstance(C_colmajor, np.ndarray)
               else C_colmajor.reshape(-1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E = st.evaluate(st.C, gamma)
    evals, gmax, it = 1, float("inf"), 0
    g = np.zeros(1)
    for it in range(1, max_iter + 1):
        # rotation from the lambda of the current orbitals (left by the last accepted evaluation)
        bd.donof_ri_rotate_orbitals_dev(eng.ctx, radius, st.C_try, g)
        gmax = float(g[0])
        if gmax <= gtol:
            it -= 1
            break
        En = st.evaluate(st.C_try, gamma)
        evals += 1
        if En < E:
            dec = E - En
            st.C, st.C_try = st.C_try, st.C
            E = En
            radius = min(1.5 * radius, r_max)
            if dec <= etol * max(1.0, abs(E)):
                break
        else:
            radius *= 0.5
            E = st.evaluate(st.C, gamma)  # restore lambda at the accepted orbitals
            evals += 1
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(C=st.C.cpu().numpy().copy(), E=E, gmax=gmax, iterations=it, evaluations=evals,
                ms_per_iteration=1000.0 * dt / max(it, 1), radius=radius)


def flambda_iterations(eng, C_colmajor, gamma, max_iter=100, gtol=1e-4, etol=1e-10, bound=0.1, bound_max=1.0):
    """Inner iterations with the paper's step (donof_ri_flambda_step): F^lambda from the
    Lagrangian, eigenvalues of the accepted step as the next diagonal (lambda_pp at the
    first), off-diagonal elements damped to `bound`; a step that raises E is rejected
    and halves the bound, an accepted one grows it by 1.5 (up to bound_max).
    Returns dict(C, E, gmax, iterations, evaluations, energies, ms_per_iteration)."""
    import torch
    st = _Inner(eng)
    nb = eng.nbf
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    st.C.copy_(torch.as_tensor(np.ascontiguousarray(C_colmajor).reshape(-1)) if isinstance(C_colmajor, np.ndarray)
               else C_colmajor.reshape(-1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E = st.evaluate(st.C, gamma)
    energies = [E]
    diag = np.zeros(nb)
    have_diag = False
    evals, gmax, it = 1, float("inf"), 0
    for it in range(1, max_iter + 1):
        trial = np.empty(nb)
        if have_diag:
            trial[:] = diag
        gmax, _ = bd.donof_ri_flambda_step(eng.ctx, trial, not have_diag, bound, st.C_try)
        if gmax <= gtol:
            it -= 1
            break
        En = st.evaluate(st.C_try, gamma)
        evals += 1
        if En < E:
            dec = E - En
            st.C, st.C_try = st.C_try, st.C
            E = En
            diag[:] = trial
            have_diag = True
            bound = min(1.5 * bound, bound_max)
            energies.append(E)
            if dec <= etol * max(1.0, abs(E)):
                break
        else:
            bound *= 0.5
            E = st.evaluate(st.C, gamma)  # the Lagrangian of the accepted orbitals
            evals += 1
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(C=st.C.cpu().numpy().copy(), E=E, gmax=gmax, iterations=it, evaluations=evals, energies=energies,
                ms_per_iteration=1000.0 * dt / max(it, 1))


def solve(eng, C0, gamma0, max_outer=10, max_inner=50, etol=1e-6, gtol=1e-4, on_max_iter=20000):
    """Outer / inner iterations from orbitals C0 ([mu, p] numpy) and angles gamma0.
    Returns dict(C, gamma, E, outer, inner_total, history)."""
    C = bd.Engine.colmajor(C0)
    gamma = np.array(gamma0, dtype=np.float64)
    hist = []
    E_prev = None
    st = _Inner(eng)
    radius = 0.05
    total_inner = 0
    for o in range(1, max_outer + 1):
        bd.donof_ri_transform(eng.ctx, C, bd.DONOF_RI_FULL)
        gamma, E_on, _, it_on, _ = eng.optimize_occupations(gamma, max_iter=on_max_iter, gtol=1e-8, etol=1e-14)
        r = orbital_iterations(eng, C, gamma, max_iter=max_inner, gtol=gtol, radius=radius, state=st)
        C, radius = r["C"], max(r["radius"], 1e-3)
        total_inner += r["iterations"]
        hist.append(dict(outer=o, E_occ=E_on, on_iterations=it_on, E=r["E"], gmax=r["gmax"],
                         inner=r["iterations"], ms_per_inner=r["ms_per_iteration"]))
        if E_prev is not None and abs(r["E"] - E_prev) < etol and r["gmax"] < gtol:
            break
        E_prev = r["E"]
    return dict(C=C.reshape(eng.nbf, eng.nbf).T.copy(), gamma=gamma, E=hist[-1]["E"], outer=len(hist),
                inner_total=total_inner, history=hist)


def main():
    """Compare the FP64 and SLICE4 engines and the learned occupation guess on one workload:
    outer / inner iterations, energies, ms per inner iteration."""
    import argparse
    import json
    from synthetic import standard_gamma
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c6h12")
    ap.add_argument("--outer", type=int, default=4)
    ap.add_argument("--inner", type=int, default=25)
    ap.add_argument("--learned", type=int, default=0, help="train the warm-start network on this many rings first")
    args = ap.parse_args()
    eng0, w = bd.engine_and_workload(args.workload, bd.DONOF_RI_FP64)
    eng0.close()
    s = w.system
    g0 = standard_gamma(s.n_strong, s.n_weak_per)
    runs = [("fp64", bd.DONOF_RI_FP64, None), ("slice4", bd.DONOF_RI_SLICE4, None)]
    net = None
    if args.learned:
        from . import warmstart
        X, Y = warmstart.training_set(args.learned)
        net, _ = warmstart.train(X, Y)
        runs.append(("slice4+learned", bd.DONOF_RI_SLICE4, net))
    out = []
    for name, prec, nn in runs:
        eng = bd.Engine(s, prec)
        start = g0
        if nn is not None:
            eng.transform(w.C, bd.DONOF_RI_FULL)
            start = eng.gamma_guess(nn)
        t0 = time.perf_counter()
        r = solve(eng, w.C, start, max_outer=args.outer, max_inner=args.inner)
        dt = time.perf_counter() - t0
        eng.close()
        out.append(dict(form=name, E=r["E"], outer=r["outer"], inner_total=r["inner_total"], seconds=dt,
                        history=r["history"]))
    print(json.dumps({"workload": args.workload, "runs": out}))


if __name__ == "__main__":
    main()
