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
    """Device state of the inner iterations of one engine.  exact: the energy and
    Lagrangian from exact four-centre J^(q), K^(q) (donof_ri_exact_jk, FP64 contexts)
    instead of the RI transforms (the paper's RI -> exact restart)."""

    def __init__(self, eng: "bd.Engine", exact: bool = False):
        import torch
        self.eng = eng
        self.exact = exact
        nb = eng.nbf
        self.dev = torch.device("cuda")
        self.C = torch.empty(nb * nb, dtype=torch.float64, device=self.dev)
        self.C_try = torch.empty_like(self.C)
        self.E = np.zeros(1)
        self.lam = np.empty(nb * nb)

    def evaluate(self, C_dev, gamma, want_lambda=False):
        """E at orbitals C_dev (also leaves lambda in the context for the next step)."""
        ctx = self.eng.ctx
        if self.exact:
            bd.donof_ri_exact_jk(ctx, C_dev)
        else:
            bd.donof_ri_transform(ctx, C_dev, bd.DONOF_RI_HALF)
            bd.donof_ri_jk_ao_batch(ctx)
        bd.donof_ri_energy_lagrangian(ctx, gamma, self.E, self.lam if want_lambda else None)
        return float(self.E[0])

    def gmax(self):
        """max |lambda - lambda^T| of the last evaluate(want_lambda=True)."""
        nb = self.eng.nbf
        lam = self.lam.reshape(nb, nb)
        return float(np.abs(lam - lam.T).max())


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


def _gap_floor(d, gapmin):
    """The aufbau diagonal with every gap raised to at least gapmin (ascending)."""
    out = np.array(d, dtype=np.float64, copy=True)
    for k in range(1, out.size):
        out[k] = max(out[k], out[k - 1] + gapmin)
    return out


def flambda_iterations(eng, C_colmajor, gamma, max_iter=100, gtol=1e-4, etol=1e-10, bound=0.1, bound_max=1.0,
                       diag0=None, gapmin=0.0, relative_bound=False, state=None):
    """Inner iterations with the paper's step (donof_ri_flambda_step): F^lambda from the
    Lagrangian, eigenvalues of the accepted step as the next diagonal (diag0, else
    lambda_pp, at the first), off-diagonal elements damped to `bound` (times the
    max |lambda - lambda^T| at the start when relative_bound); a step that raises E is
    rejected and halves the bound, an accepted one grows it by 1.5 (up to bound_max).
    gapmin > 0 raises every gap of the ascending diagonal to at least gapmin, so that
    degenerate orbitals of different pairing subspaces are not mixed by 45 degrees.
    Returns dict(C, E, gmax, iterations, evaluations, energies, ms_per_iteration, diag)."""
    import torch
    st = state or _Inner(eng)
    nb = eng.nbf
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    st.C.copy_(torch.as_tensor(np.ascontiguousarray(C_colmajor).reshape(-1)) if isinstance(C_colmajor, np.ndarray)
               else C_colmajor.reshape(-1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E = st.evaluate(st.C, gamma, want_lambda=relative_bound)
    if relative_bound:
        bound = bound * max(st.gmax(), 1e-12)
    energies = [E]
    diag = np.zeros(nb) if diag0 is None else np.array(diag0, dtype=np.float64)
    have_diag = diag0 is not None
    evals, gmax, it = 1, float("inf"), 0
    for it in range(1, max_iter + 1):
        trial = np.empty(nb)
        if have_diag:
            trial[:] = _gap_floor(diag, gapmin) if gapmin > 0 else diag
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
                ms_per_iteration=1000.0 * dt / max(it, 1), diag=diag.copy())


def lbfgs_iterations(eng, C_colmajor, gamma, eps, max_iter=200, gtol=1e-4, memory=10, max_step=0.5,
                     hmin=1e-2, state=None):
    """Quasi-Newton inner iterations (an addition beside the paper's F^lambda step): L-BFGS
    on the rotation generator, C <- C expm(kappa) (donof_ri_apply_rotation), with the
    gradient dE/dkappa_qp = 4 (lambda_qp - lambda_pq) (q > p) from the engine's
    Lagrangian and the initial inverse Hessian diag 1 / max(4 |n_p - n_q| |eps_p - eps_q|,
    hmin): the orbital-energy model of a determinant's Hessian weighted by the
    occupation difference of the pair (n = 0 outside the pairing space), eps orbital
    energies (the HF ones), n the occupations of the current angles.  Pairs are kept
    as they are (no parallel transport), a step is capped at max_step radians and an
    Armijo backtracking line search on E accepts it.  Stops when max |lambda -
    lambda^T| <= gtol.  With a mixed-precision engine, whose energy carries rounding
    noise of about 1e-11 |E| between nearby orbitals, a step that changes E by less
    than that noise is also accepted when it lowers max |lambda - lambda^T| (near
    convergence the decrease a step buys falls below the noise, and the gradient,
    good to about 1e-8, still points the way).  Returns dict(C, E, gmax, iterations,
    evaluations, ms_per_iteration)."""
    import torch
    st = state or _Inner(eng)
    nb = eng.nbf
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    C_cur = np.ascontiguousarray(C_colmajor, dtype=np.float64).reshape(-1).copy()
    il = np.tril_indices(nb, -1)
    eps = np.asarray(eps, dtype=np.float64)

    def evaluate(Ccm):
        st.C.copy_(torch.as_tensor(Ccm))
        E = st.evaluate(st.C, gamma, want_lambda=True)
        lam = st.lam.reshape(nb, nb).T  # lambda[q][p] (the ABI returns it column-major)
        G = lam - lam.T
        return E, 4.0 * G[il], float(np.abs(G).max())

    def kappa_of(x):
        K = np.zeros((nb, nb))
        K[il] = x
        return K - K.T

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, g, gmax = evaluate(C_cur)
    noise = 0.0 if getattr(eng, "precision", bd.DONOF_RI_FP64) == bd.DONOF_RI_FP64 else 1e-11 * max(1.0, abs(E))
    n = np.zeros(nb)
    n[:eng.n_omega] = eng.fetch(bd.DONOF_RI_FETCH_OCC)
    h0 = 1.0 / np.maximum(4.0 * np.abs(n[il[0]] - n[il[1]]) * np.abs(eps[il[0]] - eps[il[1]]), hmin)
    S, Y = [], []
    evals, it = 1, 0
    Ctry = np.empty(nb * nb)
    for it in range(1, max_iter + 1):
        if gmax <= gtol:
            it -= 1
            break
        # two-loop recursion
        q = g.copy()
        alphas = []
        for s_, y_ in reversed(list(zip(S, Y))):
            rho = 1.0 / float(y_ @ s_)
            a = rho * float(s_ @ q)
            alphas.append((a, rho, s_, y_))
            q -= a * y_
        if S:
            gam = float(S[-1] @ Y[-1]) / float(Y[-1] @ (h0 * Y[-1]))
            r = gam * h0 * q
        else:
            r = h0 * q
        for a, rho, s_, y_ in reversed(alphas):
            b = rho * float(y_ @ r)
            r += (a - b) * s_
        d = -r
        slope = float(g @ d)
        if not slope < 0.0:  # not a descent direction: restart from the preconditioned gradient
            S, Y = [], []
            d = -h0 * g
            slope = float(g @ d)
        dmax = float(np.abs(d).max())
        alpha = min(1.0, max_step / dmax) if dmax > 0 else 1.0
        accepted = False
        for _ in range(12):
            bd.donof_ri_apply_rotation(eng.ctx, kappa_of(alpha * d), Ctry)
            # apply_rotation rotated the context's own orbitals: start each trial from C_cur
            En, gn, gmn = evaluate(Ctry)
            evals += 1
            if En <= E + 1e-4 * alpha * slope or (noise > 0.0 and En <= E + noise and gmn < gmax):
                accepted = True
                break
            alpha *= 0.5
            st.C.copy_(torch.as_tensor(C_cur))
            bd.donof_ri_transform(eng.ctx, st.C, bd.DONOF_RI_HALF)  # back to the accepted orbitals
        if not accepted:
            evaluate(C_cur)  # leave the context at the accepted orbitals
            break
        sk, yk = alpha * d, gn - g
        if float(sk @ yk) > 1e-12 * float(yk @ yk):
            S.append(sk)
            Y.append(yk)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        C_cur, E, g, gmax = Ctry.copy(), En, gn, gmn
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(C=C_cur.copy(), E=E, gmax=gmax, iterations=it, evaluations=evals,
                ms_per_iteration=1000.0 * dt / max(it, 1))


def converge(eng, C0, gamma0, diag0, etol=1e-6, gtol=1e-4, max_outer=60, max_inner=100, gapmin=0.01, exact=False,
             on_max_iter=20000, time_limit=None, log=None, inner="flambda"):
    """The paper's outer / inner scheme to convergence with the F^lambda step: per outer
    iteration J, K of the current orbitals (one FULL transform, or exact four-centre
    integrals when exact), the occupation optimisation, then F^lambda inner iterations
    until max |lambda - lambda^T| <= gtol (at most max_inner).  Stops when an outer
    iteration changes E by less than etol with max |lambda - lambda^T| <= gtol.
    C0 [mu, p] numpy, gamma0, diag0 (the starting aufbau diagonal, e.g. the RHF orbital
    energies).  Returns dict(C, gamma, E, outer, inner_total, converged, seconds,
    ms_per_inner, history, diag).  time_limit (seconds): stop after the outer iteration
    that passes it (converged stays False); log: called with each outer iteration's
    record.  inner: "flambda" (the paper's step) or "lbfgs" (lbfgs_iterations, with
    diag0 as its orbital energies)."""
    import torch
    C = bd.Engine.colmajor(C0)
    gamma = np.array(gamma0, dtype=np.float64)
    diag = np.array(diag0, dtype=np.float64)
    st = _Inner(eng, exact=exact)
    hist, E_prev, total_inner, converged = [], None, 0, False
    t_inner = 0.0
    t0 = time.perf_counter()
    for o in range(1, max_outer + 1):
        if exact:
            bd.donof_ri_exact_jk(eng.ctx, C)
        else:
            bd.donof_ri_transform(eng.ctx, C, bd.DONOF_RI_FULL)
        gamma, E_on, _, it_on, _ = eng.optimize_occupations(gamma, max_iter=on_max_iter, gtol=1e-8, etol=1e-14)
        ti = time.perf_counter()
        if inner == "lbfgs":
            r = lbfgs_iterations(eng, C, gamma, diag0, max_iter=max_inner, gtol=gtol, state=st)
        else:
            r = flambda_iterations(eng, C, gamma, max_iter=max_inner, gtol=gtol, etol=1e-10, bound=0.1,
                                   bound_max=1.0, diag0=diag, gapmin=gapmin, relative_bound=True, state=st)
            diag = r["diag"]
        t_inner += time.perf_counter() - ti
        C = r["C"]
        total_inner += r["iterations"]
        hist.append(dict(outer=o, E_occ=E_on, on_iterations=it_on, E=r["E"], gmax=r["gmax"], inner=r["iterations"],
                         seconds=time.perf_counter() - t0))
        if log is not None:
            log(hist[-1])
        if E_prev is not None and abs(r["E"] - E_prev) < etol and r["gmax"] <= gtol:
            converged = True
            break
        E_prev = r["E"]
        if time_limit is not None and time.perf_counter() - t0 > time_limit:
            break
    torch.cuda.synchronize()
    return dict(C=C.reshape(eng.nbf, eng.nbf).T.copy(), gamma=gamma, E=hist[-1]["E"], outer=len(hist),
                inner_total=total_inner, converged=converged, seconds=time.perf_counter() - t0,
                ms_per_inner=1000.0 * t_inner / max(total_inner, 1), history=hist, diag=diag)


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
    """The paper's scheme to convergence from the RI-HF orbitals on one workload, with the
    FP64 and SLICE4 engines (and the learned occupation guess when --learned > 0):
    outer / inner iterations, energies, ms per inner iteration; with --restart, the
    converged FP64 RI run restarted with exact four-centre integrals (nbf <= 256).
    --checkpoint PATH writes the converged FP64 RI state (and, after --restart, the
    exact one to PATH_exact) as PATH.json + PATH.bin; --resume PATH starts from such a
    state instead of the RI-HF guess (with --forms "" and --restart: the exact restart
    straight from the file)."""
    import argparse
    import json
    from synthetic import standard_gamma
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c6h12")
    ap.add_argument("--outer", type=int, default=60)
    ap.add_argument("--inner", type=int, default=100)
    ap.add_argument("--etol", type=float, default=1e-6)
    ap.add_argument("--gtol", type=float, default=1e-4)
    ap.add_argument("--gapmin", type=float, default=0.01)
    ap.add_argument("--forms", default="fp64,slice4")
    ap.add_argument("--inner-step", default="flambda", choices=["flambda", "lbfgs"])
    ap.add_argument("--learned", type=int, default=0, help="train the warm-start network on this many rings first")
    ap.add_argument("--restart", action="store_true", help="restart the converged FP64 run with exact integrals")
    ap.add_argument("--time-limit", type=float, default=None, help="seconds per converge() run")
    ap.add_argument("--checkpoint", default=None, help="write the converged FP64 states to PATH.json / PATH.bin")
    ap.add_argument("--resume", default=None, help="start from a state written by --checkpoint")
    args = ap.parse_args()
    import sys

    def log(rec):
        print(json.dumps(rec), file=sys.stderr, flush=True)
    from .checkpoint import load_state, save_state
    eng0, w = bd.engine_and_workload(args.workload, bd.DONOF_RI_FP64)
    s = w.system
    state = None
    if args.resume:
        state = load_state(args.resume, workload=args.workload, nbf=s.nbf)
        C0, eps0, g0 = state["C"], state["diag"], state["gamma"]
        start_rec = {"resumed_from": args.resume, "E": state["E"], "outer": state["outer"], "form": state["form"]}
    else:
        t0 = time.perf_counter()
        C0, eps0, E_hf, it_hf, com = eng0.rhf(max_iter=200, tol=1e-8)
        t_hf = time.perf_counter() - t0
        g0 = standard_gamma(s.n_strong, s.n_weak_per)
        start_rec = {"E": E_hf, "iterations": it_hf, "commutator": com, "seconds": t_hf}
    runs = [(f, {"fp64": bd.DONOF_RI_FP64, "slice4": bd.DONOF_RI_SLICE4}[f], None)
            for f in args.forms.split(",") if f]
    if args.learned:
        from . import warmstart
        X, Y = warmstart.training_set(args.learned, orbitals="rhf")
        net, _ = warmstart.train(X, Y)
        runs.append(("slice4+learned", bd.DONOF_RI_SLICE4, net))
    out, conv64 = [], None
    for name, prec, nn in runs:
        eng = eng0 if prec == bd.DONOF_RI_FP64 else bd.Engine(s, prec)
        start = g0
        if nn is not None:
            eng.transform(C0, bd.DONOF_RI_FULL)
            start = eng.gamma_guess(nn)
        print(f"# {name}", file=sys.stderr, flush=True)
        r = converge(eng, C0, start, eps0, etol=args.etol, gtol=args.gtol, max_outer=args.outer,
                     max_inner=args.inner, gapmin=args.gapmin, time_limit=args.time_limit, log=log,
                     inner=args.inner_step)
        if prec == bd.DONOF_RI_FP64 and conv64 is None:
            conv64 = r
        else:
            eng.close()
        out.append(dict(form=name, E=r["E"], converged=r["converged"], outer=r["outer"],
                        inner_total=r["inner_total"], seconds=r["seconds"], ms_per_inner=r["ms_per_inner"],
                        history=r["history"]))
    line = {"workload": args.workload, "inner_step": args.inner_step,
            ("start" if state is not None else "rhf"): start_rec, "runs": out}
    if args.checkpoint and conv64 is not None:
        save_state(args.checkpoint, args.workload, conv64["C"], conv64["gamma"], conv64["diag"], conv64["E"],
                   conv64["outer"], conv64["converged"], "fp64")
    if conv64 is None and state is not None:
        conv64 = dict(C=C0, gamma=g0, diag=eps0, E=state["E"])  # the restart starts from the file
    if args.restart and conv64 is not None:
        print("# exact restart", file=sys.stderr, flush=True)
        r = converge(eng0, conv64["C"], conv64["gamma"], conv64["diag"], etol=args.etol, gtol=args.gtol,
                     max_outer=args.outer, max_inner=args.inner, gapmin=args.gapmin, exact=True,
                     time_limit=args.time_limit, log=log, inner=args.inner_step)
        line["restart_exact"] = dict(E=r["E"], converged=r["converged"], outer=r["outer"],
                                     inner_total=r["inner_total"], seconds=r["seconds"],
                                     ri_error=conv64["E"] - r["E"], history=r["history"])
        if args.checkpoint:
            save_state(args.checkpoint + "_exact", args.workload, r["C"], r["gamma"], r["diag"], r["E"], r["outer"],
                       r["converged"], "fp64-exact")
    eng0.close()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
