"""Learned warm start for the occupation optimisation: data, training, evaluation.

Host orchestration only; every computation runs in the library's kernels:
the engine produces J, K (donof_ri_transform), the per-subspace features
(donof_ri_on_features) and the converged angles (donof_ri_optimize_occupations,
returned folded into [0, pi/2]); the network is trained by donof_mlp_train_step
(forward, backward and Adam kernels) and applied by donof_ri_gamma_guess.

The training targets are the converged angles the method itself generates on
seeded synthetic rings (C6-C12, jitter 0.05 A, orbitals S^-1/2 Q with Q
Haar-random and S the overlap the engine evaluates for each ring), one
sample per pairing subspace; the features are z-scored with the training set's
mean and standard deviation.

    python -m paper_2012_15662_gb300.warmstart --train 300 --eval c20h40
trains on 300 rings and compares, on the evaluation workload, the iterations
and time of the occupation optimisation from the standard guess and from the
network's guess (the converged energies must agree: the plain optimiser judges).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as bd

N_HIDDEN = 64


def targets(gamma: np.ndarray, n_strong: int, n_weak_per: int) -> np.ndarray:
    """Folded angles -> rows [N_I][N_g]: strong angle, then the subspace's weak angles."""
    Y = np.empty((n_strong, n_weak_per), dtype=np.float32)
    Y[:, 0] = gamma[:n_strong]
    Y[:, 1:] = gamma[n_strong:].reshape(n_strong, n_weak_per - 1)
    return Y


def sample(n_c, seed, precision=bd.DONOF_RI_SLICE4, max_iter=20000, etol=1e-13, jitter=0.05, orbitals="random"):
    """(features, targets, iterations, energy) of one seeded ring from the standard guess;
    orbitals "random" (S^-1/2 Q) or "rhf" (the ring's RI-HF orbitals, donof_ri_rhf)."""
    from synthetic import make_system, ring_workload, standard_gamma
    eng = bd.Engine(make_system("ring", n_c=n_c, seed=seed, jitter=jitter), precision)
    try:
        workload = ring_workload(n_c, seed, eng.overlap(), jitter=jitter)
        s = workload.system
        C = workload.C if orbitals == "random" else eng.rhf(max_iter=30, tol=1e-6)[0]
        eng.transform(C, bd.DONOF_RI_FULL)
        X = eng.on_features()
        g0 = standard_gamma(s.n_strong, s.n_weak_per)
        gam, E, grad, it, reason = eng.optimize_occupations(g0, max_iter=max_iter, gtol=1e-8, etol=etol)
        return X, targets(gam, s.n_strong, s.n_weak_per), it, E
    finally:
        eng.close()


def training_set(n_systems: int, first_seed: int = 1000, n_c_range=(6, 12), precision=bd.DONOF_RI_SLICE4,
                 orbitals="random", max_seconds=None, log=None, info=None):
    """Features and targets of n_systems seeded rings (C6..C12 in turn).  max_seconds:
    stop adding rings once the data generation has taken that long (the rings used are
    the first info["rings"] of the sequence); log(k, seconds) is called every 100 rings."""
    lo, hi = n_c_range
    Xs, Ys = [], []
    t0 = time.perf_counter()
    for k in range(n_systems):
        n_c = lo + k % (hi - lo + 1)
        X, Y, _, _ = sample(n_c, first_seed + k, precision, orbitals=orbitals)
        Xs.append(X)
        Ys.append(Y)
        dt = time.perf_counter() - t0
        if log is not None and (k + 1) % 100 == 0:
            log(k + 1, dt)
        if max_seconds is not None and dt > max_seconds:
            break
    if info is not None:
        info["rings"] = len(Xs)
    return np.concatenate(Xs), np.concatenate(Ys)


def init_params(n_in, n_hidden, n_out, y_mean, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) matrices, zero hidden biases, output bias at the target mean."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (n_hidden, n_in)) / np.sqrt(n_in)
    W2 = rng.uniform(-1, 1, (n_hidden, n_hidden)) / np.sqrt(n_hidden)
    W3 = rng.uniform(-1, 1, (n_out, n_hidden)) / np.sqrt(n_hidden)
    parts = [W1, np.zeros(n_hidden), W2, np.zeros(n_hidden), W3, np.full(n_out, y_mean)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def train(X, Y, steps=6000, batch=1024, lr=3e-3, weight_decay=1e-4, seed=0, net=None):
    """Train a network on (X, Y); returns (net, final loss)."""
    n_in, n_out = X.shape[1], Y.shape[1]
    if net is None:
        net = bd.Mlp(n_in, N_HIDDEN, n_out, max_batch=max(batch, X.shape[0]))
        net.set_params(init_params(n_in, N_HIDDEN, n_out, float(Y.mean()), seed))
        mu = X.mean(axis=0)
        sd = X.std(axis=0)
        net.set_normalization(mu, 1.0 / np.where(sd > 0, sd, 1.0))
    rng = np.random.default_rng(seed + 1)
    loss = np.zeros(1, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    for step in range(steps):
        idx = rng.integers(0, X.shape[0], min(batch, X.shape[0]))
        net.train_step(X[idx], Y[idx], lr, weight_decay, loss if step == steps - 1 else None)
    return net, float(loss[0])


def compare(workload, net, precision=bd.DONOF_RI_SLICE4, clip=0.05, max_iter=20000, etol=1e-13, eng=None):
    """Occupation optimisation of one system (a synthetic.Workload) from the standard
    and from the learned guess; `eng` a context of that system (made and closed here
    when None)."""
    from synthetic import standard_gamma
    s = workload.system
    if eng is None:
        eng = bd.Engine(s, precision)
    try:
        eng.transform(workload.C, bd.DONOF_RI_FULL)
        out = {}
        for name in ("standard", "learned"):
            bd.donof_ri_sync(eng.ctx)
            t0 = time.perf_counter()
            g0 = standard_gamma(s.n_strong, s.n_weak_per) if name == "standard" else eng.gamma_guess(net, clip)
            gam, E, grad, it, reason = eng.optimize_occupations(g0, max_iter=max_iter, gtol=1e-8, etol=etol)
            dt = time.perf_counter() - t0
            _, E0, _, _, _ = eng.optimize_occupations(g0, max_iter=0)
            out[name] = {"iterations": it, "E": E, "E_start": E0, "ms": 1000.0 * dt, "stop": reason}
        return out
    finally:
        eng.close()


def loop_compare(name, net, seed=None, clip=0.05, time_limit=600.0):
    """The full mixed-precision ON + NO loop (solve.converge with the quasi-Newton orbital
    step, DONOF_RI_SLICE4) on a named workload from its RI-HF orbitals, from the standard
    occupation guess and from the network's: outer and inner iterations, the first
    occupation optimisation's iterations, seconds, converged energy."""
    from synthetic import standard_gamma
    from . import solve
    eng, w = bd.engine_and_workload(name, bd.DONOF_RI_SLICE4, seed=seed)
    s = w.system
    try:
        C0, eps0, E_hf, it_hf, _ = eng.rhf(max_iter=200, tol=1e-8)
        out = {"rhf": {"E": E_hf, "iterations": it_hf}}
        for label in ("standard", "learned"):
            if label == "standard":
                g0 = standard_gamma(s.n_strong, s.n_weak_per)
            else:
                eng.transform(C0, bd.DONOF_RI_FULL)
                g0 = eng.gamma_guess(net, clip)
            r = solve.converge(eng, C0, g0, eps0, inner="lbfgs", max_inner=300, time_limit=time_limit)
            out[label] = {"E": r["E"], "converged": r["converged"], "outer": r["outer"],
                          "inner_total": r["inner_total"], "on_iterations_first": r["history"][0]["on_iterations"],
                          "on_iterations_total": int(sum(h["on_iterations"] for h in r["history"])),
                          "seconds": r["seconds"], "ms_per_inner": r["ms_per_inner"]}
        return out
    finally:
        eng.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=300, help="number of training rings (C6..C12)")
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--eval", default="c20h40", help="evaluation workload name")
    ap.add_argument("--eval-seeds", type=int, default=3, help="evaluation systems (the named one, then reseeded)")
    ap.add_argument("--orbitals", default="random", choices=["random", "rhf"],
                    help="orbitals of the training rings and of the evaluation: S^-1/2 Q or RI-HF")
    ap.add_argument("--loop", action="store_true", help="evaluate over the full ON + NO loop (RI-HF start)")
    ap.add_argument("--loop-time-limit", type=float, default=600.0, help="seconds per loop run (--loop)")
    ap.add_argument("--max-data-seconds", type=float, default=None,
                    help="cap on the data generation time (fewer rings are used if it is reached)")
    args = ap.parse_args()
    import sys

    def log(k, dt):
        print(json.dumps({"rings": k, "seconds": dt}), file=sys.stderr, flush=True)

    t0 = time.perf_counter()
    # targets from the FP64 form (the features and converged angles of each ring)
    info = {}
    X, Y = training_set(args.train, precision=bd.DONOF_RI_FP64, orbitals=args.orbitals,
                        max_seconds=args.max_data_seconds, log=log, info=info)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, loss = train(X, Y, steps=args.steps)
    t_train = time.perf_counter() - t0
    rows = []
    for k in range(args.eval_seeds):
        seed = None if k == 0 else 900 + k
        if args.loop:
            rows.append(loop_compare(args.eval, net, seed=seed, time_limit=args.loop_time_limit))
            continue
        eng, w = bd.engine_and_workload(args.eval, bd.DONOF_RI_SLICE4, seed=seed)
        if args.orbitals == "rhf":
            w.C = eng.rhf(max_iter=200, tol=1e-8)[0]
        rows.append(compare(w, net, eng=eng))
    print(json.dumps({"train_systems": info["rings"], "requested": args.train, "orbitals": args.orbitals,
                      "samples": int(X.shape[0]), "data_s": t_data, "train_s": t_train,
                      "final_loss": loss, "eval": args.eval, "results": rows}))


if __name__ == "__main__":
    main()
