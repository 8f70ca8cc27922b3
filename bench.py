"""Benchmark: RI J/K build time per PNOF7 iteration on one GB300 (or N replicas).

One step = one pass of the whole hot path over the workload: the half and
full transforms with J_pq / K_pq (Table 2), the per-orbital AO J^(q) / K^(q)
(Table 3) and the PNOF7 energy and Lagrangian, i.e. the C-ABI sequence
  donof_ri_transform(FULL) -> donof_ri_jk_mo -> donof_ri_jk_ao_batch
  -> donof_ri_energy_lagrangian.
Inputs (orbitals C, angles gamma) are resident in device memory when the
timed region starts; L2 is flushed (256 MB write) between timed steps,
outside the per-step CUDA events.  `e2e` repeats the step through the same
entry points with pinned host buffers (host->device copy of C and gamma and
device->host copy of J, K, E, lambda inside the timed region).

Multi-GPU: the path does not shard across GPUs in this engine (replicas
only); under torchrun every rank runs an independent replica and `value` is
the effective time per iteration of the whole job (max-over-ranks time
divided by all ranks' iterations).

`--impl reference` times the FP64 CPU oracle (the only baseline: the paper
ships no code) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "RI J/K build ms per PNOF7 iteration"
UNIT = "ms/iteration"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# Nominal dense rates (TFLOP/s) used to scale the measured bf16 peak to other types.
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}

ROWS = ["half", "diag", "full_k", "j", "jao", "kao", "energy", "other"]
# Profile rows 8..13: the tensor-core GEMM kernel of a row, timed alone.
GEMMS = ["half", "full_k", "j", "jao", "kao", "fock"]
GEMM_KERNEL = {"slice4": "s4_gemm_kernel<{}>", "tf32x3": "tc_gemm_kernel<{}>"}
# Profile rows 14, 15: the memory-bound passes of SLICE4, timed alone.
MEMS = {"digits": "xf_to_digits_kernel", "split": "slice_pair_kernel"}


def algorithmic_bytes(s):
    """Bytes each memory-bound pass must move per launch (unpadded element counts).
    digits: b_half integers read (4 B), its L3 and L6 digit layouts written (8 B each),
    the diagonal partials written (8 B per 64-wide nu tile); split: J^(q), K^(q) read as
    FP32 pairs (8 B) and written as four BF16 digit planes (8 B), one exponent per row."""
    nb, nx, m = s.nbf, s.naux, s.n_omega
    return {"digits": nx * m * nb * (4 + 8 + 8) + ((nb + 63) // 64) * m * nx * 8,
            "split": 2 * m * nb * nb * (8 + 8) + 2 * m * nb * 4}


def _system(name, trim_naux=0):
    from synthetic import without_basis_functions, workload_system
    s = workload_system(name)
    if 0 < trim_naux < s.naux:
        s = without_basis_functions(s, 0, s.naux - trim_naux)
    return s


def workload_desc(name, trim_naux=0):
    s = _system(name, trim_naux)
    trimmed = f" (auxiliary set trimmed to its first {s.naux})" if 0 < trim_naux else ""
    return s, (f"{name}{trimmed}: s-type ring, nbf={s.nbf}, naux={s.naux}, N_I={s.n_strong}, "
               f"N_g={s.n_weak_per}, N_Omega={s.n_omega}")


def engine_workload(bd, name, precision, stream=None, trim_naux=0):
    """A context for the named workload and the workload itself, its orbitals
    C = S^-1/2 Q built from the overlap matrix the engine evaluated at init."""
    from synthetic import make_workload
    s = _system(name, trim_naux)
    eng = bd.Engine(s, precision, stream=stream)
    w = make_workload(name, eng.fetch(bd.DONOF_RI_FETCH_OVERLAP))
    w.system = s
    return eng, w


def algorithmic_flops(s):
    """Algorithmic FLOPs per launch group of each row (2 per multiply-add; symmetric halves not counted)."""
    nb, nx, m = s.nbf, s.naux, s.n_omega
    return {
        "half": 2.0 * nb * nb * nx * m,
        "diag": 2.0 * nb * nx * m,
        "full_k": 2.0 * nb * nx * m * m + 2.0 * nx * m * m,
        "j": 1.0 * nx * m * (m + 1),
        "jao": 1.0 * nb * (nb + 1) * nx * m,
        "kao": 1.0 * nb * (nb + 1) * nx * m,
        "energy": 4.0 * nb * nb * m * m + 2.0 * nb * nb * m,
        "fock": 4.0 * nb * nb * m * m,
    }


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return dict(FALLBACK_PEAKS), "fallback"


def _peak_value(d, key):
    v = d.get(key)
    if isinstance(v, dict):
        for k in ("value", "median", "tflops", "gbs"):
            if k in v:
                return float(v[k])
    return float(v) if v is not None else None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha(precision):
    files = {"tf32x3": ["tc.cu"], "slice4": ["s4.cu"], "fp64": ["path64.cu", "setup64.cu"]}[precision]
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2012_15662_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(workload, precision, row):
    """DRAM bytes per launch of the dominant row from a committed ncu summary, if its source hash matches."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}_{precision}.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(precision)
    for ln in open(path):
        f = dict(kv.split("=", 1) for kv in ln.split() if "=" in kv)
        if f.get("row") == row and f.get("src_sha") == sha and "bytes_per_launch" in f:
            return float(f["bytes_per_launch"])
    return None


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
# Largest auxiliary set the oracle sample evaluates whole; beyond it the sample runs
# rows a1-a6 on the leading auxiliary functions and scales them (all of a1-a6 are sums
# over the auxiliary index, so their cost is proportional to the number of P).
ORACLE_WHOLE_NAUX = 1000
ORACLE_SLICE_NAUX = 48


def _oracle_sample(name, budget_s):
    """Time the oracle on the workload until budget_s is spent; returns
    (ms per iteration, repetitions, description of the sample)."""
    from scipy.linalg import solve_triangular
    from oracle import integrals as I, pnof7, ri
    from synthetic import make_workload, pairing_columns
    w = make_workload(name, I.overlap)
    s = w.system
    H = I.core_hamiltonian(s)
    e_nuc = I.nuclear_repulsion(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    m = s.n_omega
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)

    def a7(r):
        A, Bc = pnof7.coupling(n, sub, rank)
        pnof7.lagrangian(w.C, H, r["Jao"], r["Kao"], n, A, Bc)
        Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
        pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, e_nuc)

    if s.naux <= ORACLE_WHOLE_NAUX:
        B, L, G = ri.setup(s)
        times = []
        t_end = time.perf_counter() + budget_s
        while True:
            t0 = time.perf_counter()
            a7(ri.all_rows(B, w.C, m))
            times.append(time.perf_counter() - t0)
            if time.perf_counter() > t_end:
                break
        return (1000.0 * float(np.mean(times)), len(times),
                f"{len(times)} whole iterations of {name} (all rows, FP64 numpy/BLAS) in ~{budget_s:.0f} s")
    # B^P of the leading k auxiliary functions needs only the leading block of the
    # metric's Cholesky factor and the matching (P|mu nu) (forward substitution)
    k = ORACLE_SLICE_NAUX
    G = I.metric(s)
    Lk = np.linalg.cholesky(G[:k, :k])
    e3 = I.eri3(s, slice(0, k))
    Bk = solve_triangular(Lk, e3.reshape(k, -1), lower=True).reshape(k, s.nbf, s.nbf)
    del e3
    t0 = time.perf_counter()
    r = ri.all_rows(Bk, w.C, m)
    t_rows = [time.perf_counter() - t0]
    t0 = time.perf_counter()
    a7(r)
    t_a7 = time.perf_counter() - t0
    t_end = time.perf_counter() + max(0.0, budget_s - t_rows[0] - t_a7)
    while time.perf_counter() < t_end:
        t0 = time.perf_counter()
        ri.all_rows(Bk, w.C, m)
        t_rows.append(time.perf_counter() - t0)
    scale = s.naux / k
    ms = 1000.0 * (float(np.mean(t_rows)) * scale + t_a7)
    return (ms, len(t_rows),
            f"rows a1-a6 of {name} on the first {k} of {s.naux} auxiliary functions ({len(t_rows)} repetitions, "
            f"time x {scale:.2f}) plus the energy and Lagrangian (a7) once at full size; FP64 numpy/BLAS")


def cpu_baseline(name, budget_s=12.0):
    """Time the oracle in a spawned subprocess with every host core available to BLAS."""
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench._oracle_sample({name!r}, {budget_s})))")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "error": out.stderr[-300:]}
    ms, iters, sample = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}


# ---------------------------------------------------------------------------
def job_ms_per_iteration(rank_total_ms, steps, world, device="cpu"):
    """Effective ms per iteration of the whole job (replicas): the slowest rank's
    time for its `steps` iterations, over the steps x world iterations all ranks ran."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(rank_total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        rank_total_ms = float(t.item())
    return rank_total_ms / (steps * world)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c20h40",
                    help="timed workload (default: C20H40, the largest one-GPU configuration)")
    ap.add_argument("--precision", default="slice4", choices=["slice4", "tf32x3", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch eagerly instead of replaying a CUDA graph")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default SLICE4 tile schedule")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="iterations of the plain FP64 form on the same workload (mixed vs FP64 key; 0: skip)")
    ap.add_argument("--trim-naux", type=int, default=0,
                    help="keep only the first N auxiliary functions (a reduced case of the same orbital "
                         "basis, for profiling captures; 0: the full set)")
    ap.add_argument("--extra-workloads", default="c6h12,c16h32",
                    help="comma-separated workloads also timed (CUDA-graph iterations) as extra keys")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        _, desc = workload_desc(args.workload, args.trim_naux)
        budget = max(2.0, min(20.0, 0.5 * (args.steps + args.warmup)))
        cb = cpu_baseline(args.workload, budget_s=budget)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["value"],
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": desc, "precision": "fp64 (CPU oracle)"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    from paper_2012_15662_gb300 import binding as bd

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    _, desc = workload_desc(args.workload, args.trim_naux)
    prec = {"slice4": bd.DONOF_RI_SLICE4, "tf32x3": bd.DONOF_RI_TF32X3, "fp64": bd.DONOF_RI_FP64}[args.precision]
    stream = torch.cuda.Stream(device=dev)
    eng, w = engine_workload(bd, args.workload, prec, stream=stream.cuda_stream, trim_naux=args.trim_naux)
    s = w.system
    nb, m = s.nbf, s.n_omega
    C_dev = torch.from_numpy(bd.Engine.colmajor(w.C)).to(dev)
    g_dev = torch.from_numpy(np.ascontiguousarray(w.gamma)).to(dev)
    J_dev = torch.empty((m, m), dtype=torch.float64, device=dev)
    K_dev = torch.empty((m, m), dtype=torch.float64, device=dev)
    E_dev = torch.empty(1, dtype=torch.float64, device=dev)
    L_dev = torch.empty(nb * nb, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    tuned = None
    if prec == bd.DONOF_RI_SLICE4 and not args.no_autotune:
        # tile schedule tuned on this problem before any timing (donof_ri_autotune)
        bd.donof_ri_transform(eng.ctx, C_dev, bd.DONOF_RI_FULL)
        bd.donof_ri_jk_ao_batch(eng.ctx)
        report, tried = bd.donof_ri_autotune(eng.ctx, reps=3)
        tuned = {"settings_timed": tried,
                 "per_kind": {k: {"stages": int(r[0]), "splits_or_sym": int(r[1]), "ctas": int(r[2]), "us": int(r[3])}
                              for k, r in zip(["half", "full_k", "j", "jao", "kao", "fock"], report)}}
        torch.cuda.synchronize()

    def step(graph=not args.no_graph):
        bd.donof_ri_iteration(eng.ctx, C_dev, g_dev, bd.DONOF_RI_FULL, J_dev, K_dev, E_dev, L_dev,
                              use_graph=graph)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    bd.donof_ri_sync(eng.ctx)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local_rank)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = bd.donof_ri_launch_count(eng.ctx)
    barrier()
    sampler.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
    barrier()
    clocks = sampler.stop()
    launches = bd.donof_ri_launch_count(eng.ctx) - l0
    bd.donof_ri_sync(eng.ctx)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    # Per-row kernel durations: the same steps launched eagerly with CUDA events recorded on the
    # engine's stream around every launch group of a row (graphs carry no profiling events).
    bd.donof_ri_profile(eng.ctx, True)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            step(graph=False)
    barrier()
    rows = {}
    for i, r in enumerate(ROWS):
        t, c = bd.donof_ri_profile_read(eng.ctx, i)
        rows[r] = (t, c)
    gemms = {}
    for i, r in enumerate(GEMMS):
        t, c = bd.donof_ri_profile_read(eng.ctx, len(ROWS) + i)
        if c > 0:
            gemms[r] = (t, c)
    mems = {}
    for i, r in enumerate(MEMS):
        t, c = bd.donof_ri_profile_read(eng.ctx, len(ROWS) + len(GEMMS) + i)
        if c > 0:
            mems[r] = (t, c)
    bd.donof_ri_profile(eng.ctx, False)
    ms = float(np.mean(step_ms))
    value = job_ms_per_iteration(ms * args.steps, args.steps, world, dev)

    # e2e through the same entry points with pinned host buffers
    e2e = None
    if not args.no_e2e:
        C_h = torch.from_numpy(bd.Engine.colmajor(w.C)).pin_memory()
        g_h = torch.from_numpy(np.ascontiguousarray(w.gamma)).pin_memory()
        J_h = torch.empty((m, m), dtype=torch.float64).pin_memory()
        K_h = torch.empty((m, m), dtype=torch.float64).pin_memory()
        E_h = torch.empty(1, dtype=torch.float64).pin_memory()
        L_h = torch.empty(nb * nb, dtype=torch.float64).pin_memory()

        def step_host():
            bd.donof_ri_iteration(eng.ctx, C_h, g_h, bd.DONOF_RI_FULL, J_h, K_h, E_h, L_h)

        for _ in range(args.warmup):
            step_host()
        barrier()
        tt = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            tt.append(time.perf_counter() - t0)
        barrier()
        e_ms = 1000.0 * float(np.mean(tt))
        e2e = {"value": job_ms_per_iteration(e_ms * args.steps, args.steps, world, dev), "unit": UNIT,
               "h2d_bytes_per_step": int(8 * (nb * nb + len(w.gamma))),
               "d2h_bytes_per_step": int(8 * (2 * m * m + 1 + nb * nb))}

    # roofline of the dominant kernel: the tensor-core GEMM kernel with the largest
    # share of the step (its own event pair); the FP64 form, which has no such
    # kernel, falls back to its dominant row
    flops = algorithmic_flops(s)
    if gemms:
        dom = max(gemms, key=lambda r: gemms[r][0])
        t_dom, c_dom = gemms[dom]
        kind = GEMMS.index(dom)
        kernel = GEMM_KERNEL[args.precision].format(kind)
        if args.precision == "slice4":
            # second template argument: every unit a single K chunk (the contractions over
            # the orbital basis: K = nbf <= 736; over the auxiliary index: K = naux <= 512)
            one = dom == "fock" or (dom in ("half", "full_k") and s.nbf <= 736) or (
                dom in ("jao", "kao") and s.naux <= 512)
            kernel = f"s4_gemm_kernel<{kind}, {int(one)}>"
        traffic_key = "gemm_" + dom
    else:
        dom = max((r for r in ROWS if r in flops and rows[r][1] > 0), key=lambda r: rows[r][0])
        t_dom, c_dom = rows[dom]
        kernel = "row " + dom
        traffic_key = dom
    per_launch_ms = t_dom / max(c_dom, 1)
    achieved = flops[dom] / (per_launch_ms * 1e-3) / 1e12
    peaks, peak_src = read_peaks()
    # A split-precision contraction executes several tensor-core products per
    # algorithmic product; its peak in algorithmic flops is the dtype's dense peak
    # divided by that count (3 TF32 MMAs for TF32X3, 13 BF16 digit-pair MMAs for
    # SLICE4).  executed_tflops is the tensor-core rate the kernel actually ran at.
    mult = 1
    if prec == bd.DONOF_RI_FP64:
        peak = NOMINAL["fp64"]
        bound, peak_note = "alu", "FP64 nominal 1.25 TFLOP/s (DFMA on CUDA cores; not measured)"
    elif prec == bd.DONOF_RI_TF32X3:
        bf = _peak_value(peaks, "bf16_tflops") or FALLBACK_PEAKS["bf16_tflops"]
        mult = 3
        peak = bf * NOMINAL["tf32"] / NOMINAL["bf16"] / mult
        bound, peak_note = "tensor", (f"TF32 dense = {peak_src} bf16 burst {bf:.0f} x 1.1/2.25, "
                                      "/ 3 TF32 MMAs per algorithmic product")
    else:
        bf = _peak_value(peaks, "bf16_tflops") or FALLBACK_PEAKS["bf16_tflops"]
        mult = 13
        peak = bf / mult
        bound, peak_note = "tensor", (f"BF16 dense, {peak_src} burst {bf:.0f}, / 13 BF16 digit-pair MMAs per "
                                      "algorithmic product")
    traffic = read_traffic(args.workload, args.precision, traffic_key)
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "kernel_row": dom, "launch_ms": per_launch_ms,
            "share_of_step": t_dom / args.steps / ms,
            "algorithmic_flops_per_launch": flops[dom], "executed_tflops": achieved * mult,
            "peak_source": peak_note}

    if rank != 0:
        return 0
    # the memory-bound passes against the measured copy bandwidth (algorithmic bytes
    # over each launch's own events)
    hbm_peak = _peak_value(peaks, "hbm_gbs") or FALLBACK_PEAKS["hbm_gbs"]
    nbytes = algorithmic_bytes(s)
    hbm_kernels = {}
    for r, (t, c) in mems.items():
        us = 1000.0 * t / c
        gbs = nbytes[r] / (us * 1e-6) / 1e9
        hbm_kernels[r] = {"kernel": MEMS[r], "bytes_per_launch": int(nbytes[r]), "us_per_launch": us,
                          "achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "tf32x3": "tf32x3", "slice4": "bf16x4-digits (exact sums)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": desc, "precision": args.precision,
                   "l2": "flushed between steps (256 MB write, outside the step events)",
                   "launch": "eager" if args.no_graph else "one CUDA graph per step (donof_ri_iteration)",
                   "parallelism": f"replicas x{world}", "autotune": tuned},
        "rows_ms_per_step": {r: rows[r][0] / args.steps for r in ROWS},
        "gemm_kernels_ms_per_step": {r: gemms[r][0] / args.steps for r in gemms},
        "hbm_kernels": hbm_kernels,
        "roofline": roof, "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e,
    }
    # the result of the last timed iteration (for the mixed vs FP64 comparison)
    torch.cuda.synchronize()
    res = {"E": float(E_dev.item()), "J": J_dev.cpu().numpy(), "K": K_dev.cpu().numpy(),
           "lam": L_dev.cpu().numpy()}
    eng.close()
    del flush
    torch.cuda.empty_cache()
    if args.fp64_steps > 0 and prec != bd.DONOF_RI_FP64:
        line["mixed_vs_fp64"] = fp64_comparison(bd, torch, dev, args, w, res, value)
    extra = [x for x in args.extra_workloads.split(",") if x and x not in (args.workload, "none")]
    if extra and world == 1:
        line["other_workloads"] = {x: time_workload(bd, torch, dev, x, prec) for x in extra}
    if world == 1 and not args.no_cpu_baseline and not args.trim_naux:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line))
    return 0


def _graph_iterations(bd, torch, eng, w, stream, steps, warmup):
    """ms per CUDA-graph iteration (device events, L2 flushed between steps) and the last outputs."""
    dev = torch.device("cuda", torch.cuda.current_device())
    nb, m = eng.nbf, eng.n_omega
    C_dev = torch.from_numpy(bd.Engine.colmajor(w.C)).to(dev)
    g_dev = torch.from_numpy(np.ascontiguousarray(w.gamma)).to(dev)
    J = torch.empty((m, m), dtype=torch.float64, device=dev)
    K = torch.empty((m, m), dtype=torch.float64, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    L = torch.empty(nb * nb, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            bd.donof_ri_iteration(eng.ctx, C_dev, g_dev, bd.DONOF_RI_FULL, J, K, E, L)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            bd.donof_ri_iteration(eng.ctx, C_dev, g_dev, bd.DONOF_RI_FULL, J, K, E, L)
            b.record(stream)
    torch.cuda.synchronize()
    bd.donof_ri_sync(eng.ctx)
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    return ms, {"E": float(E.item()), "J": J.cpu().numpy(), "K": K.cpu().numpy(), "lam": L.cpu().numpy()}


def fp64_comparison(bd, torch, dev, args, w, res, mixed_ms):
    """The plain FP64 GPU form on the same workload and orbitals: ms per iteration
    (one CUDA graph per iteration, like the mixed form) and the mixed form's
    deviation from it in E, J, K and lambda."""
    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64, stream=stream.cuda_stream)
    init_s = time.perf_counter() - t0
    ms, r64 = _graph_iterations(bd, torch, eng, w, stream, args.fp64_steps, 1)
    eng.close()
    torch.cuda.empty_cache()
    return {"fp64_ms_per_iteration": ms, "mixed_ms_per_iteration": mixed_ms, "speedup": ms / mixed_ms,
            "fp64_iterations_timed": args.fp64_steps, "fp64_init_s": init_s,
            "abs_dE_eh": abs(res["E"] - r64["E"]), "E_fp64_eh": r64["E"],
            "max_abs_dJ": float(np.abs(res["J"] - r64["J"]).max()),
            "max_abs_dK": float(np.abs(res["K"] - r64["K"]).max()),
            "max_abs_dlambda": float(np.abs(res["lam"] - r64["lam"]).max()),
            "note": "same orbitals and angles; FP64 form = DONOF_RI_FP64 (DFMA), mixed = the timed form"}


def time_workload(bd, torch, dev, name, prec, steps=10):
    """ms per CUDA-graph iteration of another workload (default schedule, no autotuning)."""
    stream = torch.cuda.Stream(device=dev)
    eng, w = engine_workload(bd, name, prec, stream=stream.cuda_stream)
    ms, r = _graph_iterations(bd, torch, eng, w, stream, steps, 3)
    eng.close()
    torch.cuda.empty_cache()
    s = w.system
    return {"ms_per_iteration": ms, "steps": steps, "E_eh": r["E"],
            "shape": f"nbf={s.nbf}, naux={s.naux}, N_Omega={s.n_omega}"}


if __name__ == "__main__":
    sys.exit(main())
