#!/usr/bin/env python
"""ISDF decompositions per second on GB300: weights -> weighted K-means ->
interpolation-vector fit, on seeded synthetic plane-wave orbitals.

    python bench.py [--gpus N --steps K --warmup W] [--workload silica] [--impl reference]

A step is one full decomposition (all steps of the hot path) of one orbital
pair that is already resident in HBM: the weight function, T Lloyd updates
with the final assignment and snap, the plan update (gather, M, Cholesky,
M^-1) and Theta for every grid row, fitted in row blocks of 131,072 rows into
one reused block buffer (Theta is never fully resident). The default workload
is the largest one that fits one GPU: 128^3 grid, 1024 complex64 orbitals,
4096 points, T = 100 (silica-like). Both precision modes run on the same
workload: the headline `value` is the tensor-core (split-FP16) path, the
`fp64` object the plain FP64 GPU path; both report the relative Frobenius
error of Theta and of the reconstructed Z against the CPU FP64 oracle on a
seeded 16,384-row sample. Under torchrun every rank decomposes its own
orbital pair (independent problems, no data-path collective); `value` counts
all ranks' decompositions.

`--impl reference` times the CPU FP64 oracle (the reference for this method)
on the host cores, on a bounded sample of the same workload per step (the
same sample definition as the `cpu_baseline` of the GPU line).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ISDF decompositions/sec (K-means+Θ fit), mixed vs FP64 at stated Θ error"
UNIT = "decompositions/s"
DEFAULT_WORKLOAD = "silica"
THETA_BLOCK = 131072          # Theta row block (config: fitted in grid blocks, never fully resident)
ERROR_ROWS = 16384            # oracle subsample for the Theta / Z errors (seed 2000 + s)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None,
                    help="default: silica for the decomposition, adjoint for --op adjoint, medium for "
                         "--op exchange and --study weights, kpoints for --op batch")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-graph", action="store_true", help="launch every kernel from the host instead of "
                    "replaying one captured CUDA graph per step")
    ap.add_argument("--op", choices=["decompose", "exchange", "batch", "adjoint", "gemm", "weights", "kmeans"],
                    default="decompose",
                    help="exchange: time the ISDF exchange application (FFT potentials + Eq. v2) instead; "
                         "batch: batched decompositions of several pairs on one grid (default workload kpoints); "
                         "adjoint: surrogate loss + gradients at fixed points (default workload adjoint); "
                         "gemm / weights / kmeans: one kernel family alone at the workload's shapes on a subset of "
                         "rows (--rows) or synthetic weights, small enough for a profiler capture")
    ap.add_argument("--rows", type=int, default=65536, help="grid rows of the --op gemm / weights cases")
    ap.add_argument("--batch", type=int, default=8, help="pairs per batched step (--op batch)")
    ap.add_argument("--study", choices=["weights"], default=None,
                    help="instead of timing: the weight-function accuracy study (Appendix A diagnostics)")
    return ap.parse_args()


def algorithmic_flops(w):
    """Per-row algorithmic FLOPs of the two GEMM kernels (real flops of the complex products)."""
    return {"gram": 16.0 * w.n_orb * w.n_mu, "apply": 8.0 * w.n_mu * w.n_mu}


# DRAM bytes (read + write) per launch from one ncu capture of the same kernel version on GB300 (only valid for the
# workload, launch size and kernel version profiled). Silica apply and Gram: the 32,768-row launches of `bench.py
# --op gemm --workload silica --rows 65536` (the apply on CTA pairs, tiles in groups of 8 pair rows, the peer CTA
# loading each stage as soon as its slot is empty, K segments of 1,024), scaled by rows
# to the 131,072-row launches of the step. Silica weights: the 262,144-row launch of `bench.py --op weights
# --workload silica --rows 262144`, scaled by rows to the 128^3 grid.
NCU_TRAFFIC = {("silica", "apply"): 4 * (12.530186e9 + 1.116051e9),
               ("silica", "gram"): 4 * (4.062169e9 + 1.107082e9),
               ("silica", "weights"): 8 * (4.316357e9 + 5.800448e6),
               # the five passes of one exchange potential (ncu on the x, y and fused z passes: 2 x, 2 y, z)
               ("medium", "fft_potential"): 2 * (906.020608e6 + 858.783232e6) + 2 * (906.043392e6 + 845.432320e6)
               + 906.016768e6 + 845.357056e6}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [ln.split(",") for ln in open(self.path).read().splitlines() if ln.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if "Active" == r[5 + i].strip()})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle (baseline / reference arm)
def oracle_context(w, phi, psi, log=None):
    """Inputs of the oracle sample, prepared once (not timed): the oracle's own weights over the full
    grid (computed in row chunks, so no full complex128 copy of the orbitals exists on the host), the
    seeded initial points drawn from them, and the host rows the sample's weight stage reads.
    phi, psi: the workload's orbitals (device or host tensors in their storage dtype)."""
    import numpy as np
    import torch

    import oracle as O
    from paper_2208_07731_gb300 import workload as W
    O.load()
    chunk = 65536
    wt = np.empty(w.n_r, np.float64)
    for r0 in range(0, w.n_r, chunk):
        r1 = min(w.n_r, r0 + chunk)
        wt[r0:r1] = O.weights(phi[r0:r1].cpu().numpy(), psi[r0:r1].cpu().numpy())
    init = W.init_indices(wt, w.n_mu, 1000 + w.seed)
    n_wrows = min(w.n_r, 65536)
    wrows = torch.from_numpy(W.subsample_rows(w.n_r, n_wrows, 3000 + w.seed)).to(phi.device)
    n_trows = min(w.n_r, 4096 if w.n_r * w.n_mu <= 1e9 else 2048)
    trows = W.subsample_rows(w.n_r, n_trows, 4000 + w.seed)
    return {"w": w, "wt": wt, "init": init, "phi": phi, "psi": psi,
            "wphi": phi[wrows].cpu().numpy(), "wpsi": psi[wrows].cpu().numpy(), "trows": trows}


def oracle_sample(ctx):
    """One bounded sample of the CPU FP64 oracle's decomposition, timed stage by stage and scaled to
    one full decomposition (weights + T Lloyd updates and the snap + M, Cholesky + Theta on all rows):
      weights   on a 65,536-row sample (or every row), scaled by N_r / rows;
      K-means   the oracle's Lloyd run with one update on the full grid (two assignment passes, one
                update, the snap), scaled by (T + 1) / 2 passes;
      M, L      in full at the points that run selected;
      Theta     on a 4,096-row sample (2,048 on the largest grids), scaled by N_r / rows.
    The same definition serves the GPU line's cpu_baseline and --impl reference.
    Returns (seconds per full decomposition extrapolated, seconds the sample took, stage seconds,
    description)."""
    import numpy as np

    import oracle as O
    w = ctx["w"]
    shape, cell = (w.n,) * 3, (w.L,) * 3
    t, meas = {}, {}
    t0 = time.perf_counter()
    O.weights(ctx["wphi"], ctx["wpsi"])
    meas["weights"] = time.perf_counter() - t0
    t["weights"] = meas["weights"] * w.n_r / ctx["wphi"].shape[0]
    t0 = time.perf_counter()
    km = O.kmeans(ctx["wt"], shape, cell, w.n_mu, ctx["init"], 1)
    meas["kmeans"] = time.perf_counter() - t0
    t["kmeans"] = meas["kmeans"] * (w.iters + 1) / 2.0
    idx = km["idx"]
    rows_mu = (ctx["phi"][idx].cpu().numpy(), ctx["psi"][idx].cpu().numpy())
    t0 = time.perf_counter()
    phi_mu = O.gather(rows_mu[0], rows_mu[1], np.arange(w.n_mu))
    L = O.cholesky(O.form_M(*phi_mu))
    meas["M_cholesky"] = t["M_cholesky"] = time.perf_counter() - t0
    rows = ctx["trows"]
    pr, qr = ctx["phi"][rows].cpu().numpy(), ctx["psi"][rows].cpu().numpy()
    t0 = time.perf_counter()
    O.theta_rows(pr, qr, phi_mu[0], phi_mu[1], L, np.arange(len(rows)))
    meas["theta"] = time.perf_counter() - t0
    t["theta"] = meas["theta"] * w.n_r / len(rows)
    desc = (f"weights on {ctx['wphi'].shape[0]} of {w.n_r} rows; K-means: one Lloyd update (2 assignment "
            f"passes + snap) on the full grid, scaled to T = {w.iters}; M and Cholesky in full; Theta on "
            f"{len(rows)} of {w.n_r} rows; every stage scaled to one full decomposition")
    return sum(t.values()), sum(meas.values()), t, desc


def run_reference(args):
    """The CPU FP64 oracle as the reference arm: each step is one bounded sample (oracle_sample) of the
    GPU line's workload; ms_per_step is the sample's measured time, value the decompositions/s it
    extrapolates to. The orbitals are generated on the GPU when one is present (input generation only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch

    from paper_2208_07731_gb300 import workload as W
    w = W.WORKLOADS[args.workload]
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    phi, psi = W.make_pair(w, device=dev)
    phi, psi = W.storage(phi, w).contiguous(), W.storage(psi, w).contiguous()
    ctx = oracle_context(w, phi, psi)
    full, meas, desc = [], [], ""
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        total, spent, _, desc = oracle_sample(ctx)
        if i >= args.warmup:
            full.append(total)
            meas.append(spent)
    t_all = time.perf_counter() - t_all
    sec = statistics.median(full)
    value = 1.0 / sec
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(meas) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic plane-wave orbitals (seeded)",
            "config": {"workload": w.name, "grid": f"{w.n}^3", "n_r": w.n_r, "n_orb": w.n_orb, "n_mu": w.n_mu,
                       "lloyd_iters": w.iters, "orbital_dtype": w.dtype},
            "extrapolated": True,
            "value_basis": "each step times one bounded oracle sample (ms_per_step, measured); value = 1 / its "
                           "stage times scaled to one full decomposition (median over the timed steps)",
            "seconds_per_full_decomposition": sec, "timed_region_s": t_all,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU path
def run_adjoint(args):
    """Adjoint measurement (config 3 by default; any workload with --op adjoint): the exchange-like
    surrogate L = dV sum_r Re[conj(Theta_r) K Theta_r] and its gradients dL/dPhi, dL/dPsi at fixed
    interpolation points (taken from a prior K-means), per step: plan update (gather, M, Cholesky,
    M^-1) + blocked backward in blocks of 131,072 rows that recomputes Theta (never stored) + finalize.
    Mixed is the headline; the FP64 GPU path runs on the same inputs (fewer steps where one takes
    seconds), and the relative difference of the two gradients is reported."""
    import torch

    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as isdf
    from paper_2208_07731_gb300 import workload as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    phi, psi = W.make_pair(w, device=dev)
    phi, psi = W.storage(phi, w).contiguous(), W.storage(psi, w).contiguous()
    torch.cuda.empty_cache()
    wt = isdf.weights(phi, psi)
    init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 1000 + w.seed))
    idx = isdf.kmeans(wt, (w.n,) * 3, (w.L,) * 3, w.n_mu, init, w.iters)["idx"]
    del wt
    K = torch.from_numpy(W.loss_matrix(w.n_mu, 3000 + w.seed)).to(dev)
    block = min(w.n_r, THETA_BLOCK)
    res = {}
    for mode in ("mixed",) if args.no_fp64 else ("mixed", "fp64"):
        plan = isdf.Plan(phi, psi, idx, mode=mode, max_rows=block)

        def step():
            plan.update(idx)
            return isdf.surrogate_loss_and_grad(plan, K, w.dV, block=block)

        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        t_first = time.perf_counter() - t0
        if mode == "mixed":
            warm, steps = args.warmup, args.steps
        else:
            steps = max(1, min(args.steps, int(60.0 / max(t_first, 1e-3))))
            warm = max(1, min(args.warmup, int(10.0 / max(t_first, 1e-3))))
        for _ in range(warm - 1):
            step()
        torch.cuda.synchronize()
        l0 = isdf.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(dev.index)
        clocks.start()
        e0.record()
        for _ in range(steps):
            loss, gphi, gpsi = step()
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        plan.check()
        res[mode] = {"ms": e0.elapsed_time(e1) / steps, "launches": (isdf.kernel_launches() - l0) // steps,
                     "loss": loss.item(), "steps": steps, "warmup": warm, "clocks": clk,
                     # kept in complex64 for the comparison (its ~6e-8 rounding is far below the difference)
                     "gphi": gphi.to(torch.complex64) if mode == "mixed" else gphi,
                     "gpsi": gpsi.to(torch.complex64) if mode == "mixed" else gpsi}
        del gphi, gpsi
        plan.close()
        torch.cuda.empty_cache()
    a = res["mixed"]
    line = {"metric": "ISDF Θ-fit adjoint evaluations/sec (surrogate loss + dL/dΦ, dL/dΨ at fixed points)",
            "value": 1e3 / a["ms"], "unit": "gradients/s", "n_gpus": 1, "steps": a["steps"], "warmup": a["warmup"],
            "ms_per_step": a["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 hi+lo split x3 on tcgen05 (f32 accumulate) for every adjoint GEMM; f64 M, Cholesky, M^-1 "
                     "and f64 gradient accumulation",
            "data": "synthetic: seeded random plane-wave Bloch orbitals, orthonormalised",
            "config": {"workload": w.name, "grid": f"{w.n}^3", "n_orb": w.n_orb, "n_mu": w.n_mu,
                       "block_rows": block, "theta": "recomputed per block, never stored"},
            "gpu_launches": a["launches"], "clocks": a["clocks"], "loss": {"mixed": a["loss"]}}
    if "fp64" in res:
        b = res["fp64"]
        num = den = 0.0
        for x, y in ((a["gphi"], b["gphi"]), (a["gpsi"], b["gpsi"])):
            for r0 in range(0, w.n_r, block):
                xb, yb = x[r0:r0 + block].to(torch.complex128), y[r0:r0 + block]
                num += (torch.linalg.vector_norm(xb - yb) ** 2).item()
                den += (torch.linalg.vector_norm(yb) ** 2).item()
        line["fp64"] = {"value": 1e3 / b["ms"], "ms_per_step": b["ms"], "steps": b["steps"], "warmup": b["warmup"],
                        "clocks": b["clocks"]}
        line["grad_rel_diff_mixed_vs_fp64"] = math.sqrt(num / den)
        line["loss"]["fp64"] = b["loss"]
        line["speedup_mixed_vs_fp64"] = b["ms"] / a["ms"]
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_study(args):
    """Weight-function study (Sec. 2.2, Appendix A): for SSM with alpha = 1..4, PSM, uniformly random
    points and randomized-QRCP points (Eq. QRCP), the interpolation points' fit error ||Z - Theta C||_F / ||Z||_F (FP64
    plan), the cluster residual R of Eq. errorISDF relative to ||Z||_F^2, and how delocalised the
    points are (mean density at the points over the grid's mean density). All on the GPU path."""
    import numpy as np
    import torch

    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as isdf
    from paper_2208_07731_gb300 import workload as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    phi, psi = W.make_pair(w, device=dev)
    phi, psi = W.storage(phi, w).contiguous(), W.storage(psi, w).contiguous()
    shape, cell = (w.n,) * 3, (w.L,) * 3
    rho = isdf.weights(phi, psi, "ssm", 2.0)          # |phi|^2 + |psi|^2 summed: twice the density
    rho_mean = float(rho.mean())
    rows = []
    for name, kind, alpha in [("ssm_a2", "ssm", 2.0), ("ssm_a1", "ssm", 1.0), ("ssm_a3", "ssm", 3.0),
                              ("ssm_a4", "ssm", 4.0), ("psm", "psm", 2.0), ("uniform_random", None, None)]:
        t0 = time.perf_counter()
        if kind is None:
            idx = torch.from_numpy(W.init_indices(np.ones(w.n_r), w.n_mu, 1000 + w.seed)).to(dev)
            labels = None
        else:
            wt = isdf.weights(phi, psi, kind, alpha)
            init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 1000 + w.seed)).to(dev)
            km = isdf.kmeans(wt, shape, cell, w.n_mu, init, w.iters, early_stop=True)
            idx, labels = km["idx"], km["labels"]
        plan = isdf.Plan(phi, psi, idx, mode="fp64", max_rows=min(w.n_r, 131072))
        fe = plan.fit_error()
        plan.check()
        plan.close()
        row = {"points": name, "fit_error_rel": fe["error"],
               "rho_at_points_rel": float(rho[idx].mean()) / rho_mean}
        if labels is not None:
            cr = isdf.cluster_residual(phi, psi, labels, idx)
            row["cluster_residual_rel"] = cr["R"] / cr["z2"]
        torch.cuda.synchronize()
        row["seconds"] = time.perf_counter() - t0
        rows.append(row)
    # the comparator of Sec. 2.1: randomized QRCP points (Eq. QRCP) on a sketch with p = N_mu + 16 columns;
    # one FP64 pass over the sketch per point, so only where the sketch stays below ~5 GB
    p = w.n_mu + 16
    if w.n_r * p * 16 < 5e9:
        t0 = time.perf_counter()
        rng = np.random.default_rng(5000 + w.seed)
        cr = lambda *sh: torch.from_numpy((rng.standard_normal(sh) + 1j * rng.standard_normal(sh)) / np.sqrt(2))
        q = isdf.qrcp_points(phi, psi, cr(w.n_orb, p), cr(w.n_orb, p), w.n_mu)
        plan = isdf.Plan(phi, psi, q["idx"], mode="fp64", max_rows=min(w.n_r, 131072))
        fe = plan.fit_error()
        plan.check()
        plan.close()
        torch.cuda.synchronize()
        rows.append({"points": "qrcp_randomized", "fit_error_rel": fe["error"],
                     "rho_at_points_rel": float(rho[q["idx"]].mean()) / rho_mean,
                     "seconds": time.perf_counter() - t0})
    print(json.dumps({"study": "weights", "workload": w.name, "grid": f"{w.n}^3", "n_orb": w.n_orb,
                      "n_mu": w.n_mu, "kmeans_iters": w.iters, "theta": "FP64 plan", "rows": rows}), flush=True)
    return 0


def run_exchange(args):
    """ISDF exchange application on a decomposition's output: per step the potentials V_mu of all
    interpolation vectors (five FFT passes over the N_r x N_mu matrix, Eq. V_mu) and the application
    -(V o Phi Phi_mu^H) Psi_mu (Eq. v2) for every grid row. Theta comes from a plan on the pair
    (Psi, Phi) at K-means points; the potentials overwrite a copy of it each step."""
    import torch

    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as isdf
    from paper_2208_07731_gb300 import workload as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    phi, psi = W.make_pair(w, device=dev)
    phi, psi = W.storage(phi, w).contiguous(), W.storage(psi, w).contiguous()
    shape, cell = (w.n,) * 3, (w.L,) * 3
    wt = isdf.weights(phi, psi)
    init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 1000 + w.seed))
    idx = isdf.kmeans(wt, shape, cell, w.n_mu, init, w.iters, early_stop=True)["idx"]
    pk = peaks()
    omega = 0.106          # the screening parameter of HSE06 (bohr^-1)
    res = {}
    for mode in ("mixed",) if args.no_fp64 else ("mixed", "fp64"):
        plan = isdf.Plan(psi, phi, idx, mode=mode, max_rows=min(w.n_r, 262144))
        theta = plan.fit_theta()
        plan.check()
        plan.close()
        ex = isdf.Exchange(shape, cell, w.n_mu, w.n_orb, w.n_orb, orb_dtype=phi.dtype, mode=mode, kernel="erfc",
                           omega=omega, max_rows=min(w.n_r, 131072), device=dev)
        v = torch.empty_like(theta)
        out = torch.empty((w.n_r, w.n_orb), dtype=torch.complex128, device=dev)
        steps = args.steps if mode == "mixed" else max(1, min(args.steps, 5))
        for _ in range(args.warmup):
            ex.potential(theta, out=v)
            ex.apply(phi, psi, idx, v, out=out)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        clocks = ClockSampler(dev.index)
        clocks.start()
        l0 = isdf.kernel_launches()
        for e0, e1, e2 in ev:
            e0.record()
            ex.potential(theta, out=v)
            e1.record()
            ex.apply(phi, psi, idx, v, out=out)
            e2.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ex.check()
        pot = sum(e0.elapsed_time(e1) for e0, e1, _ in ev) / steps
        app = sum(e1.elapsed_time(e2) for _, e1, e2 in ev) / steps
        res[mode] = {"ms": pot + app, "potential_ms": pot, "apply_ms": app, "steps": steps, "clocks": clk,
                     "launches": (isdf.kernel_launches() - l0) // steps, "out": out.clone(),
                     "el": 16 if mode == "fp64" else 8}
        ex.close()
        del theta, v
    a, b = res["mixed"], res.get("fp64")
    rel = (float(torch.linalg.vector_norm(a["out"] - b["out"]) / torch.linalg.vector_norm(b["out"]))
           if b else None)
    # the five FFT passes each read and write the N_r x N_mu matrix once
    fft_bytes = 5 * 2 * w.n_r * w.n_mu * a["el"]
    hbm = pk.get("hbm_gbs")
    achieved = fft_bytes / (a["potential_ms"] * 1e-3) / 1e9
    line = {"metric": "ISDF exchange applications/sec (V_mu by FFT, Eq. V_mu, + Eq. v2 on all grid rows)",
            "value": 1e3 / a["ms"], "unit": "applications/s", "n_gpus": 1, "steps": a["steps"],
            "warmup": args.warmup, "ms_per_step": a["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "mixed: complex64 V with FP32 FFT; application products split-FP16 x3 on tcgen05 (FP32 accumulate), "
                     "complex128 output",
            "data": "synthetic: seeded random plane-wave Bloch orbitals, orthonormalised; Theta from a plan on "
                    "(Psi, Phi) at K-means points",
            "config": {"workload": w.name, "grid": f"{w.n}^3", "n_orb": w.n_orb, "n_mu": w.n_mu,
                       "kernel": f"erfc, omega={omega}", "inputs_exceed_L2": True},
            "stages_ms": {"potential": a["potential_ms"], "apply": a["apply_ms"]},
            "gpu_launches": a["launches"], "clocks": a["clocks"],
            "roofline": {"kernel": "fft_lines (5 passes)", "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm if hbm else None,
                         "peak_source": "measured" if hbm else None,
                         "traffic": NCU_TRAFFIC.get((w.name, "fft_potential")),
                         "traffic_note": "DRAM bytes of the 5 passes of one potential (ncu), vs the algorithmic "
                                         "bytes below",
                         "algorithmic_bytes_per_step": fft_bytes},
            "fp64": ({"value": 1e3 / b["ms"], "ms_per_step": b["ms"], "potential_ms": b["potential_ms"],
                      "apply_ms": b["apply_ms"], "steps": b["steps"],
                      "fft_bound": "fp64 alu (complex128 FFT)"} if b else None),
            "out_rel_diff_mixed_vs_fp64": rel}
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Batched decompositions (several k-point pairs on one grid, small N): per step the shared weight
    (one accumulating weight call per pair), one K-means on it, and every pair's plan update and Theta
    fit; the batch runs the pairs on concurrent streams, the sequential variant runs the same plans one
    after another on one stream. Both steps are captured as CUDA graphs and replayed."""
    import torch

    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as isdf
    from paper_2208_07731_gb300 import workload as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    B = int(args.batch)
    pairs = [(p.contiguous(), q.contiguous()) for p, q in W.kpoint_pairs(w, B, device=dev)]
    shape, cell = (w.n,) * 3, (w.L,) * 3
    wbuf = torch.empty(w.n_r, dtype=torch.float64, device=dev)

    def shared_weight():
        for b, (p, q) in enumerate(pairs):
            isdf.weights(p, q, out=wbuf, accumulate=b > 0)

    shared_weight()
    init = torch.from_numpy(W.init_indices(wbuf.cpu().numpy(), w.n_mu, 1000 + w.seed)).to(dev)
    ws = torch.empty(isdf.kmeans_workspace_bytes(shape, w.n_mu), dtype=torch.uint8, device=dev)
    idx0 = isdf.kmeans(wbuf, shape, cell, w.n_mu, init, w.iters, workspace=ws, early_stop=True)["idx"]
    mode = "mixed"
    thetas = [torch.empty((w.n_r, w.n_mu), dtype=torch.complex64, device=dev) for _ in range(B)]
    batch = isdf.Batch(pairs, idx0, mode=mode, max_rows=w.n_r)
    plans = [isdf.Plan(p, q, idx0, mode=mode, max_rows=w.n_r) for p, q in pairs]

    def step_batched():
        shared_weight()
        km = isdf.kmeans(wbuf, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False,
                         early_stop=True)
        batch.update(km["idx"])
        batch.fit_theta(out=thetas)

    def step_sequential():
        shared_weight()
        km = isdf.kmeans(wbuf, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False,
                         early_stop=True)
        for pl, th in zip(plans, thetas):
            pl.update(km["idx"])
            pl.fit_theta(out=th)

    res = {}
    for name, fn in (("batched", step_batched), ("sequential", step_sequential)):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        l0 = isdf.kernel_launches()
        with torch.cuda.graph(graph):
            fn()
        launches = isdf.kernel_launches() - l0
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        res[name] = {"ms": e0.elapsed_time(e1) / args.steps, "launches": launches, "clocks": clocks.stop()}
        del graph
    batch.check()
    for pl in plans:
        pl.check()
    a, b = res["batched"], res["sequential"]
    line = {"metric": "ISDF batched decompositions/sec (shared weight + one K-means + per-pair plan update and "
                      "Theta fit)",
            "value": B * 1e3 / a["ms"], "unit": "decompositions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": a["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f16 hi+lo split x3 on tcgen05 (f32 accumulate) for the Gram and M^-1 GEMMs; f64 weights, "
                     "K-means, M, Cholesky, M^-1",
            "data": "synthetic: seeded random plane-wave Bloch orbitals at 8 k-points of one cell, orthonormalised",
            "config": {"workload": w.name, "grid": f"{w.n}^3", "n_orb": w.n_orb, "n_mu": w.n_mu, "pairs": B,
                       "lloyd_iters": w.iters, "launch": "one CUDA graph replay per step"},
            "gpu_launches": a["launches"], "clocks": a["clocks"],
            "sequential": {"value": B * 1e3 / b["ms"], "ms_per_step": b["ms"]},
            "speedup_vs_sequential": b["ms"] / a["ms"]}
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)
    return 0


def fp64_peak(dev):
    """Measured FP64 peak of this GPU: a cuBLAS DGEMM of 8192^3 (torch.matmul), best of 3 after a
    warm-up, timed with CUDA events on the current stream. A measurement of the FP64 pipe only
    (no kernel of the hot path runs here)."""
    import torch
    n = 8192
    g = torch.Generator(device=dev).manual_seed(7)
    a = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    b = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    c = a @ b
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return {"tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "how": "cuBLAS DGEMM 8192^3 via torch.matmul, best of 3"}


def theta_errors(theta_rows, ref, M_dev):
    """Relative Frobenius error of Theta on the sample rows and of the reconstructed Z there:
    ||(Theta - Theta_ref) C||_F / ||Theta_ref C||_F = sqrt(tr(dT M dT^H) / tr(T M T^H))."""
    import numpy as np
    import torch
    got = theta_rows.astype(np.complex128)
    d = got - ref
    err = float(np.linalg.norm(d) / np.linalg.norm(ref))
    dt = torch.from_numpy(d).to(M_dev.device)
    rt = torch.from_numpy(ref).to(M_dev.device)
    num = torch.real(torch.sum((dt @ M_dev) * dt.conj())).item()
    den = torch.real(torch.sum((rt @ M_dev) * rt.conj())).item()
    return err, math.sqrt(max(num, 0.0) / den)


def run_kernel_case(args):
    """One kernel family alone, at a workload's shapes, on inputs of a few GB (profiler-sized):
      gemm:    the split-FP16 Gram-Hadamard and M^-1 GEMMs of a mixed plan (N, N_mu of the workload) on
               --rows rows of seeded random complex64 orbitals, fitted in blocks of --rows / 2;
      weights: the weight kernel on --rows rows of seeded random orbitals of the workload's width and dtype;
      kmeans:  T Lloyd updates on the workload's grid and N_mu with a synthetic weight (a constant floor
               plus unit Gaussians on the 6 x 6 x 6 lattice of the silica-like cell).
    Prints one JSON line: time per launch (CUDA events, after warm-up) and algorithmic rates."""
    import numpy as np
    import torch

    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as isdf
    from paper_2208_07731_gb300 import workload as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    pk = peaks()
    gen = torch.Generator(device=dev).manual_seed(11)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    line = {"op": args.op, "workload": w.name}
    if args.op == "gemm":
        n_r, blk = args.rows, max(128, args.rows // 2)
        phi = (torch.randn(n_r, w.n_orb, dtype=torch.complex64, device=dev, generator=gen) / n_r ** 0.5).contiguous()
        psi = (torch.randn(n_r, w.n_orb, dtype=torch.complex64, device=dev, generator=gen) / n_r ** 0.5).contiguous()
        idx = torch.randperm(n_r, device=dev, generator=gen)[:w.n_mu].sort().values
        plan = isdf.Plan(phi, psi, idx, mode="mixed", max_rows=blk)
        theta = torch.empty((blk, w.n_mu), dtype=torch.complex64, device=dev)

        def fit():
            for r0 in range(0, n_r, blk):
                plan.fit_theta(r0, min(blk, n_r - r0), out=theta)

        for _ in range(max(1, args.warmup)):
            fit()
        torch.cuda.synchronize()
        plan.check()
        plan.enable_timing(4096)
        for k in isdf.TIMER_KINDS:
            plan.kernel_time(k)
        for _ in range(args.steps):
            fit()
        torch.cuda.synchronize()
        plan.check()
        peak = pk.get("bf16_tflops")
        for k in ("gram", "apply"):
            ms, n, rows = plan.kernel_time(k)
            fl = algorithmic_flops(w)[k] * rows / n
            a = fl / (ms / n * 1e-3) / 1e12
            line[k] = {"ms_per_launch": ms / n, "rows_per_launch": rows / n, "algorithmic_tflops": a,
                       "tensor_tflops_3_products": 3 * a, "frac_of_burst_bf16": a / peak if peak else None}
        line["config"] = {"n_r": n_r, "n_orb": w.n_orb, "n_mu": w.n_mu, "block_rows": blk,
                          "orbitals": "seeded random complex64 (shapes of the workload)"}
    elif args.op == "weights":
        n_r = args.rows
        dt = torch.complex64 if w.dtype == "c64" else torch.complex128
        phi = torch.randn(n_r, w.n_orb, dtype=dt, device=dev, generator=gen)
        psi = torch.randn(n_r, w.n_orb, dtype=dt, device=dev, generator=gen)
        out = torch.empty(n_r, dtype=torch.float64, device=dev)
        for _ in range(max(1, args.warmup)):
            isdf.weights(phi, psi, out=out)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(args.steps):
            isdf.weights(phi, psi, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        b = 2 * phi.numel() * phi.element_size() + 8 * n_r
        line.update({"ms_per_launch": ms, "bytes_per_launch": b, "gbs": b / ms / 1e6,
                     "frac_of_hbm": b / ms / 1e6 / pk["hbm_gbs"] if pk.get("hbm_gbs") else None,
                     "config": {"n_r": n_r, "n_orb": w.n_orb, "dtype": str(dt)}})
    else:
        n = w.n
        x = torch.arange(n, dtype=torch.float64, device=dev) * (w.L / n)
        X, Y, Z = torch.meshgrid(x, x, x, indexing="ij")
        wt = torch.full((n, n, n), 0.05, dtype=torch.float64, device=dev)
        for c in (np.arange(6) + 0.5) * (w.L / 6):
            for d in (np.arange(6) + 0.5) * (w.L / 6):
                for e in (np.arange(6) + 0.5) * (w.L / 6):
                    wt += torch.exp(-((X - c) ** 2 + (Y - d) ** 2 + (Z - e) ** 2) / 2.0)
        wt = wt.reshape(-1).contiguous()
        del X, Y, Z
        init = torch.from_numpy(W.init_indices(wt.cpu().numpy(), w.n_mu, 1000 + w.seed)).to(dev)
        shape, cell = (n,) * 3, (w.L,) * 3
        ws = torch.empty(isdf.kmeans_workspace_bytes(shape, w.n_mu), dtype=torch.uint8, device=dev)
        for _ in range(max(1, args.warmup)):
            km = isdf.kmeans(wt, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(args.steps):
            km = isdf.kmeans(wt, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        line.update({"ms_per_run": ms, "lloyd_updates": w.iters, "ms_per_pass": ms / (w.iters + 1),
                     "stats": km["stats"].tolist(),
                     "config": {"grid": f"{n}^3", "n_mu": w.n_mu, "weight": "0.05 + unit Gaussians on a 6^3 lattice"}})
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2208_07731_gb300 import build
    build.build()
    import paper_2208_07731_gb300 as isdf
    from paper_2208_07731_gb300 import workload as W

    from paper_2208_07731_gb300 import ranks as R
    rank, world, local = R.env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier_max(x):
        return R.max_over_ranks(x, device=dev)

    # independent problems per rank (like separate k-points): the seed differs by rank
    w = R.rank_workload(W.WORKLOADS[args.workload], rank)
    phi, psi = W.make_pair(w, device=dev)
    phi, psi = W.storage(phi, w).contiguous(), W.storage(psi, w).contiguous()
    torch.cuda.empty_cache()
    shape, cell = (w.n,) * 3, (w.L,) * 3
    wbuf = torch.empty(w.n_r, dtype=torch.float64, device=dev)
    isdf.weights(phi, psi, out=wbuf)
    init_h = W.init_indices(wbuf.cpu().numpy(), w.n_mu, 1000 + w.seed)
    init = torch.from_numpy(init_h).to(dev)  # device-resident: no host copy inside a captured step
    ws = torch.empty(isdf.kmeans_workspace_bytes(shape, w.n_mu), dtype=torch.uint8, device=dev)
    block = min(w.n_r, THETA_BLOCK)
    flops = algorithmic_flops(w)
    pk = peaks()

    def run_mode(mode):
        theta_blk = torch.empty((block, w.n_mu), dtype=torch.complex64 if mode == "mixed" else torch.complex128,
                                device=dev)
        km0 = isdf.kmeans(wbuf, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False)
        plan = isdf.Plan(phi, psi, km0["idx"], mode=mode, max_rows=block)

        def fit_all(sink=None):
            # Theta in row blocks into one reused buffer: every row is fitted, Theta is never resident
            for r0 in range(0, w.n_r, block):
                n = min(block, w.n_r - r0)
                plan.fit_theta(r0, n, out=theta_blk[:n])
                if sink is not None:
                    sink(r0, n, theta_blk[:n])

        def step():
            isdf.weights(phi, psi, out=wbuf)
            km = isdf.kmeans(wbuf, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False)
            plan.update(km["idx"])
            fit_all()
            return km

        # warm-up on a side stream (the capture below needs the library's one-time set-up done); the
        # first warm-up step is timed on the host to size the FP64 comparison run
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            t0 = time.perf_counter()
            step()
            torch.cuda.synchronize()
            t_first = time.perf_counter() - t0
            if mode == "mixed":
                warm, steps = args.warmup, args.steps
            else:
                # the FP64 path takes ~10-30 s per step on the largest grid: at least 2 timed steps,
                # at most about 60 s of them, and the warm-up count cut to fit (>= 1, the step above)
                steps = max(2, min(args.steps, int(60.0 / max(t_first, 1e-3))))
                warm = max(1, min(args.warmup, int(10.0 / max(t_first, 1e-3))))
            for _ in range(warm - 1):
                step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        plan.check()
        plan.enable_timing(4096)
        stages = None
        if mode == "mixed":
            # per-stage breakdown (one untimed step with events between stages)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[0].record()
            isdf.weights(phi, psi, out=wbuf)
            ev[1].record()
            km = isdf.kmeans(wbuf, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False)
            ev[2].record()
            plan.update(km["idx"])
            ev[3].record()
            fit_all()
            ev[4].record()
            torch.cuda.synchronize()
            stages = {k: ev[i].elapsed_time(ev[i + 1]) for i, k in enumerate(["weights", "kmeans", "plan_update",
                                                                              "fit_theta"])}
        for kind in isdf.TIMER_KINDS:
            plan.kernel_time(kind)  # reset: the capture below records one step's events
        run = step
        launches = None
        if not args.no_graph:
            # one decomposition captured as a CUDA graph; every timed step replays all of its kernels
            graph = torch.cuda.CUDAGraph()
            l0 = isdf.kernel_launches()
            with torch.cuda.graph(graph):
                km_graph = step()
            launches = isdf.kernel_launches() - l0

            def run():
                graph.replay()
                return km_graph
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        l0 = isdf.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            km = run()
        e1.record()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if launches is None:
            launches = (isdf.kernel_launches() - l0) // steps
        clk = clocks.stop()
        ms = barrier_max(e0.elapsed_time(e1)) / steps
        # kernel timings: the events of the last replay (graph) or of every timed step
        kt = {k: plan.kernel_time(k) for k in isdf.TIMER_KINDS}
        nsteps_timed = steps if args.no_graph else 1
        plan.check()
        stats = km["stats"].cpu().tolist()
        plan_stages = {k: kt[k][0] / nsteps_timed for k in ("gather_M", "cholesky", "tri_inverse", "minv",
                                                             "mixed_prep") if kt[k][1]}
        if stages is not None:
            stages["plan_update_parts"] = plan_stages
        return {"ms": ms, "stages": stages, "plan_stages": plan_stages, "kt": kt, "launches": launches,
                "clocks": clk, "plan": plan, "fit_all": fit_all, "idx": km["idx"].clone(), "stats": stats,
                "steps": steps, "warmup": warm, "first_step_s": t_first, "theta_blk": theta_blk,
                "graph": None if args.no_graph else graph}

    def roof(r, mode, fp64_pk):
        out = {}
        for name in ("apply", "gram"):
            ms_k, n_k, rows_k = r["kt"][name]
            if n_k == 0:
                continue
            per_launch_flops = flops[name] * rows_k / n_k
            achieved = per_launch_flops / (ms_k / n_k * 1e-3) / 1e12
            extra = {}
            peak = pk.get("bf16_tflops_sustained")
            src = "MEASURED_PEAKS.json bf16_tflops_sustained (of measured; fp16 dense = bf16 dense)"
            if peak is None:
                peak, src = 1700.0, "fallback sustained bf16 (no MEASURED_PEAKS.json)"
            if mode == "mixed":
                extra = {"split_products_per_product": 3,
                         "tensor_rate_tflops": 3.0 * achieved, "tensor_rate_frac": 3.0 * achieved / peak}
            else:
                # FP64 mode: the products run on tcgen05 by exact slicing, 28 FP16 digit-pair products per
                # FP64 product; the roofline counts that tensor work, the FP64-equivalent rate is info
                extra = {"fp64_equivalent_tflops": achieved, "slice_products_per_fp64_product": 28}
                achieved *= 28.0
                src += "; achieved = 28 digit-pair FP16 products per FP64 product"
            traffic = NCU_TRAFFIC.get((w.name, name)) if mode == "mixed" else None
            out[name] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": src,
                         "launches": n_k, "ms_per_launch": ms_k / n_k, "rows_per_launch": rows_k / n_k,
                         "algorithmic_flops_per_launch": per_launch_flops, **extra}
        # the FP64 factorisation and inverse (a9): Cholesky (stage 3) and the triangular inverse (stage 4,
        # folded into stage 3 when the recursive factorisation forms both), (4/3) n^3 real flops each (the
        # complex LAPACK counts). Above 512 points most of them run as exact-slicing tensor-core products,
        # so the FP64-equivalent rate can exceed the FP64 pipe; the ratio to the measured DGEMM rate is
        # reported as such.
        nt = r["kt"]["cholesky"][1]
        if nt:
            ms_chol = (r["kt"]["cholesky"][0] + r["kt"]["tri_inverse"][0]) / nt
            fl = 8.0 / 3.0 * float(w.n_mu) ** 3
            achieved = fl / (ms_chol * 1e-3) / 1e12
            out["fp64_chain"] = {"bound": "fp64-equivalent", "achieved": achieved, "peak": fp64_pk["tflops"],
                                 "unit": "TFLOP/s", "frac": achieved / fp64_pk["tflops"], "traffic": None,
                                 "peak_source": "measured in this run: " + fp64_pk["how"],
                                 "launches": nt, "ms_per_launch": ms_chol, "algorithmic_flops_per_launch": fl,
                                 "what": "Cholesky factor + triangular inverse of M (FP64 results; blocked "
                                         "16-wide FP64-pipe steps up to 512 rows, exact-slicing products above)"}
        return out

    res = {"mixed": run_mode("mixed")}
    if not args.no_fp64:
        res["fp64"] = run_mode("fp64")
    fpk = fp64_peak(dev)
    mixed = res["mixed"]
    rf = roof(mixed, "mixed", fpk)
    st = mixed["stages"]
    wbytes = w.n_r * 2 * w.n_orb * phi.element_size() + 8 * w.n_r
    hbm = pk.get("hbm_gbs")
    line = {"metric": METRIC, "value": R.job_throughput(1, world, mixed["ms"] * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": mixed["steps"], "warmup": mixed["warmup"], "ms_per_step": mixed["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 hi+lo split x3 on tcgen05 (f32 accumulate) for the Gram and M^-1 GEMMs; f64 for weights, "
                     "K-means decisions and sums, M, Cholesky, M^-1",
            "data": "synthetic: seeded random plane-wave Bloch orbitals, orthonormalised (no DFT data available)",
            "config": {"workload": w.name, "grid": f"{w.n}^3", "n_r": w.n_r, "L_bohr": w.L, "n_orb": w.n_orb,
                       "n_mu": w.n_mu, "lloyd_iters": w.iters, "orbital_dtype": w.dtype, "mode": "mixed",
                       "centres": w.centres, "theta_block_rows": block,
                       "theta": "fitted in row blocks into one reused block buffer, never fully resident",
                       "launch": "host launches" if args.no_graph else "one CUDA graph replay per step",
                       "l2": f"inputs larger than L2: Phi+Psi {2 * phi.numel() * phi.element_size() / 1e9:.2f} GB, "
                             f"Theta {w.n_r * w.n_mu * 8 / 1e9:.1f} GB written per step"},
            "roofline": None, "rooflines": rf,
            "stages_ms": st, "gpu_launches": mixed["launches"], "clocks": mixed["clocks"],
            "kmeans_stats": dict(zip(["updates", "near_ties", "empty", "fp64_decided"], mixed["stats"])),
            "fp64_peak_measured": fpk}
    if st and hbm:
        ach = wbytes / (st["weights"] * 1e-3) / 1e9
        rf["weights"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "traffic": NCU_TRAFFIC.get((w.name, "weights")), "launches": 1,
                         "ms_per_launch": st["weights"], "algorithmic_bytes_per_launch": wbytes,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "note": "stage time of one untimed step (CUDA events)"}
    # the dominant kernel by measured time per step (stage-timed entries count once per step)
    dom = max((k for k in rf if k != "weights"), key=lambda k: rf[k]["ms_per_launch"] * rf[k]["launches"])
    line["roofline"] = dict(rf[dom], kernel=dom)
    if "fp64" in res:
        f = res["fp64"]
        line["fp64"] = {"value": R.job_throughput(1, world, f["ms"] * 1e-3), "unit": UNIT, "ms_per_step": f["ms"],
                        "steps": f["steps"], "warmup": f["warmup"], "first_step_s": f["first_step_s"],
                        "rooflines": roof(f, "fp64", fpk), "plan_update_parts": f["plan_stages"],
                        "gpu_launches": f["launches"], "clocks": f["clocks"],
                        "same_idx_as_mixed": bool(torch.equal(mixed["idx"], f["idx"]))}
        line["speedup_mixed_vs_fp64"] = f["ms"] / mixed["ms"]

    # end to end through the public API: pinned host orbitals in, all of Theta and idx back in pinned host memory,
    # every step (the plan and orbital buffers of the timed run are reused). Plan.fit_theta_host fits Theta in row
    # blocks into the plan's device staging blocks and copies each block to the host array on a copy stream while
    # the next block is fitted. The split-precision fit reads only the FP16 operand copies made by the plan update,
    # so the next step's orbitals are copied in (on their own stream) while this step's Theta is fitted: each step
    # still copies its 34 GB in and its Theta out inside the timed region, one step ahead.
    plan = mixed["plan"]
    mixed["graph"] = None
    dtype_t = mixed["theta_blk"].dtype
    ph_h = phi.cpu().pin_memory()
    qh_h = psi.cpu().pin_memory()
    theta_h = torch.empty((w.n_r, w.n_mu), dtype=dtype_t, pin_memory=True)
    idx_h = torch.empty(w.n_mu, dtype=torch.int64).pin_memory()
    copy_in = torch.cuda.Stream()
    in_ready, update_done = torch.cuda.Event(), torch.cuda.Event()
    pipelined = plan.mode == isdf.MIXED              # the FP64 fit reads the orbitals themselves

    def load_inputs():
        with torch.cuda.stream(copy_in):
            phi.copy_(ph_h, non_blocking=True)
            psi.copy_(qh_h, non_blocking=True)
            in_ready.record(copy_in)

    def e2e_step():
        compute = torch.cuda.current_stream()
        if not pipelined:
            load_inputs()
        compute.wait_event(in_ready)                 # this step's orbitals have landed
        isdf.weights(phi, psi, out=wbuf)
        km = isdf.kmeans(wbuf, shape, cell, w.n_mu, init, w.iters, workspace=ws, labels=False, objective=False)
        plan.update(km["idx"])                       # the step's last reader of the orbitals
        if pipelined:
            update_done.record(compute)
            copy_in.wait_event(update_done)
            load_inputs()                            # the next step's orbitals, beside this step's fit
        plan.fit_theta_host(theta_h)
        idx_h.copy_(km["idx"], non_blocking=True)

    if pipelined:
        load_inputs()
    e2e_steps = args.steps if mixed["ms"] < 200.0 else max(3, min(args.steps, 5))
    for _ in range(max(3, min(args.warmup, 3))):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.current_stream().wait_stream(copy_in)    # the last step's input copy is inside the timed region
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = barrier_max(e0.elapsed_time(e1)) / e2e_steps
    line["e2e"] = {"value": R.job_throughput(1, world, e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                   "steps": e2e_steps, "warmup": max(3, min(args.warmup, 3)),
                   "h2d_bytes_per_step": 2 * phi.numel() * phi.element_size(),
                   "d2h_bytes_per_step": w.n_r * w.n_mu * dtype_t.itemsize + idx_h.numel() * 8,
                   "theta_block_rows": block,
                   "d2h_overlap": "Theta blocks copied from 3 device staging blocks while the next block is fitted",
                   "h2d_overlap": ("the next step's orbitals copied in while this step's Theta is fitted" if pipelined
                                   else "none")}
    del ph_h, qh_h, theta_h

    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle as O
        O.load()
        # Theta and reconstructed-Z errors of both GPU modes against the oracle on the seeded row sample
        rows = W.subsample_rows(w.n_r, min(ERROR_ROWS, w.n_r), 2000 + w.seed)
        rows_t = torch.from_numpy(rows).to(dev)
        idx = mixed["idx"]
        idx_h2 = idx.cpu().numpy()
        pm, qm = O.gather(phi[idx].cpu().numpy(), psi[idx].cpu().numpy(), np.arange(w.n_mu))
        M = O.form_M(pm, qm)
        L = O.cholesky(M)
        ref = O.theta_rows(phi[rows_t].cpu().numpy(), psi[rows_t].cpu().numpy(), pm, qm, L, np.arange(len(rows)))
        M_dev = torch.from_numpy(M).to(dev)
        # mixed: the rows of one more blocked fit (the timed step's own kernels and layout)
        got = np.empty((len(rows), w.n_mu), np.complex64)

        def sink(r0, n, blk):
            sel = np.nonzero((rows >= r0) & (rows < r0 + n))[0]
            if len(sel):
                got[sel] = blk[torch.from_numpy(rows[sel] - r0).to(dev)].cpu().numpy()

        plan.update(idx)
        mixed["fit_all"](sink)
        plan.check()
        e_t, e_z = theta_errors(got, ref, M_dev)
        errs = {"rows": len(rows), "row_seed": 2000 + w.seed, "mixed_theta": e_t, "mixed_z": e_z,
                "gate_mixed": 1e-5}
        if "fp64" in res:
            # FP64: a plan on [Phi[idx]; Phi[rows]] with points 0..N_mu-1 gives the same M, L, M^-1 and the
            # same per-row products as the full plan (FP64-mode products scale every row on its own)
            f = res["fp64"]
            f["plan"].close()
            sub_p = torch.cat([phi[idx], phi[rows_t]]).contiguous()
            sub_q = torch.cat([psi[idx], psi[rows_t]]).contiguous()
            sp = isdf.Plan(sub_p, sub_q, torch.arange(w.n_mu, device=dev), mode="fp64",
                           max_rows=min(len(rows), 8192))
            th64 = sp.fit_theta(w.n_mu, len(rows))
            sp.check()
            e_t, e_z = theta_errors(th64.cpu().numpy(), ref, M_dev)
            errs.update({"fp64_theta": e_t, "fp64_z": e_z, "gate_fp64": 1e-10,
                         "fp64_rows_via": "plan on [Phi[idx]; Phi[rows]] (row-independent FP64 products)"})
            sp.close()
            del th64, sub_p, sub_q
        line["theta_rel_err"] = errs
        del M_dev
        # the CPU oracle on a bounded sample of the same workload
        ctx = oracle_context(w, phi, psi)
        total, spent, parts, desc = oracle_sample(ctx)
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        line["cpu_baseline"] = {"value": 1.0 / total, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc, "sample_seconds": spent, "seconds_by_stage": parts}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.workload is None:
        args.workload = {"adjoint": "adjoint", "exchange": "medium", "batch": "kpoints"}.get(
            args.op, "medium" if args.study else DEFAULT_WORKLOAD)
    if args.impl == "reference":
        return run_reference(args)
    if args.study == "weights":
        return run_study(args)
    if args.op == "exchange":
        return run_exchange(args)
    if args.op == "batch":
        return run_batch(args)
    if args.op in ("gemm", "weights", "kmeans"):
        return run_kernel_case(args)
    if args.op == "adjoint" or args.workload == "adjoint":
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
