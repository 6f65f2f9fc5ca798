"""Host logic of bench.py (no GPU): the Theta / reconstructed-Z error metric,
the bounded oracle sample shared by the GPU line's cpu_baseline and the
reference arm, and the reference arm's JSON line on the tiny workload."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2208_07731_gb300 import workload as W  # noqa: E402


def test_theta_errors_metric():
    rng = np.random.default_rng(0)
    ref = rng.standard_normal((40, 12)) + 1j * rng.standard_normal((40, 12))
    A = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    M = A @ A.conj().T + 12 * np.eye(12)
    Md = torch.from_numpy(M)
    e_t, e_z = bench.theta_errors(ref.astype(np.complex64), ref, Md)
    assert e_t < 1e-7 and e_z < 1e-7
    # a relative perturbation of 1e-3 along Theta itself: both errors are exactly that size
    e_t, e_z = bench.theta_errors(ref * (1 + 1e-3), ref, Md)
    assert math.isclose(e_t, 1e-3, rel_tol=1e-9) and math.isclose(e_z, 1e-3, rel_tol=1e-9)
    # the Z error weighs the error by M: an error along M's top eigenvector counts more than along
    # the bottom one, for the same Theta error
    lam, V = np.linalg.eigh(M)
    d_top = np.outer(np.ones(40), V[:, -1].conj()) * 1e-3
    d_bot = np.outer(np.ones(40), V[:, 0].conj()) * 1e-3
    _, z_top = bench.theta_errors(ref + d_top, ref, Md)
    _, z_bot = bench.theta_errors(ref + d_bot, ref, Md)
    assert z_top > z_bot * math.sqrt(lam[-1] / lam[0]) * 0.99


def test_oracle_sample_tiny():
    w = W.WORKLOADS["tiny"]
    phi, psi = W.make_pair(w)
    ctx = bench.oracle_context(w, phi, psi)
    total, spent, parts, desc = bench.oracle_sample(ctx)
    assert set(parts) == {"weights", "kmeans", "M_cholesky", "theta"}
    assert all(v > 0 for v in parts.values()) and total >= spent > 0
    assert "scaled" in desc


def test_reference_arm_line_tiny():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "tiny", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env,
                         timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["extrapolated"] is True
    assert line["config"]["workload"] == "tiny" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    # the timed region really ran: the steps' measured sample time fits in it
    assert line["ms_per_step"] * line["steps"] / 1e3 <= line["timed_region_s"] * 1.01
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
