"""Sec. IV figures computed from a solver result: the Hamiltonian-ratio
estimate chi_hat, the estimated time-to-solution and the speed (Sec. IV-C),
and the pruning rate (Sec. IV-A)."""

from __future__ import annotations

import math

import numpy as np


def chi_hat(inst, E: float) -> float:
    """1/2 - E / (2 (sqrt(d) ||A||_F + ||b||_1)) for E written as
    s^T A s + b^T s in the paper's form (A = j_scale J, b = h in the paper
    convention; A = -j_scale J / 2, b = -h in the physics convention)."""
    if inst.convention == "paper":
        cq, ch = inst.j_scale, 1.0
    else:
        cq, ch = -0.5 * inst.j_scale, -1.0
    J = np.asarray(inst.dense(), dtype=np.float64)
    h = np.zeros(inst.n) if inst.h is None else np.asarray(inst.h, dtype=np.float64)
    scale = math.sqrt(inst.n) * abs(cq) * float(np.linalg.norm(J)) + abs(ch) * float(np.abs(h).sum())
    return 0.5 - E / (2.0 * scale)


def paper_metrics(inst, E: float, seconds: float) -> dict:
    """chi_hat, the estimated time-to-solution T log(1 - 0.99) /
    log(1 - e^chi_hat / d) and the speed v = chi_hat / T for one solve of
    duration T seconds."""
    chi = chi_hat(inst, E)
    p = math.exp(chi) / inst.n
    tts = seconds * math.log(1.0 - 0.99) / math.log(1.0 - p) if 0.0 < p < 1.0 else None
    return {"chi_hat": chi, "T_s": seconds, "tts_s": tts, "v_per_s": chi / seconds}
