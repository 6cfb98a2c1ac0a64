"""Domain selection (Sec. III-B) in float64, one column per restart.

What one step computes, for every restart b independently (theta has shape
(n, B); the paper's theta = diag(theta_1..theta_d) is one column):

1. Round the relaxed spins x = sin(theta) to the local optimum of the current
   domain (Eq. local optimal, right-hand form): s = sgn+(sin theta), with
   sgn+(0) = +1.
2. Coupling product G = J_stored s, energy E = cQ s^T G + cH h^T s (Sec. II).
3. Loss field of Eq. (loss function), taken literally with s frozen:
   F = (A - mu I) s + b = cQ G + cH h - mu s.
4. Gradient of L(theta) = 1^T sin(theta) F with s frozen: g = cos(theta) * F.
5. Adam (Kingma and Ba, the optimiser named in Sec. IV-B) with bias correction:
   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
   theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
6. Projection: theta -= 2 pi rint(theta / 2 pi), which keeps theta in
   [-pi, pi] and leaves sin and cos unchanged.

The loop runs steps t = 1..T from theta_init = asin(x0), x0 uniform in [-1, 1)
(SplitMix64, see ``rng``), m = v = 0, and evaluates the spins of theta_T once
more after the last update (step T + 1). Each restart keeps the lowest energy
seen (strict <, so the earliest step wins ties); across restarts the lowest
(energy, restart index) wins.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import ising, rng

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Params:
    restarts: int = 64
    steps: int = 100
    lr: float = 6.0
    mu: float = 0.0
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    seed: int = 0
    # "rounded": G = J s (the paper's loss field on the local optimum s of the
    # domain); "relaxed": G = J sin(theta), the coupling product on the
    # relaxed spins, with the same F = cQ G + cH h - mu s and g = cos(theta) F
    grad_mode: str = "rounded"


def round_spins(theta: np.ndarray) -> np.ndarray:
    """s = sgn+(sin theta) as float64 +-1."""
    return np.where(np.sin(theta) >= 0.0, 1.0, -1.0)


def loss_field(J, h, cq, ch, mu, s):
    """F = cQ J s + cH h - mu s, plus G = J s."""
    G = J @ s
    F = cq * G + ch * h[:, None] - mu * s
    return F, G


def loss(J, h, cq, ch, mu, theta, s):
    """L(theta) = sum_i sin(theta_i) F_i with s held fixed (Eq. loss function)."""
    F, _ = loss_field(J, h, cq, ch, mu, s)
    return np.sum(np.sin(theta) * F, axis=0)


@dataclasses.dataclass
class StepResult:
    spins: np.ndarray  # s_t, (n, B)
    G: np.ndarray
    energy: np.ndarray  # E(s_t), (B,)
    F: np.ndarray
    grad: np.ndarray
    theta: np.ndarray  # theta_t
    m: np.ndarray
    v: np.ndarray


def step(J, h, cq, ch, p: Params, theta, m, v, t: int) -> StepResult:
    """One update from (theta_{t-1}, m_{t-1}, v_{t-1}) at step number t >= 1."""
    s = round_spins(theta)
    F, G = loss_field(J, h, cq, ch, p.mu, s)
    E = cq * np.sum(s * G, axis=0) + ch * (h @ s)
    if p.grad_mode == "relaxed":
        # the product on the relaxed spins drives the update; E stays that of s
        G = J @ np.sin(theta)
        F = cq * G + ch * h[:, None] - p.mu * s
    elif p.grad_mode != "rounded":
        raise ValueError(p.grad_mode)
    g = np.cos(theta) * F
    m = p.beta1 * m + (1.0 - p.beta1) * g
    v = p.beta2 * v + (1.0 - p.beta2) * g * g
    mhat = m / (1.0 - p.beta1 ** t)
    vhat = v / (1.0 - p.beta2 ** t)
    th = theta - p.lr * mhat / (np.sqrt(vhat) + p.eps)
    th = th - TWO_PI * np.rint(th / TWO_PI)
    return StepResult(s, G, E, F, g, th, m, v)


# Convergence rule of Sec. IV-B: a restart has converged at step t when the
# spread (max - min) of its last CONV_WINDOW values is at most CONV_TOL times
# the change since the first step. Read on the energy of the rounded spins
# (at convergence sin(theta) -> s and the loss equals E - mu d).
CONV_WINDOW = 5
CONV_TOL = 0.005


def converged(window, E_t, E_1):
    """The Sec. IV-B test on the last CONV_WINDOW energies of each restart
    (`window`, shape (CONV_WINDOW, B), any order), the current energy E_t and
    the first E_1: max - min of the window <= CONV_TOL |E_t - E_1|."""
    return window.max(axis=0) - window.min(axis=0) <= CONV_TOL * np.abs(E_t - E_1)


def select_domain(inst, p: Params, trace: bool = False, theta0=None, converge: bool = False):
    """Run T steps on all restarts; return a dict with the overall best
    (energy, spins, restart, step), per-restart bests, the last-step energies
    E_{T+1} and, when ``trace``, the (T+1, B) energy trace.

    With ``converge``, each restart stops at the first step t >= CONV_WINDOW
    where max - min of E_{t-4..t} <= CONV_TOL |E_t - E_1| (Sec. IV-B): its best
    and last energy are those of steps 1..t, ``conv_step`` holds t (0 if it
    never stops), and the run ends once every restart has stopped
    (``steps_done``); the final evaluation E_{T+1} applies to the restarts
    still running after step T."""
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    J = ising.coupling_matrix(inst)
    h = ising.field(inst)
    n, B = inst.n, p.restarts
    theta = rng.theta_init(p.seed, B, n) if theta0 is None else np.array(theta0, dtype=np.float64)
    m = np.zeros((n, B))
    v = np.zeros((n, B))
    best_e = np.full(B, np.inf)
    best_t = np.zeros(B, dtype=np.int64)
    best_s = np.zeros((n, B))
    tr = np.zeros((p.steps + 1, B)) if trace else None

    conv_step = np.zeros(B, dtype=np.int64)
    ring = np.zeros((CONV_WINDOW, B))
    E_init = np.zeros(B)
    E_stop = np.zeros(B)

    def keep(E, s, t):
        better = (E < best_e) & (conv_step == 0)
        best_e[better] = E[better]
        best_t[better] = t
        best_s[:, better] = s[:, better]

    steps_done = p.steps
    for t in range(1, p.steps + 1):
        r = step(J, h, cq, ch, p, theta, m, v, t)
        keep(r.energy, r.spins, t)
        if trace:
            tr[t - 1] = r.energy
        theta, m, v = r.theta, r.m, r.v
        if converge:
            active = conv_step == 0
            ring[(t - 1) % CONV_WINDOW, active] = r.energy[active]
            if t == 1:
                E_init[:] = r.energy
            E_stop[active] = r.energy[active]
            if t >= CONV_WINDOW:
                hit = active & converged(ring, r.energy, E_init)
                conv_step[hit] = t
            if (conv_step > 0).all():
                steps_done = t
                break
    s_last = round_spins(theta)
    E_last = cq * np.sum(s_last * (J @ s_last), axis=0) + ch * (h @ s_last)
    if steps_done == p.steps:
        keep(E_last, s_last, p.steps + 1)
    if converge:
        stopped = conv_step > 0
        E_last = np.where(stopped, E_stop, E_last)
    if trace:
        tr[p.steps] = E_last
    b = int(np.lexsort((np.arange(B), best_e))[0])
    return dict(best_energy=float(best_e[b]), best_restart=b,
                best_step=int(best_t[b]), best_spins=best_s[:, b].astype(np.int8),
                restart_best_energy=best_e, restart_best_step=best_t,
                restart_best_spins=best_s.astype(np.int8),
                last_energy=E_last, last_spins=s_last.astype(np.int8),
                theta=theta, m=m, v=v, trace=tr, conv_step=conv_step, steps_done=steps_done)
