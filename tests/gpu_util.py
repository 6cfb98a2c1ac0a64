"""Shared checks for the GPU parity tests: the CUDA path's state, exported
through the C ABI, against one oracle step from the same state."""

import math

import numpy as np

from oracle import domain_selection as ods
from oracle import ising

TOL = 1e-5  # per-element bound on FP32 gradient error, relative to the row scale


def row_scale(inst, mu):
    """|cQ| sum_j |J_ij| + |cH h_i| + mu: the largest the loss field can be."""
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    J = ising.coupling_matrix(inst)
    a = np.asarray(abs(J).sum(axis=1)).ravel()
    return abs(cq) * a + abs(ch) * np.abs(ising.field(inst)) + mu


def oracle_step(inst, st, t, p):
    """One oracle step from an exported state (restart-major arrays)."""
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    J = ising.coupling_matrix(inst)
    h = ising.field(inst)
    th = st["theta"].T.astype(np.float64)
    m = st["m"].T.astype(np.float64)
    v = st["v"].T.astype(np.float64)
    return ods.step(J, h, cq, ch, p, th, m, v, t)


def wrapped_diff(a, b):
    d = a - b
    return d - 2 * math.pi * np.rint(d / (2 * math.pi))


def check_step(inst, st0, st1, last_E, p, exact_energy, tol=TOL, min_clear=0.98):
    """st0: state before step t = st0['t'] + 1, st1: after it. `tol` bounds
    the product's error relative to the row scale (TOL for FP32 arithmetic);
    `min_clear` is the fraction of next spins that must lie outside it."""
    t = st0["t"] + 1
    r = oracle_step(inst, st0, t, p)
    # spins consumed by the step are the oracle's rounding of the same theta
    np.testing.assert_array_equal(st0["spins"].T, r.spins.astype(np.int8))
    if exact_energy:
        np.testing.assert_array_equal(last_E, r.energy)
    else:
        # each G_i may be off by TOL times the row's scale (the FP32 product's
        # bound, also the gradient's below), and the tensor cores' rounding of
        # the accumulation is not unbiased, so the errors of a local optimum's
        # terms s_i G_i can add up: bound |dE| by the sum of the row scales
        bound = TOL * (np.sum(row_scale(inst, 0.0)) + 1.0)
        assert np.all(np.abs(last_E - r.energy) <= bound)
    sc = row_scale(inst, p.mu)[:, None]
    m0 = st0["m"].T.astype(np.float64)
    v0 = st0["v"].T.astype(np.float64)
    # gradient recovered from the first moment: g = (m1 - b1 m0) / (1 - b1)
    m1 = st1["m"].T.astype(np.float64)
    v1 = st1["v"].T.astype(np.float64)
    assert np.all(np.abs(m1 - r.m) <= tol * (np.abs(m0) + (1 - p.beta1) * sc) + 1e-30)
    assert np.all(np.abs(v1 - r.v) <= tol * (v0 + 2 * (1 - p.beta2) * sc * sc) + 1e-30)
    if np.all(m0 == 0):
        g = m1 / (1 - p.beta1)
        assert np.all(np.abs(g - r.grad) <= tol * sc)
    th1 = st1["theta"].T.astype(np.float64)
    # Adam divides by sqrt(v): a gradient error dg moves theta by sens * dg,
    # sens = lr * d(mhat / (sqrt(vhat) + eps)) / dg, evaluated at the oracle's values
    c1 = 1.0 / (1.0 - p.beta1 ** t)
    c2 = 1.0 / (1.0 - p.beta2 ** t)
    mhat, vhat = r.m * c1, r.v * c2
    rv = np.sqrt(vhat)
    with np.errstate(divide="ignore", invalid="ignore"):
        sens = p.lr * ((1 - p.beta1) * c1 / (rv + p.eps) +
                       np.abs(mhat) * (1 - p.beta2) * c2 * np.abs(r.grad) /
                       np.maximum(rv * (rv + p.eps) ** 2, 1e-300))
    # gradient error: for integer instances F is exact and only cos(theta) is
    # approximated (absolute error <= 2^-21.41 < 4e-7 on [-pi, pi]); otherwise
    # the FP32 product bounds it
    dg = np.abs(r.F) * 4e-7 if (exact_energy and tol == TOL and p.grad_mode == "rounded") else tol * sc
    tol_th = tol * (1 + p.lr) * (1 + np.abs(mhat) / (rv + p.eps)) + sens * dg
    assert np.all(np.abs(wrapped_diff(th1, r.theta)) <= tol_th)
    # next spins: identical wherever the rounding is not within the tolerance
    clear = np.abs(np.sin(r.theta)) > 2 * tol_th
    nxt = st1["spins"].T
    assert np.array_equal(nxt[clear], ods.round_spins(r.theta)[clear].astype(np.int8))
    assert clear.mean() > min_clear, clear.mean()
    return r
