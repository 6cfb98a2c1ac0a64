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


def grad_from_moments(m0, m1, p):
    """The gradient the kernel used, recovered from its first moments: the
    kernel forms m1 = fma(b1, m0, (1 - b1) g) in FP32 with b1 and 1 - b1
    rounded to FP32 (1 - b1 formed in FP64 first), so g = (m1 - b1 m0) / (1 - b1)
    up to the two roundings, |err| <= 2^-24 (|g| + |m1| / (1 - b1))."""
    b1 = float(np.float32(p.beta1))
    omb1 = float(np.float32(1.0 - p.beta1))
    return (m1 - b1 * m0) / omb1, omb1


def energy_bound(inst, G, Gref, mu=0.0):
    """Bound on the step energies' error for non-integer couplings, derived
    from the measured product error: E_b = sum_i s_i (cQ G_i + cH h_i), each
    term formed by one FMA (error 2^-24 |term|) and summed in FP32 over a
    warp's 32 rows by a 5-level tree before the FP64 sum of the partial rows,
    so |dE_b| <= |cQ| sum_i |dG_bi| + 7 2^-24 sum_i |cQ G_bi + cH h_i|.
    G, Gref: restart-major [B][n]."""
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    h = ising.field(inst)[None, :]
    return abs(cq) * np.abs(G - Gref).sum(axis=1) + 7 * 2.0 ** -24 * np.abs(cq * G + ch * h).sum(axis=1)


def check_step(inst, st0, st1, last_E, p, exact_energy, tol=TOL, min_clear=0.98, G0=None):
    """st0: state before step t = st0['t'] + 1, st1: after it. `tol` bounds
    the product's error relative to the row scale (TOL for FP32 arithmetic);
    `min_clear` is the fraction of next spins that must lie outside it. G0
    (restart-major [B][n]), when given, is the coupling product the kernel
    forms at st0 (read through ising_ds_coupling): it is held to `tol` of the
    row scale itself and sets the energy bound of non-integer instances."""
    t = st0["t"] + 1
    r = oracle_step(inst, st0, t, p)
    # spins consumed by the step are the oracle's rounding of the same theta
    np.testing.assert_array_equal(st0["spins"].T, r.spins.astype(np.int8))
    sc = row_scale(inst, p.mu)[:, None]
    if G0 is not None and p.grad_mode == "rounded":
        # the product in stored units, against sum_j |J_ij|
        a = np.asarray(abs(ising.coupling_matrix(inst)).sum(axis=1)).ravel()[None, :]
        assert np.all(np.abs(G0 - r.G.T) <= tol * a + 1e-30)
    if exact_energy:
        np.testing.assert_array_equal(last_E, r.energy)
    elif G0 is not None and p.grad_mode == "rounded":
        bound = energy_bound(inst, G0.astype(np.float64), r.G.T)
        assert np.all(np.abs(last_E - r.energy) <= bound + 1e-12 * np.abs(r.energy))
    else:
        # without the product: each G_i may be off by TOL times the row's
        # scale (the FP32 product's bound, also the gradient's below), and the
        # errors of a local optimum's terms s_i G_i can share a sign, so bound
        # |dE| by the sum of the row scales (the worst case)
        bound = TOL * (np.sum(row_scale(inst, 0.0)) + 1.0)
        assert np.all(np.abs(last_E - r.energy) <= bound)
    m0 = st0["m"].T.astype(np.float64)
    v0 = st0["v"].T.astype(np.float64)
    m1 = st1["m"].T.astype(np.float64)
    v1 = st1["v"].T.astype(np.float64)
    assert np.all(np.abs(m1 - r.m) <= tol * (np.abs(m0) + (1 - p.beta1) * sc) + 1e-30)
    assert np.all(np.abs(v1 - r.v) <= tol * (v0 + 2 * (1 - p.beta2) * sc * sc) + 1e-30)
    # the kernel's own gradient at every step, recovered from m0 and m1,
    # against the oracle's, at tol of the row scale plus the recovery's rounding
    g, omb1 = grad_from_moments(m0, m1, p)
    rec = 2.0 ** -24 * (np.abs(r.grad) + tol * sc + np.abs(m1) / omb1) * 1.01
    assert np.all(np.abs(g - r.grad) <= tol * sc + rec + 1e-30)
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
