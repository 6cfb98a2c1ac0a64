"""Ising energy, single-flip difference and max-cut value (Sec. II, Sec. III-A).

The paper writes the energy as E(s) = s^T J s + h^T s with J symmetric and
zero on the diagonal (Sec. II, scalar form of the Hamiltonian). Instances are
stored as (J_stored, h, j_scale, convention); both conventions reduce to the
paper's form with

    A = cQ * J_stored,  b = cH * h,   E(s) = s^T A s + b^T s,

where (cQ, cH) = (j_scale, +1) for the paper convention and
(-j_scale / 2, -1) for the physics convention E = -1/2 s^T J s - h^T s.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def coefficients(j_scale: float, convention: str) -> tuple[float, float]:
    """(cQ, cH) such that E(s) = cQ * s^T J_stored s + cH * h^T s."""
    if convention == "paper":
        return float(j_scale), 1.0
    if convention == "physics":
        return -0.5 * float(j_scale), -1.0
    raise ValueError(convention)


def coupling_matrix(inst):
    """Stored couplings as float64: dense ndarray or scipy CSR (exact copy)."""
    if inst.layout == "dense":
        return np.asarray(inst.J, dtype=np.float64)
    return sp.csr_matrix((np.asarray(inst.data, dtype=np.float64),
                          np.asarray(inst.indices), np.asarray(inst.indptr)),
                         shape=(inst.n, inst.n))


def field(inst) -> np.ndarray:
    if inst.h is None:
        return np.zeros(inst.n, dtype=np.float64)
    return np.asarray(inst.h, dtype=np.float64)


def paper_form(inst):
    """(A, b) of E(s) = s^T A s + b^T s as dense float64 arrays."""
    cq, ch = coefficients(inst.j_scale, inst.convention)
    J = coupling_matrix(inst)
    J = J.toarray() if sp.issparse(J) else J
    return cq * J, ch * field(inst)


def energy(inst, s) -> np.ndarray:
    """E(s) = cQ s^T J s + cH h^T s in float64. s: (n,) or (n, B) of +-1."""
    cq, ch = coefficients(inst.j_scale, inst.convention)
    J = coupling_matrix(inst)
    s = np.asarray(s, dtype=np.float64)
    Js = J @ s
    q = np.sum(s * Js, axis=0)
    return cq * q + ch * (field(inst) @ s)


def energy_edges(inst, s) -> np.ndarray:
    """Same energy as a sum over couplings: E = sum_{i<j} J_hat_ij s_i s_j +
    sum_i h_hat_i s_i with J_hat = 2 A (Eq. ising hamiltonian), by an explicit
    loop over the stored entries of the upper triangle."""
    cq, ch = coefficients(inst.j_scale, inst.convention)
    s = np.asarray(s, dtype=np.float64)
    one = s.ndim == 1
    if one:
        s = s[:, None]
    csr = inst if inst.layout == "csr" else inst.to_csr()
    e = np.zeros(s.shape[1])
    hh = field(inst)
    for i in range(inst.n):
        for k in range(int(csr.indptr[i]), int(csr.indptr[i + 1])):
            j = int(csr.indices[k])
            if j > i:
                e += 2.0 * cq * float(csr.data[k]) * s[i] * s[j]
        e += ch * hh[i] * s[i]
    return e[0] if one else e


def energy_exact(inst, s):
    """Exact energy of an integer instance: (E, Q, H) with Q = s^T J s and
    H = h^T s as Python ints and E = cQ Q + cH H (exact in float64 when cQ is
    dyadic and |Q|, |H| < 2^52)."""
    cq, ch = coefficients(inst.j_scale, inst.convention)
    s = np.asarray(s, dtype=np.int64)
    one = s.ndim == 1
    if one:
        s = s[:, None]
    if inst.layout == "dense":
        J = np.asarray(inst.J, dtype=np.int64)
        Q = np.einsum("ib,ib->b", s, J @ s)
    else:
        J = sp.csr_matrix((np.asarray(inst.data, dtype=np.int64), inst.indices,
                           inst.indptr), shape=(inst.n, inst.n))
        Q = np.einsum("ib,ib->b", s, J @ s)
    H = (np.zeros(s.shape[1], dtype=np.int64) if inst.h is None
         else np.asarray(inst.h, dtype=np.int64) @ s)
    E = cq * Q.astype(np.float64) + ch * H.astype(np.float64)
    if one:
        return float(E[0]), int(Q[0]), int(H[0])
    return E, Q, H


def flip_delta(inst, s, i: int) -> float:
    """Single-flip energy change from Sec. III-A:
    E(X_i s) - E(s) = -4 s_i sum_j A_ij s_j - 2 b_i s_i."""
    A, b = paper_form(inst)
    s = np.asarray(s, dtype=np.float64)
    return float(-4.0 * s[i] * (A[i] @ s) - 2.0 * b[i] * s[i])


def maxcut_value(edges: np.ndarray, weights: np.ndarray, s) -> float:
    """Total weight of edges whose endpoints lie on opposite sides."""
    s = np.asarray(s)
    cut = s[edges[:, 0]] != s[edges[:, 1]]
    return float(np.sum(np.asarray(weights, dtype=np.float64)[cut]))
