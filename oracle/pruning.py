"""Pruning (Sec. III-A, Algorithm 1) and reconstruction, in float64.

Written in the paper's form E(s) = s^T A s + b^T s (A = cQ J_stored,
b = cH h, see ``ising``). One round r of Algorithm 1, all spins at once from
the state at the start of the round:

1. Determined spins (Eq. determined spin): alive i with
   2 |cQ| S_i < |b'_i|, S_i = sum of |J_ij| over alive neighbours in row
   order; fixed to s_i = -sgn(b'_i). The constant gains b'_i s_i for each and
   A_ij s_i s_j for every ordered pair inside the set; every alive spin j
   outside it gains b'_j += sum_{i in D} (2 cQ J_ji) s_i, summed in row order
   from zero and then added once.
2. (Extension, on by default) alive spins left with no alive neighbour and
   b' = 0 are fixed to +1; no rule of the paper reaches them and either value
   is optimal.
3. Semi-determined spins (Eq. semi determined spin), on the graph left after
   step 1: alive k with exactly one alive neighbour p and
   2 |cQ| |J_kp| >= |b'_k| (b' already folded in step 1). Then
   s_k = -sgn(cQ J_kp) s_p, the constant gains -2 |cQ| |J_kp| and p gains
   b'_p += -sgn(cQ J_kp) b'_k (summed over p's children in row order). When k
   and p are each other's only neighbour and both qualify, only the larger
   index is taken.
4. Stop when a round fixes nothing.

The constant is accumulated term by term as above rather than from the
closed-form expression printed after the simplified problem, whose last lines
omit several of these terms. The reduced problem keeps the alive spins in
increasing original index, the stored couplings among them, and the folded
field (returned in the input's convention).

Reconstruction walks the rounds backwards: fixed spins take their value,
semi-determined spins take sign * (their parent's spin).
"""

from __future__ import annotations

import dataclasses
from types import SimpleNamespace

import numpy as np

from . import ising

KIND_G, KIND_D, KIND_Z, KIND_S = 0, 1, 2, 3


@dataclasses.dataclass
class PruneResult:
    n: int
    G: np.ndarray  # original indices of the kept spins, increasing
    gidx: np.ndarray  # original -> reduced index, -1 if pruned
    reduced: SimpleNamespace  # instance-like: n, layout, J / CSR, h, j_scale, convention
    constant: float
    eta: float
    rounds: int  # rounds that fixed at least one spin
    kind: np.ndarray  # int8 per spin: 0 kept, 1 determined, 2 isolated-zero, 3 semi
    rnd: np.ndarray  # int32 round in which the spin was fixed (0 if kept)
    value: np.ndarray  # int8 value of determined / isolated spins
    parent: np.ndarray  # int64 parent of semi-determined spins (-1 otherwise)
    psign: np.ndarray  # int8 s_k = psign_k * s_parent


def _csr_arrays(inst):
    csr = inst if inst.layout == "csr" else inst.to_csr()
    indptr = np.asarray(csr.indptr, dtype=np.int64)
    cols = np.asarray(csr.indices, dtype=np.int64)
    rows = np.repeat(np.arange(inst.n, dtype=np.int64), np.diff(indptr))
    return rows, cols, np.asarray(csr.data), indptr


def prune(inst, zero_rule: bool = True) -> PruneResult:
    n = inst.n
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    rows, cols, data, indptr = _csr_arrays(inst)
    Jv = data.astype(np.float64)
    absJ = np.abs(Jv)
    nz = Jv != 0.0
    twocq = 2.0 * cq
    twocq_abs = abs(twocq)
    b = ch * ising.field(inst)
    alive = np.ones(n, dtype=bool)
    kind = np.zeros(n, dtype=np.int8)
    rnd = np.zeros(n, dtype=np.int32)
    value = np.zeros(n, dtype=np.int8)
    parent = np.full(n, -1, dtype=np.int64)
    psign = np.zeros(n, dtype=np.int8)
    C = 0.0
    r = 0
    rounds = 0
    while True:
        r += 1
        changed = False
        # 1. determined spins
        live = nz & alive[rows] & alive[cols]
        S = np.bincount(rows[live], weights=absJ[live], minlength=n)
        D = alive & (twocq_abs * S < np.abs(b))
        if D.any():
            changed = True
            sD = np.where(b < 0.0, 1.0, -1.0)  # -sgn(b'), b' != 0 on D
            C += float(np.sum(b[D] * sD[D]))
            dd = live & D[rows] & D[cols]
            C += float(np.sum(cq * Jv[dd] * sD[rows[dd]] * sD[cols[dd]]))
            fe = live & ~D[rows] & D[cols]
            acc = np.bincount(rows[fe], weights=(twocq * Jv[fe]) * sD[cols[fe]],
                              minlength=n)
            recv = np.bincount(rows[fe], minlength=n) > 0
            b[recv] = b[recv] + acc[recv]
            kind[D] = KIND_D
            rnd[D] = r
            value[D] = sD[D].astype(np.int8)
            alive &= ~D
        # 2. isolated spins with zero field
        live = nz & alive[rows] & alive[cols]
        deg = np.bincount(rows[live], minlength=n)
        if zero_rule:
            Z = alive & (deg == 0) & (b == 0.0)
            if Z.any():
                changed = True
                kind[Z] = KIND_Z
                rnd[Z] = r
                value[Z] = 1
                alive &= ~Z
        # 3. semi-determined spins
        deg1 = alive & (deg == 1)
        e1 = live & deg1[rows]
        par = np.full(n, -1, dtype=np.int64)
        jkp = np.zeros(n)
        par[rows[e1]] = cols[e1]
        jkp[rows[e1]] = Jv[e1]
        cand = deg1 & (twocq_abs * np.abs(jkp) >= np.abs(b))
        ks = np.nonzero(cand)[0]
        ps = par[ks]
        mutual = cand[ps] & (par[ps] == ks)
        Sm = cand.copy()
        Sm[ks[mutual & (ks < ps)]] = False
        if Sm.any():
            changed = True
            ks = np.nonzero(Sm)[0]
            sg = -np.sign(cq * jkp[ks])
            C += float(np.sum(-twocq_abs * np.abs(jkp[ks])))
            sgn_all = np.zeros(n)
            sgn_all[ks] = sg
            fe = live & Sm[cols]
            acc = np.bincount(rows[fe], weights=sgn_all[cols[fe]] * b[cols[fe]],
                              minlength=n)
            recv = np.bincount(rows[fe], minlength=n) > 0
            b[recv] = b[recv] + acc[recv]
            kind[ks] = KIND_S
            rnd[ks] = r
            parent[ks] = par[ks]
            psign[ks] = sg.astype(np.int8)
            alive &= ~Sm
        if not changed:
            break
        rounds = r
    G = np.nonzero(alive)[0]
    gidx = np.full(n, -1, dtype=np.int64)
    gidx[G] = np.arange(G.shape[0])
    keep = nz & alive[rows] & alive[cols]
    nG = G.shape[0]
    h_red = ch * b[G]
    if inst.layout == "dense":
        Jd = np.asarray(inst.J)
        red = SimpleNamespace(n=nG, layout="dense", J=Jd[np.ix_(G, G)].copy(),
                              indptr=None, indices=None, data=None, h=h_red,
                              j_scale=inst.j_scale, convention=inst.convention)
    else:
        rr = gidx[rows[keep]]
        ip = np.zeros(nG + 1, dtype=np.int64)
        np.cumsum(np.bincount(rr, minlength=nG), out=ip[1:])
        red = SimpleNamespace(n=nG, layout="csr", J=None, indptr=ip,
                              indices=gidx[cols[keep]].astype(np.int32),
                              data=data[keep].copy(), h=h_red,
                              j_scale=inst.j_scale, convention=inst.convention)
    eta = 1.0 - nG / n if n else 0.0
    return PruneResult(n=n, G=G, gidx=gidx, reduced=red, constant=C, eta=eta,
                       rounds=rounds, kind=kind, rnd=rnd, value=value,
                       parent=parent, psign=psign)


def reconstruct(res: PruneResult, s_reduced) -> np.ndarray:
    """Full spin vector from the reduced problem's spins."""
    s = np.zeros(res.n, dtype=np.int8)
    s[res.G] = np.asarray(s_reduced, dtype=np.int8)
    fixed = (res.kind == KIND_D) | (res.kind == KIND_Z)
    s[fixed] = res.value[fixed]
    for r in range(res.rounds, 0, -1):
        k = np.nonzero((res.kind == KIND_S) & (res.rnd == r))[0]
        s[k] = res.psign[k] * s[res.parent[k]]
    return s


def first_round_rate(inst) -> float:
    """Fraction of spins fixed as determined in round 1 (the eta_1 of Sec. IV-A)."""
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    rows, cols, data, _ = _csr_arrays(inst)
    S = np.bincount(rows, weights=np.abs(data.astype(np.float64)), minlength=inst.n)
    b = ch * ising.field(inst)
    return float(np.mean(2.0 * abs(cq) * S < np.abs(b)))
