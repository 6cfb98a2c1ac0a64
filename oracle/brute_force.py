"""Exhaustive ground state for n <= 20 (the primal problem of Sec. II).

Every one of the 2^n spin vectors is evaluated with the plain quadratic form
E(s) = s^T A s + b^T s in chunks; the lowest energy and the first state that
reaches it (in enumeration order, state k has s_i = +1 iff bit i of k is 0)
are returned.
"""

from __future__ import annotations

import numpy as np

from . import ising


def ground_state(inst, chunk_bits: int = 14):
    n = inst.n
    if n > 22:
        raise ValueError("brute force is for n <= 22")
    A, b = ising.paper_form(inst)
    best_e = np.inf
    best_s = None
    total = 1 << n
    chunk = 1 << min(chunk_bits, n)
    bit = (np.uint64(1) << np.arange(n, dtype=np.uint64))[None, :]
    for start in range(0, total, chunk):
        k = np.arange(start, min(start + chunk, total), dtype=np.uint64)[:, None]
        s = np.where((k & bit) != 0, -1.0, 1.0)  # (chunk, n)
        E = np.einsum("ci,ci->c", s @ A, s) + s @ b
        j = int(np.argmin(E))
        if E[j] < best_e:
            best_e = float(E[j])
            best_s = s[j].astype(np.int8)
    return best_e, best_s
