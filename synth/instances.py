"""Seeded generators for the Ising instances used by tests and the benchmark.

An instance stores couplings J (dense row-major, or CSR with both (i,j) and
(j,i) present, columns increasing within a row), an optional field h, a scale
``j_scale`` applied to the stored couplings, and the energy convention the
numbers are meant in:

* ``"physics"``: E(s) = -1/2 * j_scale * s^T J s - h^T s  (max-cut is J = -W/2,
  stored here as the integer matrix -W with j_scale = 1/2);
* ``"paper"``:   E(s) = j_scale * s^T J s + h^T s, the form of Sec. II where the
  pairwise coupling of the Hamiltonian is split symmetrically (J = J_hat / 2,
  stored as J_hat with j_scale = 1/2).

The shapes and value distributions follow the workloads of Sec. IV
(6-regular Table-1 families, complete graphs, max-cut) and the synthetic
stand-ins for the benchmark suites of Table 3 (Erdos-Renyi max-cut,
Sherrington-Kirkpatrick glasses, a 2D torus and an ER graph with pendant trees).
Nothing here evaluates an energy or applies a solver rule.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Instance:
    n: int
    layout: str  # "dense" | "csr"
    J: Optional[np.ndarray] = None  # dense (n, n) stored couplings
    indptr: Optional[np.ndarray] = None  # int64 (n + 1,)
    indices: Optional[np.ndarray] = None  # int32 (nnz,)
    data: Optional[np.ndarray] = None  # (nnz,) stored couplings
    h: Optional[np.ndarray] = None  # (n,) field, None means zero
    j_scale: float = 1.0
    convention: str = "physics"
    name: str = ""

    @property
    def nnz(self) -> int:
        if self.layout == "csr":
            return int(self.indptr[-1])
        return int(np.count_nonzero(self.J))

    @property
    def integer(self) -> bool:
        jd = self.J if self.layout == "dense" else self.data
        ok = np.issubdtype(jd.dtype, np.integer)
        if self.h is not None:
            ok = ok and np.issubdtype(self.h.dtype, np.integer)
        return bool(ok)

    def dense(self) -> np.ndarray:
        """Stored couplings as a dense array (same dtype)."""
        if self.layout == "dense":
            return self.J
        out = np.zeros((self.n, self.n), dtype=self.data.dtype)
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        out[rows, self.indices] = self.data
        return out

    def to_csr(self) -> "Instance":
        """Same instance with CSR layout (zero couplings dropped)."""
        if self.layout == "csr":
            return self
        r, c = np.nonzero(self.J)
        order = np.lexsort((c, r))
        r, c = r[order], c[order]
        indptr = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(np.bincount(r, minlength=self.n), out=indptr[1:])
        return dataclasses.replace(
            self, layout="csr", J=None, indptr=indptr,
            indices=c.astype(np.int32), data=self.J[r, c].copy())

    def to_dense(self) -> "Instance":
        if self.layout == "dense":
            return self
        return dataclasses.replace(self, layout="dense", J=self.dense(),
                                   indptr=None, indices=None, data=None)


# --------------------------------------------------------------------------- graphs

def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def er_graph_edges(n: int, seed: int, p: Optional[float] = None,
                   mean_degree: Optional[float] = None) -> np.ndarray:
    """Erdos-Renyi G(n, p) edge list (i < j), shape (m, 2) int64."""
    if p is None:
        p = float(mean_degree) / (n - 1)
    rng = _rng(seed, 1)
    if n <= 4096:
        iu, ju = np.triu_indices(n, k=1)
        keep = rng.random(iu.shape[0]) < p
        return np.stack([iu[keep], ju[keep]], axis=1).astype(np.int64)
    total = n * (n - 1) // 2
    m = int(rng.binomial(total, p))
    got = np.empty(0, dtype=np.int64)
    while got.shape[0] < m:
        need = (m - got.shape[0]) * 11 // 10 + 16
        a = rng.integers(0, n, need)
        b = rng.integers(0, n, need)
        ok = a != b
        lo = np.minimum(a, b)[ok]
        hi = np.maximum(a, b)[ok]
        key = lo * n + hi
        got = np.unique(np.concatenate([got, key]))
    got = rng.permutation(got)[:m]
    got.sort()
    return np.stack([got // n, got % n], axis=1).astype(np.int64)


def regular_graph_edges(n: int, k: int, seed: int) -> np.ndarray:
    """Simple k-regular graph: configuration-model pairing repaired by random
    double-edge swaps until no loop or repeated edge is left."""
    assert (n * k) % 2 == 0 and k < n
    rng = _rng(seed, 2)
    stubs = np.repeat(np.arange(n, dtype=np.int64), k)
    rng.shuffle(stubs)
    pairs = stubs.reshape(-1, 2).copy()
    m = pairs.shape[0]

    def key(a, b):
        return (min(a, b), max(a, b))

    for _ in range(100000):
        seen = {}
        bad = []
        for e in range(m):
            a, b = int(pairs[e, 0]), int(pairs[e, 1])
            kk = key(a, b)
            if a == b or kk in seen:
                bad.append(e)
            else:
                seen[kk] = e
        if not bad:
            break
        for e in bad:
            f = int(rng.integers(0, m))
            if f == e:
                continue
            a, b = pairs[e]
            c, d = pairs[f]
            if rng.random() < 0.5:
                pairs[e] = (a, c)
                pairs[f] = (b, d)
            else:
                pairs[e] = (a, d)
                pairs[f] = (b, c)
    else:  # pragma: no cover
        raise RuntimeError("regular graph repair did not converge")
    lo = np.minimum(pairs[:, 0], pairs[:, 1])
    hi = np.maximum(pairs[:, 0], pairs[:, 1])
    order = np.lexsort((hi, lo))
    return np.stack([lo[order], hi[order]], axis=1)


def torus_edges(rows: int, cols: int) -> np.ndarray:
    """2D periodic square lattice, rows x cols sites, 2 * rows * cols edges."""
    idx = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    right = np.stack([idx.ravel(), np.roll(idx, -1, axis=1).ravel()], axis=1)
    down = np.stack([idx.ravel(), np.roll(idx, -1, axis=0).ravel()], axis=1)
    e = np.concatenate([right, down])
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    order = np.lexsort((hi, lo))
    return np.stack([lo[order], hi[order]], axis=1)


def pendant_tree_edges(n_base: int, n_extra: int, max_depth: int, seed: int,
                       mean_tree_size: float = 4.0) -> np.ndarray:
    """Trees of depth <= max_depth hanging off uniformly chosen base vertices.

    Spins n_base .. n_base + n_extra - 1 are added one at a time; each either
    starts a new tree (attached to a random base vertex, depth 1) or joins the
    current tree under a node of depth < max_depth."""
    rng = _rng(seed, 3)
    edges = np.empty((n_extra, 2), dtype=np.int64)
    depth = np.zeros(n_extra, dtype=np.int64)
    cur: list[int] = []
    p_new = 1.0 / mean_tree_size
    for t in range(n_extra):
        v = n_base + t
        open_nodes = [u for u in cur if depth[u - n_base] < max_depth]
        if not open_nodes or rng.random() < p_new:
            parent = int(rng.integers(0, n_base))
            depth[t] = 1
            cur = [v]
        else:
            parent = open_nodes[int(rng.integers(0, len(open_nodes)))]
            depth[t] = depth[parent - n_base] + 1
            cur.append(v)
        edges[t] = (parent, v)
    return edges


# --------------------------------------------------------------------------- layouts

def csr_from_edges(n: int, edges: np.ndarray, weights: np.ndarray):
    """Symmetric CSR (indptr int64, indices int32, data) from i<j edges."""
    rows = np.concatenate([edges[:, 0], edges[:, 1]])
    cols = np.concatenate([edges[:, 1], edges[:, 0]])
    vals = np.concatenate([weights, weights])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.shape[0] > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate edge")
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=indptr[1:])
    return indptr, cols.astype(np.int32), vals


def dense_from_edges(n: int, edges: np.ndarray, weights: np.ndarray) -> np.ndarray:
    J = np.zeros((n, n), dtype=weights.dtype)
    J[edges[:, 0], edges[:, 1]] = weights
    J[edges[:, 1], edges[:, 0]] = weights
    return J


def _pm1(rng, m, dtype=np.int8):
    return (2 * rng.integers(0, 2, m) - 1).astype(dtype)


# --------------------------------------------------------------------------- families

def sk_dense(n: int, seed: int, std: float = 1.0, dtype=np.float64,
             h_std: Optional[float] = None, name: str = "") -> Instance:
    """Sherrington-Kirkpatrick glass: J_ij ~ N(0, std^2) for i<j, mirrored,
    zero diagonal; h ~ N(0, h_std^2) or absent. Physics convention."""
    rng = _rng(seed, 4)
    g = rng.standard_normal((n, n)) * std
    J = np.triu(g, k=1)
    J = (J + J.T).astype(dtype)
    h = None
    if h_std is not None:
        h = (rng.standard_normal(n) * h_std).astype(dtype)
    return Instance(n=n, layout="dense", J=J, h=h, j_scale=1.0,
                    convention="physics", name=name or f"sk{n}")


def er_dense(n: int, seed: int, p: Optional[float] = None,
             mean_degree: Optional[float] = None, weights: str = "one",
             name: str = "") -> Instance:
    """Max-cut on an Erdos-Renyi graph written as an Ising instance: J = -W/2,
    stored as the int8 matrix -W with j_scale 1/2, h = 0, physics convention."""
    edges = er_graph_edges(n, seed, p=p, mean_degree=mean_degree)
    rng = _rng(seed, 5)
    if weights == "one":
        w = np.ones(edges.shape[0], dtype=np.int8)
    else:
        w = _pm1(rng, edges.shape[0])
    J = dense_from_edges(n, edges, (-w).astype(np.int8))
    return Instance(n=n, layout="dense", J=J, h=None, j_scale=0.5,
                    convention="physics", name=name or f"er{n}")


def torus_csr(rows: int, cols: int, seed: int, name: str = "") -> Instance:
    """2D torus with couplings uniform in {+1, -1}, int8 CSR, h = 0."""
    n = rows * cols
    edges = torus_edges(rows, cols)
    w = _pm1(_rng(seed, 6), edges.shape[0])
    indptr, indices, data = csr_from_edges(n, edges, w)
    return Instance(n=n, layout="csr", indptr=indptr, indices=indices,
                    data=data, h=None, j_scale=1.0, convention="physics",
                    name=name or f"torus{rows}x{cols}")


def er_pendant_csr(n_base: int, mean_degree: float, n_extra: int,
                   max_depth: int, seed: int, h_mode: str = "zero",
                   name: str = "") -> Instance:
    """ER graph (couplings +/-1) plus pendant trees of depth <= max_depth on
    n_extra extra spins, int8 CSR. h_mode 'zero' or 'int2' (h_i uniform in
    {-2..2}, int32)."""
    e1 = er_graph_edges(n_base, seed, mean_degree=mean_degree)
    e2 = pendant_tree_edges(n_base, n_extra, max_depth, seed)
    edges = np.concatenate([e1, e2])
    n = n_base + n_extra
    rng = _rng(seed, 7)
    w = _pm1(rng, edges.shape[0])
    indptr, indices, data = csr_from_edges(n, edges, w)
    h = None
    if h_mode == "int2":
        h = rng.integers(-2, 3, n).astype(np.int32)
    return Instance(n=n, layout="csr", indptr=indptr, indices=indices,
                    data=data, h=h, j_scale=1.0, convention="physics",
                    name=name or f"er{n_base}+trees{n_extra}")


def regular_instance(n: int, k: int, seed: int, j_values, h_values,
                     name: str = "") -> Instance:
    """k-regular graph with given per-edge couplings and fields, paper
    convention: E = sum_{i>j} J_hat_ij s_i s_j + sum_i h_i s_i."""
    edges = regular_graph_edges(n, k, seed)
    indptr, indices, data = csr_from_edges(n, edges, np.asarray(j_values))
    return Instance(n=n, layout="csr", indptr=indptr, indices=indices,
                    data=data, h=np.asarray(h_values), j_scale=0.5,
                    convention="paper", name=name)


def table1_instance(dist: str, seed: int, n: int = 1000, k: int = 6) -> Instance:
    """The three 6-regular families of Table 1 (same mean and variance):
    uniform  J_hat ~ U(-1, 1),        h_hat ~ U(-6, 6);
    gaussian J_hat ~ N(0, 1/3),       h_hat ~ N(0, 12);
    binary   J_hat in {+-1/sqrt 3},   h_hat in {+-2 sqrt 3};
    binary_int: the binary family times sqrt 3 (J_hat in {+-1}, h in {+-6}),
    which keeps every ratio and is exact in integers."""
    rng = _rng(seed, 8)
    m = n * k // 2
    if dist == "uniform":
        jv = rng.uniform(-1.0, 1.0, m)
        hv = rng.uniform(-6.0, 6.0, n)
    elif dist == "gaussian":
        jv = rng.standard_normal(m) * math.sqrt(1.0 / 3.0)
        hv = rng.standard_normal(n) * math.sqrt(12.0)
    elif dist == "binary":
        jv = _pm1(rng, m, np.float64) / math.sqrt(3.0)
        hv = _pm1(rng, n, np.float64) * 2.0 * math.sqrt(3.0)
    elif dist == "binary_int":
        jv = _pm1(rng, m, np.int32)
        hv = _pm1(rng, n, np.int32) * 6
    else:
        raise ValueError(dist)
    return regular_instance(n, k, seed, jv, hv, name=f"table1-{dist}")


def table2_instance(dist: str, seed: int, n: int = 1000) -> Instance:
    """The complete-graph family of the solver comparison (Sec. IV-C), paper
    convention E = sum_{i>j} J_hat_ij s_i s_j + sum_i h_i s_i:
    uniform  J_hat_ij, h_i ~ U(-1000, 1000);
    gaussian J_hat_ij, h_i ~ N(0, alpha^2) with alpha ~ U(0, 1000) drawn once
    per instance. Dense FP32."""
    rng = _rng(seed, 10)
    if dist == "uniform":
        g = rng.uniform(-1000.0, 1000.0, (n, n))
        hv = rng.uniform(-1000.0, 1000.0, n)
    elif dist == "gaussian":
        alpha = rng.uniform(0.0, 1000.0)
        g = rng.standard_normal((n, n)) * alpha
        hv = rng.standard_normal(n) * alpha
    else:
        raise ValueError(dist)
    J = np.triu(g, k=1)
    J = (J + J.T).astype(np.float32)
    return Instance(n=n, layout="dense", J=J, h=hv.astype(np.float32), j_scale=0.5,
                    convention="paper", name=f"table2-{dist}")


def random_sparse_instance(n: int, seed: int, p: float = 0.3, kind: str = "int",
                           h: str = "int", convention: str = "physics",
                           j_scale: float = 1.0, layout: str = "csr",
                           jmax: int = 3) -> Instance:
    """Small mixed instance for exhaustive checks: G(n, p) edges with integer
    couplings in [-jmax, jmax] \\ {0} (kind 'int') or N(0, 1) (kind 'float');
    fields integer in [-2 jmax, 2 jmax], Gaussian, or zero."""
    edges = er_graph_edges(n, seed, p=p)
    rng = _rng(seed, 9)
    m = edges.shape[0]
    if kind == "int":
        w = rng.integers(1, jmax + 1, m) * _pm1(rng, m, np.int64)
        w = w.astype(np.int32)
    else:
        w = rng.standard_normal(m)
    if h == "int":
        hv = rng.integers(-2 * jmax, 2 * jmax + 1, n).astype(np.int32)
    elif h == "float":
        hv = rng.standard_normal(n) * 2.0
    else:
        hv = None
    indptr, indices, data = csr_from_edges(n, edges, w)
    inst = Instance(n=n, layout="csr", indptr=indptr, indices=indices,
                    data=data, h=hv, j_scale=j_scale, convention=convention,
                    name=f"rand{n}")
    return inst.to_dense() if layout == "dense" else inst


def workload(name: str, seed: int = 0) -> Instance:
    """Named benchmark-shaped instances (see the workload table in the design notes)."""
    if name == "sk100":
        return sk_dense(100, seed, 1.0, np.float64, name="sk100")
    if name == "er800":
        return er_dense(800, seed, p=0.06, weights="one", name="er800")
    if name == "er2000":
        return er_dense(2000, seed, mean_degree=10.0, weights="pm1", name="er2000")
    if name == "table2_uniform":
        return table2_instance("uniform", seed)
    if name == "table2_gaussian":
        return table2_instance("gaussian", seed)
    if name == "sk4096":
        return sk_dense(4096, seed, math.sqrt(1.0 / 4096), np.float32,
                        h_std=math.sqrt(0.1), name="sk4096")
    if name == "torus20k":
        return torus_csr(100, 200, seed, name="torus20k")
    if name == "er100k_pendant":
        return er_pendant_csr(100000, 4.0, 20000, 3, seed, name="er100k_pendant")
    if name == "er100k_pendant_h":
        return er_pendant_csr(100000, 4.0, 20000, 3, seed, h_mode="int2",
                              name="er100k_pendant_h")
    raise KeyError(name)


def serving_stream(count: int, seed: int, rate: float = 200.0, n_min: int = 64,
                   n_max: int = 8192, dense_fraction: float = 0.5, sparse_degree: float = 8.0):
    """Request stream shaped like the serving workload: Poisson arrivals at
    `rate` per second, N log-uniform in [n_min, n_max], a `dense_fraction` of
    dense Gaussian SK instances (J ~ N(0, 1/N), h ~ N(0, 0.1)) and the rest
    sparse ER graphs of the given mean degree with couplings +-1. Returns a
    list of (arrival time in seconds, Instance)."""
    rng = _rng(seed, 10)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        if rng.random() < dense_fraction:
            inst = sk_dense(n, seed * 100003 + k, math.sqrt(1.0 / n), np.float32,
                            h_std=math.sqrt(0.1), name=f"req{k}-sk{n}")
        else:
            e = er_graph_edges(n, seed * 100003 + k, mean_degree=min(sparse_degree, n - 1))
            w = _pm1(_rng(seed * 100003 + k, 11), e.shape[0])
            indptr, indices, data = csr_from_edges(n, e, w)
            inst = Instance(n=n, layout="csr", indptr=indptr, indices=indices, data=data,
                            j_scale=1.0, convention="physics", name=f"req{k}-er{n}")
        out.append((t, inst))
    return out


def serving_stream_pooled(count: int, seed: int, rate: float = 200.0, n_min: int = 64,
                          n_max: int = 8192, dense_fraction: float = 0.5,
                          sparse_degree: float = 8.0, pool: int = 24):
    """The serving stream of serving_stream at a scale whose instances do not
    all fit host memory: `pool` dense SK and `pool` sparse ER instances at
    log-spaced sizes in [n_min, n_max] are generated once, and each request
    (Poisson arrivals at `rate`, N drawn log-uniformly, dense with
    probability `dense_fraction`) takes the pooled instance of the nearest
    size on the log scale. Returns a list of (arrival time in seconds,
    Instance); requests share Instance objects."""
    sizes = np.unique(np.round(np.exp(np.linspace(math.log(n_min), math.log(n_max), pool))).astype(int))
    dense = [sk_dense(int(n), seed * 100003 + 7 * k, math.sqrt(1.0 / n), np.float32,
                      h_std=math.sqrt(0.1), name=f"pool-sk{n}") for k, n in enumerate(sizes)]
    sparse = []
    for k, n in enumerate(sizes):
        e = er_graph_edges(int(n), seed * 100003 + 7 * k + 1, mean_degree=min(sparse_degree, n - 1))
        w = _pm1(_rng(seed * 100003 + 7 * k + 1, 11), e.shape[0])
        indptr, indices, data = csr_from_edges(int(n), e, w)
        sparse.append(Instance(n=int(n), layout="csr", indptr=indptr, indices=indices, data=data,
                               j_scale=1.0, convention="physics", name=f"pool-er{n}"))
    logs = np.log(sizes)
    rng = _rng(seed, 12)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        x = rng.uniform(math.log(n_min), math.log(n_max))
        k = int(np.argmin(np.abs(logs - x)))
        out.append((t, dense[k] if rng.random() < dense_fraction else sparse[k]))
    return out
