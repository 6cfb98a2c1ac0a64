"""Pins for the oracle's pruning (Sec. III-A, Algorithm 1) and reconstruction."""

import json
import os

import numpy as np
import pytest

import synth
from oracle import brute_force, ising, metrics, pruning

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_pruning.json")


def _with_pendants(n_core, n_extra, seed, kind="int", h="int", conv="physics", j_scale=0.5):
    """Small core graph plus pendant chains so that both rules fire."""
    core = synth.random_sparse_instance(n_core, seed, p=0.35, kind=kind, h=h,
                                        convention=conv, j_scale=j_scale)
    r = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n_core), np.diff(core.indptr))
    e = [(int(a), int(b)) for a, b in zip(rows, core.indices) if a < b]
    w = [core.data[k] for k in range(len(rows)) if rows[k] < core.indices[k]]
    for t in range(n_extra):
        v = n_core + t
        u = int(r.integers(0, v))
        e.append((u, v))
        w.append(type(w[0])(r.integers(1, 4) * (2 * r.integers(0, 2) - 1)) if kind == "int"
                 else r.standard_normal())
    n = n_core + n_extra
    indptr, indices, data = synth.csr_from_edges(n, np.array(e), np.array(w, dtype=core.data.dtype))
    if h == "int":
        hv = r.integers(-4, 5, n).astype(np.int32)
    elif h == "float":
        hv = r.standard_normal(n) * 2
    else:
        hv = None
    return synth.Instance(n=n, layout="csr", indptr=indptr, indices=indices, data=data,
                          h=hv, j_scale=j_scale, convention=conv)


CASES = [(kind, h, conv, js) for kind, h in [("int", "int"), ("int", "zero"), ("float", "float")]
         for conv, js in [("physics", 0.5), ("paper", 0.5), ("physics", 1.0)]]


@pytest.mark.parametrize("kind,h,conv,js", CASES)
def test_pruning_is_exact_against_brute_force(kind, h, conv, js):
    fired = 0
    for seed in range(6):
        inst = _with_pendants(9, 6, seed, kind, h, conv, js)
        res = pruning.prune(inst)
        e0, _ = brute_force.ground_state(inst)
        if res.reduced.n:
            eg, sg = brute_force.ground_state(res.reduced)
        else:
            eg, sg = 0.0, np.zeros(0, np.int8)
        assert eg + res.constant == pytest.approx(e0, abs=1e-9 if kind == "float" else 0)
        full = pruning.reconstruct(res, sg)
        assert ising.energy(inst, full) == pytest.approx(e0, abs=1e-9 if kind == "float" else 0)
        fired += res.n - res.reduced.n
    assert fired > 0


@pytest.mark.parametrize("seed", range(4))
def test_reconstruct_invariant_on_random_reduced_states(seed):
    inst = synth.er_pendant_csr(300, 2.5, 120, 3, seed, h_mode="int2")
    res = pruning.prune(inst)
    assert 0 < res.reduced.n < inst.n
    r = np.random.default_rng(seed)
    for _ in range(5):
        sg = (2 * r.integers(0, 2, res.reduced.n) - 1).astype(np.int8)
        full = pruning.reconstruct(res, sg)
        # the reduced field holds halves (j_scale 1/2): float64 is exact here
        eg = float(ising.energy(res.reduced, sg))
        assert ising.energy_exact(inst, full)[0] == eg + res.constant


def test_zero_field_reduces_to_two_core():
    nx = pytest.importorskip("networkx")
    for seed in range(3):
        inst = synth.er_pendant_csr(400, 2.2, 150, 3, seed)
        res = pruning.prune(inst)
        g = nx.Graph()
        g.add_nodes_from(range(inst.n))
        rows = np.repeat(np.arange(inst.n), np.diff(inst.indptr))
        g.add_edges_from((int(a), int(b)) for a, b in zip(rows, inst.indices) if a < b)
        core = sorted(nx.k_core(g, 2).nodes())
        np.testing.assert_array_equal(res.G, np.array(core, dtype=np.int64))
        assert res.constant == -0.5 * np.sum(np.abs(inst.data[np.isin(rows, res.G, invert=True)
                                                            | np.isin(inst.indices, res.G, invert=True)]))


def test_tree_prunes_completely_to_its_ground_state():
    # a tree with h = 0 has ground energy -sum |J_eff| (every bond satisfied)
    n = 200
    edges = synth.pendant_tree_edges(1, n - 1, 50, 3, mean_tree_size=1e9)
    w = (2 * np.random.default_rng(1).integers(0, 2, n - 1) - 1).astype(np.int8) * 3
    indptr, indices, data = synth.csr_from_edges(n, edges, w)
    inst = synth.Instance(n=n, layout="csr", indptr=indptr, indices=indices, data=data,
                          j_scale=0.5, convention="physics")
    res = pruning.prune(inst)
    assert res.reduced.n == 0 and res.eta == 1.0
    full = pruning.reconstruct(res, np.zeros(0, np.int8))
    e = ising.energy_exact(inst, full)[0]
    assert e == res.constant == -0.5 * 3 * (n - 1)


def test_binary_family_prunes_nothing():
    g = json.load(open(GOLDEN))
    for dist in ["binary", "binary_int"]:
        for seed in range(3):
            res = pruning.prune(synth.table1_instance(dist, seed))
            assert res.eta == g["binary_eta"]


def test_first_round_rate_closed_form_and_monte_carlo():
    g = json.load(open(GOLDEN))["uniform_first_round"]
    est = metrics.eta1_estimate(g["k"], g["alpha"], g["beta"])
    assert est == pytest.approx(g["eta1"], abs=1e-6)
    rates = [pruning.first_round_rate(synth.table1_instance("uniform", s)) for s in range(12)]
    assert np.mean(rates) == pytest.approx(est, abs=0.01)
    # Gaussian family: same rule against a direct draw of the two distributions
    rates = [pruning.first_round_rate(synth.table1_instance("gaussian", s)) for s in range(12)]
    r = np.random.default_rng(0)
    a = np.abs(r.standard_normal((400000, 6)) * np.sqrt(1 / 3)).sum(1)
    b = np.abs(r.standard_normal(400000) * np.sqrt(12))
    assert np.mean(rates) == pytest.approx(np.mean(b > a), abs=0.01)


def test_determined_rule_is_strict_and_semi_rule_is_not():
    # paper form with A = J: spin 0 has |h_0| = 2 sum_j |A_0j| = 4 exactly, so the
    # strict determined rule does not fire in round 1, while the semi rule
    # (2 |A_01| >= |h_0|) does fire on the pair
    J = np.array([[0, 2], [2, 0]], dtype=np.int32)
    inst = synth.Instance(n=2, layout="dense", J=J, h=np.array([4, 0], np.int32),
                          j_scale=1.0, convention="paper")
    res = pruning.prune(inst, zero_rule=False)
    assert not (res.kind[0] == pruning.KIND_D and res.rnd[0] == 1)
    assert res.kind[1] == pruning.KIND_S and res.rnd[1] == 1 and res.parent[1] == 0
    assert res.kind[0] == pruning.KIND_D and res.rnd[0] == 2
    assert res.reduced.n == 0
    e0, _ = brute_force.ground_state(inst)
    full = pruning.reconstruct(res, np.zeros(0, np.int8))
    assert ising.energy(inst, full) == e0 == res.constant == -8


def test_row_sums_are_sequential_in_row_order():
    # the oracle's per-row sums (np.bincount) add entries one by one in row
    # order starting from 0.0, the order the folds of a round are defined in
    w = np.array([1e16, 1.0, -1e16, 3.0])
    assert np.bincount(np.zeros(4, np.int64), weights=w)[0] == ((1e16 + 1.0) - 1e16) + 3.0
    r = np.random.default_rng(0)
    w = r.standard_normal(5000) * 10.0 ** r.integers(-8, 8, 5000)
    acc = 0.0
    for x in w:
        acc += x
    assert np.bincount(np.zeros(5000, np.int64), weights=w)[0] == acc
