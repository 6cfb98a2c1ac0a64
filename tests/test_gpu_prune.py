"""K1 pruning and K5 reconstruction through the C ABI: decisions, record,
reduced instance and reconstruction bit-exact against the oracle (Sec. III-A,
Algorithm 1)."""

import numpy as np
import pytest

import synth
from oracle import ising, pruning
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu


def _compare(ctx, inst, zero_rule=True, float_const=False):
    res = pruning.prune(inst, zero_rule=zero_rule)
    pr = api.prune(ctx, inst, zero_rule=zero_rule)
    rec = pr.record()
    np.testing.assert_array_equal(rec["kind"], res.kind)
    np.testing.assert_array_equal(rec["round"], res.rnd)
    np.testing.assert_array_equal(rec["value"], res.value)
    np.testing.assert_array_equal(rec["sign"], res.psign)
    np.testing.assert_array_equal(rec["parent"], res.parent.astype(np.int32))
    np.testing.assert_array_equal(rec["g_index"], res.gidx)
    assert pr.n_reduced == res.reduced.n
    assert pr.rounds == res.rounds
    assert pr.eta == res.eta
    if float_const:
        assert pr.constant == pytest.approx(res.constant, rel=1e-12, abs=1e-12)
    else:
        assert pr.constant == res.constant
    red = pr.reduced()
    np.testing.assert_array_equal(red.h, res.reduced.h)  # bitwise: FP64 folds in row order
    if inst.layout == "dense":
        np.testing.assert_array_equal(red.J, res.reduced.J)
    else:
        np.testing.assert_array_equal(red.indptr, res.reduced.indptr)
        np.testing.assert_array_equal(red.indices, res.reduced.indices)
        np.testing.assert_array_equal(red.data, res.reduced.data)
    r = np.random.default_rng(0)
    for _ in range(3):
        sg = (2 * r.integers(0, 2, res.reduced.n) - 1).astype(np.int8)
        np.testing.assert_array_equal(pr.reconstruct(sg), pruning.reconstruct(res, sg))
    pr.close()
    return res


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("h_mode", ["zero", "int2"])
def test_pendant_trees(gpu_ctx, seed, h_mode):
    inst = synth.er_pendant_csr(500, 2.5, 200, 3, seed, h_mode=h_mode)
    res = _compare(gpu_ctx, inst)
    assert res.eta > 0.1


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "binary", "binary_int"])
def test_table1_families_float_decisions(gpu_ctx, dist):
    for seed in range(2):
        _compare(gpu_ctx, synth.table1_instance(dist, seed), float_const=dist != "binary_int")


@pytest.mark.parametrize("kind,h", [("int", "int"), ("float", "float"), ("int", "zero")])
@pytest.mark.parametrize("conv,js", [("physics", 0.5), ("paper", 0.5), ("physics", 1.0)])
def test_random_small(gpu_ctx, kind, h, conv, js):
    for seed in range(3):
        inst = synth.random_sparse_instance(40, seed, p=0.06, kind=kind, h=h, convention=conv,
                                            j_scale=js)
        _compare(gpu_ctx, inst, float_const=kind == "float")
        _compare(gpu_ctx, inst, zero_rule=False, float_const=kind == "float")


def test_dense_input(gpu_ctx):
    inst = synth.random_sparse_instance(120, 9, p=0.03, kind="int", h="int", layout="dense")
    res = _compare(gpu_ctx, inst)
    assert 0 < res.reduced.n < 120


def test_single_spin_and_all_pruned(gpu_ctx):
    one = synth.Instance(n=1, layout="dense", J=np.zeros((1, 1), np.int32),
                         h=np.array([2], np.int32), convention="physics")
    res = _compare(gpu_ctx, one)
    assert res.reduced.n == 0
    tree = synth.er_pendant_csr(2, 0.0, 60, 3, 1)
    _compare(gpu_ctx, tree)


def test_full_size_pendant_instance(gpu_ctx):
    inst = synth.workload("er100k_pendant_h", 0)
    res = _compare(gpu_ctx, inst)
    assert res.eta > 0.15


def test_solve_energy_matches_reconstruction(gpu_ctx):
    inst = synth.er_pendant_csr(400, 2.5, 150, 3, 4, h_mode="int2")
    out = api.solve(gpu_ctx, inst, restarts=128, steps=60, lr=6.0, seed=2)
    e = ising.energy_exact(inst, out["best_spins"])[0]
    assert out["best_energy"] == e
    # pruned spins are those the record implies for the returned kept spins
    res = pruning.prune(inst)
    sg = out["best_spins"][res.G]
    np.testing.assert_array_equal(pruning.reconstruct(res, sg), out["best_spins"])
