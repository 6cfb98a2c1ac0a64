"""Pins for the oracle's energy (Sec. II) and flip identity (Sec. III-A)."""

import numpy as np
import pytest

import synth
from oracle import brute_force, ising


def _rand_spins(n, B, seed):
    r = np.random.default_rng(seed)
    return (2 * r.integers(0, 2, (n, B)) - 1).astype(np.int64)


@pytest.mark.parametrize("convention,j_scale", [("physics", 0.5), ("physics", 1.0),
                                                ("paper", 0.5), ("paper", 2.0)])
@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_three_forms_agree_exactly_on_integer_instances(convention, j_scale, layout):
    inst = synth.random_sparse_instance(30, 3, p=0.3, kind="int", h="int",
                                        convention=convention, j_scale=j_scale,
                                        layout=layout)
    s = _rand_spins(30, 7, 1)
    e1 = ising.energy(inst, s)
    e2 = ising.energy_edges(inst, s)
    e3, Q, H = ising.energy_exact(inst, s)
    np.testing.assert_array_equal(e1, e2)
    np.testing.assert_array_equal(e1, e3)
    # exact integer parts: Q is even (zero diagonal, symmetric)
    assert np.all(Q % 2 == 0)


def test_float_forms_agree():
    inst = synth.random_sparse_instance(25, 4, p=0.4, kind="float", h="float")
    s = _rand_spins(25, 5, 2)
    np.testing.assert_allclose(ising.energy(inst, s), ising.energy_edges(inst, s),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("convention", ["physics", "paper"])
def test_single_flip_identity(convention):
    inst = synth.random_sparse_instance(20, 5, p=0.3, kind="int", h="int",
                                        convention=convention, j_scale=0.5)
    s = _rand_spins(20, 1, 3)[:, 0]
    e0 = ising.energy_exact(inst, s)[0]
    for i in range(20):
        t = s.copy()
        t[i] = -t[i]
        assert ising.energy_exact(inst, t)[0] - e0 == ising.flip_delta(inst, s, i)


def test_maxcut_identity():
    # J = -W/2 with h = 0: cut(s) = W_total / 2 - E(s)
    inst = synth.er_dense(60, 7, p=0.2, weights="pm1")
    W = -inst.J.astype(np.int64)
    iu, ju = np.nonzero(np.triu(W, 1))
    edges = np.stack([iu, ju], 1)
    w = W[iu, ju]
    s = _rand_spins(60, 9, 4)
    for b in range(9):
        cut = ising.maxcut_value(edges, w, s[:, b])
        assert cut == pytest.approx(w.sum() / 2.0 - ising.energy_exact(inst, s[:, b])[0],
                                    abs=0)


def test_conventions_match_hamiltonian():
    # Table-1 style instance in the paper's convention: E = sum_{i>j} J_hat s s + sum h s
    inst = synth.table1_instance("binary_int", 0, n=40, k=4)
    s = _rand_spins(40, 1, 5)[:, 0]
    Jh = inst.dense().astype(np.int64)
    direct = sum(Jh[i, j] * s[i] * s[j] for i in range(40) for j in range(i)) + inst.h @ s
    assert ising.energy_exact(inst, s)[0] == direct
    # the same couplings as a physics instance: J = -J_hat, h = -h_hat
    phys = synth.Instance(n=40, layout="dense", J=-Jh, h=-inst.h, j_scale=1.0,
                          convention="physics")
    assert ising.energy_exact(phys, s)[0] == direct


def test_brute_force_hand_cases():
    # ferromagnet on 5 spins: E = -sum_{i<j} s_i s_j, ground -10 at all-equal
    J = np.ones((5, 5), dtype=np.int32) - np.eye(5, dtype=np.int32)
    inst = synth.Instance(n=5, layout="dense", J=J, j_scale=1.0, convention="physics")
    e, s = brute_force.ground_state(inst)
    assert e == -10 and abs(int(s.sum())) == 5
    # antiferromagnetic triangle is frustrated: ground -1
    inst = synth.Instance(n=3, layout="dense", J=-(np.ones((3, 3), np.int32) - np.eye(3, dtype=np.int32)),
                          j_scale=1.0, convention="physics")
    assert brute_force.ground_state(inst)[0] == -1
    # single spin in a field h = 3: E = -3 s -> s = +1
    inst = synth.Instance(n=1, layout="dense", J=np.zeros((1, 1), np.int32),
                          h=np.array([3], np.int32), convention="physics")
    e, s = brute_force.ground_state(inst)
    assert e == -3 and s[0] == 1
