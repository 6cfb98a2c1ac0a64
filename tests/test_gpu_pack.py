"""Batching: sessions of different sizes and restart counts advanced together
by packed launches (one step launch over all members' tiles, one tracking
launch over all their restarts) compute exactly what each computes alone:
state, spins, per-restart bests and the result are bit-identical to the same
session run by itself, and the result's energy is the oracle's energy of its
spins (Sec. III-B; restarts batched across instances as in Sec. IV-C)."""

import math

import numpy as np
import pytest

import synth
from oracle import ising
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu


def _fp16_members():
    # float couplings: two FP16 planes; ragged n and B, one to several tiles
    return [(synth.sk_dense(300, 31, 1 / math.sqrt(300), np.float32, h_std=0.3), 200),
            (synth.sk_dense(129, 32, 1 / math.sqrt(129), np.float32), 96),
            (synth.sk_dense(700, 33, 1 / math.sqrt(700), np.float64, h_std=math.sqrt(0.1)), 256),
            (synth.sk_dense(64, 34, 0.2, np.float32, h_std=0.1), 130)]


def _e4m3_members():
    # integer couplings: exact E4M3, integer energies
    return [(synth.er_dense(500, 41, p=0.02, weights="pm1"), 256),
            (synth.er_dense(150, 42, p=0.08, weights="pm1"), 100),
            (synth.random_sparse_instance(260, 43, p=0.1, kind="int", h="int", layout="dense",
                                          jmax=7), 160)]


def _state(s):
    st = s.export_state()
    E, t, sp = s.restart_best()
    return st, E, t, sp


@pytest.mark.parametrize("members", [_fp16_members, _e4m3_members])
@pytest.mark.parametrize("steps", [7, 60])
def test_packed_members_match_each_alone(gpu_ctx, members, steps):
    mem = members()
    prec = "auto"
    # one restart-tile width for every member, chosen by the pack (the
    # members alone keep their own)
    packed = [api.Session(gpu_ctx, inst, restarts=B, steps=steps, seed=5 + k, precision=prec,
                          streaming=True) for k, (inst, B) in enumerate(mem)]
    pk = api.Pack(gpu_ctx, packed)
    pk.run(steps)
    pk.close()
    for k, ((inst, B), s) in enumerate(zip(mem, packed)):
        alone = api.Session(gpu_ctx, inst, restarts=B, steps=steps, seed=5 + k, precision=prec)
        alone.run(steps)
        a_st, a_E, a_t, a_sp = _state(alone)
        p_st, p_E, p_t, p_sp = _state(s)
        assert p_st["t"] == a_st["t"] == steps
        for key in ["theta", "m", "v", "spins"]:
            np.testing.assert_array_equal(p_st[key], a_st[key], err_msg=f"member {k} {key}")
        np.testing.assert_array_equal(p_E, a_E)
        np.testing.assert_array_equal(p_t, a_t)
        np.testing.assert_array_equal(p_sp, a_sp)
        s.finish()
        alone.finish()
        rp, ra = s.result(), alone.result()
        assert rp["best_energy"] == ra["best_energy"]
        np.testing.assert_array_equal(rp["best_spins"], ra["best_spins"])
        e = ising.energy(inst, rp["best_spins"].astype(np.float64))
        assert rp["best_energy"] == pytest.approx(float(e), rel=1e-12, abs=1e-9)
        s.close()
        alone.close()


def test_members_at_different_steps_and_graph_replay(gpu_ctx):
    """Members joined at different points of their runs (their own step
    counters differ) advance correctly through the graph-replayed packed
    step loop (a pack captures its graph on its second call; two graphs of
    steps here), and a member's later own steps continue from where the pack
    left it, with the same per-restart bests (energy, step, spins)."""
    mem = _fp16_members()[:3]
    ses = [api.Session(gpu_ctx, inst, restarts=B, steps=140, seed=9, streaming=True)
           for inst, B in mem]
    ses[1].run(13)
    ses[2].run(2)
    pk = api.Pack(gpu_ctx, ses)
    pk.run(10)
    pk.run(70)
    pk.close()
    ses[0].run(5)
    for k, ((inst, B), s) in enumerate(zip(mem, ses)):
        done = 80 + {0: 5, 1: 13, 2: 2}[k]
        alone = api.Session(gpu_ctx, inst, restarts=B, steps=140, seed=9)
        alone.run(done)
        a, p = alone.export_state(), s.export_state()
        assert a["t"] == p["t"] == done
        for key in ["theta", "m", "v", "spins"]:
            np.testing.assert_array_equal(p[key], a[key], err_msg=f"member {k} {key}")
        # best energies, their steps and spins: the tracking done inside the
        # packed and the single launches, and their closing tracking launches
        for x, y in zip(s.restart_best(), alone.restart_best()):
            np.testing.assert_array_equal(x, y, err_msg=f"member {k} bests")
        alone.close()
        s.close()


def test_pack_rejects_mixed_and_unsupported_members(gpu_ctx):
    f = api.Session(gpu_ctx, _fp16_members()[0][0], restarts=200, steps=5, streaming=True)
    i = api.Session(gpu_ctx, _e4m3_members()[0][0], restarts=256, steps=5, streaming=True)
    with pytest.raises(api.IsingError):
        api.Pack(gpu_ctx, [f, i])  # E4M3 and 16-bit operands in one launch
    # integer couplings: |J| <= 100 in one BF16 plane, up to 3000 in two FP16
    # planes (a launch's stages hold one plane count)
    one = api.Session(gpu_ctx, synth.random_sparse_instance(200, 44, p=0.1, kind="int", h="int",
                                                            layout="dense", jmax=100),
                      restarts=128, steps=5, streaming=True)
    two = api.Session(gpu_ctx, synth.random_sparse_instance(200, 45, p=0.1, kind="int", h="int",
                                                            layout="dense", jmax=3000),
                      restarts=128, steps=5, streaming=True)
    one.run(1)
    two.run(1)
    assert (one.result()["operand_planes"], two.result()["operand_planes"]) == (1, 2)
    with pytest.raises(api.IsingError):
        api.Pack(gpu_ctx, [one, two])
    one.close()
    two.close()
    r = api.Session(gpu_ctx, _e4m3_members()[1][0], restarts=100, steps=5)  # resident form
    with pytest.raises(api.IsingError):
        api.Pack(gpu_ctx, [r])
    sp = api.Session(gpu_ctx, synth.torus_csr(10, 13, 5), restarts=64, steps=5)
    with pytest.raises(api.IsingError):
        api.Pack(gpu_ctx, [sp])
    pk = api.Pack(gpu_ctx, [f])
    with pytest.raises(api.IsingError):
        pk.run(6)  # more steps than the member has left
    pk.close()
    for s in (f, i, r, sp):
        s.close()
