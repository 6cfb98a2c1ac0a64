"""The request server (continuous batching of independent solves): each
result equals the same request solved alone, admission follows the memory
budget, and oversized requests are refused."""

import math
import time

import numpy as np
import pytest

import synth
from oracle import ising
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu


def _mix():
    return [
        (synth.er_dense(300, 1, p=0.05, weights="pm1"), dict(restarts=256, steps=300)),
        (synth.sk_dense(200, 2, 1 / math.sqrt(200), np.float32, h_std=0.3),
         dict(restarts=200, steps=260, precision="tc")),
        (synth.torus_csr(20, 30, 3), dict(restarts=256, steps=333)),
        (synth.er_pendant_csr(400, 3.0, 100, 3, 4, h_mode="int2"), dict(restarts=128, steps=280)),
        (synth.er_dense(520, 5, mean_degree=8, weights="pm1"), dict(restarts=300, steps=250)),
        (synth.random_sparse_instance(90, 6, p=0.1, kind="int", h="int", layout="dense"),
         dict(restarts=64, steps=500, precision="fp32")),
        (synth.er_dense(180, 7, p=0.05, weights="pm1"), dict(restarts=100, steps=300)),
    ]


@pytest.mark.parametrize("pack", [False, True])
def test_results_in_the_mix_equal_results_alone(gpu_ctx, pack):
    """With packing, the dense tensor-core requests of one kind that are
    ready together advance in packed launches (the three E4M3 max-cut ones
    here share a pack, different sizes and restart counts)."""
    mix = _mix()
    alone = [api.solve(gpu_ctx, inst, seed=11 + k, **kw) for k, (inst, kw) in enumerate(mix)]
    srv = api.Server(gpu_ctx, budget_bytes=8 << 30, max_active=4 if not pack else 6,
                     chunk_steps=64, pack=pack)
    ids = [srv.submit(inst, seed=11 + k, **kw) for k, (inst, kw) in enumerate(mix)]
    for k, rid in enumerate(ids):
        res = srv.wait(rid, timeout=300)
        assert res["status"] == 0 and res["done"] == 1
        np.testing.assert_array_equal(res["best_spins"], alone[k]["best_spins"])
        assert res["best_energy"] == alone[k]["best_energy"]
        e = ising.energy(mix[k][0], res["best_spins"].astype(np.float64))
        assert res["best_energy"] == pytest.approx(float(e), rel=1e-12, abs=1e-9)
        assert res["t_submit_ms"] <= res["t_admit_ms"] <= res["t_done_ms"]
    srv.close()


def test_admission_follows_the_budget(gpu_ctx):
    mix = _mix()[:4]
    srv = api.Server(gpu_ctx, budget_bytes=8 << 30, max_active=4, chunk_steps=100)
    fps = []
    for inst, kw in mix:
        rid = srv.submit(inst, **kw)
        fps.append(srv.wait(rid)["footprint"])
    srv.close()
    # a budget that holds any one request but no two: requests run one at a time
    budget = max(fps) + min(fps) // 2
    srv = api.Server(gpu_ctx, budget_bytes=budget, max_active=4, chunk_steps=100)
    ids = [srv.submit(inst, **kw) for inst, kw in mix]
    res = [srv.wait(r, timeout=300) for r in ids]
    for a, b in zip(res, res[1:]):
        assert b["t_admit_ms"] >= a["t_done_ms"] - 1e-6
    assert all(r["status"] == 0 for r in res)
    srv.close()


def test_oversized_request_is_refused_and_unknown_ids_are_errors(gpu_ctx):
    srv = api.Server(gpu_ctx, budget_bytes=1 << 20, max_active=2, chunk_steps=10)
    with pytest.raises(api.IsingError) as e:
        srv.submit(synth.er_dense(300, 1, p=0.05), restarts=256, steps=10)
    assert e.value.code == 5
    with pytest.raises(api.IsingError):
        srv.poll(12345)
    srv.close()


@pytest.mark.parametrize("pack", [False, True])
def test_time_to_target_queries(gpu_ctx, pack):
    """ising_server_submit_target: a target every spin vector meets stops the
    request after its first chunk; an unreachable one runs every step and
    gives the plain request's result; a target between the two stops it at
    the first chunk whose best meets it, with fewer steps and an energy at or
    below the target (exact on the full instance)."""
    inst = synth.sk_dense(300, 9, 1 / math.sqrt(300), np.float32, h_std=0.3)
    kw = dict(restarts=256, steps=400, seed=5, precision="fp8")
    chunk = 50
    plain = api.solve(gpu_ctx, inst, **kw)
    srv = api.Server(gpu_ctx, budget_bytes=8 << 30, max_active=4, chunk_steps=chunk, pack=pack)
    # the plain run's energy after its first chunk of steps bounds a target it meets early
    s = api.Session(gpu_ctx, inst, streaming=True, **kw)
    s.run(2 * chunk)
    early = s.result()["best_energy"]
    s.close()
    mid = early + 1e-9 * abs(early)
    ids = [srv.submit(inst, target=math.inf, **kw), srv.submit(inst, target=-math.inf, **kw),
           srv.submit(inst, target=mid, **kw)]
    r_inf, r_none, r_mid = [srv.wait(r, timeout=300) for r in ids]
    st = srv.stats()
    srv.close()
    for r in (r_inf, r_none, r_mid):
        assert r["status"] == 0 and r["done"] == 1, r["error"]
        e = ising.energy(inst, r["best_spins"].astype(np.float64))
        assert r["best_energy"] == pytest.approx(float(e), rel=1e-12, abs=1e-9)
    assert r_inf["reached"] == 1 and r_inf["steps_done"] == chunk
    assert r_none["reached"] == 0 and r_none["steps_done"] == kw["steps"]
    np.testing.assert_array_equal(r_none["best_spins"], plain["best_spins"])
    assert r_none["best_energy"] == plain["best_energy"]
    assert r_mid["reached"] == 1 and r_mid["best_energy"] <= mid
    assert r_mid["steps_done"] <= 2 * chunk
    assert st["completed"] == 3 and st["target_checks"] >= 1 + kw["steps"] // chunk
    for key in ("setup_ms", "advance_ms", "check_ms", "finish_ms", "release_ms", "idle_ms"):
        assert 0.0 <= st[key] <= st["elapsed_ms"]


def test_cancel(gpu_ctx):
    """ising_server_cancel: an admitted request ends at the end of its chunk
    with the best of the steps it ran (an exact result, cancelled = 1); a
    queued one is dropped at once without spins; a finished one is left as
    it is."""
    inst = synth.er_dense(400, 3, p=0.05, weights="pm1")
    srv = api.Server(gpu_ctx, budget_bytes=8 << 30, max_active=1, chunk_steps=20, pack=False)
    a = srv.submit(inst, restarts=256, steps=1000000, seed=1)
    b = srv.submit(inst, restarts=256, steps=100, seed=2)
    srv.cancel(b)  # still queued behind a (one slot)
    rb = srv.wait(b, timeout=60)
    assert rb["done"] == 1 and rb["cancelled"] == 1 and rb["steps_done"] == 0
    assert rb["best_spins"] is None and math.isnan(rb["best_energy"])
    time.sleep(0.3)  # (set up, and running its chunks)
    srv.cancel(a)
    ra = srv.wait(a, timeout=120)
    assert ra["status"] == 0 and ra["cancelled"] == 1 and 0 < ra["steps_done"] < 1000000
    assert ra["steps_done"] % 20 == 0
    e = ising.energy(inst, ra["best_spins"].astype(np.float64))
    assert ra["best_energy"] == float(e)
    srv.cancel(a)  # finished: nothing happens
    assert srv.poll(a)["steps_done"] == ra["steps_done"]
    srv.close()
