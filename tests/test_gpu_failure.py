"""Failure handling without a GPU fault: device waits that nothing completes
give up after their clock budget and report a status the host reads, after
which the context keeps working; the server reports a request that is not
done in time and refuses what it cannot hold."""

import numpy as np
import pytest

import synth
from oracle import ising
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu


def test_bounded_waits_give_up_and_the_context_survives(gpu_ctx):
    rc, mask = api.selftest_waits(gpu_ctx, 20_000_000)  # ~10 ms of SM clock
    assert rc == 4 and mask == 3
    inst = synth.er_dense(64, 1, p=0.2, weights="pm1")
    r = api.select_domain(gpu_ctx, inst, restarts=8, steps=10, seed=1)
    assert r["best_energy"] == float(ising.energy(inst, r["best_spins"].astype(np.float64)))


def test_bad_limits_are_rejected(gpu_ctx):
    for bad in [0, -5, 1 << 40]:
        rc, mask = api.selftest_waits(gpu_ctx, bad)
        assert rc == 1 and mask == -1


def test_server_wait_reports_a_request_still_running(gpu_ctx):
    inst = synth.er_dense(800, 2, p=0.06, weights="one")
    srv = api.Server(gpu_ctx, budget_bytes=4 << 30, max_active=2, chunk_steps=50)
    rid = srv.submit(inst, restarts=1024, steps=4000, seed=1)
    with pytest.raises(api.IsingError) as e:
        srv.wait(rid, timeout=1e-4)
    assert e.value.code == 4
    res = srv.wait(rid, timeout=300)
    assert res["status"] == 0 and res["done"] == 1
    srv.close()
