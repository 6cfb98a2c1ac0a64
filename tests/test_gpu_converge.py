"""The convergence rule of Sec. IV-B (ISING_DS_CONVERGE, read on the energy
of the rounded spins) on every step-kernel path: each restart stops at the
first step where the window rule holds on its own energy trace, its best is
the minimum of the trace up to there, and the run ends once every restart
has stopped."""

import numpy as np
import pytest

import synth
from oracle import ising
from oracle import domain_selection as ods
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu

CASES = [
    ("er_int", synth.er_dense(150, 1, p=0.08, weights="pm1"), dict(precision="fp8")),
    ("er_int_stream", synth.er_dense(150, 1, p=0.08, weights="pm1"), dict(precision="fp8", streaming=True)),
    ("int_h_fp32", synth.random_sparse_instance(130, 4, p=0.1, kind="int", h="int", layout="dense"),
     dict(precision="fp32")),
    ("torus", synth.torus_csr(10, 13, 5), dict()),
    ("table1_binary_int", synth.table1_instance("binary_int", 3, n=200), dict()),
]


def _rule_steps(trace, T):
    """First t in [5, T] where max - min of E_{t-4..t} <= 0.005 |E_t - E_1|."""
    out = np.zeros(trace.shape[1], dtype=np.int64)
    for b in range(trace.shape[1]):
        for t in range(ods.CONV_WINDOW, T + 1):
            w = trace[t - ods.CONV_WINDOW:t, b]
            if w.max() - w.min() <= ods.CONV_TOL * abs(trace[t - 1, b] - trace[0, b]):
                out[b] = t
                break
    return out


@pytest.mark.parametrize("name,inst,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("lr", [0.05, 6.0])
def test_stops_where_the_rule_holds_on_the_trace(gpu_ctx, name, inst, kw, lr):
    B, T = 40, 150
    plain = api.Session(gpu_ctx, inst, restarts=B, steps=T, lr=lr, seed=2, **kw)
    trace = np.zeros((T, B))
    for t in range(T):
        plain.run(1)
        trace[t] = plain.last_energies()
    plain.close()
    s = api.Session(gpu_ctx, inst, restarts=B, steps=T, lr=lr, seed=2, converge=True, **kw)
    s.run(T)
    s.finish()
    conv = s.convergence()
    want = _rule_steps(trace, T)
    np.testing.assert_array_equal(conv, want)
    E, step, spins = s.restart_best()
    for b in range(B):
        upto = want[b] if want[b] else T
        assert E[b] == trace[:upto, b].min() or (not want[b] and E[b] <= trace[:, b].min())
        if want[b]:
            assert step[b] == int(np.argmin(trace[:want[b], b])) + 1
    e = ising.energy(inst, spins.T.astype(np.float64))
    np.testing.assert_allclose(E, e, rtol=1e-12, atol=1e-9)
    res = s.result()
    if want.all():
        assert res["steps_done"] < T or want.max() > T - 48
    s.close()


@pytest.mark.parametrize("kw", [dict(precision="fp8"), dict(precision="fp32"), dict()],
                         ids=["resident", "plain", "auto"])
def test_no_motion_stops_everything_at_step_five(gpu_ctx, kw):
    """lr = 0: theta never moves, every window is flat, all restarts stop at
    step 5 with the first step's energy as their best; the run ends at the
    first check (48 steps) instead of T."""
    inst = synth.er_dense(150, 1, p=0.08, weights="pm1") if kw else synth.torus_csr(10, 13, 5)
    B, T = 33, 500
    s = api.Session(gpu_ctx, inst, restarts=B, steps=T, lr=0.0, seed=4, converge=True, **kw)
    first = api.Session(gpu_ctx, inst, restarts=B, steps=T, lr=0.0, seed=4, **kw)
    first.run(1)
    E1 = first.last_energies()
    first.close()
    s.run(T)
    s.finish()
    np.testing.assert_array_equal(s.convergence(), 5)
    E, step, _ = s.restart_best()
    np.testing.assert_array_equal(E, E1)
    np.testing.assert_array_equal(step, 1)
    assert s.result()["steps_done"] == 48
    s.close()


def test_server_request_with_the_rule_matches_the_session(gpu_ctx):
    inst = synth.er_dense(300, 1, p=0.05, weights="pm1")
    kw = dict(restarts=64, steps=400, lr=0.05, seed=9, converge=True)
    alone = api.solve(gpu_ctx, inst, **kw)
    srv = api.Server(gpu_ctx, budget_bytes=4 << 30, max_active=2, chunk_steps=48)
    rid = srv.submit(inst, **kw)
    res = srv.wait(rid, timeout=120)
    srv.close()
    assert res["status"] == 0
    assert res["best_energy"] == alone["best_energy"]
    np.testing.assert_array_equal(res["best_spins"], alone["best_spins"])


@pytest.mark.parametrize("name,inst,kw,width", [
    ("tc_stream", synth.er_dense(150, 1, p=0.08, weights="pm1"),
     dict(precision="fp8", streaming=True), 128),
    ("plain", synth.random_sparse_instance(130, 4, p=0.1, kind="int", h="int", layout="dense"),
     dict(precision="fp32"), 128),
    ("sparse", synth.torus_csr(10, 13, 5), dict(), 128),
])
def test_retired_tiles_are_skipped(gpu_ctx, name, inst, kw, width):
    """Early retirement: a tile (or slice) of restarts is computed at step t
    exactly when one of its restarts is still running then, i.e. has not
    stopped or stopped at a step >= t. The restart-steps the kernels report
    equal that count over the steps run, below B x steps, and the results
    are those of the rule (the trace test above)."""
    B, T = 520, 400
    s = api.Session(gpu_ctx, inst, restarts=B, steps=T, lr=0.05, seed=3, converge=True,
                    autotune=False, **kw)
    s.run(T)
    done = s.result()["steps_done"]
    conv = s.convergence()
    last = np.where(conv > 0, conv, np.iinfo(np.int64).max)
    want = 0
    for b0 in range(0, B, width):
        b1 = min(b0 + width, B)
        want += (b1 - b0) * min(int(last[b0:b1].max()), done)
    got = s.work()
    assert got == want, (got, want, done)
    assert got < B * done
    s.close()
