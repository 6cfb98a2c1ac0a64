"""Domain-selection step kernels (K2p plain FP32, K2s sparse, K2 tensor core)
through the C ABI against one oracle step from the same state (Sec. III-B),
plus integer-exact energies, best tracking and edge cases."""

import math

import numpy as np
import pytest

import synth
from oracle import brute_force, ising, rng
from oracle import domain_selection as ods
from paper_2312_05837_gb300 import api

import gpu_util as U

pytestmark = pytest.mark.gpu


def _instances():
    return {
        "er_int": synth.er_dense(150, 1, p=0.08, weights="pm1"),
        "sk_float": synth.sk_dense(140, 2, 1.0, np.float64),
        "sk_float_h": synth.sk_dense(133, 3, 1 / math.sqrt(133), np.float32, h_std=math.sqrt(0.1)),
        "rand_int_h_paper": synth.random_sparse_instance(130, 4, p=0.1, kind="int", h="int",
                                                         convention="paper", j_scale=0.5,
                                                         layout="dense"),
        "torus_small": synth.torus_csr(10, 13, 5),
        "er_pendant_h": synth.er_pendant_csr(200, 3.0, 60, 3, 6, h_mode="int2"),
        "csr_float_h": synth.random_sparse_instance(170, 7, p=0.05, kind="float", h="float"),
        # n <= 128: the tensor-core path's small form (one k-block in E4M3, one
        # or two in BF16; 77 and 100 leave ragged row and K tails)
        "er_small_int": synth.er_dense(77, 22, p=0.1, weights="pm1"),
        "sk_small_h": synth.sk_dense(100, 21, 0.1, np.float32, h_std=math.sqrt(0.1)),
        "rand_small_int_h": synth.random_sparse_instance(128, 23, p=0.15, kind="int", h="int",
                                                         convention="paper", j_scale=0.5,
                                                         layout="dense"),
    }


INSTANCES = _instances()
# (instance, precision) pairs exercised by the parity tests
CASES = [("er_int", "fp32"), ("sk_float", "fp32"), ("sk_float_h", "fp32"),
         ("rand_int_h_paper", "fp32"), ("torus_small", "auto"), ("er_pendant_h", "auto"),
         ("csr_float_h", "auto"), ("er_int", "tc"), ("sk_float", "tc"), ("sk_float_h", "tc"),
         ("rand_int_h_paper", "tc"), ("er_int", "fp8"), ("rand_int_h_paper", "auto"),
         ("er_int", "fp8-stream"), ("sk_float_h", "tc-stream"), ("rand_int_h_paper", "tc-stream"),
         ("er_small_int", "auto"), ("sk_small_h", "tc"), ("rand_small_int_h", "tc"),
         ("sk_small_h", "fp32")]


def _exact(inst):
    return bool(inst.integer)


def _kw(prec):
    """'tc-stream' / 'fp8-stream' force the tensor-core path's streaming form
    (state in device memory between steps) instead of the resident one."""
    if prec.endswith("-stream"):
        return dict(precision=prec[: -len("-stream")], streaming=True)
    return dict(precision=prec)


@pytest.mark.parametrize("name,prec", CASES)
def test_initial_state_is_the_oracle_draw(gpu_ctx, name, prec):
    inst = INSTANCES[name]
    s = api.Session(gpu_ctx, inst, restarts=37, steps=5, seed=9, **_kw(prec))
    st = s.export_state()
    th0 = rng.theta_init(9, 37, inst.n).T
    np.testing.assert_allclose(st["theta"], th0, rtol=0, atol=4e-7)
    np.testing.assert_array_equal(st["spins"], np.where(rng.uniform_pm1(9, 37, inst.n).T >= 0, 1, -1))
    assert st["t"] == 0 and not st["m"].any() and not st["v"].any()
    s.close()


@pytest.mark.parametrize("name,prec", CASES)
@pytest.mark.parametrize("lr,mu", [(6.0, 0.0), (0.1, 0.7)])
def test_one_step_parity_along_a_run(gpu_ctx, name, prec, lr, mu):
    inst = INSTANCES[name]
    p = ods.Params(restarts=40, steps=12, lr=lr, mu=mu, seed=3)
    s = api.Session(gpu_ctx, inst, restarts=40, steps=12, lr=lr, mu=mu, seed=3, **_kw(prec))
    st = s.export_state()
    for _ in range(12):
        G0 = s.coupling()
        s.run(1)
        nxt = s.export_state()
        U.check_step(inst, st, nxt, s.last_energies(), p, _exact(inst), G0=G0)
        st = nxt
    s.close()


@pytest.mark.parametrize("name,prec", CASES)
def test_one_step_parity_from_an_imported_state(gpu_ctx, name, prec):
    inst = INSTANCES[name]
    B, n = 33, inst.n
    r = np.random.default_rng(11)
    th = r.uniform(-math.pi, math.pi, (B, n)).astype(np.float32)
    m = (r.standard_normal((B, n)) * 0.3).astype(np.float32)
    v = (r.random((B, n)) * 0.5).astype(np.float32)
    p = ods.Params(restarts=B, steps=20, lr=0.5, mu=0.2, seed=1)
    s = api.Session(gpu_ctx, inst, restarts=B, steps=20, lr=0.5, mu=0.2, seed=1, **_kw(prec))
    s.import_state(th, m, v, 7)
    st0 = s.export_state()
    assert st0["t"] == 7
    np.testing.assert_array_equal(st0["theta"], th)
    s.run(1)
    U.check_step(inst, st0, s.export_state(), s.last_energies(), p, _exact(inst))
    s.close()


@pytest.mark.parametrize("name,prec", CASES)
def test_bests_after_an_imported_state_cover_the_steps_run(gpu_ctx, name, prec):
    """A state imported at step t0 has no energies of its own, so the bests
    of a fresh session afterwards are those of the steps it then runs: per
    restart the earliest minimum of their energies (strict <), whether the
    steps run one call at a time or in one call with graph replays, on every
    path (the streaming tensor-core update launches track the step before
    theirs, and must not track the imported one)."""
    inst = INSTANCES[name]
    B, n, t0, K = 24, inst.n, 7, 100
    r = np.random.default_rng(12)
    th = r.uniform(-math.pi, math.pi, (B, n)).astype(np.float32)
    m = (r.standard_normal((B, n)) * 0.3).astype(np.float32)
    v = (r.random((B, n)) * 0.5).astype(np.float32)
    kw = dict(restarts=B, steps=t0 + K + 5, lr=0.5, mu=0.2, seed=1, **_kw(prec))
    a = api.Session(gpu_ctx, inst, **kw)
    a.import_state(th, m, v, t0)
    trace = np.empty((K, B))
    for k in range(K):
        a.run(1)
        trace[k] = a.last_energies()
    b = api.Session(gpu_ctx, inst, **kw)
    b.import_state(th, m, v, t0)
    b.run(K)
    for s_ in (a, b):
        E, step, _ = s_.restart_best()
        np.testing.assert_array_equal(E, trace.min(axis=0))
        np.testing.assert_array_equal(step, t0 + 1 + trace.argmin(axis=0))
    np.testing.assert_array_equal(b.last_energies(), trace[-1])
    a.close()
    b.close()


@pytest.mark.parametrize("name,prec", CASES)
def test_best_tracking_and_result(gpu_ctx, name, prec):
    inst = INSTANCES[name]
    B, T = 24, 30
    s = api.Session(gpu_ctx, inst, restarts=B, steps=T, lr=6.0, seed=5, **_kw(prec))
    trace = np.full((T + 1, B), np.inf)
    for t in range(T):
        s.run(1)
        trace[t] = s.last_energies()
    s.finish()
    trace[T] = s.last_energies()
    E, step, spins = s.restart_best()
    np.testing.assert_array_equal(E, trace.min(axis=0))
    np.testing.assert_array_equal(step, trace.argmin(axis=0) + 1)
    Eo = ising.energy(inst, spins.T.astype(np.float64))
    if _exact(inst):
        np.testing.assert_array_equal(E, Eo)
    else:
        np.testing.assert_allclose(E, Eo, rtol=1e-5)
    res = s.result()
    e_full = ising.energy(inst, res["best_spins"].astype(np.float64))
    assert res["best_energy"] == pytest.approx(e_full, rel=1e-12, abs=1e-12)
    assert res["best_energy"] <= E.min() + 1e-4 * abs(E.min())
    assert res["last_best_energy"] == trace[T].min()
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "auto", "tc"])
def test_reaches_brute_force_ground_states(gpu_ctx, prec):
    hits = 0
    for seed in range(4):
        inst = synth.sk_dense(16, 100 + seed, 1.0)
        if prec == "auto":
            inst = inst.to_csr()
        e0, _ = brute_force.ground_state(inst)
        out = api.select_domain(gpu_ctx, inst, restarts=256, steps=150, lr=6.0, seed=seed,
                                precision=prec)
        assert out["best_energy"] >= e0 - 1e-9
        hits += abs(out["best_energy"] - e0) < 1e-9
    assert hits >= 3


@pytest.mark.parametrize("prec,layout", [("fp32", "dense"), ("auto", "csr"), ("tc", "dense"),
                                         ("fp8", "dense")])
@pytest.mark.parametrize("n,B,T", [(1, 1, 3), (1, 5, 0), (2, 1, 4), (129, 130, 3), (257, 3, 2)])
def test_edge_sizes(gpu_ctx, prec, layout, n, B, T):
    inst = synth.random_sparse_instance(n, n + B, p=0.2, kind="int", h="int", layout=layout)
    out = api.select_domain(gpu_ctx, inst, restarts=B, steps=T, lr=1.0, seed=4, precision=prec)
    assert out["best_energy"] == ising.energy_exact(inst, out["best_spins"])[0]
    assert out["steps_done"] == T
    # the same run through the oracle reaches the same kind of answer: never below the ground
    if n <= 16:
        assert out["best_energy"] >= brute_force.ground_state(inst)[0]


def test_invalid_parameters(gpu_ctx):
    inst = INSTANCES["er_int"]
    for kw in [dict(restarts=0, steps=3), dict(restarts=4, steps=-1),
               dict(restarts=4, steps=3, beta1=1.0), dict(restarts=4, steps=3, eps=0.0),
               dict(restarts=4, steps=3, mu=-1.0)]:
        with pytest.raises(api.IsingError) as e:
            api.select_domain(gpu_ctx, inst, **kw)
        assert e.value.code == 1
    with pytest.raises(api.IsingError) as e:
        api.select_domain(gpu_ctx, INSTANCES["torus_small"], restarts=4, steps=2, precision="bf16")
    assert e.value.code == 6


@pytest.mark.parametrize("name,prec", [("er_int", "tc"), ("sk_float_h", "tc"), ("er_int", "fp32"),
                                       ("torus_small", "auto"), ("er_int", "fp8"),
                                       ("er_int", "fp8-stream"), ("sk_float_h", "tc-stream")])
def test_graph_replay_equals_step_by_step(gpu_ctx, name, prec):
    """Long runs replay a captured CUDA graph of the step loop; the state and
    the bests must be bit-identical to launching the steps one by one."""
    inst = INSTANCES[name]
    T = 230
    a = api.Session(gpu_ctx, inst, restarts=70, steps=T, seed=2, **_kw(prec))
    b = api.Session(gpu_ctx, inst, restarts=70, steps=T, seed=2, **_kw(prec))
    a.run(T)
    for _ in range(T):
        b.run(1)
    sa, sb = a.export_state(), b.export_state()
    for k in ["theta", "m", "v", "spins"]:
        np.testing.assert_array_equal(sa[k], sb[k])
    assert sa["t"] == sb["t"] == T
    for x, y in zip(a.restart_best(), b.restart_best()):
        np.testing.assert_array_equal(x, y)
    a.close()
    b.close()



@pytest.mark.parametrize("name,prec,B", [("er_int", "fp8", 300), ("sk_float_h", "tc", 200),
                                         ("rand_int_h_paper", "tc", 1),
                                         ("er_int", "fp8", 9000), ("sk_float_h", "tc", 9000),
                                         ("er_small_int", "fp8", 1), ("er_small_int", "auto", 65),
                                         ("rand_small_int_h", "tc", 64), ("sk_small_h", "tc", 300),
                                         ("er_small_int", "fp8", 6000), ("sk_small_h", "tc", 20000),
                                         ("er_small_int", "fp8", 20000)])
def test_resident_equals_streaming(gpu_ctx, name, prec, B):
    """The resident tensor-core forms (state in tensor memory, one launch for
    the whole run, tracking inside) give the same state and bests bit for bit
    as the streaming form (one launch per step). B = 9000 on two row tiles
    makes 142 tiles of 128 restarts, nearly one per SM, with a ragged last
    column. For n <= 128 the small form runs with blocks of 32 restarts up to
    B = 32 x SMs (B = 1, 64, 65, 300: one to ten CTAs, ragged), of 64 beyond
    (B = 6000) and of 128 beyond 64 x SMs (B = 20000: more CTAs than SMs, so
    CTAs start after others have finished)."""
    inst = INSTANCES[name]
    T = 57
    a = api.Session(gpu_ctx, inst, restarts=B, steps=T, seed=4, precision=prec)
    b = api.Session(gpu_ctx, inst, restarts=B, steps=T, seed=4, precision=prec, streaming=True)
    a.run(20)
    a.run(T - 20)
    b.run(T)
    sa, sb = a.export_state(), b.export_state()
    for k in ["theta", "m", "v", "spins"]:
        np.testing.assert_array_equal(sa[k], sb[k])
    for x, y in zip(a.restart_best(), b.restart_best()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.last_energies(), b.last_energies())
    a.finish()
    b.finish()
    ra, rb = a.result(), b.result()
    assert (ra["resident"], rb["resident"]) == (2 if inst.n <= 128 else 1, 0)
    assert ra["best_energy"] == rb["best_energy"]
    np.testing.assert_array_equal(ra["best_spins"], rb["best_spins"])
    a.close()
    b.close()


def test_autotuned_sparse_equals_fixed_shape(gpu_ctx):
    """The autotuner only changes the launch shape: state and bests match a
    run with the default shape bit for bit."""
    inst = INSTANCES["er_pendant_h"]
    a = api.Session(gpu_ctx, inst, restarts=256, steps=30, seed=6)
    b = api.Session(gpu_ctx, inst, restarts=256, steps=30, seed=6, autotune=False)
    a.run(30)
    b.run(30)
    sa, sb = a.export_state(), b.export_state()
    for k in ["theta", "m", "v", "spins"]:
        np.testing.assert_array_equal(sa[k], sb[k])
    for x, y in zip(a.restart_best(), b.restart_best()):
        np.testing.assert_array_equal(x, y)
    a.close()
    b.close()


_FORCED_SHAPE = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import synth
from paper_2312_05837_gb300 import api
inst = synth.random_sparse_instance(300, 9, p=0.02, kind="float", h="float")
ctx = api.Context(0)
a = api.Session(ctx, inst, restarts=256, steps=12, seed=3)            # shape from the cache file
b = api.Session(ctx, inst, restarts=256, steps=12, seed=3, autotune=False)
a.run(12); b.run(12)
sa, sb = a.export_state(), b.export_state()
ok = all(np.array_equal(sa[k], sb[k]) for k in ["theta", "m", "v", "spins"])
ok = ok and all(np.array_equal(x, y) for x, y in zip(a.restart_best(), b.restart_best()))
a.close(); b.close(); ctx.close()
print("EQUAL" if ok else "DIFFERENT")
"""


def test_two_slice_shape_equals_one_slice_shape(tmp_path):
    """Forces the 256-restart slice shape through the tuning cache file in a
    fresh process and compares it with the default 128-restart shape."""
    import os
    import subprocess
    import sys
    import synth as S
    inst = S.random_sparse_instance(300, 9, p=0.02, kind="float", h="float")
    key = f"sparse n=300 nnz={int(inst.indptr[-1])} Bp=256 i8=0 ie=0"
    cache = tmp_path / "tune.txt"
    cache.write_text(key + "|2\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, ISING_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", _FORCED_SHAPE.format(root=root)], env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().endswith("EQUAL"), out.stdout[-500:]
