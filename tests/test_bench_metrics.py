"""The library's Sec. IV-C figures (chi_hat, estimated TTS, speed), which
bench.py and the experiments report, against the oracle's metrics module,
on both conventions and layouts."""

import os
import sys

import numpy as np
import pytest

import synth
from oracle import domain_selection as ods
from oracle import metrics

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.mark.parametrize("inst", [synth.table2_instance("uniform", 0, n=60),
                                  synth.table2_instance("gaussian", 1, n=40),
                                  synth.table1_instance("gaussian", 2, n=50),
                                  synth.er_dense(70, 3, p=0.1, weights="pm1")])
def test_paper_metrics_match_the_oracle(inst):
    from paper_2312_05837_gb300.metrics import paper_metrics
    r = ods.select_domain(inst, ods.Params(restarts=8, steps=30, seed=1))
    E = float(r["best_energy"])
    got = paper_metrics(inst, E, 0.25)
    chi = metrics.chi_hat(inst, E)
    assert got["chi_hat"] == pytest.approx(chi, rel=1e-12)
    assert got["tts_s"] == pytest.approx(metrics.tts(0.25, chi, inst.n), rel=1e-9)
    assert got["v_per_s"] == pytest.approx(metrics.speed(0.25, chi), rel=1e-12)
    assert got["chi_hat"] > 0.5  # E < 0 for a found optimum of a random instance


def test_table2_family_shapes():
    u = synth.table2_instance("uniform", 5, n=200)
    assert u.convention == "paper" and u.j_scale == 0.5 and u.J.dtype == np.float32
    assert np.array_equal(u.J, u.J.T) and not np.diag(u.J).any()
    assert np.abs(u.J).max() <= 1000 and np.abs(u.h).max() <= 1000
    g = synth.table2_instance("gaussian", 5, n=200)
    assert np.array_equal(g.J, g.J.T)


def test_traffic_figure_only_for_its_workload_and_source():
    """bench.py reports the committed ncu DRAM figure of the dominant kernel
    only for the workload it was captured on and while the kernel's source
    is the one profiled."""
    import json
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kernel, e in d.items():
        src = {"sparse_step_kernel": "paper_2312_05837_gb300/csrc/ds_sparse.cu"}.get(
            kernel, "paper_2312_05837_gb300/csrc/ds_tc.cu")
        other = "er2000" if e["workload"] != "er2000" else "sk4096"
        assert bench.traffic_for(kernel, src, other) is None
        got = bench.traffic_for(kernel, src, e["workload"])
        assert got in (None, e["bytes_per_launch"])
    assert bench.traffic_for("no_such_kernel", "bench.py", "er2000") is None


def test_serving_capacity_at_the_roofline():
    """The serving leg's capacity figure: a dense request takes the longer of
    its E4M3 flop time and its state + J traffic time, a sparse one its
    24.25 B per padded update; the capacity is requests over their summed
    times."""
    import types
    import bench
    pk = {"bf16_tflops_sustained": 1000.0, "hbm_gbs": 5000.0}
    B, T = 256, 2000
    dense = types.SimpleNamespace(n=1000, layout="dense")
    sparse = types.SimpleNamespace(n=3000, layout="csr")
    t_dense = max(2.0 * 1000 ** 2 * B * T / 2e15, (24.0 * 1000 * B + 1000 ** 2) * T / 5e12)
    t_sparse = 24.25 * 3000 * 256 * T / 5e12
    got = bench.serving_capacity([(0.0, dense), (0.1, sparse)], B, T, pk)
    assert got == pytest.approx(2.0 / (t_dense + t_sparse), rel=1e-12)
    # restarts pad to 128 on the sparse path
    got_pad = bench.serving_capacity([(0.0, sparse)], 129, T, pk)
    assert got_pad == pytest.approx(1.0 / (24.25 * 3000 * 256 * T / 5e12), rel=1e-12)


def test_launch_count_model_of_a_solve():
    """bench.py's count of the library's kernel launches in one solve: the
    streaming tensor-core path takes one launch per step (each tracks the
    step before it) plus one tracking launch after the last; the other
    non-resident paths a step and a tracking launch per step (the sparse path
    also a spin copy); a resident form one launch for all steps."""
    import bench
    T, rounds = 50, 2
    base = bench.launches_per_solve(0, rounds, 0, False, False, False)
    assert bench.launches_per_solve(T, rounds, 1, False, False, False) - \
        bench.launches_per_solve(0, rounds, 1, False, False, False) == T
    assert bench.launches_per_solve(T, rounds, 0, False, False, False) - base == 2 * T
    assert bench.launches_per_solve(T, rounds, 2, False, False, False) - \
        bench.launches_per_solve(0, rounds, 2, False, False, False) == 3 * T
    assert bench.launches_per_solve(T, rounds, 1, True, False, False) == \
        bench.launches_per_solve(2 * T, rounds, 1, True, False, False)
    # set-up: the integer row-sum bound and the per-row scales add a launch each
    assert bench.launches_per_solve(T, rounds, 1, False, True, True) == \
        bench.launches_per_solve(T, rounds, 1, False, False, False) + 2
