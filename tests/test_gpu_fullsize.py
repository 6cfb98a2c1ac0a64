"""Parity at the full workload sizes the benchmark times, in the same launch
configuration (precision AUTO, so the resident FP8 tensor-core form for the
N=2000 max-cut, the sparse kernel for the torus and the pruned ER graph, the
streaming two-plane FP16 form for N=4096 SK, the resident two-plane form for
the complete 1000-spin graphs of Sec. IV-C): after a run of steps, one step
of all restarts (a sample of 256 on the largest) is checked against the oracle element by
element (Sec. III-B), and the reduced-precision operand forms are held to the
plain FP32 path's best energy (Sec. IV)."""

import math

import numpy as np
import pytest

import synth
from oracle import domain_selection as ods
from oracle import ising
from paper_2312_05837_gb300 import api

import gpu_util as U

pytestmark = pytest.mark.gpu


def _sample(st, idx):
    return dict(theta=st["theta"][idx], m=st["m"][idx], v=st["v"][idx],
                spins=st["spins"][idx], t=st["t"])


@pytest.mark.parametrize("name,B,warm,path,prec", [
    ("er2000", 1024, 300, 1, 4),
    ("torus20k", 512, 200, 2, 1),
    ("sk4096", 4096, 40, 1, 2),
    ("er100k_pendant", 512, 60, 2, 1),
    ("table2_uniform", 1024, 100, 1, 2),
])
def test_bench_workload_sampled_one_step_parity(gpu_ctx, name, B, warm, path, prec):
    inst = synth.workload(name, 0)
    lr, mu = 6.0, 0.0
    s = api.Session(gpu_ctx, inst, restarts=B, steps=warm + 2, lr=lr, mu=mu, seed=17)
    s.run(warm)
    st0 = s.export_state()
    G0 = s.coupling()
    s.run(1)
    st1 = s.export_state()
    E = s.last_energies()
    # every restart where the oracle's FP64 step over all of them stays within
    # a few GB of host memory; else the first, last, ragged-tile and 251 random ones
    if inst.n * B <= 20_000_000:
        idx = np.arange(B)
    else:
        r = np.random.default_rng(B + warm)
        idx = np.unique(np.concatenate([[0, 1, B - 1, B // 2 - 1, B // 2],
                                        r.choice(B, 251, replace=False)]))
    p = ods.Params(restarts=len(idx), steps=warm + 2, lr=lr, mu=mu, seed=17)
    U.check_step(inst, _sample(st0, idx), _sample(st1, idx), E[idx], p, bool(inst.integer),
                 G0=G0[idx])
    s.finish()
    res = s.result()
    assert (res["path"], res["precision"]) == (path, prec)
    if name in ("er2000", "table2_uniform"):
        assert res["resident"] == 1
    e = ising.energy(inst, res["best_spins"].astype(np.float64))
    assert res["best_energy"] == pytest.approx(float(e), rel=1e-12, abs=1e-9)
    s.close()


def test_reduced_precision_reaches_the_plain_fp32_best(gpu_ctx):
    """SK couplings J ~ N(0, 1/N) with fields h ~ N(0, 0.1) (a smaller case of
    the N=4096 workload): the BF16 single-plane and the row-scaled E4M3
    operands change G by up to 2^-8 and 2^-4 of the row's absolute sum, yet
    the best energy over the restarts (re-evaluated exactly in FP64), averaged
    over four seeds, stays within 0.5 % of the plain FP32 path's on the same
    seeds. (At lr = 6 the trajectories of different operand precisions part
    after some steps, so single runs differ like runs of different seeds: the
    oracle's spread over seeds 4..7 is 0.7 % for one run.)"""
    n = 768
    inst = synth.sk_dense(n, 21, 1 / math.sqrt(n), np.float32, h_std=math.sqrt(0.1))
    seeds = [4, 5, 6, 7]

    def mean_best(prec):
        tot = 0.0
        for seed in seeds:
            out = api.select_domain(gpu_ctx, inst, restarts=1024, steps=800, lr=6.0, seed=seed,
                                    precision=prec)
            e = ising.energy(inst, out["best_spins"].astype(np.float64))
            assert out["best_energy"] == pytest.approx(float(e), rel=1e-12)
            tot += out["best_energy"]
        return tot / len(seeds)

    ref = mean_best("fp32")
    gaps = {prec: (mean_best(prec) - ref) / abs(ref) for prec in ["tc", "bf16", "fp8"]}
    print("mean best-energy gap vs plain FP32:", {k: f"{v:+.4%}" for k, v in gaps.items()})
    assert all(abs(g) <= 0.005 for g in gaps.values()), gaps
