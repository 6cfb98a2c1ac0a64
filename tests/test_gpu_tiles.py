"""Launch shapes of the tensor-core streaming step (Sec. III-B) give the same
results: every tile width, tiles shared by a cluster of two CTAs (each
loads half of the spin tile and multicasts it to both), and tiles whose MMAs
a CTA pair issues as one (each CTA keeps its half; cta_group::2, M 256),
bit-identical to the default shape in state, spins, bests and result,
including odd numbers of row tiles (the last pair's second tile lies past n)
and ragged restart tiles; and both pair forms pass the one-step oracle
parity at full size."""

import math

import numpy as np
import pytest

import synth
from oracle import domain_selection as ods
from paper_2312_05837_gb300 import api

import gpu_util as U

pytestmark = pytest.mark.gpu


def _run(ctx, inst, B, T, shape, **kw):
    s = api.Session(ctx, inst, restarts=B, steps=T, seed=6, streaming=True, autotune=False, **kw)
    if shape is not None:
        s.set_tiles(*shape)
    s.run(T)
    st = s.export_state()
    best = s.restart_best()
    s.finish()
    res = s.result()
    s.close()
    return st, best, res


@pytest.mark.parametrize("inst,B", [
    (synth.sk_dense(300, 51, 1 / math.sqrt(300), np.float32, h_std=0.3), 500),   # 3 row tiles
    (synth.sk_dense(640, 52, 1 / math.sqrt(640), np.float64), 449),              # 5 row tiles
    (synth.er_dense(520, 53, mean_degree=8, weights="pm1"), 700),                # E4M3, 5 row tiles
])
@pytest.mark.parametrize("shape", [(64, 0), (224, 0), (256, 0), (224, 1), (256, 1), (224, 2),
                                   (256, 2)])
def test_shapes_are_bit_identical(gpu_ctx, inst, B, shape):
    T = 25
    ref_st, ref_best, ref_res = _run(gpu_ctx, inst, B, T, (128, 0))
    st, best, res = _run(gpu_ctx, inst, B, T, shape)
    for k in ["theta", "m", "v", "spins"]:
        np.testing.assert_array_equal(st[k], ref_st[k], err_msg=k)
    for a, b in zip(best, ref_best):
        np.testing.assert_array_equal(a, b)
    assert res["best_energy"] == ref_res["best_energy"]
    np.testing.assert_array_equal(res["best_spins"], ref_res["best_spins"])


@pytest.mark.parametrize("pair", [1, 2])
def test_pairs_at_full_size_match_the_oracle(gpu_ctx, pair):
    inst = synth.workload("sk4096", 0)
    B, warm = 4096, 20
    s = api.Session(gpu_ctx, inst, restarts=B, steps=warm + 2, lr=6.0, seed=17, streaming=True)
    s.set_tiles(224, pair)
    s.run(warm)
    st0 = s.export_state()
    G0 = s.coupling()
    s.run(1)
    st1 = s.export_state()
    p = ods.Params(restarts=B, steps=warm + 2, lr=6.0, mu=0.0, seed=17)
    U.check_step(inst, st0, st1, s.last_energies(), p, False, G0=G0)
    s.close()


def test_unavailable_shapes_are_refused(gpu_ctx):
    inst = synth.sk_dense(100, 54, 0.1, np.float32)
    s = api.Session(gpu_ctx, inst, restarts=300, steps=5, streaming=True)
    with pytest.raises(api.IsingError):
        s.set_tiles(224, 1)  # one row tile: nothing to pair
    with pytest.raises(api.IsingError):
        s.set_tiles(96)
    s.close()
    r = api.Session(gpu_ctx, synth.er_dense(150, 1, p=0.08, weights="pm1"), restarts=64, steps=5)
    with pytest.raises(api.IsingError):
        r.set_tiles(128)  # resident form
    r.close()
