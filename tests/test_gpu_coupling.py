"""The coupling product G = J s (Sec. III-B) of each step kernel, read back
through ising_ds_coupling, against the oracle's matrix product."""

import math

import numpy as np
import pytest

import synth
from oracle import ising
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu


def _check(ctx, inst, B, prec, exact):
    s = api.Session(ctx, inst, restarts=B, steps=3, seed=1, precision=prec)
    st = s.export_state()
    G = s.coupling()
    J = ising.coupling_matrix(inst)
    ref = np.asarray(J @ st["spins"].T.astype(np.float64)).T
    if exact:
        np.testing.assert_array_equal(G, ref)
    else:
        scale = np.asarray(abs(J).sum(axis=1)).ravel()[None, :]
        assert np.max(np.abs(G - ref) / scale) <= 1e-5
    # after a step the product follows the new spins
    s.run(1)
    st = s.export_state()
    ref = np.asarray(J @ st["spins"].T.astype(np.float64)).T
    G = s.coupling()
    if exact:
        np.testing.assert_array_equal(G, ref)
    s.close()


def test_tc_single_tile(gpu_ctx):
    _check(gpu_ctx, synth.er_dense(128, 0, p=0.2, weights="pm1"), 128, "tc", True)


@pytest.mark.parametrize("prec", ["tc", "fp32", "fp8", "auto"])
@pytest.mark.parametrize("n,B", [(200, 130), (64, 1), (1, 3), (300, 512), (129, 257)])
def test_dense_integer_exact(gpu_ctx, prec, n, B):
    inst = synth.random_sparse_instance(n, n + B, p=0.3, kind="int", h="int", layout="dense",
                                        jmax=7)
    _check(gpu_ctx, inst, B, prec, True)


@pytest.mark.parametrize("prec", ["tc", "fp32"])
def test_dense_float_three_planes(gpu_ctx, prec):
    inst = synth.sk_dense(333, 5, 1 / math.sqrt(333), np.float32, h_std=0.3)
    _check(gpu_ctx, inst, 200, prec, False)
    inst = synth.sk_dense(100, 6, 1.0, np.float64)
    _check(gpu_ctx, inst, 64, prec, False)


def test_bf16_single_plane_error_is_bf16_sized(gpu_ctx):
    inst = synth.sk_dense(256, 7, 1 / 16, np.float32)
    s = api.Session(gpu_ctx, inst, restarts=128, steps=1, seed=1, precision="bf16")
    st = s.export_state()
    G = s.coupling()
    J = ising.coupling_matrix(inst)
    ref = (J @ st["spins"].T.astype(np.float64)).T
    scale = np.abs(J).sum(axis=1)[None, :]
    err = np.max(np.abs(G - ref) / scale)
    assert 1e-6 < err <= 2.0 ** -8
    s.close()


@pytest.mark.parametrize("name,B", [("torus_small", 128), ("csr_float_h", 300)])
def test_sparse(gpu_ctx, name, B):
    inst = {"torus_small": synth.torus_csr(10, 13, 5),
            "csr_float_h": synth.random_sparse_instance(170, 7, p=0.05, kind="float",
                                                        h="float")}[name]
    _check(gpu_ctx, inst, B, "auto", inst.integer)


def test_bench_size_tc(gpu_ctx):
    _check(gpu_ctx, synth.workload("er2000", 0), 1024, "tc", True)


def test_fp8_row_scaled_error_is_e4m3_sized(gpu_ctx):
    """Non-integer J in E4M3 with one scale per row: each coupling is rounded
    to 3 mantissa bits (relative error <= 2^-4), so |dG_i| <= 2^-4 sum_j |J_ij|."""
    inst = synth.sk_dense(300, 8, 1 / math.sqrt(300), np.float32)
    s = api.Session(gpu_ctx, inst, restarts=96, steps=1, seed=1, precision="fp8")
    st = s.export_state()
    G = s.coupling()
    J = ising.coupling_matrix(inst)
    ref = (J @ st["spins"].T.astype(np.float64)).T
    scale = np.abs(J).sum(axis=1)[None, :]
    err = np.max(np.abs(G - ref) / scale)
    assert 1e-4 < err <= 2.0 ** -4
    s.close()


def test_bench_size_fp8(gpu_ctx):
    _check(gpu_ctx, synth.workload("er2000", 0), 1024, "fp8", True)


@pytest.mark.parametrize("n,B,prec,jmax,rel", [(300, 96, "fp8", 40, 2.0 ** -4),
                                               (120, 40, "fp8", 40, 2.0 ** -4),
                                               (300, 96, "bf16", 400, 2.0 ** -8)])
def test_rounded_integer_couplings(gpu_ctx, n, B, prec, jmax, rel):
    """Integer couplings beyond the operand type's exact range (E4M3 row-scaled
    above 16, one BF16 plane above 256) are rounded, so the products are no
    longer the instance's integers: the coupling error is the type's, the
    step energies are FP32 partials (within that error), the run stays
    deterministic between the resident and streaming forms, and the result's
    energy is the exact energy of its spins (n = 120 runs the small form)."""
    inst = synth.random_sparse_instance(n, 12, p=0.1, kind="int", h="int", layout="dense", jmax=jmax)
    s = api.Session(gpu_ctx, inst, restarts=B, steps=1, seed=1, precision=prec)
    st = s.export_state()
    G = s.coupling()
    J = ising.coupling_matrix(inst)
    ref = (J @ st["spins"].T.astype(np.float64)).T
    scale = np.abs(J).sum(axis=1)[None, :]
    assert np.max(np.abs(G - ref) / scale) <= rel
    s.run(1)
    E = s.last_energies()
    Eo = ising.energy(inst, st["spins"].T.astype(np.float64))
    assert np.all(np.abs(E - Eo) <= rel * (np.sum(np.abs(J)) + np.abs(inst.h).sum() + 1.0))
    s.close()
    a = api.Session(gpu_ctx, inst, restarts=B, steps=30, seed=2, precision=prec)
    b = api.Session(gpu_ctx, inst, restarts=B, steps=30, seed=2, precision=prec, streaming=True)
    a.run(30)
    b.run(30)
    sa, sb = a.export_state(), b.export_state()
    for k in ["theta", "m", "v", "spins"]:
        np.testing.assert_array_equal(sa[k], sb[k])
    a.finish()
    res = a.result()
    assert res["best_energy"] == pytest.approx(float(ising.energy(inst, res["best_spins"].astype(np.float64))),
                                               rel=1e-12, abs=1e-9)
    a.close()
    b.close()
