"""K3 energy kernel through the C ABI against the oracle (Sec. II)."""

import numpy as np
import pytest

import synth
from oracle import ising
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu


def _spins(count, n, seed):
    r = np.random.default_rng(seed)
    return (2 * r.integers(0, 2, (count, n)) - 1).astype(np.int8)


@pytest.mark.parametrize("layout", ["dense", "csr"])
@pytest.mark.parametrize("conv,js", [("physics", 0.5), ("paper", 0.5), ("physics", 1.0)])
@pytest.mark.parametrize("hmode", ["int", "zero"])
@pytest.mark.parametrize("n", [1, 67, 300])
def test_integer_energy_is_bit_exact(gpu_ctx, layout, conv, js, hmode, n):
    inst = synth.random_sparse_instance(n, n, p=0.2, kind="int", h=hmode, convention=conv,
                                        j_scale=js, layout=layout)
    s = _spins(9, n, 1)
    E, Q, H = api.energy(gpu_ctx, inst, s, exact_parts=True)
    Eo, Qo, Ho = ising.energy_exact(inst, s.T)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(Q, Qo)
    np.testing.assert_array_equal(H, Ho)


@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_float_energy_fp64(gpu_ctx, layout):
    inst = synth.random_sparse_instance(150, 4, p=0.3, kind="float", h="float", layout=layout)
    s = _spins(5, 150, 2)
    E = api.energy(gpu_ctx, inst, s)
    np.testing.assert_allclose(E, ising.energy(inst, s.T), rtol=1e-12, atol=1e-10)


def test_bench_sized_instances(gpu_ctx):
    inst = synth.workload("er2000", 0)
    s = _spins(4, 2000, 3)
    np.testing.assert_array_equal(api.energy(gpu_ctx, inst, s), ising.energy_exact(inst, s.T)[0])
    inst = synth.workload("sk4096", 0)
    s = _spins(2, 4096, 4)
    np.testing.assert_allclose(api.energy(gpu_ctx, inst, s), ising.energy(inst, s.T), rtol=1e-12)


def test_device_memory_inputs(gpu_ctx):
    torch = pytest.importorskip("torch")
    inst = synth.random_sparse_instance(90, 5, p=0.2, kind="int", h="int", layout="dense")
    dev = synth.Instance(n=90, layout="dense", J=torch.tensor(inst.J).cuda(),
                         h=torch.tensor(inst.h).cuda(), j_scale=inst.j_scale,
                         convention=inst.convention)
    s = _spins(3, 90, 5)
    E = api.energy(gpu_ctx, dev, torch.tensor(s).cuda())
    np.testing.assert_array_equal(E.cpu().numpy(), ising.energy_exact(inst, s.T)[0])


def test_invalid_instances_are_rejected(gpu_ctx):
    inst = synth.random_sparse_instance(20, 6, p=0.4, kind="int", h="int", layout="dense")
    bad = synth.Instance(n=20, layout="dense", J=inst.J.copy(), h=inst.h, convention="physics")
    bad.J[0, 1] += 1
    with pytest.raises(api.IsingError, match="not symmetric"):
        api.energy(gpu_ctx, bad, _spins(1, 20, 0))
    bad.J = inst.J.copy()
    bad.J[3, 3] = 2
    with pytest.raises(api.IsingError, match="diagonal"):
        api.energy(gpu_ctx, bad, _spins(1, 20, 0))
    csr = inst.to_csr()
    bad = synth.Instance(n=20, layout="csr", indptr=csr.indptr, indices=csr.indices[::-1].copy(),
                         data=csr.data, convention="physics")
    with pytest.raises(api.IsingError):
        api.energy(gpu_ctx, bad, _spins(1, 20, 0))
