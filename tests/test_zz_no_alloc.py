"""ising_energy_noalloc, the energy entry point that allocates nothing (for
callers that cannot allocate device memory), against ising_energy on the
same inputs. This file is collected last on purpose."""

import dataclasses

import numpy as np
import pytest

import synth
from paper_2312_05837_gb300 import api

pytestmark = pytest.mark.gpu


def _device(inst, torch):
    def t(x):
        return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return dataclasses.replace(inst, J=t(inst.J), indptr=t(inst.indptr),
                               indices=t(inst.indices), data=t(inst.data), h=t(inst.h))


def _cases():
    return [
        ("dense_int8", synth.er_dense(300, 1, p=0.05, weights="pm1"), True),
        ("csr_int_h", synth.random_sparse_instance(257, 2, p=0.05, kind="int", h="int",
                                                   convention="paper", j_scale=0.5), True),
        ("dense_float_h", synth.sk_dense(190, 3, 0.1, np.float32, h_std=0.3), False),
        ("csr_float", synth.random_sparse_instance(222, 4, p=0.04, kind="float", h="float"),
         False),
    ]


@pytest.mark.parametrize("name,inst,exact", _cases())
def test_matches_the_allocating_entry_point_on_two_calls(gpu_ctx, name, inst, exact):
    torch = pytest.importorskip("torch")
    dev = _device(inst, torch)
    r = np.random.default_rng(7)
    for call in range(2):  # the second call reuses the scratch the first one left behind
        count = 5 + 3 * call
        s = (2 * r.integers(0, 2, (count, inst.n)) - 1).astype(np.int8)
        ref = api.energy(gpu_ctx, inst, s)
        out = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
        api.energy_noalloc(dev, torch.from_numpy(s).cuda(), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if exact:
            np.testing.assert_array_equal(got, ref)
        else:
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_rejects_work_beyond_the_scratch(gpu_ctx):
    torch = pytest.importorskip("torch")
    inst = synth.er_dense(4096, 5, p=0.001, weights="one")
    dev = _device(inst, torch)
    count = 3000  # 3000 * 64 chunks * 16 bytes > 2 MiB
    s = torch.ones((count, inst.n), dtype=torch.int8, device="cuda")
    out = torch.empty(count, dtype=torch.float64, device="cuda")
    with pytest.raises(api.IsingError, match="2 MiB"):
        api.energy_noalloc(dev, s, out)
