"""The seeded generators produce valid leaf-only octrees (checked by the
oracle's validation), sources on the 2^-53 lattice inside the box, and the
stated field statistics."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import torchgen


def test_numpy_workloads_are_valid():
    c, src, nside = synth.workload_uniform32()
    assert c.n_leaves == 32 ** 3 and nside == 1
    assert oracle.validate(c.keys, c.levels, c.extent) == oracle.OK
    assert abs(np.log(c.n_total).std() - 1.0) < 1e-9
    a = synth.amr_cloud(24, 2, 80.0, 1.5, 7, fracs=(1.0, 0.4))
    assert oracle.validate(a.keys, a.levels, a.extent) == oracle.OK
    s = synth.mass_weighted_sources(a, 500, 3)
    q = s * 2.0 ** 53
    assert np.all(q == np.floor(q)) and np.all(s >= 0) and np.all(s < a.extent[0] * 2.0 ** -21)


@pytest.mark.parametrize("base,nref,pct", [(16, 2, 80.0), (24, 3, 80.0), (32, 1, 85.0)])
def test_torch_amr_clouds_are_valid(base, nref, pct):
    k, l, d, n, ext = torchgen.amr_cloud(base, nref, pct, 1.5, 5, fracs=(1.0, 0.4), device="cpu", max_field=64)
    assert oracle.validate(k.numpy().view(np.uint64), l.numpy(), ext) == oracle.OK
    assert d.shape == (k.numel(), 2) and torch.all(d > 0)
    c = torchgen.leaf_centres(k, l)
    assert torch.all(c >= 0) and torch.all(c < ext[0] * 2.0 ** -21)
    s = torchgen.mass_weighted_sources(k, l, n, 2000, 9)
    q = s * 2.0 ** 53
    assert torch.all(q == torch.floor(q)) and torch.all(s < ext[0] * 2.0 ** -21)


def test_torch_uniform_cloud_is_morton_ordered():
    k, l, d, n = torchgen.uniform_cloud(4, 2.0, 5, device="cpu")
    assert oracle.validate(k.numpy().view(np.uint64), l.numpy()) == oracle.OK
    assert abs(float(torch.log(n).std()) - 2.0) < 1e-9
    cen = torchgen.uniform_centres(4, torch.arange(16 ** 3))
    want = synth.leaf_centres(synth.Cloud(k.numpy().view(np.uint64), l.numpy(), np.zeros((4096, 1)), (1 << 21,) * 3))
    assert np.array_equal(cen.numpy(), want)
