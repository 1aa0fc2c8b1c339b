"""Key searches inside mixed coarse cells: with the coarse table capped
shallow, most lookups of a deep random octree search the sorted keys; the
search must find the oracle's leaves (paths bit-exact, FP64 columns bitwise,
F32-Kahan within 1e-5), for sources on and off the leaf lattice, in both ray
orders."""
import numpy as np
import pytest

import oracle
from tinytrees import leaf_boxes, random_octree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_09882_gb300 as rt
    yield rt
    rt.set_table_cap(-1)


def _dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


@pytest.mark.parametrize("cap", [0, 2, 4])
def test_search_forms_match_oracle(rt, cap):
    rng = np.random.default_rng(1500 + cap)
    keys, lev, _ = random_octree(rng, 1, 8, 0.42)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2))
    lo, hi = leaf_boxes(keys, lev)
    src = np.concatenate([rng.random((300, 3)), 0.5 * (lo + hi)[::7]])
    rt.set_table_cap(cap)
    tree = rt.Octree(_dev(keys), _dev(lev))
    rt.set_table_cap(-1)
    for nside in (1, 2):
        dirs = oracle.healpix(nside)
        want, h_or, n_or = oracle.trace(keys, lev, dens, src, dirs)
        for sel in (slice(None), slice(0, 20)):  # direction-major and source-major ray orders
            for mode in ("fp64", "f32k"):
                nseg, hsh = rt.trace_paths(tree, _dev(src[sel]), nside, mode)
                np.testing.assert_array_equal(nseg.cpu().numpy().astype(np.uint64), n_or[sel])
                np.testing.assert_array_equal(hsh.cpu().numpy().view(np.uint64), h_or[sel])
                d = _dev(dens if mode == "fp64" else dens.astype(np.float32))
                got = rt.trace_columns(tree, _dev(src[sel]), nside, d, mode).double().cpu().numpy()
                if mode == "fp64":
                    np.testing.assert_array_equal(got, want[sel])
                else:
                    assert np.all(np.abs(got - want[sel]) <= 1e-5 * np.abs(want[sel]) + 1e-30)
        assert tree.stats()["status"] == 0
    tree.close()
