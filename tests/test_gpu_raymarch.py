"""The GPU ray marching baseline (Section II): its exact Euclidean distance
transform and its march, bit-exact against the oracle's."""
import numpy as np
import pytest
import torch

from paper_1705_01167_gb300 import synth
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01167_gb300 import cddt
    cddt.load()
    return cddt


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _maps():
    one = np.zeros((70, 301), np.uint8)  # columns without an occupied cell
    one[40, 17] = 1
    return gc.tiny_maps(4, seed=41) + [
        synth.rect_map(256, 256),
        synth.rect_map(333, 197, n_rects=20, seed=42),
        one,
        np.zeros((33, 65), np.uint8),
        np.ones((9, 5), np.uint8),
    ]


@pytest.mark.parametrize("mi", range(10))
def test_distance_transform_matches_oracle(G, mi):
    from oracle import oracle as O
    g = _maps()[mi]
    d = G.CDDT(dev(g), 36, 200.0)
    rm = G.RayMarch(d)
    got = rm.distances().cpu().numpy()
    assert np.array_equal(got.view(np.uint32), O.edt(g).view(np.uint32))


@pytest.mark.parametrize("mi", [5, 6, 7, 8])
def test_raymarch_matches_oracle(G, mi):
    from oracle import oracle as O
    g = _maps()[mi]
    H, W = g.shape
    mr = 300.0
    d = G.CDDT(dev(g), 108, mr)
    rm = G.RayMarch(d)
    q = np.concatenate([gc.special_queries(W, H), gc.random_queries(W, H, 20000, 43 + mi)])
    steps = torch.empty(q.shape[0], dtype=torch.int32, device="cuda")
    got = rm.calc_range_many(dev(q), steps=steps).cpu().numpy()
    want, wsteps = O.raymarch(O.edt(g), q, mr)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.array_equal(steps.cpu().numpy(), wsteps)
    # without the optional step counts, the same ranges
    got2 = rm.calc_range_many(dev(q)).cpu().numpy()
    assert np.array_equal(got2.view(np.uint32), got.view(np.uint32))


def test_raymarch_corridor_full_size(G):
    """The 2000 x 2000 corridor map of the bench: the whole transform, and
    sampled filter rays and uniform rays marched one by one by the oracle."""
    from oracle import oracle as O
    g = synth.corridor_map(2000, 2000)
    mr = 500.0
    d = G.CDDT(dev(g), 108, mr)
    rm = G.RayMarch(d)
    E = O.edt(g)
    assert np.array_equal(rm.distances().cpu().numpy().view(np.uint32), E.view(np.uint32))
    q = np.concatenate([synth.uniform_queries(g, 30000, seed=44), gc.special_queries(2000, 2000)])
    steps = torch.empty(q.shape[0], dtype=torch.int32, device="cuda")
    got = rm.calc_range_many(dev(q), steps=steps).cpu().numpy()
    want, wsteps = O.raymarch(E, q, mr)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.array_equal(steps.cpu().numpy(), wsteps)


def test_raymarch_empty_and_rebuild_after_update(G):
    """n = 0 launches nothing; the transform is a snapshot of the grid when it
    was built, and one built after an update follows the new grid."""
    from oracle import oracle as O
    g = synth.rect_map(128, 96, n_rects=10, seed=45)
    d = G.CDDT(dev(g), 36, 200.0)
    rm = G.RayMarch(d)
    out = rm.calc_range_many(torch.empty((0, 3), dtype=torch.float32, device="cuda"))
    assert out.numel() == 0
    before = rm.distances().cpu().numpy()
    xy = np.array([[5, 7], [60, 50], [100, 3]], np.int32)
    occ = np.array([1, 1, 0], np.uint8)
    d.update_cells(dev(xy), dev(occ))
    g2 = synth.apply_writes(g, xy, occ)
    assert np.array_equal(rm.distances().cpu().numpy(), before)
    rm2 = G.RayMarch(d)
    assert np.array_equal(rm2.distances().cpu().numpy().view(np.uint32), O.edt(g2).view(np.uint32))
