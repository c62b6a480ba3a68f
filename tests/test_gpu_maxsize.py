"""Maps at the largest side the library accepts (32767 cells): the store,
random casts, the ray marcher's distance transform (its row pass then holds
three 32767-entry arrays, 196 KB, in shared memory) and march, and the
Bresenham caster, bit-exact against the oracle, in both orientations."""
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


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


@pytest.mark.parametrize("H, W", [(3, 32767), (32767, 3)])
def test_maximum_map_side(G, oracle, H, W):
    from oracle import oracle as O
    rs = synth.Stream(77)
    g = (rs.uniform(W * H) < 0.05).astype(np.uint8).reshape(H, W)
    N, mr = 16, 40000.0
    q = np.concatenate([gc.special_queries(W, H), gc.random_queries(W, H, 20000, 78)])
    for u16 in (False, True):
        d = G.CDDT(dev(g), N, mr, u16=u16)
        o = oracle.OracleCDDT(g, N, mr, u16=u16)
        _, bs, zp = d.export()
        obs_, ozp = o.export()
        assert np.array_equal(bs, obs_) and np.array_equal(bits(zp), bits(ozp)), u16
        assert np.array_equal(bits(d.calc_range_many(dev(q)).cpu().numpy()), bits(o.calc_range(q))), u16
        d.close()
    d = G.CDDT(dev(g), N, mr)
    rm = G.RayMarch(d)
    E = O.edt(g)
    assert np.array_equal(bits(rm.distances().cpu().numpy()), bits(E))
    want, wsteps = O.raymarch(E, q, mr)
    steps = torch.empty(q.shape[0], dtype=torch.int32, device="cuda")
    assert np.array_equal(bits(rm.calc_range_many(dev(q), steps=steps).cpu().numpy()), bits(want))
    assert np.array_equal(steps.cpu().numpy(), wsteps)
    assert np.array_equal(bits(d.cast_bresenham(dev(q)).cpu().numpy()), bits(O.cast_bresenham(g, q, mr)))


@pytest.mark.parametrize("H, W", [(3, 32767), (32767, 3)])
def test_maximum_map_side_prune_and_update(G, oracle, H, W):
    """Pruning and a batch of cell writes on the largest maps: the
    prune's strip enumeration and the update's merge at coordinates up to
    32767, both bit-exact against the oracle's prune and update."""
    rs = synth.Stream(79)
    g = (rs.uniform(W * H) < 0.5).astype(np.uint8).reshape(H, W)  # dense: the prune drops ~2 % of the keys
    N, mr = 36, 40000.0
    q = np.concatenate([gc.special_queries(W, H), gc.random_queries(W, H, 20000, 80)])
    xy, occ = synth.cell_toggles(g, 400, 400, seed=81)
    for u16 in (False, True):
        d = G.CDDT(dev(g), N, mr, u16=u16)
        o = oracle.OracleCDDT(g, N, mr, u16=u16)
        d.update_cells(dev(xy), dev(occ))
        assert d.status() == G.CDDT_OK
        assert o.update(xy, occ) == 0
        _, bs, zp = d.export()
        obs_, ozp = o.export()
        assert np.array_equal(bs, obs_) and np.array_equal(bits(zp), bits(ozp)), ("update", u16)
        d.prune()
        o.prune()
        _, bs, zp = d.export()
        obs_, ozp = o.export()
        assert np.array_equal(bs, obs_) and np.array_equal(bits(zp), bits(ozp)), ("prune", u16)
        assert np.array_equal(bits(d.calc_range_many(dev(q)).cpu().numpy()), bits(o.calc_range(q))), u16
        d.close()
