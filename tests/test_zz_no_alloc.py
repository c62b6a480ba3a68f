"""cddt_calc_range_many_noalloc: slice-sorted ray casting for callers that
cannot allocate device memory while they run (a host application that hands
the library a fixed memory budget, or a real-time loop that forbids
allocation after start-up).  Its scratch lives in a fixed buffer of the
library; the ranges must equal those of cddt_calc_range_many bit for bit,
call after call, whatever an earlier call left in the shared buffer.

Collected last on purpose: a run that stops at its first failure has then
already run every other test."""
import ctypes as C

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


def _noalloc(G, d, poses, out):
    """The new entry point, called through the C ABI."""
    L = G.load()
    return L.cddt_calc_range_many_noalloc(d.handle, C.c_void_p(poses.data_ptr()), C.c_void_p(out.data_ptr()),
                                          poses.shape[0], C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _reference(G, d, poses):
    """The existing entry point: cddt_calc_range_many with the slice sort."""
    L = G.load()
    out = torch.empty(poses.shape[0], dtype=torch.float32, device="cuda")
    rc = L.cddt_calc_range_many(d.handle, C.c_void_p(poses.data_ptr()), C.c_void_p(out.data_ptr()),
                                poses.shape[0], 1, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == G.CDDT_OK
    return out


def _bits(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("u16", [False, True])
def test_two_calls_in_a_row_match_the_existing_entry_point(G, oracle, u16):
    g = synth.corridor_map(512, 512, seed=61, r_min=48)
    d = G.CDDT(torch.from_numpy(g).cuda(), 200, 600.0, u16=u16)
    first_h = np.concatenate([synth.uniform_queries(g, 200000, seed=62), gc.special_queries(512, 512)])
    first = torch.from_numpy(first_h).cuda()
    second = torch.from_numpy(gc.random_queries(512, 512, 70001, 63)).cuda()
    # a small call first: it sets up the buffer's address and loads the
    # kernels, so that what follows measures the call alone
    warm = torch.empty(64, device="cuda")
    assert _noalloc(G, d, first[:64], warm) == G.CDDT_OK
    torch.cuda.synchronize()
    for i, poses in enumerate((first, second)):  # the second call is smaller than the first
        out = torch.full((poses.shape[0],), float("nan"), device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        assert _noalloc(G, d, poses, out) == G.CDDT_OK
        torch.cuda.synchronize()
        # nothing was allocated: the sorted path of cddt_calc_range_many
        # would have taken 16 bytes per query (3.2 MB here) from the device
        assert torch.cuda.mem_get_info()[0] == free_before
        want = _reference(G, d, poses)
        torch.cuda.synchronize()
        assert np.array_equal(_bits(out), _bits(want))
        if i == 0:  # and straight against the CPU oracle
            o = oracle.OracleCDDT(g, 200, 600.0, u16=u16)
            assert np.array_equal(_bits(out), o.calc_range(first_h).view(np.uint32))
    d.close()


def test_largest_batch_and_limits(G):
    g = synth.rect_map(256, 256)
    d = G.CDDT(torch.from_numpy(g).cuda(), G.NOALLOC_MAX_THETA_DISC, 300.0)
    n = G.NOALLOC_MAX_QUERIES
    poses = torch.from_numpy(gc.random_queries(256, 256, n, 64)).cuda()
    out = torch.empty(n, device="cuda")
    assert _noalloc(G, d, poses, out) == G.CDDT_OK
    assert np.array_equal(_bits(out), _bits(_reference(G, d, poses)))
    # one query past the limit is refused before any launch
    big = torch.zeros((n + 1, 3), device="cuda")
    assert _noalloc(G, d, big, torch.empty(n + 1, device="cuda")) == G.CDDT_ERR_ARG
    # an empty batch is accepted
    assert _noalloc(G, d, poses[:0], out[:0]) == G.CDDT_OK
    d.close()
    d2 = G.CDDT(torch.from_numpy(g).cuda(), G.NOALLOC_MAX_THETA_DISC + 2, 300.0)
    assert _noalloc(G, d2, poses[:10], out[:10]) == G.CDDT_ERR_ARG
    d2.close()
