"""The filter steps around the sensor model (motion model, low-variance
resampling) against the oracle, and one full step (motion, sensor weights,
resampling) captured in a CUDA graph."""
import numpy as np
import pytest
import torch

from paper_1705_01167_gb300 import synth

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


def _case(seed, sizes):
    rs = np.random.default_rng(seed)
    P = int(sum(sizes))
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    parts = np.stack([rs.uniform(0, 500, P), rs.uniform(0, 400, P), rs.uniform(0, 2 * np.pi, P)], 1)
    parts[::7, 2] = rs.uniform(-0.3, 0.0, parts[::7].shape[0])  # headings just below 0 and past 2 pi
    parts[1::7, 2] = rs.uniform(6.2, 6.5, parts[1::7].shape[0])
    odom = np.stack([rs.normal(0, 1.5, len(sizes)), rs.normal(0, 0.5, len(sizes)),
                     rs.normal(0, 0.2, len(sizes))], 1)
    noise = rs.normal(0, 0.1, (P, 3))
    return (parts.astype(np.float32), seg, odom.astype(np.float32), noise.astype(np.float32))


def test_motion_matches_oracle(G, oracle):
    parts, seg, odom, noise = _case(1, [1, 33, 0, 500, 1200, 7])
    got = G.motion(dev(parts), dev(seg), dev(odom), dev(noise)).cpu().numpy()
    want = oracle.motion(parts, seg, odom, noise)
    # float32 evaluation (sincosf, 2 ulp; 6 rounded operations) against the
    # float64 form rounded once
    f = np.searchsorted(seg, np.arange(parts.shape[0]), side="right") - 1
    mag = np.abs(parts[:, :2]).max(1) + np.abs(odom[f, :2]).sum(1) + np.abs(noise[:, :2]).sum(1) + 1.0
    tol = 16 * 2.0 ** -24 * mag
    assert (np.abs(got[:, 0] - want[:, 0]) <= tol).all()
    assert (np.abs(got[:, 1] - want[:, 1]) <= tol).all()
    dth = np.abs(np.mod(got[:, 2].astype(np.float64) - want[:, 2] + np.pi, 2 * np.pi) - np.pi)
    assert (dth <= 16 * 2.0 ** -24 * 8.0).all()
    assert (got[:, 2] >= 0).all() and (got[:, 2] < np.float32(2 * np.pi) + 1e-6).all()


def test_resampling_matches_oracle(G, oracle):
    sizes = [1, 2, 64, 0, 2500, 777]
    parts, seg, _, _ = _case(2, sizes)
    rs = np.random.default_rng(3)
    logw = rs.normal(-300.0, 4.0, parts.shape[0]).astype(np.float32)
    logw[5::11] = -np.inf  # zero weights
    u0 = rs.uniform(0, 1, len(sizes)).astype(np.float32)
    idx_t = torch.empty(parts.shape[0], dtype=torch.int32, device="cuda")
    out, idx = G.resample(dev(parts), dev(logw), dev(seg), dev(u0), index=idx_t)
    got = idx.cpu().numpy().astype(np.int64)
    want, margin = oracle.resample_indices(logw, seg, u0)
    bad = got != want
    # only decisions at a near-tie of a running sum may differ (another
    # summation order rounds them otherwise)
    assert (margin[bad] < 1e-12).all(), (np.flatnonzero(bad)[:5], margin[bad][:5])
    f = np.searchsorted(seg, np.arange(parts.shape[0]), side="right") - 1
    assert np.array_equal(out.cpu().numpy(), parts[seg[f] + got])
    assert np.isfinite(logw[seg[f] + got]).all()  # zero-weight particles are never drawn
    out2, idx2 = G.resample(dev(parts), dev(logw), dev(seg), dev(u0),
                            index=torch.empty_like(idx_t))
    assert torch.equal(idx2, idx) and torch.equal(out2, out)


def test_resampling_of_undefined_weights(G, oracle):
    """Filters whose log-weights are all -inf, all NaN, partly NaN and partly
    +inf: the same indices as the oracle (reading R1), and no NaN in the
    output."""
    sizes = [33, 40, 257, 64]
    parts, seg, _, _ = _case(3, sizes)
    rs = np.random.default_rng(9)
    logw = rs.normal(-50.0, 3.0, parts.shape[0]).astype(np.float32)
    logw[seg[0]:seg[1]] = -np.inf
    logw[seg[1]:seg[2]] = np.nan
    logw[seg[2]:seg[3]:4] = np.nan
    logw[seg[3] + 7] = logw[seg[3] + 50] = np.inf
    u0 = rs.uniform(0, 1, len(sizes)).astype(np.float32)
    idx_t = torch.empty(parts.shape[0], dtype=torch.int32, device="cuda")
    out, idx = G.resample(dev(parts), dev(logw), dev(seg), dev(u0), index=idx_t)
    got = idx.cpu().numpy().astype(np.int64)
    want, margin = oracle.resample_indices(logw, seg, u0)
    assert np.array_equal(got[margin >= 1e-12], want[margin >= 1e-12])
    assert np.array_equal(got[seg[0]:seg[2]], np.concatenate([np.arange(33), np.arange(40)]))
    assert np.isfinite(out.cpu().numpy()).all()


def test_filter_step_in_a_graph(G, oracle):
    """Motion, batched sensor weights and resampling of 3 filters as one
    CUDA graph, replayed: the same as the steps run one by one."""
    g = synth.rect_map(200, 160, seed=81)
    mr = 250.0
    d = G.CDDT(dev(g), 72, mr)
    o = oracle.OracleCDDT(g, 72, mr)
    bo_np = synth.beam_offsets(61)
    bo = dev(bo_np)
    D = synth.pair_offset(61)
    sizes = [300, 1000, 450]
    P = sum(sizes)
    seg = dev(np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64))
    gts = synth.uniform_particles(g, 3, seed=82)
    parts0 = np.concatenate([synth.tracking_particles(gts[f].astype(np.float64), n, seed=83 + f)
                             for f, n in enumerate(sizes)])
    from tests import gpu_cases as gc
    obs = torch.stack([dev(gc.observations(o, gts[f], bo_np, mr, seed=90 + f)) for f in range(3)])
    odom = dev(np.array([[1.0, 0.0, 0.05], [0.5, 0.2, -0.1], [0.0, 0.0, 0.0]], np.float32))
    noise = dev(np.random.default_rng(4).normal(0, 0.05, (P, 3)).astype(np.float32))
    u0 = dev(np.array([0.25, 0.5, 0.75], np.float32))
    m = G.beam_model(mr)
    offs = np.concatenate([[0], np.cumsum(sizes)])

    def make():
        a = dev(parts0)
        b = torch.empty_like(a)
        logw = torch.empty(P, device="cuda")
        plan = G.Plan([dict(map=d, particles=a[offs[f]:offs[f + 1]], beam_off=bo, obs=obs[f], model=m,
                            logw=logw[offs[f]:offs[f + 1]], pair_offset=D) for f in range(3)])
        scratch = torch.empty(P, dtype=torch.float64, device="cuda")

        def step():
            G.motion(a, seg, odom, noise)
            plan.run()
            G.resample(a, logw, seg, u0, out=b, scratch=scratch)
        return a, b, logw, plan, step

    a1, b1, lw1, p1, step1 = make()
    step1()
    torch.cuda.synchronize()
    a2, b2, lw2, p2, step2 = make()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p2.run()  # builds the plan's items outside the capture
    torch.cuda.current_stream().wait_stream(s)
    a2.copy_(dev(parts0))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step2()
    a2.copy_(dev(parts0))
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(a1, a2) and torch.equal(lw1, lw2) and torch.equal(b1, b2)
    # the sensor weights of the moved particles match the oracle's
    want = np.concatenate([o.sensor_weights(a1[offs[f]:offs[f + 1]].cpu().numpy(), bo_np,
                                            obs[f].cpu().numpy(), oracle.beam_model(mr))
                           for f in range(3)])
    got = lw1.cpu().numpy().astype(np.float64)
    assert (np.abs(got - want) <= 1e-5 * np.maximum(1.0, np.abs(want))).all()
    p1.close()
    p2.close()
