"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times, on outputs the oracle can compute one by one
(sampled particles, queries and bins) or in full where it is fast enough.
Observed ranges are cast by the oracle (brute force on the largest maps)."""
import math

import numpy as np
import pytest
import torch

from paper_1705_01167_gb300 import synth, workloads as WL

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


def bits_equal(a, b):
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def logw_close(got, want, rtol=1e-5):
    got = np.asarray(got, np.float64)
    return np.all(np.abs(got - want) <= rtol * np.maximum(1.0, np.abs(want)))


def grad_close(got, want, scale, rtol=1e-5):
    """Within rtol of the float64 oracle relative to the sum of the per-beam
    term magnitudes, and relative to |g| where that sum is at most 10 |g|."""
    err = np.linalg.norm(np.asarray(got, np.float64) - want, axis=1)
    gn, sn = np.linalg.norm(want, axis=1), np.linalg.norm(scale, axis=1)
    mild = (gn > 0) & (sn <= 10 * gn)
    return (np.all(err <= rtol * np.maximum(sn, 1e-6)) and mild.sum() >= len(gn) // 2
            and np.all(err[mild] <= rtol * gn[mild]))


def obs_from(ranges, noise, mr):
    return np.clip(ranges.astype(np.float64) + noise, 0, mr).astype(np.float32)


# ------------------------------------------------------------------ 2000 x 2000

@pytest.fixture(scope="module")
def corridor(G, oracle):
    w = WL.corridor2000(sweep=200_000)
    o = oracle.OracleCDDT(w["grid"], w["theta_disc"], w["max_range"])
    r = o.calc_range(WL.gt_queries(w["gt"], w["beam_off"]), nthreads=16).reshape(len(w["gt"]), -1)
    w["obs"] = obs_from(r, w["noise"], w["max_range"])
    return w, o


def test_corridor2000_store_and_sweep(G, oracle, corridor):
    w, o = corridor
    d = G.CDDT(dev(w["grid"]), w["theta_disc"], w["max_range"])
    sb, bs, zp = d.export()
    obs_, ozp = o.export()
    assert np.array_equal(bs, obs_)
    assert bits_equal(zp, ozp)
    q = w["sweep"]
    want = o.calc_range(q, nthreads=16)
    qd = dev(q)
    assert bits_equal(d.calc_range_many(qd).cpu().numpy(), want)
    assert bits_equal(d.calc_range_many(qd, sort_by_slice=True).cpu().numpy(), want)
    d.set_search(G.SEARCH_BINARY)
    assert bits_equal(d.calc_range_many(qd).cpu().numpy(), want)


def test_corridor2000_batched_plan(G, oracle, corridor):
    """The benchmark's launch: 200 filter steps x 2500 particles in one
    autotuned persistent launch; every 37th particle checked."""
    w, o = corridor
    d = G.CDDT(dev(w["grid"]), w["theta_disc"], w["max_range"])
    S, P = w["parts"].shape[:2]
    parts = dev(w["parts"].reshape(-1, 3))
    bo = dev(w["beam_off"])
    obs = dev(w["obs"])
    logw = torch.full((S * P,), float("nan"), device="cuda")
    m = G.beam_model(w["max_range"])
    plan = G.Plan([dict(map=d, particles=parts[t * P:(t + 1) * P], beam_off=bo, obs=obs[t], model=m,
                        logw=logw[t * P:(t + 1) * P], pair_offset=w["D"]) for t in range(S)])
    plan.autotune()
    plan.run()
    got = logw.cpu().numpy().reshape(S, P)
    om = oracle.beam_model(w["max_range"])
    for t in range(0, S, 7):
        idx = np.arange(t % 37, P, 37)
        want = o.sensor_weights(w["parts"][t][idx], w["beam_off"], w["obs"][t], om, nthreads=16)
        assert logw_close(got[t][idx], want), t
    plan.close()


def test_corridor2000_u16(G, oracle, corridor):
    """The 16-bit store at full size (reading S7): the zero points, the
    200 000-query sweep by tree and binary search, and the fused plan in its
    autotuned shape on sampled particles, against the oracle's 16-bit CDDT."""
    w, _ = corridor
    o = oracle.OracleCDDT(w["grid"], w["theta_disc"], w["max_range"], u16=True)
    d = G.CDDT(dev(w["grid"]), w["theta_disc"], w["max_range"], u16=True)
    _, bs, zp = d.export()
    obs_, ozp = o.export()
    assert np.array_equal(bs, obs_)
    assert bits_equal(zp, ozp)
    q = w["sweep"]
    want = o.calc_range(q, nthreads=16)
    qd = dev(q)
    assert bits_equal(d.calc_range_many(qd).cpu().numpy(), want)
    d.set_search(G.SEARCH_BINARY)
    assert bits_equal(d.calc_range_many(qd).cpu().numpy(), want)
    d.set_search(G.SEARCH_TREE)
    S, P = w["parts"].shape[:2]
    parts = dev(w["parts"].reshape(-1, 3))
    bo = dev(w["beam_off"])
    obs = dev(w["obs"])
    logw = torch.full((S * P,), float("nan"), device="cuda")
    m = G.beam_model(w["max_range"])
    plan = G.Plan([dict(map=d, particles=parts[t * P:(t + 1) * P], beam_off=bo, obs=obs[t], model=m,
                        logw=logw[t * P:(t + 1) * P], pair_offset=w["D"]) for t in range(S)])
    plan.autotune()
    plan.run()
    got = logw.cpu().numpy().reshape(S, P)
    om = oracle.beam_model(w["max_range"])
    for t in range(3, S, 11):
        idx = np.arange(t % 41, P, 41)
        want = o.sensor_weights(w["parts"][t][idx], w["beam_off"], w["obs"][t], om, nthreads=16)
        assert logw_close(got[t][idx], want), t
    plan.close()


def test_corridor2000_pruned(G, oracle, corridor):
    w, o = corridor
    d = G.CDDT(dev(w["grid"]), w["theta_disc"], w["max_range"])
    q = dev(w["sweep"])
    before = d.calc_range_many(q).cpu().numpy()
    sb0, bs0, zp0 = d.export()
    d.prune()
    sb, bs, zp = d.export()
    assert d.stats()["n_zero_points"] < zp0.size
    # sampled bins against the pruning rule evaluated for that bin alone
    eps = oracle.prune_eps(2000, 2000)
    obs_, ozp = o.export()
    rs = synth.Stream(5150)
    nonempty = np.flatnonzero(np.diff(obs_) > 0)
    for g in nonempty[rs.integers(40, 0, nonempty.size - 1)]:
        sl = int(np.searchsorted(sb0, g, side="right") - 1)
        b = int(g - sb0[sl])
        keep = o.params.prune_bin(w["grid"], sl, b, ozp[obs_[g]:obs_[g + 1]], eps)
        assert bits_equal(zp[bs[g]:bs[g + 1]], ozp[obs_[g]:obs_[g + 1]][keep]), (sl, b)
    after = d.calc_range_many(q).cpu().numpy()
    assert bits_equal(after, before)  # every sweep query starts in a free cell


def test_corridor2000_differentiation(G, oracle):
    """4096 x 61 and 1024 x 1081 beams: log-weights and the adjoint against
    the float64 oracle, then 10 gradient refinement steps x += eta g/|g|
    taken on the GPU, checked again at the refined poses."""
    w = WL.diff2000()
    o = oracle.OracleCDDT(w["grid"], w["theta_disc"], w["max_range"])
    d = G.CDDT(dev(w["grid"]), w["theta_disc"], w["max_range"])
    m, om = G.beam_model(w["max_range"]), oracle.beam_model(w["max_range"])
    for sc in w["scans"]:
        r = o.calc_range(WL.gt_queries(w["gt"], sc["beam_off"]), nthreads=16)
        obs = obs_from(r, sc["noise"], w["max_range"])
        parts = dev(sc["parts"]).requires_grad_(True)
        bo, ob = dev(sc["beam_off"]), dev(obs)
        logw = G.SensorWeights.apply(parts, d, bo, ob, m, sc["D"])
        assert logw_close(logw.detach().cpu().numpy(), o.sensor_weights(sc["parts"], sc["beam_off"], obs, om, nthreads=16))
        logw.sum().backward()
        want, scale = o.sensor_grad(sc["parts"], sc["beam_off"], obs, om, nthreads=16)
        assert grad_close(parts.grad[:, :2].cpu().numpy(), want, scale)
        x = parts.detach().clone()
        for _ in range(w["refine_steps"]):
            lw, g = d.sensor_weights_fwd_bwd(x, bo, ob, m, sc["D"])
            n = torch.linalg.norm(g, dim=1, keepdim=True).clamp_min(1e-12)
            x[:, :2] += w["eta"] * g / n
        xs = x.cpu().numpy()
        lw, g = d.sensor_weights_fwd_bwd(x, bo, ob, m, sc["D"])
        want, scale = o.sensor_grad(xs, sc["beam_off"], obs, om, nthreads=16)
        assert grad_close(g.cpu().numpy(), want, scale)
        assert logw_close(lw.cpu().numpy(), o.sensor_weights(xs, sc["beam_off"], obs, om, nthreads=16))


def refine_move(x, g, eta):
    """One refinement step as cddt_plan_refine takes it, in float32:
    (x, y) += eta g / max(|g|, 1e-12), each operation correctly rounded."""
    x = np.array(x, np.float32, copy=True)
    gx, gy = g[:, 0].astype(np.float32), g[:, 1].astype(np.float32)
    n = np.sqrt(gx * gx + gy * gy)
    s = np.float32(eta) / np.maximum(n, np.float32(1e-12))
    x[:, 0] = x[:, 0] + gx * s
    x[:, 1] = x[:, 1] + gy * s
    return x


def test_corridor2000_plan_refinement(G, oracle):
    """The diff2000 workload through one plan: both filters (4096 x 61 and
    1024 x 1081 beams) take their 10 gradient refinement steps in one launch
    (cddt_plan_refine).  Every step is checked: the run of k steps ends at the
    pose of the run of k - 1 steps moved by that run's own gradient (bit for
    bit), and its log-weights and gradients match the float64 oracle at that
    pose; lanes per particle 1, 8, 128, 256 (a particle over several warps)
    and the automatic choice agree."""
    w = WL.diff2000()
    o = oracle.OracleCDDT(w["grid"], w["theta_disc"], w["max_range"])
    d = G.CDDT(dev(w["grid"]), w["theta_disc"], w["max_range"])
    m, om = G.beam_model(w["max_range"]), oracle.beam_model(w["max_range"])
    filters, host = [], []
    for sc in w["scans"]:
        r = o.calc_range(WL.gt_queries(w["gt"], sc["beam_off"]), nthreads=16)
        obs = obs_from(r, sc["noise"], w["max_range"])
        P = sc["parts"].shape[0]
        filters.append(dict(map=d, particles=dev(sc["parts"]), beam_off=dev(sc["beam_off"]), obs=dev(obs), model=m,
                            logw=torch.empty(P, device="cuda"), pair_offset=sc["D"],
                            grad_xy=torch.empty((P, 2), device="cuda"),
                            particles_out=torch.empty((P, 3), device="cuda")))
        host.append((sc, obs))
    plan = G.Plan(filters)
    eta = w["eta"]
    for tpp in (0, 1, 8, 128, 256):
        prev = None
        for k in range(w["refine_steps"] + 1 if tpp == 0 else 3):
            plan.refine(k, eta, tpp=tpp)
            torch.cuda.synchronize()
            cur = []
            for f, (sc, obs) in zip(filters, host):
                x = f["particles_out"].cpu().numpy()
                g = f["grad_xy"].cpu().numpy()
                lw = f["logw"].cpu().numpy()
                assert np.array_equal(x[:, 2].view(np.uint32), sc["parts"][:, 2].view(np.uint32))
                want, scale = o.sensor_grad(x, sc["beam_off"], obs, om, nthreads=16)
                assert grad_close(g, want, scale), (tpp, k, sc["B"])
                assert logw_close(lw, o.sensor_weights(x, sc["beam_off"], obs, om, nthreads=16)), (tpp, k, sc["B"])
                cur.append((x, g))
            if prev is not None:
                for (x0, g0), (x1, _) in zip(prev, cur):
                    assert bits_equal(x1, refine_move(x0, g0, eta)), (tpp, k)
            prev = cur
        if tpp == 0:  # the refined poses moved: ten steps of 0.1 cell
            moved = np.linalg.norm(prev[0][0][:, :2] - host[0][0]["parts"][:, :2], axis=1)
            assert np.median(moved) > 0.5
    plan.close()
    d.close()


# ------------------------------------------------------------------ 4000 x 4000 updates

def test_update4000(G, oracle):
    """4000 x 4000, theta_disc 360: three steps of 5000 inserts + 5000
    removes through cddt_update_cells, each followed by sampled checks of
    bins (the definition scanned over the map) and ray casts (brute force);
    the final store equals a fresh GPU build of the final grid."""
    w = WL.update4000(steps=3, particles=100_000)
    N, mr = w["theta_disc"], w["max_range"]
    d = G.CDDT(dev(w["grid"]), N, mr)
    p = oracle.Params(4000, 4000, N, mr)
    cur = w["grid"]
    rs = synth.Stream(4001)
    for t, (xy, occ) in enumerate(w["writes"]):
        d.update_cells(dev(xy), dev(occ))
        assert d.status() == G.CDDT_OK
        cur = synth.apply_writes(cur, xy, occ)
        sb, bs, zp = d.export()
        # bins touched by the writes, and random ones
        k = rs.integers(6, 0, xy.shape[0] - 1)
        picks = []
        for (x, y) in xy[k]:
            sl = int(rs.integers(1, 0, N // 2 - 1)[0])
            yr = np.float32(np.float32(y) * p.c[sl]) - np.float32(np.float32(x) * p.s[sl])
            picks.append((sl, int(np.floor(yr + np.float32(0.5))) + int(p.T[sl])))
        for g in rs.integers(4, 0, int(sb[-1]) - 1):
            sl = int(np.searchsorted(sb, g, side="right") - 1)
            picks.append((sl, int(g - sb[sl])))
        for sl, b in picks:
            g = int(sb[sl]) + b
            assert bits_equal(zp[bs[g]:bs[g + 1]], p.bin_brute(cur, sl, b)), (t, sl, b)
    # sampled sensor-model ranges against the brute-force caster
    parts = w["parts"]
    r = p.calc_range_brute(cur, WL.gt_queries(w["gt"], w["beam_off"]), nthreads=16)
    obs = obs_from(r.reshape(1, -1), w["noise"], mr)[0]
    m = G.beam_model(mr)
    logw, ranges = d.sensor_weights(dev(parts), dev(w["beam_off"]), dev(obs), m, w["D"], want_ranges=True)
    ranges = ranges.cpu().numpy()
    sel = rs.integers(96, 0, parts.shape[0] - 1)
    q = np.concatenate([np.stack([np.full(61, parts[i, 0]), np.full(61, parts[i, 1]),
                                  (parts[i, 2] + w["beam_off"]).astype(np.float32)], 1) for i in sel]).astype(np.float32)
    want = p.calc_range_brute(cur, q, nthreads=16)
    assert bits_equal(ranges[sel].reshape(-1), want)
    fresh = G.CDDT(dev(cur), N, mr)
    a, b = d.export(), fresh.export()
    assert np.array_equal(a[1], b[1]) and bits_equal(a[2], b[2])


# ------------------------------------------------------------------ 64 batched maps

def test_batched64(G, oracle):
    """64 maps 512^2 .. 4096^2, theta_disc 100 .. 360, 500 .. 10000
    particles: one autotuned persistent launch (and its graph replay) against
    per-filter launches on every map, and against the oracle on the six
    smallest maps."""
    w = WL.batched64()
    bo = dev(w["beam_off"])
    D = w["D"]
    filters, handles, per = [], [], []
    small = sorted(range(len(w["maps"])), key=lambda i: w["maps"][i]["grid"].size)[:6]
    for mi, mp in enumerate(w["maps"]):
        g = mp["grid"]
        d = G.CDDT(dev(g), mp["theta_disc"], mp["max_range"])
        p = oracle.Params(g.shape[1], g.shape[0], mp["theta_disc"], mp["max_range"])
        r = p.calc_range_brute(g, WL.gt_queries(mp["gt"], w["beam_off"]), nthreads=16)
        obs = obs_from(r.reshape(1, -1), mp["noise"], mp["max_range"])[0]
        parts = mp["parts"][0]
        m = G.beam_model(mp["max_range"])
        logw = torch.full((parts.shape[0],), float("nan"), device="cuda")
        filters.append(dict(map=d, particles=dev(parts), beam_off=bo, obs=dev(obs), model=m, logw=logw, pair_offset=D))
        handles.append(d)
        per.append((parts, obs))
    plan = G.Plan(filters)
    plan.autotune()
    plan.run()
    torch.cuda.synchronize()
    got = [f["logw"].cpu().numpy() for f in filters]
    for f in filters:
        f["logw"].fill_(float("nan"))
    plan.launch_graph()
    torch.cuda.synchronize()
    for f, g0 in zip(filters, got):
        assert np.array_equal(f["logw"].cpu().numpy(), g0)  # the replay is the same launch
    for f, g0 in zip(filters, got):
        single = f["map"].sensor_weights(f["particles"], bo, f["obs"], f["model"], D).cpu().numpy()
        assert logw_close(g0, single.astype(np.float64))
    for mi in small:
        mp = w["maps"][mi]
        o = oracle.OracleCDDT(mp["grid"], mp["theta_disc"], mp["max_range"])
        parts, obs = per[mi]
        idx = np.arange(0, parts.shape[0], 11)
        want = o.sensor_weights(parts[idx], w["beam_off"], obs, oracle.beam_model(mp["max_range"]), nthreads=16)
        assert logw_close(got[mi][idx], want), mi
    # the largest map (side 4096 if drawn, the largest theta_disc among the
    # largest sides): 96 sampled particles' ranges against the brute-force
    # definition (every edge cell scanned, no store) bit for bit, and the
    # batched launch's log-weights against the float64 beam model of them
    big = max(range(len(w["maps"])), key=lambda i: (w["maps"][i]["grid"].size, w["maps"][i]["theta_disc"]))
    mp = w["maps"][big]
    parts, obs = per[big]
    sel = np.unique(np.linspace(0, parts.shape[0] - 1, 96).astype(np.int64))
    f = filters[big]
    _, ranges = f["map"].sensor_weights(dev(parts[sel]), bo, f["obs"], f["model"], D, want_ranges=True)
    q = np.concatenate([np.stack([np.full(61, parts[i, 0]), np.full(61, parts[i, 1]),
                                  (parts[i, 2] + w["beam_off"]).astype(np.float32)], 1) for i in sel]).astype(np.float32)
    p = oracle.Params(mp["grid"].shape[1], mp["grid"].shape[0], mp["theta_disc"], mp["max_range"])
    brute = p.calc_range_brute(mp["grid"], q, nthreads=16)
    assert bits_equal(ranges.cpu().numpy().reshape(-1), brute), (big, mp["grid"].shape, mp["theta_disc"])
    pz, _ = oracle.beam_eval(oracle.beam_model(mp["max_range"]), np.tile(obs, sel.size), brute.astype(np.float64))
    assert logw_close(got[big][sel], np.log(pz).reshape(sel.size, -1).sum(1)), big
    plan.close()
