"""The persistent batched launch (many maps and filters of uneven sizes in one
launch, optionally replayed as a CUDA graph) against the CPU oracle."""
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


def _close(got, want, rtol=1e-5):
    got = np.asarray(got, np.float64)
    assert np.all(np.abs(got - want) <= rtol * np.maximum(1.0, np.abs(want))), (got[:4], want[:4])


@pytest.fixture(scope="module")
def batch(G, oracle):
    """Maps of different sizes, theta discretisations and key types, each
    with one or more filters of different particle counts and scans."""
    specs = [  # (generator, W, H, N, max_range, u16, [(P, B), ...])
        ("rect", 256, 256, 108, 300.0, False, [(1000, 61), (33, 61), (1, 7)]),
        ("corr", 512, 384, 120, 400.0, False, [(2500, 61), (517, 1081)]),
        ("corr", 320, 320, 64, 250.0, True, [(700, 61), (5, 2)]),
        ("rect", 64, 64, 16, 80.0, False, [(0, 61), (64, 61)]),
    ]
    maps, filters, refs = [], [], []
    for mi, (kind, W, H, N, mr, u16, fl) in enumerate(specs):
        g = synth.rect_map(W, H, seed=900 + mi) if kind == "rect" else synth.corridor_map(W, H, seed=900 + mi, r_min=48)
        d = G.CDDT(dev(g), N, mr, u16=u16)
        o = oracle.OracleCDDT(g, N, mr, u16=u16)
        maps.append((d, o))
        for fi, (P, B) in enumerate(fl):
            bo = synth.beam_offsets(B)
            D = synth.pair_offset(B)
            gt = synth.uniform_particles(g, 1, seed=1000 + 10 * mi + fi)[0]
            obs = gc.observations(o, gt, bo, mr, seed=2000 + 10 * mi + fi)
            parts = synth.tracking_particles(gt.astype(np.float64), P, seed=3000 + 10 * mi + fi) if P else np.zeros((0, 3), np.float32)
            m = G.beam_model(mr)
            f = dict(map=d, particles=dev(parts).reshape(-1, 3), beam_off=dev(bo), obs=dev(obs), model=m,
                     logw=torch.full((max(P, 1),), float("nan"), device="cuda")[:P], pair_offset=D)
            filters.append(f)
            want = o.sensor_weights(parts, bo, obs, oracle.beam_model(mr), nthreads=8) if P else np.zeros(0)
            refs.append(want)
    return maps, filters, refs


def _check(filters, refs):
    torch.cuda.synchronize()
    for f, want in zip(filters, refs):
        _close(f["logw"].cpu().numpy(), want)


def test_plan_run_matches_oracle(G, batch):
    maps, filters, refs = batch
    plan = G.Plan(filters)
    assert plan.items > len([f for f in filters if f["particles"].shape[0]])
    for tpp in (1, 2, 4, 8, 16, 32):
        for block in (256, 512):
            for regcap in (0, 1):
                for f in filters:
                    f["logw"].fill_(float("nan"))
                plan.set_shape(tpp, block // tpp * 2 if tpp < 8 else 64 if tpp == 8 else block // tpp, block, regcap)
                plan.run()
                _check(filters, refs)
    plan.close()


def test_plan_autotune_and_graph(G, batch):
    maps, filters, refs = batch
    plan = G.Plan(filters)
    shape = plan.autotune()
    assert shape["tpp"] in (1, 2, 4, 8, 16, 32)
    for f in filters:
        f["logw"].fill_(float("nan"))
    plan.launch_graph()
    _check(filters, refs)
    for f in filters:
        f["logw"].fill_(float("nan"))
    plan.launch_graph()  # replay
    _check(filters, refs)
    # a new shape drops the captured graph; the next launch captures it
    other = dict(tpp=4 if shape["tpp"] != 4 else 8, ppi=128, block=512 if shape["block"] != 512 else 256, regcap=0)
    plan.set_shape(**other)
    assert plan.shape() == other
    for f in filters:
        f["logw"].fill_(float("nan"))
    plan.launch_graph()
    _check(filters, refs)
    plan.close()


def test_plan_follows_handle_changes(G, batch):
    """A plan re-reads its handles after a change (here the search layout),
    so later runs use the current store."""
    maps, filters, refs = batch
    plan = G.Plan(filters)
    plan.run()
    _check(filters, refs)
    g0 = plan.groups()
    assert g0[1] == 0 and g0[3] == 0 and g0[0] > 0 and g0[2] > 0
    for d, _ in maps:
        d.set_search(G.SEARCH_BINARY)
    for f in filters:
        f["logw"].fill_(float("nan"))
    plan.run()
    _check(filters, refs)
    g1 = plan.groups()
    assert g1[0] == 0 and g1[2] == 0 and g1[1] == g0[0] and g1[3] == g0[2]
    for f in filters:
        f["logw"].fill_(float("nan"))
    plan.launch_graph()
    _check(filters, refs)
    for d, _ in maps:
        d.set_search(G.SEARCH_TREE)
    plan.close()


def test_plan_argument_errors(G, batch):
    maps, filters, refs = batch
    plan = G.Plan(filters[:2])
    with pytest.raises(G.CDDTError):
        plan.set_shape(3, 64, 256)
    with pytest.raises(G.CDDTError):
        plan.set_shape(1, 64, 300)
    plan.close()


def test_plan_more_filters_than_one_launch(G, oracle):
    """More filters than one launch's parameter table holds: the plan splits
    them over several launches, each with its own table and queue."""
    g = synth.rect_map(96, 80, seed=950)
    mr = 120.0
    d = G.CDDT(dev(g), 36, mr)
    o = oracle.OracleCDDT(g, 36, mr)
    n = 2 * 220 + 17
    filters, refs = [], []
    for fi in range(n):
        B = 5 + fi % 7
        P = 1 + (7 * fi) % 23
        bo = synth.beam_offsets(B)
        D = synth.pair_offset(B)
        gt = synth.uniform_particles(g, 1, seed=5000 + fi)[0]
        obs = gc.observations(o, gt, bo, mr, seed=6000 + fi)
        parts = synth.tracking_particles(gt.astype(np.float64), P, seed=7000 + fi)
        filters.append(dict(map=d, particles=dev(parts).reshape(-1, 3), beam_off=dev(bo), obs=dev(obs),
                            model=G.beam_model(mr), logw=torch.full((P,), float("nan"), device="cuda"),
                            pair_offset=D))
        refs.append(o.sensor_weights(parts, bo, obs, oracle.beam_model(mr), nthreads=1))
    plan = G.Plan(filters)
    assert plan.groups()[0] == n  # one item per filter at the default shape
    plan.run()
    _check(filters, refs)
    for f in filters:
        f["logw"].fill_(float("nan"))
    plan.launch_graph()
    _check(filters, refs)
    plan.close()


def test_plan_on_pinned_host_buffers(G, batch):
    """A plan may take page-locked host tensors for particles, scans and
    log-weights: the kernel reads and writes them itself, bit for bit as on
    device buffers."""
    maps, filters, refs = batch
    dev_plan = G.Plan(filters)
    dev_plan.run()
    torch.cuda.synchronize()
    host = []
    for f in filters:
        h = dict(f)
        h["particles"] = f["particles"].cpu().pin_memory()
        h["obs"] = f["obs"].cpu().pin_memory()
        h["beam_off"] = f["beam_off"].cpu().pin_memory()
        h["logw"] = torch.full(f["logw"].shape, float("nan")).pin_memory()
        host.append(h)
    plan = G.Plan(host)
    plan.run()
    torch.cuda.synchronize()
    for f, h in zip(filters, host):
        assert torch.equal(h["logw"], f["logw"].cpu())
    for h in host:
        h["logw"].fill_(float("nan"))
    plan.launch_graph()
    torch.cuda.synchronize()
    for f, h in zip(filters, host):
        assert torch.equal(h["logw"], f["logw"].cpu())
    with pytest.raises(ValueError):  # pageable host memory is refused
        bad = dict(filters[0])
        bad["logw"] = torch.empty(filters[0]["logw"].shape)
        G.Plan([bad])
    plan.close()
    dev_plan.close()


def test_plan_refine_lanes_and_arguments(G, batch):
    """cddt_plan_refine over the batch's filters: with no step (one forward +
    adjoint evaluation at the given poses) every lane count, up to a
    particle over eight warps, gives the log-weights of cddt_plan_run and the
    same gradients to float32 rounding of the sums; bad lane counts, steps
    and step sizes are refused."""
    maps, filters, refs = batch
    fl = [dict(f, grad_xy=torch.empty((f["particles"].shape[0], 2), device="cuda"),
               particles_out=torch.empty((f["particles"].shape[0], 3), device="cuda")) for f in filters]
    plan = G.Plan(fl)
    grads = {}
    for tpp in (1, 32, 64, 128, 256, 0):
        for f in fl:
            f["logw"].fill_(float("nan"))
        plan.refine(0, 0.1, tpp=tpp)
        torch.cuda.synchronize()
        for f, want in zip(fl, refs):
            _close(f["logw"].cpu().numpy(), want)
            assert torch.equal(f["particles_out"], f["particles"])  # no step: the poses stay
        grads[tpp] = [f["grad_xy"].cpu().numpy().astype(np.float64) for f in fl]
    for tpp, gs in grads.items():
        for g, g1 in zip(gs, grads[1]):
            if g1.size == 0:  # the filter without particles
                continue
            scale = np.maximum(np.abs(g1).max(), 1.0)
            assert np.abs(g - g1).max() <= 1e-4 * scale, tpp
    for bad in (dict(tpp=3), dict(tpp=512), dict(steps=-1), dict(eta=-1.0)):
        args = dict(steps=1, eta=0.1, tpp=0)
        args.update(bad)
        with pytest.raises(G.CDDTError):
            plan.refine(args["steps"], args["eta"], tpp=args["tpp"])
    plan.close()
