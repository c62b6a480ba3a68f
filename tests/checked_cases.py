"""A fixed set of calls through the public binding whose outputs a
bounds-checked build (CDDT_CHECKED=1) must reproduce bit for bit, with no
bounds check tripped.  Run in a child process, since the library variant is
chosen when the binding first loads it.

    python -m tests.checked_cases OUT.npz
"""
import sys

import numpy as np
import torch

from paper_1705_01167_gb300 import cddt as G
from paper_1705_01167_gb300 import synth
from tests import gpu_cases as gc


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_cases() -> dict:
    out, status = {}, {}

    def rec(name, d, t):
        out[name] = t.cpu().numpy() if isinstance(t, torch.Tensor) else t
        status[name] = d.status() if d is not None else 0

    g = synth.rect_map(256, 256)
    mr = 300.0
    q = np.concatenate([gc.special_queries(256, 256), gc.random_queries(256, 256, 20000, 501)])
    bo = synth.beam_offsets(61)
    D = synth.pair_offset(61)
    parts = synth.uniform_particles(g, 2000, seed=502)
    obs = np.clip(synth.noise(61, 40.0, seed=503) + 60.0, 0, mr).astype(np.float32)
    m = G.beam_model(mr)
    tq, tp, tb, to = dev(q), dev(parts), dev(bo), dev(obs)
    for u16 in (False, True):
        d = G.CDDT(dev(g), 108, mr, u16=u16)
        for search in (G.SEARCH_TREE, G.SEARCH_BINARY):
            d.set_search(search)
            rec(f"range_u{int(u16)}_s{search}", d, d.calc_range_many(tq))
        d.set_search(G.SEARCH_TREE)
        rec(f"sorted_u{int(u16)}", d, d.calc_range_many(tq, sort_by_slice=True))
        lw, rg = d.sensor_weights(tp, tb, to, m, D, want_ranges=True)
        rec(f"logw_u{int(u16)}", d, lw)
        rec(f"ranges_u{int(u16)}", d, rg)
        rec(f"grad_u{int(u16)}", d, d.sensor_weights_backward(tp, tb, to, m, torch.ones(2000, device="cuda"), D))
        lut = G.Lut(d)
        rec(f"lut_u{int(u16)}", d, lut.calc_range_many(tq))
        lut.close()
        d.close()
    # many filters in one persistent launch
    d = G.CDDT(dev(g), 108, mr)
    logw = torch.empty(3 * 2000, dtype=torch.float32, device="cuda")
    plan = G.Plan([dict(map=d, particles=tp, beam_off=tb, obs=to, model=m, logw=logw[f * 2000:(f + 1) * 2000],
                        pair_offset=D) for f in range(3)])
    plan.run()
    rec("plan", d, logw)
    plan.close()
    # prune, then update another handle and cast again
    d.prune()
    rec("pruned", d, d.calc_range_many(tq))
    d.close()
    d = G.CDDT(dev(g), 108, mr)
    xy, occ = synth.cell_toggles(g, 300, 300, seed=504)
    d.update_cells(dev(xy.astype(np.int32)), dev(occ.astype(np.uint8)))
    rec("updated", d, d.calc_range_many(tq))
    rm = G.RayMarch(d)
    rec("raymarch", d, rm.calc_range_many(tq))
    rm.close()
    d.close()
    return out, status


def main(path: str):
    assert torch.cuda.is_available()
    out, status = run_cases()
    np.savez(path, checked=np.int32(G.load().cddt_checked_build()),
             **{f"out_{k}": v for k, v in out.items()}, **{f"st_{k}": np.int32(v) for k, v in status.items()})


if __name__ == "__main__":
    main(sys.argv[1])
