"""The bounds-checked build (CDDT_CHECKED=1): on valid inputs it trips no
check and reproduces the normal build bit for bit; with the store's extent
under-reported (CDDT_FAULT=bounds, so valid reads fall outside the extent the
checks see) every cast still returns and the handle reports CDDT_ERR_BOUNDS."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def _child(env_extra, code, timeout=900):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=timeout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return r


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01167_gb300 import build
    build.build_checked()


def test_checked_build_matches_normal_build(built, tmp_path):
    from tests import checked_cases
    out = tmp_path / "checked.npz"
    _child({"CDDT_CHECKED": "1"}, f"from tests import checked_cases as c; c.main({str(out)!r})")
    z = np.load(out)
    assert int(z["checked"]) == 1
    want, st = checked_cases.run_cases()
    from paper_1705_01167_gb300 import cddt as G
    assert G.load().cddt_checked_build() == 0
    for k, v in want.items():
        assert int(z[f"st_{k}"]) == 0, (k, int(z[f"st_{k}"]))
        assert st[k] == 0, k
        got = z[f"out_{k}"]
        assert got.shape == v.shape and np.array_equal(got.view(np.uint32), v.view(np.uint32)), k


def test_checked_build_flags_out_of_extent_reads(built, tmp_path):
    code = """
import numpy as np, torch
from paper_1705_01167_gb300 import cddt as G, synth
from tests import gpu_cases as gc
assert G.load().cddt_checked_build() == 1
g = synth.rect_map(256, 256)
q = torch.from_numpy(gc.random_queries(256, 256, 20000, 505)).cuda()
for u16 in (False, True):
    d = G.CDDT(torch.from_numpy(g).cuda(), 108, 300.0, u16=u16)
    for s in (G.SEARCH_TREE, G.SEARCH_BINARY):
        d.set_search(s)
        r = d.calc_range_many(q)
        torch.cuda.synchronize()
        st = d.status()
        assert st == G.CDDT_ERR_BOUNDS, (u16, s, st)
        assert d.status() == 0                  # read and cleared
        assert torch.isfinite(r).all()
    d.close()
print("flagged")
"""
    r = _child({"CDDT_CHECKED": "1", "CDDT_FAULT": "bounds"}, code)
    assert "flagged" in r.stdout
