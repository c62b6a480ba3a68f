"""The C ABI from plain C on the GPU: the example builds a CDDT of a box with
a pillar through include/cddt.h and checks 16 axis-aligned casts (unsorted
and slice-sorted) against their closed forms."""
import subprocess

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_c_example_on_gpu(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests.c_example.build_example import build_example
    exe = build_example(str(tmp_path))
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "16 ray casts match their closed forms" in r.stdout
