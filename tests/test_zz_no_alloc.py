"""The allocation-free M^dagger M entry point (hqmc_apply_MdagM_static).

It is for callers that cannot allocate device memory: code that runs while
another component owns the device allocator (a memory pool that must not be
bypassed, or a budget that is already handed out), plug-ins that are handed only
device pointers, and code that must not let cudaMalloc/cudaFree synchronise the
device.  Its only scratch is a fixed device array inside the library.

This file is collected last, so that a run stopping at the first failure has
run every other test before it.  The comparison with the config-based
hqmc_apply_MdagM (two calls in a row) runs here, after the other tests, and once
more in a fresh Python interpreter started by the test, where the entry point's
first call on the device does its one-time set-up.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def compare_twice(hq, L, N):
    """Two static calls in a row (sharing the scratch array), each against the
    config-based apply at 1e-12 (FP64 rounding of the same fused kernel family)."""
    with hq.Config(L, N) as cfg:
        for call in range(2):
            th = torch.from_numpy(inputs.theta_hot(L, N, seed=300 + call)).cuda()
            x = torch.from_numpy(inputs.complex_gaussian(L, N, seed=400 + call)).cuda()
            y_static = hq.apply_MdagM_static(L, N, th, x).cpu().numpy()
            y_cfg = hq.apply_MdagM(cfg, th, x).cpu().numpy()
            assert rel(y_static, y_cfg) < 1e-12, (L, N, call)


@pytest.mark.parametrize("L,N", [(8, 40), (24, 240)])
def test_static_apply_matches_config_apply_twice(hq, L, N):
    compare_twice(hq, L, N)


def test_static_apply_allocates_nothing(hq):
    """After the first call (which loads the module holding the scratch array),
    further calls leave the device's free memory unchanged."""
    L, N = 24, 240
    th = torch.from_numpy(inputs.theta_hot(L, N, seed=310)).cuda()
    x = torch.from_numpy(inputs.complex_gaussian(L, N, seed=410)).cuda()
    y = torch.empty_like(x)
    hq.apply_MdagM_static(L, N, th, x, y=y)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        hq.apply_MdagM_static(L, N, th, x, y=y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_apply_in_a_fresh_process():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2508_16298_gb300 import hqmc\n"
            "import tests.test_zz_no_alloc as t\n"
            "t.compare_twice(hqmc, 8, 40)\n"
            "print('fresh process ok')\n") % ROOT
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0 and "fresh process ok" in res.stdout, res.stdout + res.stderr


def test_static_apply_rejects_lattices_beyond_its_scratch(hq):
    L, N = 66, 660  # 2,874,960 sites > 262,144
    assert L * L * N > hq.STATIC_MAX_SITES
    th = torch.zeros((N, L, L, 2), dtype=torch.float64, device="cuda")
    x = torch.zeros((N, L, L), dtype=torch.complex128, device="cuda")
    with pytest.raises(hq.HQMCError) as e:
        hq.apply_MdagM_static(L, N, th, x)
    assert e.value.status == hq.EUNSUPPORTED


def test_static_apply_rejects_a_non_finite_hopping(hq):
    L, N = 8, 40
    th = torch.zeros((N, L, L, 2), dtype=torch.float64, device="cuda")
    x = torch.zeros((N, L, L), dtype=torch.complex128, device="cuda")
    for t in (float("nan"), float("inf"), 0.0):
        with pytest.raises(hq.HQMCError) as e:
            hq.apply_MdagM_static(L, N, th, x, t=t)
        assert e.value.status == hq.EINVAL
