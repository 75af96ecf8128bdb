"""The allocation-free M^dagger M entry point (hqmc_apply_MdagM_static).

It serves callers that cannot allocate device memory (another component owns
the allocator, only device pointers are handed in, or cudaMalloc's device-wide
synchronisation is not allowed): its scratch is a fixed device array inside the
library.  This file is collected last on purpose.  The test runs alone in a
fresh process and after the other tests, and compares the static entry point
with the config-based hqmc_apply_MdagM on two calls in a row.
"""
import numpy as np
import pytest
import torch

from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("L,N", [(8, 40), (24, 240)])
def test_static_apply_matches_config_apply_twice(hq, L, N):
    with hq.Config(L, N) as cfg:
        for call in range(2):  # two calls in a row share the static scratch
            th = torch.from_numpy(inputs.theta_hot(L, N, seed=300 + call)).cuda()
            x = torch.from_numpy(inputs.complex_gaussian(L, N, seed=400 + call)).cuda()
            y_static = hq.apply_MdagM_static(L, N, th, x).cpu().numpy()
            y_cfg = hq.apply_MdagM(cfg, th, x).cpu().numpy()
            assert rel(y_static, y_cfg) < 1e-12, (L, N, call)


def test_static_apply_rejects_lattices_beyond_its_scratch(hq):
    L, N = 66, 660  # 2,874,960 sites > 262,144
    assert L * L * N > hq.STATIC_MAX_SITES
    th = torch.zeros((N, L, L, 2), dtype=torch.float64, device="cuda")
    x = torch.zeros((N, L, L), dtype=torch.complex128, device="cuda")
    with pytest.raises(hq.HQMCError) as e:
        hq.apply_MdagM_static(L, N, th, x)
    assert e.value.status == hq.EUNSUPPORTED
