"""The library's per-rank operator of the slab decomposition (LibrarySlabOperator:
the fused M^dagger M and the force on a config of n_local + 2 slices) against the
FP64 oracle.  One rank runs the whole decomposition (halos from its own ends);
several slabs are evaluated one after another in one process, each with its
halo slices cut from the global field (signed at the wrap as the exchange signs
them), so no kernel waits on another."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu

L, NTAU = 8, 24


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def test_one_rank_solve_and_force(hq):
    from paper_2508_16298_gb300 import tauslab
    th = inputs.theta_hot(L, NTAU, 5)
    phi = inputs.complex_gaussian(L, NTAU, 6)
    lat = oracle.Lattice(L, NTAU)
    lay = tauslab.SlabLayout(NTAU, 1, 0)
    op = tauslab.LibrarySlabOperator(L, NTAU)
    try:
        th_ext = tauslab.halo(torch.from_numpy(th).cuda(), lay, antiperiodic=False)
        X = torch.zeros((NTAU, L, L), dtype=torch.complex128, device="cuda")
        its, res = tauslab.cg(op, th_ext, torch.from_numpy(phi).cuda(), X, lay, tol=1e-11)
        F = tauslab.force(op, th_ext, X, lay).cpu().numpy()
    finally:
        op.close()
    X = X.cpu().numpy()
    assert res <= 1e-11
    r = phi - oracle.apply_MdagM(lat, th, X)
    assert np.linalg.norm(r) <= 1.01e-11 * np.linalg.norm(phi)
    Fo = -oracle.fermion_dS(lat, th, X) - oracle.bosonic_dS(lat, th)
    assert np.max(np.abs(F - Fo)) < 1e-12 * np.max(np.abs(Fo))


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_evaluated_in_turn(hq, world):
    from paper_2508_16298_gb300 import tauslab
    th = inputs.theta_hot(L, NTAU, 7)
    x = inputs.complex_gaussian(L, NTAU, 8)
    lat = oracle.Lattice(L, NTAU)
    ys, fs = [], []
    for rank in range(world):
        lay = tauslab.SlabLayout(NTAU, world, rank)
        idx = [(t % NTAU) for t in range(lay.tau0 - 1, lay.tau1 + 1)]
        th_ext = torch.from_numpy(th[idx].copy()).cuda()
        x_ext = x[idx].copy()
        if lay.tau0 == 0:
            x_ext[0] = -x_ext[0]
        if lay.tau1 == NTAU:
            x_ext[-1] = -x_ext[-1]
        op = tauslab.LibrarySlabOperator(L, lay.n_local)
        try:
            ys.append(op.apply_MdagM_ext(th_ext, torch.from_numpy(x_ext).cuda())[1:-1].cpu().numpy())
            fs.append(op.force_ext(th_ext, torch.from_numpy(x_ext).cuda())[1:-1].cpu().numpy())
        finally:
            op.close()
    y, F = np.concatenate(ys), np.concatenate(fs)
    want = oracle.apply_MdagM(lat, th, x)
    assert np.max(np.abs(y - want)) < 1e-12 * np.max(np.abs(want))
    Fo = -oracle.fermion_dS(lat, th, x) - oracle.bosonic_dS(lat, th)
    assert np.max(np.abs(F - Fo)) < 1e-12 * np.max(np.abs(Fo))
