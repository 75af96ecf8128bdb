"""The imaginary-time slab decomposition (paper_2508_16298_gb300/tauslab.py) on two
and three gloo ranks on CPU, against the FP64 oracle's global operators: the
distributed M^dagger M apply, CG solve and force equal the global ones.  The
per-rank operator in these CPU runs is the oracle on the extended slab (the test
supplies it); on GPUs it is the library's (LibrarySlabOperator)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
L, NTAU = 4, 12


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


class OracleSlabOperator:
    """The oracle on a lattice of n_local + 2 slices (test infrastructure)."""

    def __init__(self, n_local):
        import oracle
        self.oracle = oracle
        self.lat = oracle.Lattice(L, n_local + 2)

    def apply_MdagM_ext(self, theta_ext, x_ext):
        import torch
        return torch.from_numpy(self.oracle.apply_MdagM(self.lat, theta_ext.numpy(), x_ext.numpy()))

    def force_ext(self, theta_ext, X_ext):
        import torch
        th, X = theta_ext.numpy(), X_ext.numpy()
        return torch.from_numpy(-self.oracle.fermion_dS(self.lat, th, X) - self.oracle.bosonic_dS(self.lat, th))


def global_inputs():
    sys.path.insert(0, ROOT)
    from paper_2508_16298_gb300 import inputs
    th = inputs.theta_hot(L, NTAU, 3)
    phi = inputs.complex_gaussian(L, NTAU, 4)
    return th, phi


def run_slabs(rank, world):
    """One rank's part: returns its rows of O phi, X and F."""
    import torch
    from paper_2508_16298_gb300 import tauslab
    th, phi = global_inputs()
    lay = tauslab.SlabLayout(NTAU, world, rank)
    sl = slice(lay.tau0, lay.tau1)
    th_loc = torch.from_numpy(th[sl].copy())
    phi_loc = torch.from_numpy(phi[sl].copy())
    op = OracleSlabOperator(lay.n_local)
    th_ext = tauslab.halo(th_loc, lay, antiperiodic=False)
    Ophi = tauslab.apply_MdagM(op, th_ext, phi_loc, lay)
    X = torch.zeros_like(phi_loc)
    its, res = tauslab.cg(op, th_ext, phi_loc, X, lay, tol=1e-12)
    F = tauslab.force(op, th_ext, X, lay)
    return lay.tau0, lay.tau1, Ophi.numpy(), X.numpy(), F.numpy(), its, res


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + run_slabs(rank, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def check_against_oracle(parts):
    import oracle
    th, phi = global_inputs()
    lat = oracle.Lattice(L, NTAU)
    Ophi = np.concatenate([p[3] for p in parts])
    X = np.concatenate([p[4] for p in parts])
    F = np.concatenate([p[5] for p in parts])
    assert [p[1] for p in parts] == sorted(p[1] for p in parts) and parts[-1][2] == NTAU
    want = oracle.apply_MdagM(lat, th, phi)
    assert np.max(np.abs(Ophi - want)) < 1e-13 * np.max(np.abs(want))
    Xo, _, _, _ = oracle.cg(lat, th, phi, tol=1e-13)
    assert np.max(np.abs(X - Xo)) < 1e-9 * np.max(np.abs(Xo))
    assert all(p[7] <= 1e-12 for p in parts)  # every rank sees the same global true residual
    assert len({p[6] for p in parts}) == 1    # and the same iteration count
    Fo = -oracle.fermion_dS(lat, th, X) - oracle.bosonic_dS(lat, th)
    assert np.max(np.abs(F - Fo)) < 1e-12 * np.max(np.abs(Fo))


@pytest.mark.parametrize("world", [2, 3])
def test_slab_decomposition_on_gloo_ranks(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    check_against_oracle(parts)


def test_single_rank_slab_is_the_whole_lattice():
    sys.path.insert(0, ROOT)
    check_against_oracle([(0,) + run_slabs(0, 1)])


def test_layout_is_contiguous_and_balanced():
    sys.path.insert(0, ROOT)
    from paper_2508_16298_gb300.tauslab import SlabLayout
    for n, w in ((12, 2), (13, 3), (660, 8)):
        lays = [SlabLayout(n, w, r) for r in range(w)]
        assert lays[0].tau0 == 0 and lays[-1].tau1 == n
        assert all(a.tau1 == b.tau0 for a, b in zip(lays, lays[1:]))
        assert max(l.n_local for l in lays) - min(l.n_local for l in lays) <= 1
