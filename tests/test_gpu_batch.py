"""Batched chains of uneven lattices (one launch per CG iteration for all chains)
against independent single-chain runs with the same kernels: bit for bit."""
import numpy as np
import pytest
import torch

from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu

LATS = [(8, 16), (12, 24), (16, 32), (10, 40)]


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def test_batched_cg_equals_independent_solves(hq):
    thetas = [torch.from_numpy(inputs.theta_hot(L, N, 500 + i)).cuda() for i, (L, N) in enumerate(LATS)]
    phis = [torch.from_numpy(inputs.complex_gaussian(L, N, 600 + i)).cuda() for i, (L, N) in enumerate(LATS)]
    with hq.Batch(LATS) as b:
        xs, infos = b.cg_solve(thetas, phis, tol=1e-10)
        n_launch = b.launch_count()
    for i, (L, N) in enumerate(LATS):
        with hq.Config(L, N, variant=1) as cfg:
            x1, info1 = hq.cg_solve(cfg, thetas[i], phis[i], tol=1e-10)
        assert infos[i]["status"] == 0 and infos[i]["iterations"] == info1["iterations"]
        assert torch.equal(xs[i], x1), i
        assert infos[i]["true_residual"] == info1["true_residual"]
    assert n_launch > 0


def test_batched_trajectory_equals_independent_trajectories(hq):
    th0 = [inputs.theta_hot(L, N, 700 + i) for i, (L, N) in enumerate(LATS)]
    seeds = [11 + i for i in range(len(LATS))]
    dts = [0.02, 0.015, 0.01, 0.02]
    with hq.Batch(LATS) as b:
        thetas = [torch.from_numpy(t).cuda() for t in th0]
        infos = b.trajectory(thetas, seeds, traj_counter=3, nsteps=3, dts=dts, tol=1e-10)
    for i, (L, N) in enumerate(LATS):
        with hq.Config(L, N, variant=1) as cfg:
            t1 = torch.from_numpy(th0[i]).cuda()
            info1 = hq.trajectory(cfg, t1, seed=seeds[i], traj_counter=3, nsteps=3, dt=dts[i], tol=1e-10)
        assert infos[i]["dH"] == info1["dH"] and infos[i]["accepted"] == info1["accepted"], i
        assert infos[i]["cg_iterations"] == info1["cg_iterations"]
        assert torch.equal(thetas[i], t1), i


def test_autotuned_batch_equals_independent_solves(hq):
    """The batch autotuner picks a cluster size and tile order; the results stay those
    of single-chain runs bit for bit, whatever it picks."""
    thetas = [torch.from_numpy(inputs.theta_hot(L, N, 540 + i)).cuda() for i, (L, N) in enumerate(LATS)]
    phis = [torch.from_numpy(inputs.complex_gaussian(L, N, 640 + i)).cuda() for i, (L, N) in enumerate(LATS)]
    with hq.Batch(LATS, autotune=True) as b:
        shape = b.launch_shape()
        xs, infos = b.cg_solve(thetas, phis, tol=1e-10)
    print("autotuned batch shape:", shape)
    assert shape["cluster"] in (1, 2, 4, 8) and shape["order"] in (0, 1, 2) and shape["tuned_us"] > 0
    for i, (L, N) in enumerate(LATS):
        with hq.Config(L, N, variant=1) as cfg:
            x1, info1 = hq.cg_solve(cfg, thetas[i], phis[i], tol=1e-10)
        assert infos[i]["status"] == 0 and infos[i]["iterations"] == info1["iterations"]
        assert torch.equal(xs[i], x1), i
        assert infos[i]["true_residual"] == info1["true_residual"]


def test_batch_rejects_bad_lattice(hq):
    with pytest.raises(hq.HQMCError):
        hq.Batch([(8, 16), (9, 16)])


def test_batched_preconditioned_cg_equals_independent_solves(hq):
    """The tau-line preconditioner in the batch: one launch over every chain's tiles,
    bit for bit the results of single-chain PCG64 solves (variant 1 keeps the same
    separate update and preconditioner kernels)."""
    thetas = [torch.from_numpy(inputs.theta_ordered(L, N, 800 + i, tau_walk=0.0)).cuda()
              for i, (L, N) in enumerate(LATS)]
    phis = [torch.from_numpy(inputs.complex_gaussian(L, N, 900 + i)).cuda() for i, (L, N) in enumerate(LATS)]
    with hq.Batch(LATS) as b:
        xs0, infos0 = b.cg_solve(thetas, phis, tol=1e-10)
        b.set_solver("pcg64")
        xs, infos = b.cg_solve(thetas, phis, tol=1e-10)
    for i, (L, N) in enumerate(LATS):
        with hq.Config(L, N, variant=1) as cfg:
            x1, info1 = hq.cg_solve(cfg, thetas[i], phis[i], tol=1e-10, solver="pcg64")
        assert infos[i]["status"] == 0 and infos[i]["iterations"] == info1["iterations"]
        assert infos[i]["iterations"] < infos0[i]["iterations"]
        assert torch.equal(xs[i], x1), i
        assert infos[i]["true_residual"] == info1["true_residual"]


def test_batched_preconditioned_trajectory_equals_independent_trajectories(hq):
    th0 = [inputs.theta_hot(L, N, 1000 + i) for i, (L, N) in enumerate(LATS)]
    seeds = [31 + i for i in range(len(LATS))]
    dts = [0.02, 0.015, 0.01, 0.02]
    with hq.Batch(LATS) as b:
        b.set_solver("pcg64")
        thetas = [torch.from_numpy(t).cuda() for t in th0]
        infos = b.trajectory(thetas, seeds, traj_counter=5, nsteps=3, dts=dts, tol=1e-10)
        with pytest.raises(hq.HQMCError):
            b.set_solver("mixed")
    for i, (L, N) in enumerate(LATS):
        with hq.Config(L, N, variant=1) as cfg:
            t1 = torch.from_numpy(th0[i]).cuda()
            info1 = hq.trajectory(cfg, t1, seed=seeds[i], traj_counter=5, nsteps=3, dt=dts[i], tol=1e-10,
                                  solver="pcg64")
        assert infos[i]["dH"] == info1["dH"] and infos[i]["accepted"] == info1["accepted"], i
        assert infos[i]["cg_iterations"] == info1["cg_iterations"]
        assert torch.equal(thetas[i], t1), i


def test_batched_trajectory_graph_replays_with_new_counters(hq):
    """The trajectory graph is captured once and replayed: the trajectory counter,
    seeds and dt are read from device memory at every launch, so two trajectories
    in a row still equal two single-chain trajectories in a row."""
    th0 = [inputs.theta_hot(L, N, 1100 + i) for i, (L, N) in enumerate(LATS)]
    seeds = [41 + i for i in range(len(LATS))]
    dts = [0.02, 0.015, 0.01, 0.02]
    with hq.Batch(LATS) as b:
        thetas = [torch.from_numpy(t).cuda() for t in th0]
        inf_a = b.trajectory(thetas, seeds, traj_counter=7, nsteps=2, dts=dts, tol=1e-10)
        inf_b = b.trajectory(thetas, seeds, traj_counter=8, nsteps=2, dts=[d * 0.5 for d in dts], tol=1e-10)
    for i, (L, N) in enumerate(LATS):
        with hq.Config(L, N, variant=1) as cfg:
            t1 = torch.from_numpy(th0[i]).cuda()
            a = hq.trajectory(cfg, t1, seed=seeds[i], traj_counter=7, nsteps=2, dt=dts[i], tol=1e-10)
            bb = hq.trajectory(cfg, t1, seed=seeds[i], traj_counter=8, nsteps=2, dt=dts[i] * 0.5, tol=1e-10)
        assert inf_a[i]["dH"] == a["dH"] and inf_b[i]["dH"] == bb["dH"], i
        assert inf_a[i]["u"] == a["u"] and inf_b[i]["u"] == bb["u"]
        assert torch.equal(thetas[i], t1), i


@pytest.mark.parametrize("solver", ["cg64", "pcg64"])
def test_batched_trajectory_against_oracle(hq, solver):
    """Each chain of a batched trajectory against the FP64 oracle's trajectory with the
    same Philox draws (p, R, u from oracle/philox.py) and CG at 1e-12: dH to 1e-7 and
    the field to 1e-8, as for single-chain trajectories."""
    import oracle
    from oracle import philox
    lats = [(4, 8), (6, 12), (8, 16)]
    th0 = [inputs.theta_ordered(L, N, 1200 + i, tau_walk=0.0) for i, (L, N) in enumerate(lats)]
    seeds = [51 + i for i in range(len(lats))]
    dts = [0.02, 0.02, 0.015]
    ctr = 9
    with hq.Batch(lats) as b:
        b.set_solver(solver)
        thetas = [torch.from_numpy(t).cuda() for t in th0]
        infos = b.trajectory(thetas, seeds, traj_counter=ctr, nsteps=3, dts=dts, tol=1e-12)
    for i, (L, N) in enumerate(lats):
        lat = oracle.Lattice(L, N)
        p = philox.draw_momenta(seeds[i], ctr, L, N)
        R = philox.draw_pseudofermion(seeds[i], ctr, L, N)
        u = philox.draw_metropolis(seeds[i], ctr)
        ref = oracle.trajectory(lat, th0[i], p, R, u=u, nsteps=3, dt=dts[i], tol=1e-12)
        assert infos[i]["status"] == 0 and infos[i]["max_true_residual"] <= 1e-12
        assert abs(infos[i]["u"] - u) == 0.0
        assert abs(infos[i]["dH"] - ref["dH"]) < 1e-7, (i, infos[i]["dH"], ref["dH"])
        assert bool(infos[i]["accepted"]) == ref["accepted"]
        want = ref["theta"] if ref["accepted"] else th0[i]
        assert np.max(np.abs(thetas[i].cpu().numpy() - want)) < 1e-8
