"""Chronological initial guess of leapfrog solves (hqmc_set_guess_history): a
trajectory with the guess is the oracle's trajectory (same draws, CG to 1e-12:
dH to 1e-7, the field to 1e-8, as without it), and it needs fewer iterations."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("solver", ["cg64", "pmixed"])
def test_guess_keeps_the_oracle_trajectory(hq, solver):
    L, N, nsteps, dt = 8, 16, 6, 0.02
    lat = oracle.Lattice(L, N)
    th0 = inputs.theta_hot(L, N, 71)
    p0 = inputs.momenta(L, N, 72)
    R = inputs.complex_gaussian(L, N, 73)
    tol = 1e-12 if solver == "cg64" else 1e-10
    ref = oracle.trajectory(lat, th0, p0, R, u=0.5, nsteps=nsteps, dt=dt, tol=1e-12)
    out = {}
    with hq.Config(L, N) as cfg:
        for k in (0, 4):
            hq.set_guess_history(cfg, k)
            th = cuda(th0)
            out[k] = (hq.trajectory(cfg, th, p_in=cuda(p0), R_in=cuda(R), u_in=0.5, nsteps=nsteps, dt=dt, tol=tol,
                                    solver=solver), th.cpu().numpy())
    for k, (info, th) in out.items():
        assert info["status"] == 0 and info["max_true_residual"] <= tol
        assert abs(info["dH"] - ref["dH"]) < 1e-7, (k, info["dH"], ref["dH"])
        assert bool(info["accepted"]) == ref["accepted"]
        want = ref["theta"] if ref["accepted"] else th0
        assert np.max(np.abs(th - want)) < 1e-8
    print(solver, "iterations without / with the guess:", out[0][0]["cg_iterations"], out[4][0]["cg_iterations"])
    assert out[4][0]["cg_iterations"] < out[0][0]["cg_iterations"]


def test_guess_cuts_iterations_on_a_smooth_field(hq):
    """20 leapfrog steps on an L = 16 ordered field: the guess from the last four
    solutions at least halves the iterations of the solves after the first three."""
    L, N = 16, 160
    th0 = inputs.theta_ordered(L, N, 74, tau_walk=0.0)
    its = {}
    with hq.Config(L, N) as cfg:
        for k in (0, 4):
            hq.set_guess_history(cfg, k)
            th = cuda(th0)
            info = hq.trajectory(cfg, th, seed=3, traj_counter=1, nsteps=20, dt=0.002, tol=1e-8, solver="pmixed")
            assert info["status"] == 0 and info["max_true_residual"] <= 1e-8
            its[k] = info
    print("iterations without / with the guess:", its[0]["cg_iterations"], its[4]["cg_iterations"])
    assert its[4]["cg_iterations"] < 0.7 * its[0]["cg_iterations"]
    assert abs(its[4]["dH"] - its[0]["dH"]) < 1e-5 and its[4]["accepted"] == its[0]["accepted"]


def test_guess_history_arguments(hq):
    with hq.Config(8, 16) as cfg:
        for bad in (-1, 9):
            with pytest.raises(hq.HQMCError) as e:
                hq.set_guess_history(cfg, bad)
            assert e.value.status == hq.EINVAL
        hq.set_guess_history(cfg, 3)
        hq.set_guess_history(cfg, 2)  # smaller: no new allocation
        hq.set_guess_history(cfg, 0)


def test_learned_guess_gives_way_to_the_chronological_guess(hq):
    """A net equal to minus the identity is rejected on every solve (||r0 - O z|| =
    ||r0 + O r0|| > ||r0||).  With the chronological guess the learned solver stops
    trying it after two consecutive tries that do not halve the residual; without it,
    it tries every solve.  Either way the trajectory is the oracle's."""
    from oracle import net as onet
    L, N, nsteps, dt = 8, 16, 6, 0.02
    lat = oracle.Lattice(L, N)
    th0 = inputs.theta_hot(L, N, 81)
    p0 = inputs.momenta(L, N, 82)
    R = inputs.complex_gaussian(L, N, 83)
    ref = oracle.trajectory(lat, th0, p0, R, u=0.5, nsteps=nsteps, dt=dt, tol=1e-12)
    ws = onet.identity_weights(onet.LAYERS)
    ws[0] = -ws[0]
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    with hq.Config(L, N) as cfg:
        net = hq.Net(seed=0)
        net.set_weights(flat)
        hq.set_preconditioner(cfg, net)
        out = {}
        for k in (0, 4):
            hq.set_guess_history(cfg, k)
            th = cuda(th0)
            out[k] = hq.trajectory(cfg, th, p_in=cuda(p0), R_in=cuda(R), u_in=0.5, nsteps=nsteps, dt=dt, tol=1e-10,
                                   solver="plearned"), th.cpu().numpy()
        hq.set_preconditioner(cfg, None)
        net.close()
    for k, (info, th) in out.items():
        assert info["status"] == 0 and info["max_true_residual"] <= 1e-10
        assert info["net_guesses_used"] == 0
        assert info["net_guesses_tried"] == (2 if k else nsteps + 1), (k, info["net_guesses_tried"])
        assert abs(info["dH"] - ref["dH"]) < 1e-7 and bool(info["accepted"]) == ref["accepted"]
        want = ref["theta"] if ref["accepted"] else th0
        assert np.max(np.abs(th - want)) < 1e-8
