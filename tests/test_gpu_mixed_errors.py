"""Errors of the mixed-precision solvers against the FP64 oracle: the solution X,
the fermion force computed from it, and dH of a trajectory with the same draws.

Both sides stop at a true FP64 residual: the mixed solve at tol = 1e-8, the
oracle at 1e-12.  The error of X is then bounded by kappa(M^dagger M) * 1e-8;
the force is linear in X (and in Y = M X), dH's fermion part is phi^dagger X.
The bounds below follow from the stopping rule (stated at each assertion);
the measured values, printed with -s, are well inside them.
"""
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


@pytest.mark.parametrize("solver", ["mixed", "pmixed"])
def test_solution_and_force_errors_against_the_oracle(hq, solver):
    L, N = 16, 160
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 91, tau_walk=0.0)
    R = inputs.complex_gaussian(L, N, 92)
    phi = oracle.apply_M(lat, th, R, dagger=True)
    Xo, _, _, _ = oracle.cg(lat, th, phi, tol=1e-12)
    Fo = oracle.fermion_dS(lat, th, Xo)
    with hq.Config(L, N) as cfg:
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver=solver)
        F = torch.zeros((N, L, L, 2), dtype=torch.float64, device="cuda")
        dSf = torch.zeros_like(F)
        hq.force(cfg, cuda(th), X, F=F, dSf=dSf)
        X, dSf = X.cpu().numpy(), dSf.cpu().numpy()
    assert info["status"] == 0 and info["true_residual"] <= 1e-8
    ex = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    ef = np.max(np.abs(dSf - Fo)) / np.max(np.abs(Fo))
    print(f"{solver}: |dX|/|X| = {ex:.2e}, max|dF|/max|F| = {ef:.2e}")
    assert ex < 1e-5 and ef < 1e-5


def test_trajectory_dH_error_against_the_oracle(hq):
    L, N, nsteps, dt = 12, 120, 5, 0.001
    lat = oracle.Lattice(L, N)
    th0 = inputs.theta_ordered(L, N, 93, tau_walk=0.0)
    p0 = inputs.momenta(L, N, 94)
    R = inputs.complex_gaussian(L, N, 95)
    ref = oracle.trajectory(lat, th0, p0, R, u=0.5, nsteps=nsteps, dt=dt, tol=1e-12)
    with hq.Config(L, N) as cfg:
        for solver in ("mixed", "pmixed"):
            th = cuda(th0.copy())
            info = hq.trajectory(cfg, th, p_in=cuda(p0), R_in=cuda(R), u_in=0.5, nsteps=nsteps, dt=dt, tol=1e-8,
                                 solver=solver)
            eth = np.max(np.abs(th.cpu().numpy() - ref["theta"]))
            edh = abs(info["dH"] - ref["dH"])
            print(f"{solver}: |dH - dH_oracle| = {edh:.2e} (dH = {ref['dH']:.3e}), max|theta - theta_oracle| = {eth:.2e}")
            assert info["status"] == 0 and bool(info["accepted"]) == ref["accepted"]
            # the fermion part of H is phi^dagger X; a solve stopped at ||r|| <= tol ||phi|| changes it
            # by |X^dagger r| <= tol ||X|| ||phi||, of the order tol * |H| (H0 = S_B + p^2 + R^dagger R here)
            assert edh < 1e-8 * abs(ref["H0"]) and eth < 1e-8
