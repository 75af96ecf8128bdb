"""The tau-line preconditioner and the preconditioned solvers (through the C ABI)
against the FP64 oracle of oracle/precond.py.

Tolerances: the preconditioner apply is a sum of W + 1 = 34 scaled shifts per
pass, evaluated as a sliding-window recursion on the GPU and as explicit sums in
the oracle; FP64 agrees to a few 1e-15 relative (1e-12 required), FP32 to float
rounding of ~70 dependent operations (1e-5 required).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import precond as opc
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


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


@pytest.mark.parametrize("L,N", [(4, 6), (6, 2), (6, 33), (8, 40), (10, 9), (24, 240), (66, 660)])
def test_coefficients_and_apply(hq, L, N):
    """Ntau < W + 1 makes the window wrap the tau line several times (sign per wrap)."""
    lat = oracle.Lattice(L, N)
    c = opc.coefficients(lat)
    r = inputs.complex_gaussian(L, N, 300 + L)
    want = opc.apply(c, r)
    with hq.Config(L, N) as cfg:
        got = hq.get_precond(cfg)
        z64 = hq.apply_precond(cfg, cuda(r)).cpu().numpy()
        z32 = hq.apply_precond(cfg, cuda(r.astype(np.complex64))).cpu().numpy()
    assert abs(got["a"] - c.a) < 1e-13 and abs(got["b"] - c.b) < 1e-13
    assert abs(got["rho"] - c.rho) < 1e-13 and got["W"] == c.W
    assert rel(z64, want) < 1e-12
    assert z32.dtype == np.complex64 and rel(z32, opc.apply(c, r.astype(np.complex64).astype(np.complex128))) < 1e-5


@pytest.mark.parametrize("L,N", [(24, 240), (66, 660)])
def test_tile_height_and_autotuned_parity(hq, L, N):
    """The separate kernel's FP32 tile height is chosen per config (all tiles
    resident at once where a height allows it; timed by the autotuner when it
    runs); the result does not depend on it.  FP64 tiles are the tallest that
    leave two per SM on large lattices, else 64 slices."""
    lat = oracle.Lattice(L, N)
    c = opc.coefficients(lat)
    r = inputs.complex_gaussian(L, N, 700 + L).astype(np.complex64)
    want = opc.apply(c, r.astype(np.complex128))
    for autotune in (False, True):
        with hq.Config(L, N, autotune=autotune) as cfg:
            sh = hq.get_precond_shape(cfg, hq.FP32)
            assert 16 <= sh["tile_slices"] <= 256 and sh["fused"] in (False, True)
            assert hq.get_precond_shape(cfg, hq.FP64)["tile_slices"] == (220 if L == 66 else 64)
            z = hq.apply_precond(cfg, cuda(r)).cpu().numpy()
            z64 = hq.apply_precond(cfg, cuda(r.astype(np.complex128))).cpu().numpy()
        assert rel(z, want) < 1e-5
        assert rel(z64, want) < 1e-12


@pytest.mark.parametrize("L,N,start", [(4, 6, "hot"), (8, 40, "hot"), (8, 40, "cold"), (12, 24, "warm")])
def test_pcg64_matches_oracle_pcg(hq, L, N, start):
    lat = oracle.Lattice(L, N)
    th = {"hot": inputs.theta_hot(L, N, 31), "cold": inputs.theta_ordered(L, N, 31, tau_walk=0.0),
          "warm": inputs.theta_warm(L, N, 31)}[start]
    phi = inputs.complex_gaussian(L, N, 32)
    Xo, it_o, res_o = opc.pcg(lat, th, phi, opc.coefficients(lat), tol=1e-12)
    with hq.Config(L, N) as cfg:
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-12, solver="pcg64")
    assert info["status"] == 0 and info["true_residual"] <= 1e-12
    assert abs(info["iterations"] - it_o) <= 2
    assert rel(X.cpu().numpy(), Xo) < 1e-7


@pytest.mark.parametrize("L,N", [(24, 240), (48, 480)])
def test_preconditioned_mixed_solver(hq, L, N):
    """FP32 pCG with FP64 reliable updates reaches the FP64 true residual in far
    fewer iterations than plain mixed CG on a tau-smooth field."""
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 41, tau_walk=0.0)
    R = inputs.complex_gaussian(L, N, 42)
    phi = oracle.apply_M(lat, th, R, dagger=True)
    with hq.Config(L, N) as cfg:
        Xp, infop = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver="pmixed")
        Xm, infom = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver="mixed")
        Xp = Xp.cpu().numpy()
    assert infop["status"] == 0 and infop["true_residual"] <= 1e-8 and infop["fp64_fallback"] == 0
    assert infop["iterations"] * 3 < infom["iterations"]
    r = phi - oracle.apply_MdagM(lat, th, Xp)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi)


def test_preconditioned_learned_solver(hq):
    L, N = 12, 48
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 51, tau_walk=0.0)
    phi = inputs.complex_gaussian(L, N, 52)
    with hq.Config(L, N) as cfg:
        net = hq.Net(seed=3)
        hq.set_preconditioner(cfg, net)
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-9, solver="plearned")
        hq.set_preconditioner(cfg, None)
        net.close()
        X = X.cpu().numpy()
    assert info["status"] == 0 and info["true_residual"] <= 1e-9
    r = phi - oracle.apply_MdagM(lat, th, X)
    assert np.linalg.norm(r) <= 1.01e-9 * np.linalg.norm(phi)


def test_trajectory_with_preconditioned_solvers_matches_oracle(hq):
    """The solver changes only how X is reached: with tight tolerances the
    trajectory (same p, R, u) matches the oracle's plain-CG trajectory."""
    L, N, nsteps, dt = 8, 40, 5, 0.02
    lat = oracle.Lattice(L, N)
    th0 = inputs.theta_hot(L, N, 61)
    p0 = inputs.momenta(L, N, 62)
    R = inputs.complex_gaussian(L, N, 63)
    u = 0.5
    ref = oracle.trajectory(lat, th0, p0, R, u=u, nsteps=nsteps, dt=dt, tol=1e-12)
    with hq.Config(L, N) as cfg:
        for solver in ("pcg64", "pmixed"):
            th = cuda(th0.copy())
            tol = 1e-12 if solver == "pcg64" else 1e-9
            info = hq.trajectory(cfg, th, p_in=cuda(p0), R_in=cuda(R), u_in=u, nsteps=nsteps, dt=dt, tol=tol,
                                 solver=solver)
            assert info["status"] == 0 and bool(info["accepted"]) == ref["accepted"]
            assert abs(info["dH"] - ref["dH"]) < (1e-7 if solver == "pcg64" else 1e-4) * max(1.0, abs(ref["dH"]))
            assert np.max(np.abs(th.cpu().numpy() - ref["theta"])) < (1e-8 if solver == "pcg64" else 1e-5)


def test_preconditioned_edge_cases(hq):
    L, N = 8, 16
    th = cuda(inputs.theta_hot(L, N, 71))
    phi = cuda(inputs.complex_gaussian(L, N, 72))
    with hq.Config(L, N) as cfg:
        for solver in ("pcg64", "pmixed"):
            Z, info = hq.cg_solve(cfg, th, torch.zeros_like(phi), solver=solver)
            assert info["status"] == 0 and info["iterations"] == 0 and not Z.abs().max().item()
            X, info = hq.cg_solve(cfg, th, phi, tol=1e-14, maxit=3, solver=solver, raise_on_fail=False)
            assert info["status"] == hq.ENOTCONV and info["iterations"] <= 3 + 2
            assert info["true_residual"] > 1e-14
        with pytest.raises(hq.HQMCError) as e:
            hq.apply_precond(cfg, phi, z=phi)
        assert e.value.status == hq.EINVAL


@pytest.mark.parametrize("reliable", [25, 50])
def test_fused_and_separate_preconditioned_updates_agree(hq, reliable):
    """An odd reliable-update period keeps the separate update and preconditioner
    (the fused form alternates two residual buffers and needs an even loop body);
    both reach the same solution."""
    L, N = 12, 48
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 81, tau_walk=0.0)
    phi = inputs.complex_gaussian(L, N, 82)
    Xo, _, _ = opc.pcg(lat, th, phi, opc.coefficients(lat), tol=1e-12)
    with hq.Config(L, N, reliable_interval=reliable) as cfg:
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-9, solver="pmixed")
    assert info["status"] == 0 and info["true_residual"] <= 1e-9
    assert rel(X.cpu().numpy(), Xo) < 1e-5
