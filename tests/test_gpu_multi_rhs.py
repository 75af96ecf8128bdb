"""Systems solved together on one field (hqmc_cg_solve_multi, hqmc_estimate_multi,
through the C ABI) against the FP64 oracle.

Methods, "Stochastic estimation of fermionic observables": the N_rv systems
(M^dagger M) X_k = R_k of an estimate share theta.  The library advances them
together (one tau-walking M^dagger M launch over all systems per CG iteration,
batched updates, preconditioner and FP64 reliable updates), each with its own
scalars and convergence test.  What is checked:

* every solution has a true residual ||phi_k - O_oracle X_k|| <= 1.01 tol ||phi_k||
  with O_oracle the oracle's FP64 M^dagger M (the factor 1.01 covers the FP64
  rounding of the two residual evaluations), on lattices whose slice ranges per
  CTA are ragged, and at the bench's own size L = 66, Ntau = 660;
* two preconditioned iterations of every system from pinned guesses equal the
  oracle's two pCG iterations (Eq. (pCG)) element by element within FP32
  rounding: the second direction holds z_1 = Otilde^{-1}(r_0 - alpha_0 q_0), so
  this checks each system's q_0 = O p_0 of the multi-system launch element-wise
  through an invertible map, with every system's own alpha and beta;
* the estimate equals the oracle's (same Philox draws) within kappa * tol, and
  the sequential estimate of hqmc_estimate to the solves' accuracy;
* edge cases: no workspace, too many systems, an unsupported solver, a zero
  right-hand side among others, maxit = 0, groups of systems smaller than nrv.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import estimate as oest
from oracle import philox
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


def sources(L, N, th, nrhs, seed):
    lat = oracle.Lattice(L, N)
    return np.stack([oracle.apply_M(lat, th, inputs.complex_gaussian(L, N, seed + k), dagger=True)
                     for k in range(nrhs)])


# ranges: slice ranges per system of the walk launch (0: the default model, which on
# these small lattices gives one slice per CTA); 3 on Ntau = 70 gives ragged ranges
# of 23 and 24 slices, 1 one range of all Ntau slices per system (its halo is the
# antiperiodic wrap).
@pytest.mark.parametrize("L,N,solver,ranges", [(8, 40, "pmixed", 0), (6, 30, "mixed", 0), (10, 70, "pmixed", 3),
                                               (10, 70, "mixed", 7), (8, 40, "pmixed", 1), (4, 6, "pmixed", 4)])
def test_solutions_against_oracle(hq, L, N, solver, ranges):
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, 11)
    nrhs, tol = 5, 1e-9
    phi = sources(L, N, th, nrhs, 40)
    with hq.Config(L, N) as cfg:
        hq.set_multi_rhs(cfg, nrhs)
        hq.set_multi_ranges(cfg, ranges)
        shape = hq.multi_launch_shape(cfg, nrhs)
        assert ranges == 0 or shape["ranges"] == ranges
        X, infos = hq.cg_solve_multi(cfg, cuda(th), cuda(phi), tol=tol, solver=solver)
    print(L, N, solver, shape, [i["iterations"] for i in infos])
    X = X.cpu().numpy()
    for k in range(nrhs):
        assert infos[k]["status"] == 0 and infos[k]["true_residual"] <= tol, infos[k]
        r = phi[k] - oracle.apply_MdagM(lat, th, X[k])
        assert np.linalg.norm(r) <= 1.01 * tol * np.linalg.norm(phi[k])


@pytest.mark.parametrize("L,N,ranges", [(8, 40, 0), (10, 50, 3), (10, 50, 1)])
def test_two_iterations_elementwise(hq, L, N, ranges):
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 3, tau_walk=0.1)
    nrhs = 3
    phi = sources(L, N, th, nrhs, 60)
    X0 = np.stack([0.1 * inputs.complex_gaussian(L, N, 80 + k) for k in range(nrhs)])
    with hq.Config(L, N) as cfg:
        hq.set_multi_rhs(cfg, nrhs)
        hq.set_multi_ranges(cfg, ranges)
        Xg, infos = hq.cg_solve_multi(cfg, cuda(th), cuda(phi), x=cuda(X0), tol=1e-12, maxit=2, solver="pmixed",
                                      raise_on_fail=False)
    Xg = Xg.cpu().numpy()
    c = opc.coefficients(lat)
    for k in range(nrhs):
        assert infos[k]["iterations"] == 2 and infos[k]["status"] == 2, infos[k]  # HQMC_ENOTCONV after maxit
        Xo, it, _ = opc.pcg(lat, th, phi[k], c, x0=X0[k], tol=1e-30, maxit=2)
        assert it == 2
        dg, do = Xg[k] - X0[k], Xo - X0[k]
        err = np.max(np.abs(dg - do)) / np.max(np.abs(do))
        print("system", k, "two pCG iterations, FP32 vs oracle:", err)
        assert err < 1e-4


def test_same_solutions_as_one_at_a_time(hq):
    """On a tau-smooth field (a few hundred iterations), against hqmc_cg_solve with the
    same separate update and preconditioner launches: the same solutions to the
    solves' accuracy and the same iteration counts up to FP32 rounding of the sums.
    On a hot field (a few thousand iterations) the solutions still agree."""
    L, N, nrhs, tol = 12, 120, 4, 1e-9
    for start in ("ordered", "hot"):
        th = inputs.theta_ordered(L, N, 12, tau_walk=0.1) if start == "ordered" else inputs.theta_hot(L, N, 12)
        phi = cuda(sources(L, N, th, nrhs, 50))
        tht = cuda(th)
        with hq.Config(L, N) as cfg:
            hq.set_precond_fused(cfg, False)
            hq.set_multi_rhs(cfg, nrhs)
            X, infos = hq.cg_solve_multi(cfg, tht, phi, tol=tol, solver="pmixed")
            for k in range(nrhs):
                x1, i1 = hq.cg_solve(cfg, tht, phi[k].clone(), tol=tol, solver="pmixed")
                err = (torch.linalg.vector_norm(x1 - X[k]) / torch.linalg.vector_norm(x1)).item()
                print(start, k, infos[k]["iterations"], i1["iterations"], err)
                assert err < 1e-5  # both within kappa * tol of the exact solution
                if start == "ordered":
                    assert abs(infos[k]["iterations"] - i1["iterations"]) <= 0.02 * i1["iterations"] + 3


def test_event_timing_path(hq):
    """With event timing on, the systems' loop bodies are enqueued from the host (no
    graph) with events around every launch: the same solutions, and timed launches."""
    L, N, nrhs, tol = 8, 40, 3, 1e-9
    th = inputs.theta_hot(L, N, 13)
    phi = cuda(sources(L, N, th, nrhs, 20))
    with hq.Config(L, N) as cfg:
        hq.set_multi_rhs(cfg, nrhs)
        X0, i0 = hq.cg_solve_multi(cfg, cuda(th), phi, tol=tol, solver="pmixed")
        hq.set_timing(cfg, True)
        X1, i1 = hq.cg_solve_multi(cfg, cuda(th), phi, tol=tol, solver="pmixed")
        n, ms = hq.get_timing(cfg, hq.TIMER_MDAGM32)
        hq.set_timing(cfg, False)
    assert [i["iterations"] for i in i0] == [i["iterations"] for i in i1]
    assert torch.equal(X0, X1)  # the same kernels in the same order
    assert n >= max(i["iterations"] for i in i1) and ms > 0


@pytest.mark.parametrize("L,N,solver,tol,cap", [(8, 40, "pmixed", 1e-9, 5), (8, 40, "mixed", 1e-9, 2)])
def test_estimate_against_oracle(hq, L, N, solver, tol, cap):
    """cap 2 with 5 vectors: groups of 2, 2 and 1 systems."""
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, 21)
    g_o, X_o, _ = oest.estimate(lat, th, seed=5, counter=100, nrv=5, tol=1e-13)
    with hq.Config(L, N) as cfg:
        hq.set_multi_rhs(cfg, cap)
        g, infos, Gxi, xi = hq.estimate(cfg, cuda(th), 5, seed=5, counter=100, tol=tol, solver=solver,
                                        want_vectors=True, together=True)
    assert all(i["status"] == 0 and i["true_residual"] <= tol for i in infos)
    for k in range(5):
        assert np.max(np.abs(xi[k].cpu().numpy() - philox.draw_random_vector(5, 100, k, L, N))) < 1e-13
    scale = np.max(np.abs(X_o))
    assert np.max(np.abs(Gxi.cpu().numpy() - X_o)) < 1e4 * tol * scale  # kappa < 1e4 here
    assert abs(g - g_o) < 1e4 * tol


def test_estimate_agrees_with_sequential(hq):
    """24 vectors on one L = 24 field: the estimate with the systems solved together
    equals hqmc_estimate's (same draws) to the solves' accuracy, and is centred on
    the exact 1/2."""
    L, N, nrv = 24, 240, 24
    th = cuda(inputs.theta_ordered(L, N, 32, tau_walk=0.0))
    with hq.Config(L, N) as cfg:
        hq.set_multi_rhs(cfg, nrv)
        g0, inf0, G0, _ = hq.estimate(cfg, th, nrv, seed=9, tol=1e-8, solver="pmixed", want_vectors=True)
        g1, inf1, G1, xi = hq.estimate(cfg, th, nrv, seed=9, tol=1e-8, solver="pmixed", want_vectors=True,
                                       together=True)
        per = (xi.conj() * G1).sum(dim=(1, 2, 3)).cpu().numpy() / (L * L * N)
    assert all(i["status"] == 0 and i["true_residual"] <= 1e-8 for i in inf0 + inf1)
    print("iterations per vector: one at a time", np.mean([i["iterations"] for i in inf0]),
          "together", np.mean([i["iterations"] for i in inf1]))
    assert abs(g1 - g0) < 1e-5
    rel = (torch.linalg.vector_norm(G1 - G0) / torch.linalg.vector_norm(G0)).item()
    assert rel < 1e-5
    sem = per.real.std(ddof=1) / np.sqrt(nrv)
    assert abs(g1.real - 0.5) < 5 * sem


def test_edge_cases(hq):
    L, N = 8, 40
    th = inputs.theta_hot(L, N, 31)
    phi = sources(L, N, th, 3, 90)
    phi[1] = 0.0
    tht, ph = cuda(th), cuda(phi)
    with hq.Config(L, N) as cfg:
        with pytest.raises(hq.HQMCError) as e:  # no workspace yet
            hq.cg_solve_multi(cfg, tht, ph)
        assert e.value.status == hq.EINVAL
        hq.set_multi_rhs(cfg, 2)
        with pytest.raises(hq.HQMCError) as e:  # 3 systems, room for 2
            hq.cg_solve_multi(cfg, tht, ph)
        assert e.value.status == hq.EINVAL
        hq.set_multi_rhs(cfg, 3)  # grows
        with pytest.raises(hq.HQMCError) as e:
            hq.cg_solve_multi(cfg, tht, ph, solver="cg64")
        assert e.value.status == hq.EUNSUPPORTED
        x0 = torch.randn(ph.shape, dtype=torch.complex128, device="cuda")
        X, infos = hq.cg_solve_multi(cfg, tht, ph, x=x0.clone(), tol=1e-9)
        assert all(i["status"] == 0 for i in infos)
        assert torch.count_nonzero(X[1]).item() == 0  # phi = 0: X = 0 whatever the guess
        assert infos[1]["iterations"] == 0
        X, infos = hq.cg_solve_multi(cfg, tht, ph, x=x0.clone(), tol=1e-9, maxit=0, raise_on_fail=False)
        assert [i["status"] for i in infos] == [hq.ENOTCONV, hq.OK, hq.ENOTCONV]
        assert infos[0]["true_residual"] > 1e-9
        hq.set_multi_rhs(cfg, 1)  # a smaller request keeps the workspace
        X, infos = hq.cg_solve_multi(cfg, tht, ph, tol=1e-9)
        assert all(i["status"] == 0 for i in infos)
        hq.set_multi_rhs(cfg, 0)  # frees it
        with pytest.raises(hq.HQMCError) as e:
            hq.cg_solve_multi(cfg, tht, ph[:1].clone())
        assert e.value.status == hq.EINVAL


def test_bench_size_against_oracle(hq):
    """L = 66, Ntau = 660 (2,874,960 sites per system), the autotuned config of the
    bench, three systems on a tau-dependent field: each X_k meets the true residual
    against the oracle's operator."""
    L, N, nrhs = 66, 660, 3
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 2, tau_walk=0.1)
    phi = sources(L, N, th, nrhs, 70)
    with hq.Config(L, N, autotune=True) as cfg:
        hq.set_multi_rhs(cfg, nrhs)
        print("multi-system launch shape at 40 systems:", hq.multi_launch_shape(cfg, 40),
              "at 3:", hq.multi_launch_shape(cfg, nrhs))
        X, infos = hq.cg_solve_multi(cfg, cuda(th), cuda(phi), tol=1e-8, solver="pmixed")
    X = X.cpu().numpy()
    for k in range(nrhs):
        print(infos[k])
        assert infos[k]["status"] == 0 and infos[k]["true_residual"] <= 1e-8
        r = phi[k] - oracle.apply_MdagM(lat, th, X[k])
        assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi[k])
