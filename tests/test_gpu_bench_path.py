"""The benchmark's solver path at its own size, L = 66, Ntau = 660 (2,874,960 sites),
against the FP64 oracle.

The bench runs an autotuned config: the tau-walking FP32 M^dagger M in
CG-direction mode, the FP32 tau-line preconditioner in the autotuner's tile
height, and the autotuner's choice between the fused and the separate
preconditioned update.  These tests use that same config and check, for both
update forms and for a tau-independent and a tau-dependent field:

* the solution of the preconditioned mixed solver (and of the learned one) has
  a true residual ||phi - O_oracle X|| <= 1.01e-8 ||phi|| with O_oracle the
  oracle's FP64 M^dagger M (the factor 1.01 covers the FP64 rounding of the two
  residual evaluations, ~1e-14 relative each);
* the force computed from that X equals the oracle's dS_f/dtheta at the same X
  to 1e-12 relative (an FP64 kernel: rounding of ~200 operations per bond);
* two preconditioned CG iterations from a pinned guess give the oracle's two
  pCG iterations (Eq. (pCG)) element by element within FP32 rounding: the
  second direction contains z_1 = Otilde^{-1}(r_0 - alpha_0 q_0), so this checks
  the CG-direction launch's q_0 = O p_0 element-wise through an invertible map,
  and the update and preconditioner launches that follow it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import precond as opc
from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu

L, N = 66, 660
LAT = oracle.Lattice(L, N)


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


@pytest.fixture(scope="module")
def cfg(hq):
    c = hq.Config(L, N, autotune=True)  # as bench.py makes it
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def field(start):
    if start == "cold":  # tau-independent ordered start
        return inputs.theta_ordered(L, N, 1, tau_walk=0.0)
    return inputs.theta_ordered(L, N, 2, tau_walk=0.1)  # smooth walk in tau


@pytest.fixture(scope="module")
def sources():
    out = {}
    for k, start in enumerate(("cold", "walk")):
        th = field(start)
        R = inputs.complex_gaussian(L, N, 70 + k)
        out[start] = (th, oracle.apply_M(LAT, th, R, dagger=True))
    return out


def test_bench_launch_shapes(hq, cfg):
    sh = cfg.launch_shape(hq.FP32)
    pcs = hq.get_precond_shape(cfg, hq.FP32)
    print("FP32 fused M^dagger M:", sh, "preconditioner:", pcs)
    assert sh["variant"] >= 100, sh  # the persistent tau-walking kernel
    assert 16 <= pcs["tile_slices"] <= 256


@pytest.mark.parametrize("start", ["cold", "walk"])
@pytest.mark.parametrize("fused", [False, True])
def test_pmixed_solution_against_oracle(hq, cfg, sources, start, fused):
    th, phi = sources[start]
    hq.set_precond_fused(cfg, fused)
    X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver="pmixed")
    X = X.cpu().numpy()
    print(start, "fused" if fused else "separate", info)
    assert info["status"] == 0 and info["true_residual"] <= 1e-8
    r = phi - oracle.apply_MdagM(LAT, th, X)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi)


@pytest.mark.parametrize("start", ["cold", "walk"])
def test_force_on_the_solution_against_oracle(hq, cfg, sources, start):
    th, phi = sources[start]
    X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver="pmixed")
    assert info["status"] == 0
    dSf = torch.empty((N, L, L, 2), dtype=torch.float64, device="cuda")
    hq.force(cfg, cuda(th), X, dSf=dSf)
    want = oracle.fermion_dS(LAT, th, X.cpu().numpy())
    err = np.max(np.abs(dSf.cpu().numpy() - want)) / np.max(np.abs(want))
    assert err < 1e-12, err


@pytest.mark.parametrize("fused", [False, True])
def test_two_preconditioned_iterations_elementwise(hq, cfg, sources, fused):
    th, phi = sources["walk"]
    X0 = 0.1 * inputs.complex_gaussian(L, N, 81)
    hq.set_precond_fused(cfg, fused)
    Xg, info = hq.cg_solve(cfg, cuda(th), cuda(phi), x=cuda(X0), tol=1e-12, maxit=2, solver="pmixed",
                           raise_on_fail=False)
    assert info["iterations"] == 2 and info["status"] == 2  # HQMC_ENOTCONV after maxit
    Xo, it, _ = opc.pcg(LAT, th, phi, opc.coefficients(LAT), x0=X0, tol=1e-30, maxit=2)
    assert it == 2
    dg, do = Xg.cpu().numpy() - X0, Xo - X0
    err = np.max(np.abs(dg - do)) / np.max(np.abs(do))
    print("two pCG iterations, FP32 vs oracle:", err)
    # FP32 rounding (6e-8) of ~70 dependent operations per element, amplified by the
    # cancellation ||r_0|| / ||r_1|| in the first update
    assert err < 1e-4


def test_plearned_solution_against_oracle(hq, cfg, sources):
    th, phi = sources["cold"]
    net = hq.Net(seed=5)
    hq.set_preconditioner(cfg, net)
    try:
        tht = cuda(th)
        trips = []
        for k in range(2):
            ph = hq.apply_M(cfg, tht, cuda(inputs.complex_gaussian(L, N, 90 + k)), dagger=True)
            x, _ = hq.cg_solve(cfg, tht, ph, tol=1e-8, solver="pmixed")
            trips.append((ph, x))
        for _ in range(3):
            for ph, x in trips:
                net.train_step(cfg, tht, ph, x, lr=1e-3, want_loss=False)
        for start in ("cold", "walk"):
            th2, phi2 = sources[start]
            X, info = hq.cg_solve(cfg, cuda(th2), cuda(phi2), tol=1e-8, solver="plearned")
            X = X.cpu().numpy()
            print(start, "plearned", info)
            assert info["status"] == 0 and info["true_residual"] <= 1e-8
            r = phi2 - oracle.apply_MdagM(LAT, th2, X)
            assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi2)
    finally:
        hq.set_preconditioner(cfg, None)
        net.close()


def test_cg64_solution_against_oracle(hq, cfg, sources):
    """The plain FP64 comparator of the bench at the same size."""
    th, phi = sources["cold"]
    X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver="cg64")
    assert info["status"] == 0 and info["true_residual"] <= 1e-8
    r = phi - oracle.apply_MdagM(LAT, th, X.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi)
