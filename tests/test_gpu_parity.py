"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  * FP64 operators and force: max |gpu - oracle| <= 1e-12 * max |oracle|.  Both
    sides evaluate the same products in a different order (factored tanh form and
    fused kernels on the GPU, cosh/sinh factors and two applications of M in the
    oracle); the observed gap is a few 1e-15.
  * FP32 operators: 1e-5 relative (float rounding of ~30 dependent operations).
  * Solves: both sides stop at a true residual <= tol, so
    ||x_gpu - x_oracle|| / ||x|| <= 2 tol kappa(M^dagger M); the tests use tol = 1e-12
    on lattices with kappa < 1e4 and require 1e-7.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import philox
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


# several tiles and ragged cluster tails: Ntau not a multiple of the cluster size,
# Ntau below it, the smallest lattice, and the configs' sizes
APPLY_CASES = [(4, 2), (4, 5), (6, 7), (8, 13), (8, 40), (12, 17), (16, 160), (24, 240), (48, 480), (66, 660)]


@pytest.mark.parametrize("L,N", APPLY_CASES)
@pytest.mark.parametrize("variant", [1, 0])
def test_apply_MdagM_fp64(hq, L, N, variant):
    """variant 1: generic kernel; 0: the register-blocked one where a strip shape fits."""
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=1000 + 7 * L + N)
    x = inputs.complex_gaussian(L, N, seed=2000 + 7 * L + N)
    with hq.Config(L, N, variant=variant) as cfg:
        y = hq.apply_MdagM(cfg, cuda(th), cuda(x)).cpu().numpy()
    assert rel(y, oracle.apply_MdagM(lat, th, x)) < 1e-12


@pytest.mark.parametrize("L,N", [(4, 3), (8, 40), (10, 9), (24, 240)])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_M_fp64(hq, L, N, dagger):
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=3000 + L + N)
    x = inputs.complex_gaussian(L, N, seed=4000 + L + N)
    with hq.Config(L, N) as cfg:
        y = hq.apply_M(cfg, cuda(th), cuda(x), dagger=dagger).cpu().numpy()
    assert rel(y, oracle.apply_M(lat, th, x, dagger=dagger)) < 1e-12


FP32_CASES = [(4, 5), (6, 2), (8, 40), (10, 9), (12, 7), (24, 240), (48, 480), (66, 660)]


@pytest.mark.parametrize("L,N", FP32_CASES)
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_apply_fp32(hq, L, N, variant):
    """variant 1: generic kernel; 2: register-blocked; 3: persistent tau-walking
    (Ntau below, equal to and above the SM count: one slice per CTA and uneven ranges)."""
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=5000 + L)
    x = inputs.complex_gaussian(L, N, seed=6000 + L).astype(np.complex64)
    xo = x.astype(np.complex128)
    try:
        cfg = hq.Config(L, N, variant=variant)
    except hq.HQMCError as e:
        assert e.status == hq.EUNSUPPORTED and variant == 2  # no FP64 strip shape at this L
        pytest.skip("no register-blocked shape for this L")
    with cfg:
        if variant == 3:
            assert cfg.launch_shape(hq.FP32)["variant"] > 100
        y = hq.apply_MdagM(cfg, cuda(th), cuda(x)).cpu().numpy()
        ym = hq.apply_M(cfg, cuda(th), cuda(x), dagger=True).cpu().numpy()
    assert y.dtype == np.complex64
    assert rel(y, oracle.apply_MdagM(lat, th, xo)) < 1e-5
    assert rel(ym, oracle.apply_M(lat, th, xo, dagger=True)) < 1e-5


def test_special_gauge_fields(hq):
    """theta = 0, pi flux and a large-angle field (theta + 2 pi n) on the GPU path."""
    L, N = 8, 12
    lat = oracle.Lattice(L, N)
    x = inputs.complex_gaussian(L, N, seed=77)
    with hq.Config(L, N) as cfg:
        for th in (inputs.theta_zero(L, N), inputs.theta_pi_flux(L, N),
                   inputs.theta_hot(L, N, 78) + 2 * np.pi * inputs.rng(79).integers(-5, 6, (N, L, L, 2))):
            y = hq.apply_MdagM(cfg, cuda(th), cuda(x)).cpu().numpy()
            assert rel(y, oracle.apply_MdagM(lat, th, x)) < 1e-12


def test_other_model_parameters(hq):
    L, N = 6, 9
    lat = oracle.Lattice(L, N, dtau=0.05, t=1.7)
    th = inputs.theta_hot(L, N, seed=81)
    x = inputs.complex_gaussian(L, N, seed=82)
    with hq.Config(L, N, dtau=0.05, t=1.7) as cfg:
        y = hq.apply_MdagM(cfg, cuda(th), cuda(x)).cpu().numpy()
    assert rel(y, oracle.apply_MdagM(lat, th, x)) < 1e-12


@pytest.mark.parametrize("L,N", [(4, 6), (8, 40)])
def test_cg_solve_fp64(hq, L, N):
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=91)
    R = inputs.complex_gaussian(L, N, seed=92)
    phi = oracle.apply_M(lat, th, R, dagger=True)
    Xo, it_o, res_o, st_o = oracle.cg(lat, th, phi, tol=1e-12)
    with hq.Config(L, N) as cfg:
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-12)
        X = X.cpu().numpy()
    assert st_o == 0 and info["status"] == 0
    assert info["true_residual"] <= 1e-12
    assert abs(info["iterations"] - it_o) <= 2
    # the oracle's operator confirms the GPU residual
    r = phi - oracle.apply_MdagM(lat, th, X)
    assert np.linalg.norm(r) <= 1.5e-12 * np.linalg.norm(phi)
    assert rel(X, Xo) < 1e-7
    # phi^dagger X = R^dagger R (Eq. (H_hmc) at the draw point)
    assert abs(np.vdot(phi, X).real - np.vdot(R, R).real) < 1e-9 * np.vdot(R, R).real


def test_cg_iterations_match_oracle_on_a_tau_smooth_field(hq):
    """L = 12, Ntau = 120 (several thousand iterations): the GPU recurrence follows the
    oracle's, so both stop at the same iteration up to rounding."""
    L, N = 12, 120
    lat = oracle.Lattice(L, N)
    th = inputs.theta_warm(L, N, seed=201)
    phi = oracle.apply_M(lat, th, inputs.complex_gaussian(L, N, seed=202), dagger=True)
    Xo, it_o, res_o, st_o = oracle.cg(lat, th, phi, tol=1e-8, maxit=50000)
    with hq.Config(L, N) as cfg:
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, maxit=50000)
    assert st_o == 0 and info["status"] == 0
    assert abs(info["iterations"] - it_o) <= 0.01 * it_o + 2, (info["iterations"], it_o)
    r = phi - oracle.apply_MdagM(lat, th, X.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi)


def test_cg_warm_start_and_edge_cases(hq):
    L, N = 8, 16
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=101)
    phi = inputs.complex_gaussian(L, N, seed=102)
    with hq.Config(L, N) as cfg:
        tht, phit = cuda(th), cuda(phi)
        X, info = hq.cg_solve(cfg, tht, phit, tol=1e-10)
        assert info["status"] == 0
        # warm start at the solution converges with at most one more iteration
        X2, info2 = hq.cg_solve(cfg, tht, phit, x=X.clone(), tol=1e-10)
        assert info2["iterations"] <= 1 and info2["status"] == 0
        # exhausted budget
        _, info3 = hq.cg_solve(cfg, tht, phit, tol=1e-12, maxit=5, raise_on_fail=False)
        assert info3["status"] == hq.ENOTCONV and info3["iterations"] == 5
        _, it_o, res_o, st_o = oracle.cg(lat, th, phi, tol=1e-12, maxit=5)
        assert abs(info3["true_residual"] - res_o) < 1e-9 * res_o
        # zero right-hand side gives zero whatever the guess
        Z, info4 = hq.cg_solve(cfg, tht, torch.zeros_like(phit), x=torch.ones_like(phit))
        assert info4["status"] == 0 and info4["iterations"] == 0 and not Z.abs().max().item()


@pytest.mark.parametrize("L,N", [(8, 40), (24, 240)])
def test_cg_mixed_precision(hq, L, N):
    """FP32 M^dagger M inside CG with FP64 reliable updates reaches the FP64 true residual."""
    lat = oracle.Lattice(L, N)
    # fields smooth in tau, as in equilibrium (a hot start at this size needs > 6e4 iterations)
    th = inputs.theta_warm(L, N, seed=111) if L > 8 else inputs.theta_hot(L, N, seed=111)
    R = inputs.complex_gaussian(L, N, seed=112)
    phi = oracle.apply_M(lat, th, R, dagger=True)
    with hq.Config(L, N) as cfg:
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver="mixed")
        X64, info64 = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-12)
        X, X64 = X.cpu().numpy(), X64.cpu().numpy()
    assert info["status"] == 0 and info["true_residual"] <= 1e-8 and info["reliable_updates"] >= 1
    r = phi - oracle.apply_MdagM(lat, th, X)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi)
    # ||X - X64|| / ||X|| <= kappa * 1e-8; kappa < 1e5 at L = 8
    if L == 8:
        assert rel(X, X64) < 1e-3


@pytest.mark.parametrize("L,N", [(4, 3), (8, 40), (24, 240)])
@pytest.mark.parametrize("noncompact,K", [(False, 0.0), (True, 0.9)])
def test_force(hq, L, N, noncompact, K):
    lat = oracle.Lattice(L, N, J=1.25, K=K, noncompact=noncompact)
    th = inputs.theta_hot(L, N, seed=121)
    X = inputs.complex_gaussian(L, N, seed=122)  # the force formula holds for any X
    dSf_o = oracle.fermion_dS(lat, th, X)
    F_o = -dSf_o - oracle.bosonic_dS(lat, th)
    with hq.Config(L, N, J=1.25, K=K, noncompact=noncompact) as cfg:
        dSf = torch.empty((N, L, L, 2), dtype=torch.float64, device="cuda")
        F = hq.force(cfg, cuda(th), cuda(X), dSf=dSf).cpu().numpy()
        dSf = dSf.cpu().numpy()
    assert rel(dSf, dSf_o) < 1e-12
    assert rel(F, F_o) < 1e-12


def test_action_terms(hq):
    L, N = 8, 10
    lat = oracle.Lattice(L, N, J=0.8, K=0.3)
    th = inputs.theta_hot(L, N, seed=131)
    p = inputs.momenta(L, N, seed=132)
    a = inputs.complex_gaussian(L, N, seed=133)
    b = inputs.complex_gaussian(L, N, seed=134)
    with hq.Config(L, N, J=0.8, K=0.3) as cfg:
        SB, pp, ab = hq.action_terms(cfg, cuda(th), cuda(p), cuda(a), cuda(b))
    assert abs(SB - oracle.bosonic_action(lat, th)) < 1e-12 * abs(SB)
    assert abs(pp - np.sum(p * p)) < 1e-12 * pp
    assert abs(ab - np.vdot(a, b).real) < 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)


def test_draws_match_philox_definition(hq):
    L, N = 8, 40
    with hq.Config(L, N) as cfg:
        p, R, u = hq.draw(cfg, seed=0x1234_5678_9ABC, traj_counter=7)
        p, R = p.cpu().numpy(), R.cpu().numpy()
    assert np.max(np.abs(p - philox.draw_momenta(0x1234_5678_9ABC, 7, L, N))) < 1e-14
    assert np.max(np.abs(R - philox.draw_pseudofermion(0x1234_5678_9ABC, 7, L, N))) < 1e-14
    assert u == philox.draw_metropolis(0x1234_5678_9ABC, 7)


def test_trajectory_matches_oracle(hq):
    """Config-1 sized trajectory with supplied draws: same dH, end point and decision."""
    L, N = 8, 40
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=141)
    p = inputs.momenta(L, N, seed=142)
    R = inputs.complex_gaussian(L, N, seed=143)
    for u in (0.3, 0.999999):
        ref = oracle.trajectory(lat, th, p, R, u=u, nsteps=10, dt=0.02, tol=1e-12)
        with hq.Config(L, N) as cfg:
            tht = cuda(th)
            info = hq.trajectory(cfg, tht, p_in=cuda(p), R_in=cuda(R), u_in=u, nsteps=10, dt=0.02, tol=1e-12)
            th_out = tht.cpu().numpy()
        assert info["status"] == 0 and info["cg_solves"] == 11
        assert abs(info["H0"] - ref["H0"]) < 1e-12 * abs(ref["H0"])
        assert abs(info["dH"] - ref["dH"]) < 1e-7
        assert bool(info["accepted"]) == ref["accepted"]
        assert np.max(np.abs(th_out - ref["theta"])) < 1e-8
        assert abs(info["cg_iterations"] - ref["cg_iterations"]) <= 2 * 11


def test_trajectory_with_device_draws(hq):
    """Draws made inside the library reproduce the oracle's Philox draws."""
    L, N = 6, 12
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=151)
    seed, ctr = 99, 5
    ref = oracle.trajectory(lat, th, philox.draw_momenta(seed, ctr, L, N), philox.draw_pseudofermion(seed, ctr, L, N),
                            u=philox.draw_metropolis(seed, ctr), nsteps=5, dt=0.03, tol=1e-12)
    with hq.Config(L, N) as cfg:
        tht = cuda(th)
        info = hq.trajectory(cfg, tht, seed=seed, traj_counter=ctr, nsteps=5, dt=0.03, tol=1e-12)
    assert abs(info["dH"] - ref["dH"]) < 1e-7
    assert info["u"] == philox.draw_metropolis(seed, ctr)
    assert bool(info["accepted"]) == ref["accepted"]


def test_leapfrog_reversible(hq):
    """Integrate, flip p, integrate back (L = 24; Ntau = 48 keeps kappa small enough for
    CG to reach a true residual of 1e-11, which reversibility to 1e-9 needs)."""
    L, N = 24, 48
    th = inputs.theta_warm(L, N, seed=161)
    p = inputs.momenta(L, N, seed=162)
    R = inputs.complex_gaussian(L, N, seed=163)
    with hq.Config(L, N) as cfg:
        tht, pt = cuda(th), cuda(p)
        phi = hq.apply_M(cfg, tht, cuda(R), dagger=True)
        X = torch.zeros_like(phi)
        i1 = hq.leapfrog(cfg, tht, pt, phi, X, nsteps=3, dt=0.01, tol=1e-11)
        pt.neg_()
        i2 = hq.leapfrog(cfg, tht, pt, phi, X, nsteps=3, dt=0.01, tol=1e-11)
        assert i1["status"] == 0 and i2["status"] == 0
        assert (tht.cpu().numpy() - th).__abs__().max() < 1e-9
        assert (pt.cpu().numpy() + p).__abs__().max() < 1e-9


def test_leapfrog_reversible_to_1e10(hq):
    """The reversibility check as the oracle pins it: CG to a true residual of 1e-12
    and theta, p back to 1e-10 (L = 8, Ntau = 16: kappa small enough for FP64 CG to
    reach 1e-12)."""
    L, N = 8, 16
    th = inputs.theta_warm(L, N, seed=171)
    p = inputs.momenta(L, N, seed=172)
    R = inputs.complex_gaussian(L, N, seed=173)
    with hq.Config(L, N) as cfg:
        tht, pt = cuda(th), cuda(p)
        phi = hq.apply_M(cfg, tht, cuda(R), dagger=True)
        X = torch.zeros_like(phi)
        i1 = hq.leapfrog(cfg, tht, pt, phi, X, nsteps=3, dt=0.02, tol=1e-12)
        pt.neg_()
        i2 = hq.leapfrog(cfg, tht, pt, phi, X, nsteps=3, dt=0.02, tol=1e-12)
        assert i1["status"] == 0 and i2["status"] == 0
        assert (tht.cpu().numpy() - th).__abs__().max() <= 1e-10
        assert (pt.cpu().numpy() + p).__abs__().max() <= 1e-10


def test_energy_conservation_at_config2_size(hq):
    """At L = 24, Ntau = 240 from a cold start: dH shrinks ~4x when dt halves at fixed
    trajectory length (leapfrog error O(dt^2))."""
    L, N = 24, 240
    th = inputs.theta_ordered(L, N, seed=171, tau_walk=0.0)
    p = inputs.momenta(L, N, seed=172)
    R = inputs.complex_gaussian(L, N, seed=173)
    dHs = []
    with hq.Config(L, N) as cfg:
        for ns, dt in ((4, 0.002), (8, 0.001)):
            info = hq.trajectory(cfg, cuda(th), p_in=cuda(p), R_in=cuda(R), u_in=0.0, nsteps=ns, dt=dt, tol=1e-8)
            assert info["status"] == 0 and info["max_true_residual"] <= 1e-8
            dHs.append(abs(info["dH"]))
    assert 2.5 < dHs[0] / dHs[1] < 6.0, dHs


def test_invalid_arguments(hq):
    for L, N in ((5, 8), (2, 8), (4, 1), (70, 10)):
        with pytest.raises(hq.HQMCError) as e:
            hq.Config(L, N)
        assert e.value.status == hq.EINVAL
    with hq.Config(4, 4) as cfg:
        th = torch.zeros((4, 4, 4, 2), dtype=torch.float64, device="cuda")
        x = torch.zeros((4, 4, 4), dtype=torch.complex128, device="cuda")
        with pytest.raises(hq.HQMCError) as e:
            hq.apply_MdagM(cfg, th, x, y=x)
        assert e.value.status == hq.EINVAL
        with pytest.raises(ValueError):
            hq.apply_MdagM(cfg, th, torch.zeros((4, 4, 5), dtype=torch.complex128, device="cuda"))


@pytest.mark.parametrize("L,N", [(8, 13), (24, 240), (48, 480), (66, 660)])
def test_autotuned_shapes_keep_parity(hq, L, N):
    """The autotuner picks kernel variant and cluster size; results must not change."""
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=181)
    x = inputs.complex_gaussian(L, N, seed=182)
    with hq.Config(L, N, autotune=True) as cfg:
        for prec in (hq.FP64, hq.FP32):
            sh = cfg.launch_shape(prec)
            assert sh["tuned_us"] > 0 and 1 <= sh["cluster"] <= 8
        y = hq.apply_MdagM(cfg, cuda(th), cuda(x)).cpu().numpy()
        y32 = hq.apply_MdagM(cfg, cuda(th), cuda(x.astype(np.complex64))).cpu().numpy()
    yo = oracle.apply_MdagM(lat, th, x)
    assert rel(y, yo) < 1e-12
    assert rel(y32, oracle.apply_MdagM(lat, th, x.astype(np.complex64).astype(np.complex128))) < 1e-5


def test_cg_with_each_kernel_variant(hq):
    L, N = 8, 40
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, seed=191)
    phi = inputs.complex_gaussian(L, N, seed=192)
    Xo, it_o, _, _ = oracle.cg(lat, th, phi, tol=1e-12)
    for variant in (1, 2, 3):
        with hq.Config(L, N, variant=variant) as cfg:
            X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-12)
            Xm, infom = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-9, solver="mixed")
        assert info["status"] == 0 and abs(info["iterations"] - it_o) <= 2
        assert rel(X.cpu().numpy(), Xo) < 1e-7
        assert infom["status"] == 0 and infom["true_residual"] <= 1e-9


def test_configs_of_different_sizes_coexist(hq):
    """A small config made after a large one must not shrink kernel limits the large one needs."""
    big, small = hq.Config(48, 16), hq.Config(8, 8)
    try:
        for cfg, (L, N) in ((big, (48, 16)), (small, (8, 8)), (big, (48, 16))):
            lat = oracle.Lattice(L, N)
            th = inputs.theta_hot(L, N, seed=211)
            x = inputs.complex_gaussian(L, N, seed=212)
            y = hq.apply_MdagM(cfg, cuda(th), cuda(x)).cpu().numpy()
            assert rel(y, oracle.apply_MdagM(lat, th, x)) < 1e-12
    finally:
        big.close()
        small.close()


def test_timing_counters(hq):
    L, N = 8, 16
    with hq.Config(L, N) as cfg:
        th = cuda(inputs.theta_hot(L, N, 171))
        x = cuda(inputs.complex_gaussian(L, N, 172))
        hq.set_timing(cfg, True)
        for _ in range(3):
            hq.apply_MdagM(cfg, th, x)
        n, ms = hq.get_timing(cfg, hq.TIMER_MDAGM)
        hq.set_timing(cfg, False)
    assert n == 3 and ms > 0


def test_resume_from_checkpoint_is_bit_exact(hq, tmp_path):
    """Every random number of trajectory k is a function of (seed, k): a chain saved
    after two trajectories and resumed continues bit for bit."""
    L, N = 8, 16
    th = cuda(inputs.theta_hot(L, N, 61))
    kw = dict(nsteps=3, dt=0.02, tol=1e-10)
    path = str(tmp_path / "chain.ckp")
    with hq.Config(L, N) as cfg:
        acc = 0
        for k in range(2):
            acc += hq.trajectory(cfg, th, seed=9, traj_counter=k, **kw)["accepted"]
        hq.save_checkpoint(path, th, seed=9, traj_counter=2, dt=0.02, nsteps=3, trajectories=2, accepted=acc)
        a = hq.trajectory(cfg, th, seed=9, traj_counter=2, **kw)
        hdr, th_b, _ = hq.load_checkpoint(path)
        th_b = th_b.cuda()
        b = hq.trajectory(cfg, th_b, seed=hdr["seed"], traj_counter=hdr["traj_counter"], nsteps=hdr["nsteps"],
                          dt=hdr["dt"], tol=1e-10)
    assert a["dH"] == b["dH"] and a["accepted"] == b["accepted"]
    assert torch.equal(th, th_b)
