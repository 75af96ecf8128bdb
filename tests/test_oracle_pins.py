"""Pins of the FP64 CPU oracle against the mathematics (no GPU).

Each test checks the oracle against something other than itself: dense matrices
exponentiated with scipy, closed-form spectra, the determinant identity of
Eq. (eq4), gauge covariance, finite differences and integrator invariants.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2508_16298_gb300 import inputs
from tests import dense

LAT = oracle.Lattice(L=4, Ntau=5, dtau=0.1, t=1.0, J=1.0)


def oracle_matrix(fn, n):
    """Columns of a linear map given as a function on flat vectors."""
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1.0
        cols.append(fn(e).reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("L", [4, 6])
def test_B_equals_product_of_matrix_exponentials(L):
    """Eq. (eq24) with each e^{V_f/2} computed by expm of the dense hopping matrix."""
    lat = oracle.Lattice(L=L, Ntau=2, dtau=0.1, t=1.0)
    th = inputs.theta_hot(L, 1, seed=11)[0]
    B = oracle_matrix(lambda v: oracle.apply_B(lat, th, v.reshape(L, L)), L * L)
    Bd = dense.dense_B(L, th, lat.dtau * lat.t)
    assert np.max(np.abs(B - Bd)) < 1e-14 * np.max(np.abs(Bd)) * 10
    # B^dagger through the adjoint path, and B itself Hermitian with det 1
    Bh = oracle_matrix(lambda v: oracle.apply_B(lat, th, v.reshape(L, L), adjoint=True), L * L)
    assert np.max(np.abs(Bh - Bd.conj().T)) < 1e-13
    assert np.max(np.abs(B - B.conj().T)) < 1e-13
    assert abs(np.linalg.det(B) - 1.0) < 1e-12


def test_B_hopping_nonunit_t():
    """The exponent is dtau * t * T_ij: scaling t by 2 equals scaling dtau by 2."""
    th = inputs.theta_hot(4, 1, seed=3)[0]
    v = inputs.complex_gaussian(4, 1, seed=4)[0]
    a = oracle.apply_B(oracle.Lattice(L=4, Ntau=2, dtau=0.05, t=2.0), th, v)
    b = oracle.apply_B(oracle.Lattice(L=4, Ntau=2, dtau=0.1, t=1.0), th, v)
    assert np.allclose(a, b, rtol=1e-14, atol=1e-14)


def test_symmetric_checkerboard_is_second_order():
    """Symmetric splitting: ||B - e^{dtau H}|| = O(dtau^3); halving dtau divides it by ~8."""
    L = 6
    th = inputs.theta_hot(L, 1, seed=5)[0]
    H = dense.hopping(L, th)
    errs = []
    for dtau in (0.2, 0.1, 0.05):
        lat = oracle.Lattice(L=L, Ntau=2, dtau=dtau)
        B = oracle_matrix(lambda v: oracle.apply_B(lat, th, v.reshape(L, L)), L * L)
        errs.append(np.linalg.norm(B - sla.expm(dtau * H), 2))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 < r1 < 9.0 and 7.5 < r2 < 8.5, errs


def test_M_and_Mdag_match_dense():
    th = inputs.theta_hot(LAT.L, LAT.Ntau, seed=21)
    x = inputs.complex_gaussian(LAT.L, LAT.Ntau, seed=22)
    Md = dense.dense_M(LAT.L, LAT.Ntau, th, LAT.dtau * LAT.t)
    y = oracle.apply_M(LAT, th, x).reshape(-1)
    yd = oracle.apply_M(LAT, th, x, dagger=True).reshape(-1)
    assert np.allclose(y, Md @ x.reshape(-1), rtol=0, atol=1e-13)
    assert np.allclose(yd, Md.conj().T @ x.reshape(-1), rtol=0, atol=1e-13)
    z = oracle.apply_MdagM(LAT, th, x).reshape(-1)
    assert np.allclose(z, Md.conj().T @ Md @ x.reshape(-1), rtol=0, atol=1e-12)


def test_logdet_identity():
    """Eq. (eq4): det M = det(1 + B_{Ntau-1} ... B_0), real and positive here."""
    lat = oracle.Lattice(L=4, Ntau=6, dtau=0.1)
    th = inputs.theta_hot(4, 6, seed=31)
    n = lat.n_sites
    M = oracle_matrix(lambda v: oracle.apply_M(lat, th, v.reshape(6, 4, 4)), n)
    s1, ld1 = np.linalg.slogdet(M)
    P = np.eye(16, dtype=complex)
    for tau in range(6):
        Bt = oracle_matrix(lambda v: oracle.apply_B(lat, th[tau], v.reshape(4, 4)), 16)
        P = Bt @ P
    s2, ld2 = np.linalg.slogdet(np.eye(16) + P)
    assert abs(ld1 - ld2) < 1e-12 * max(1.0, abs(ld1))
    assert abs(s1 - s2) < 1e-12
    assert abs(s1.imag) < 1e-10  # det M real (Methods, sign-problem-free)


def _chain_mu(L, a):
    q = 2 * np.pi * np.arange(L // 2) / (L // 2)
    # cosh^2 a - sinh^2 a = 1 at q = pi; rounding can land just below 1
    return np.arccosh(np.maximum(1.0, np.cosh(a) ** 2 + np.sinh(a) ** 2 * np.cos(q)))


def test_zero_flux_spectrum_closed_form():
    """theta = 0: spec(B) = {e^{+-mu(qx) +- mu(qy)}} with cosh mu = cosh^2 a + sinh^2 a cos q,
    and spec(M^dagger M) = {1 + b^2 - 2 b cos((2n+1) pi / Ntau)}."""
    L, N = 4, 6
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1)
    th = inputs.theta_zero(L, N)
    a = lat.dtau * lat.t
    mu = _chain_mu(L, a)
    ex = np.concatenate([mu, -mu])
    bvals = np.sort(np.exp(ex[:, None] + ex[None, :]).reshape(-1))
    B = oracle_matrix(lambda v: oracle.apply_B(lat, th[0], v.reshape(L, L)), L * L)
    assert np.allclose(np.sort(np.linalg.eigvalsh(B)), bvals, rtol=1e-13, atol=0)
    w = (2 * np.arange(N) + 1) * np.pi / N
    lam = np.sort((1 + bvals[:, None] ** 2 - 2 * bvals[:, None] * np.cos(w[None, :])).reshape(-1))
    O = oracle_matrix(lambda v: oracle.apply_MdagM(lat, th, v.reshape(N, L, L)), lat.n_sites)
    assert np.allclose(np.sort(np.linalg.eigvalsh(O)), lam, rtol=1e-12, atol=1e-13)


def test_plane_wave_eigenvector_in_time():
    """At tau-independent theta, x_tau = e^{i w tau} u with B u = b u and
    w = (2n+1) pi / Ntau is an eigenvector of M^dagger M with 1 + b^2 - 2 b cos w."""
    L, N = 4, 8
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1)
    th1 = inputs.theta_hot(L, 1, seed=41)[0]
    th = np.broadcast_to(th1, (N, L, L, 2)).copy()
    B = dense.dense_B(L, th1, lat.dtau)
    bs, U = np.linalg.eigh(B)
    k = 3
    for n in (0, 2):
        w = (2 * n + 1) * np.pi / N
        x = np.exp(1j * w * np.arange(N))[:, None] * U[:, k][None, :]
        y = oracle.apply_MdagM(lat, th, x.reshape(N, L, L)).reshape(N, -1)
        lam = 1 + bs[k] ** 2 - 2 * bs[k] * np.cos(w)
        assert np.allclose(y, lam * x, rtol=0, atol=1e-13)


def test_pi_flux_small_dtau_limit():
    """pi flux: the hopping spectrum is +-2t sqrt(cos^2 kx + cos^2 ky) over the magnetic
    zone (the pi-flux background of the Methods' preconditioner); the checkerboard B has
    log-eigenvalues dtau times that, to O(dtau^3)."""
    L = 8
    lat = oracle.Lattice(L=L, Ntau=2, dtau=0.05)
    th = inputs.theta_pi_flux(L, 1)[0]
    k = 2 * np.pi * np.arange(L) / L
    e = 2 * np.sqrt(np.cos(k)[:, None] ** 2 + np.cos(k)[None, :] ** 2).reshape(-1)
    ev = np.sort(np.linalg.eigvalsh(dense.hopping(L, th)))
    # over the full zone every magnetic-zone level appears twice: {ev, ev} = {e, -e}
    assert np.allclose(np.sort(np.concatenate([ev, ev])), np.sort(np.concatenate([e, -e])), atol=1e-12)
    B = oracle_matrix(lambda v: oracle.apply_B(lat, th, v.reshape(L, L)), L * L)
    got = np.sort(np.log(np.linalg.eigvalsh(B)))
    assert np.allclose(got, lat.dtau * ev, atol=5 * lat.dtau ** 3)


def test_gauge_covariance_and_2pi_periodicity():
    """theta'_ij = theta_ij + l_i - l_j (l tau-independent): O(theta') D x = D O(theta) x."""
    L, N = 4, 5
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1)
    th = inputs.theta_hot(L, N, seed=51)
    lam = inputs.rng(52).uniform(-np.pi, np.pi, size=(L, L))  # [y, x]
    thg = th.copy()
    thg[..., 0] += lam[None, :, :] - np.roll(lam, -1, axis=1)[None, :, :]
    thg[..., 1] += lam[None, :, :] - np.roll(lam, -1, axis=0)[None, :, :]
    D = np.exp(1j * lam)[None, :, :]
    x = inputs.complex_gaussian(L, N, seed=53)
    lhs = oracle.apply_MdagM(lat, thg, D * x)
    rhs = D * oracle.apply_MdagM(lat, th, x)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-13)
    shift = 2 * np.pi * inputs.rng(54).integers(-3, 4, size=th.shape)
    assert np.allclose(oracle.apply_MdagM(lat, th + shift, x), oracle.apply_MdagM(lat, th, x),
                       rtol=0, atol=1e-12)
    # the fermion force is gauge invariant
    R = inputs.complex_gaussian(L, N, seed=55)
    eta = oracle.apply_M(lat, th, R, dagger=True)
    X, *_ = oracle.cg(lat, th, eta, tol=1e-13)
    etag = D * eta
    Xg, *_ = oracle.cg(lat, thg, etag, tol=1e-13)
    assert np.allclose(oracle.fermion_dS(lat, th, X), oracle.fermion_dS(lat, thg, Xg), atol=1e-9)


def test_MdagM_hermitian_positive():
    th = inputs.theta_hot(LAT.L, LAT.Ntau, seed=61)
    x = inputs.complex_gaussian(LAT.L, LAT.Ntau, seed=62)
    y = inputs.complex_gaussian(LAT.L, LAT.Ntau, seed=63)
    Ox, Oy = oracle.apply_MdagM(LAT, th, x), oracle.apply_MdagM(LAT, th, y)
    assert abs(oracle.dot(y, Ox) - np.conj(oracle.dot(x, Oy))) < 1e-12 * abs(oracle.dot(y, Ox))
    xo = oracle.dot(x, Ox)
    assert xo.real > 0 and abs(xo.imag) < 1e-12 * xo.real


def test_cg_matches_dense_solve_and_R_norm():
    """CG solution against numpy.linalg.solve; eta^dagger X = R^dagger R for eta = M^dagger R."""
    L, N = 4, 6
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1)
    th = inputs.theta_hot(L, N, seed=71)
    R = inputs.complex_gaussian(L, N, seed=72)
    eta = oracle.apply_M(lat, th, R, dagger=True)
    X, it, res, st = oracle.cg(lat, th, eta, tol=1e-13)
    assert st == 0 and res <= 1e-13 and it > 0
    Md = dense.dense_M(L, N, th, lat.dtau)
    Xd = np.linalg.solve(Md.conj().T @ Md, eta.reshape(-1))
    assert np.allclose(X.reshape(-1), Xd, rtol=0, atol=1e-10 * np.max(np.abs(Xd)))
    # M X = R exactly when eta = M^dagger R
    assert np.allclose(oracle.apply_M(lat, th, X), R, atol=1e-10)
    assert abs(oracle.fermion_action(lat, eta, X) - np.vdot(R, R).real) < 1e-10 * np.vdot(R, R).real
    # warm start from the solution converges at once
    X2, it2, res2, st2 = oracle.cg(lat, th, eta, x0=X, tol=1e-12)
    assert st2 == 0 and it2 <= 2
    # an exhausted budget reports failure
    _, it3, res3, st3 = oracle.cg(lat, th, eta, tol=1e-14, maxit=3)
    assert st3 == 1 and it3 == 3 and res3 > 1e-14


def test_cg_zero_rhs():
    th = inputs.theta_hot(4, 4, seed=81)
    lat = oracle.Lattice(L=4, Ntau=4)
    X, it, res, st = oracle.cg(lat, th, np.zeros((4, 4, 4), complex))
    assert st == 0 and it == 0 and not X.any()


@pytest.mark.parametrize("L,N", [(4, 4), (4, 3)])
def test_fermion_force_finite_differences(L, N):
    """Supplement SI: dS_f/dtheta against central differences of eta^dagger (M^dagger M)^{-1} eta
    computed with dense matrices, on every bond (including the wrap bonds and tau = Ntau-1)."""
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1)
    th = inputs.theta_hot(L, N, seed=91)
    R = inputs.complex_gaussian(L, N, seed=92)
    eta = oracle.apply_M(lat, th, R, dagger=True)
    X, *_ = oracle.cg(lat, th, eta, tol=1e-14)
    g = oracle.fermion_dS(lat, th, X)
    h = 1e-5
    fd = np.zeros_like(th)
    for idx in np.ndindex(th.shape):
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        fd[idx] = (dense.fermion_action_dense(L, N, tp, lat.dtau, eta)
                   - dense.fermion_action_dense(L, N, tm, lat.dtau, eta)) / (2 * h)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(g - fd)) < 1e-6 * scale, np.max(np.abs(g - fd)) / scale


@pytest.mark.parametrize("noncompact,K", [(False, 0.0), (False, 0.7), (True, 0.0), (True, 1.0)])
def test_bosonic_action_and_force(noncompact, K):
    L, N = 4, 3
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1, J=1.25, K=K, noncompact=noncompact)
    th = inputs.theta_hot(L, N, seed=101)
    S = oracle.bosonic_action(lat, th)
    Sd = dense.bosonic_action_direct(L, N, th, lat.dtau, lat.J, lat.K, noncompact)
    assert abs(S - Sd) < 1e-12 * abs(Sd)
    g = oracle.bosonic_dS(lat, th)
    h = 1e-6
    for idx in list(np.ndindex(th.shape))[::5]:
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        fd = (oracle.bosonic_action(lat, tp) - oracle.bosonic_action(lat, tm)) / (2 * h)
        assert abs(g[idx] - fd) < 1e-6 * max(1.0, abs(fd))


def _traj_inputs(L, N, seed):
    th = inputs.theta_hot(L, N, seed)
    p = inputs.momenta(L, N, seed + 1)
    R = inputs.complex_gaussian(L, N, seed + 2)
    return th, p, R


@pytest.mark.slow
def test_energy_violation_scales_as_dt_squared():
    """Leapfrog at fixed trajectory length: |dH| ~ dt^2 (slope 2 on a log-log plot)."""
    L, N = 4, 8
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1, J=1.0)
    th, p, R = _traj_inputs(L, N, 200)
    T = 0.2
    dts, dHs = [], []
    for ns in (4, 8, 16, 32):
        out = oracle.trajectory(lat, th, p, R, u=0.0, nsteps=ns, dt=T / ns, tol=1e-13)
        dts.append(T / ns)
        dHs.append(abs(out["dH"]))
    slope = np.polyfit(np.log(dts), np.log(dHs), 1)[0]
    assert 1.9 < slope < 2.1, (dts, dHs, slope)


def test_leapfrog_reversibility():
    L, N = 4, 6
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1)
    th, p, R = _traj_inputs(L, N, 300)
    eta = oracle.apply_M(lat, th, R, dagger=True)
    th1, p1, X1, it, bad = oracle.leapfrog(lat, th, p, eta, nsteps=6, dt=0.03, tol=1e-13)
    assert bad == 0
    th2, p2, X2, it2, bad2 = oracle.leapfrog(lat, th1, -p1, eta, X0=X1, nsteps=6, dt=0.03, tol=1e-13)
    assert np.max(np.abs(th2 - th)) < 1e-10
    assert np.max(np.abs(p2 + p)) < 1e-10


def test_trajectory_accept_reject_and_H0():
    L, N = 4, 4
    lat = oracle.Lattice(L=L, Ntau=N, dtau=0.1)
    th, p, R = _traj_inputs(L, N, 400)
    acc = oracle.trajectory(lat, th, p, R, u=0.0, nsteps=3, dt=0.05)
    assert acc["accepted"] and not np.array_equal(acc["theta"], th)
    rej = oracle.trajectory(lat, th, p, R, u=np.nextafter(1.0, 0.0), nsteps=3, dt=0.05)
    if rej["dH"] > 0:
        assert not rej["accepted"] and np.array_equal(rej["theta"], th)
    # H0 = S_B + sum p^2 + R^dagger R
    H0 = oracle.bosonic_action(lat, th) + np.sum(p * p) + np.vdot(R, R).real
    assert abs(acc["H0"] - H0) < 1e-12 * abs(H0)
    # identical inputs give identical results (deterministic reductions)
    again = oracle.trajectory(lat, th, p, R, u=0.0, nsteps=3, dt=0.05)
    assert again["H1"] == acc["H1"] and np.array_equal(again["theta"], acc["theta"])
