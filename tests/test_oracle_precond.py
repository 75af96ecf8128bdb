"""Pins of the oracle's tau-line preconditioner (oracle/precond.py) to
mathematics that does not go through its own code paths."""
import numpy as np
import pytest

import oracle
from oracle import precond as pc
from paper_2508_16298_gb300 import inputs


def antiperiodic_shift(N):
    """Dense S: (S u)_tau = u_{tau-1}, (S u)_0 = -u_{N-1}."""
    S = np.zeros((N, N))
    for t in range(1, N):
        S[t, t - 1] = 1.0
    S[0, N - 1] = -1.0
    return S


def line_matrix(c, N):
    S = antiperiodic_shift(N)
    return c.a * np.eye(N) - c.b * (S + S.T)


def test_coefficients_small_dtau_closed_form():
    """B = exp(dtau K) + O(dtau^3) with K the hopping matrix (4 neighbours, |K_ij| = t):
    B_ss = 1 + dtau^2 * 4 t^2 / 2 and sum_j |B_js|^2 = (B^2)_ss = 1 + 2 dtau^2 * 4 t^2,
    up to O(dtau^4) (Methods, Eq. (eq24); the pi flux only enters at order dtau^4)."""
    for dtau in (0.01, 0.02):
        c = pc.coefficients(oracle.Lattice(8, 4, dtau=dtau, t=1.0))
        assert abs(c.b - (1 + 2 * dtau ** 2)) < 5 * dtau ** 4
        assert abs(c.a - (2 + 8 * dtau ** 2)) < 20 * dtau ** 4


def test_coefficients_do_not_depend_on_size():
    """The bulk entries are the same for every lattice large enough to hold B's range."""
    c8 = pc.coefficients(oracle.Lattice(8, 4))
    c12 = pc.coefficients(oracle.Lattice(12, 4))
    assert abs(c8.a - c12.a) < 1e-14 and abs(c8.b - c12.b) < 1e-14 and c8.W == c12.W


def test_bulk_cholesky_factor_reproduces_the_line_matrix():
    """(b/rho)(1 - rho S)(1 - rho S^dagger) = a - b (S + S^dagger) exactly (S unitary)."""
    c = pc.coefficients(oracle.Lattice(8, 12))
    N = 12
    S = antiperiodic_shift(N)
    lhs = (c.b / c.rho) * (np.eye(N) - c.rho * S) @ (np.eye(N) - c.rho * S.T)
    assert np.max(np.abs(lhs - line_matrix(c, N))) < 1e-13
    assert 0 < c.rho < 1


def test_untruncated_series_is_the_exact_line_inverse():
    """With all N powers kept (rho^N ~ 1e-18) (rho/b) F^dagger F equals the inverse of T."""
    lat = oracle.Lattice(4, 200)
    c0 = pc.coefficients(lat)
    c = pc.LineCoefficients(c0.a, c0.b, c0.rho, lat.Ntau - 1)
    N = lat.Ntau
    e = np.zeros((N, 4, 4), dtype=np.complex128)
    cols = []
    for t in range(N):
        e[:] = 0
        e[t, 1, 2] = 1.0
        cols.append(pc.apply(c, e)[:, 1, 2])
    dense = np.array(cols).T
    assert np.max(np.abs(dense - np.linalg.inv(line_matrix(c, N)))) < 1e-12


def test_truncation_rule():
    """L^{-1} keeps exactly the entries sqrt(rho/b) rho^m >= 1e-3."""
    c = pc.coefficients(oracle.Lattice(8, 4))
    pref = np.sqrt(c.rho / c.b)
    assert pref * c.rho ** c.W >= 1e-3 > pref * c.rho ** (c.W + 1)
    # F_W as a dense matrix: rho^m on the m-th subdiagonal, sign -1 past the wrap
    N = 50
    cw = pc.LineCoefficients(c.a, c.b, c.rho, c.W)
    F = np.array([pc.apply_F(cw, np.eye(N)[:, j].astype(complex)) for j in range(N)]).T.real
    for i in range(N):
        for j in range(N):
            m = (i - j) % N
            want = c.rho ** m if m <= c.W else 0.0
            if i - j < 0 and m <= c.W:
                want = -want
            assert abs(F[i, j] - want) < 1e-15


def test_preconditioner_is_hermitian_positive_and_site_diagonal():
    lat = oracle.Lattice(4, 40)
    c = pc.coefficients(lat)
    rng = np.random.default_rng(3)
    x = inputs.complex_gaussian(4, 40, 4)
    y = inputs.complex_gaussian(4, 40, 5)
    Px, Py = pc.apply(c, x), pc.apply(c, y)
    assert abs(np.vdot(y, Px) - np.vdot(Py, x)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    assert np.vdot(x, Px).real > 0
    # a vector on one site's tau line stays there
    e = np.zeros((40, 4, 4), dtype=np.complex128)
    e[:, 2, 3] = rng.standard_normal(40)
    Pe = pc.apply(c, e)
    mask = np.ones((4, 4), bool)
    mask[2, 3] = False
    assert np.max(np.abs(Pe[:, mask])) == 0.0
    # smallest eigenvalue of the line operator (dense) is positive
    N = 40
    dense = np.array([pc.apply(c, np.tile(np.eye(N)[:, j][:, None, None], (1, 4, 4)).astype(complex))[:, 0, 0]
                      for j in range(N)]).T
    assert np.min(np.linalg.eigvalsh(0.5 * (dense + dense.T))) > 0


def test_pcg_solves_the_system_exactly_on_a_tiny_lattice():
    lat = oracle.Lattice(4, 6)
    th = inputs.theta_hot(4, 6, 11)
    phi = inputs.complex_gaussian(4, 6, 12)
    n = lat.n_sites
    cols = [oracle.apply_MdagM(lat, th, np.eye(n)[:, j].reshape(6, 4, 4).astype(complex)).reshape(-1)
            for j in range(n)]
    X_dense = np.linalg.solve(np.array(cols).T, phi.reshape(-1)).reshape(6, 4, 4)
    X, its, res = pc.pcg(lat, th, phi, pc.coefficients(lat), tol=1e-13)
    assert res <= 1e-13
    assert np.max(np.abs(X - X_dense)) < 1e-9 * np.max(np.abs(X_dense))


def test_pcg_cuts_iterations_on_a_tau_smooth_field():
    """The tau lines carry the near-singular low Matsubara modes; preconditioning them
    cuts the iteration count several-fold (measured 348 -> 47 here)."""
    lat = oracle.Lattice(8, 80)
    th = inputs.theta_ordered(8, 80, 3, tau_walk=0.0)
    phi = inputs.complex_gaussian(8, 80, 5)
    X, its, res = pc.pcg(lat, th, phi, pc.coefficients(lat), tol=1e-8)
    X2, its2, _, _ = oracle.cg(lat, th, phi, tol=1e-8)
    assert res <= 1e-8 and its * 4 < its2
    assert np.linalg.norm(X - X2) < 1e-6 * np.linalg.norm(X2)


def test_F_and_its_adjoint_against_the_dense_shift():
    """F_W and F_W^dagger as dense polynomials in the antiperiodic shift matrix: apply_F
    is sum rho^m S^m and apply_F_adj its transpose, on lines short enough to wrap
    several times (N < W)."""
    for N in (5, 12, 40):
        lat = oracle.Lattice(4, N)
        c = pc.coefficients(lat)
        S = antiperiodic_shift(N)
        F = sum(c.rho ** m * np.linalg.matrix_power(S, m) for m in range(c.W + 1))
        u = inputs.complex_gaussian(4, N, 500 + N)
        Fu = np.einsum("ts,s...->t...", F, u)
        Ftu = np.einsum("st,s...->t...", F, u)
        assert np.max(np.abs(pc.apply_F(c, u) - Fu)) < 1e-12 * np.max(np.abs(Fu))
        assert np.max(np.abs(pc.apply_F_adj(c, u) - Ftu)) < 1e-12 * np.max(np.abs(Ftu))


def test_rz_is_the_scaled_norm_of_F_r():
    """<r, Otilde^{-1} r> = (rho/b) ||F_W r||^2, the form in which the GPU sums the
    pCG step length (each tile adds |x_tau|^2 of its own slices in the forward pass)."""
    lat = oracle.Lattice(4, 40)
    c = pc.coefficients(lat)
    r = inputs.complex_gaussian(4, 40, 611)
    rz = np.vdot(r.reshape(-1), pc.apply(c, r).reshape(-1))
    x = pc.apply_F(c, r)
    assert abs(rz.imag) < 1e-12 * abs(rz.real)
    assert abs(rz.real - c.scale * np.vdot(x.reshape(-1), x.reshape(-1)).real) < 1e-12 * rz.real
