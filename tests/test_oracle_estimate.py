"""Pins of the oracle's stochastic estimator (oracle/estimate.py) to mathematics
outside its own code: a dense inverse, particle-hole symmetry at half filling,
and the statistics of the estimate."""
import numpy as np

import oracle
from oracle import estimate as oest
from oracle import philox
from paper_2508_16298_gb300 import inputs


def dense_M(lat, th):
    n = lat.n_sites
    shape = (lat.Ntau, lat.L, lat.L)
    return np.array([oracle.apply_M(lat, th, np.eye(n)[:, j].reshape(shape).astype(complex)).reshape(-1)
                     for j in range(n)]).T


def test_diagonal_of_M_inverse_is_one_half():
    """Half filling on the bipartite lattice: c_i -> (-1)^i c_i^dagger maps the
    problem to its complex conjugate, so Re (M^{-1})_ii = 1/2 for every site and
    every gauge field (dense LU inverse, three fields)."""
    for L, N, th in [(4, 6, inputs.theta_hot(4, 6, 1)), (6, 4, inputs.theta_hot(6, 4, 3)),
                     (4, 8, inputs.theta_ordered(4, 8, 5, tau_walk=1.0))]:
        G = np.linalg.inv(dense_M(oracle.Lattice(L, N), th))
        assert np.max(np.abs(np.diag(G).real - 0.5)) < 1e-12


def test_solutions_are_M_inverse_times_the_draws():
    lat = oracle.Lattice(4, 6)
    th = inputs.theta_hot(4, 6, 7)
    g, X, xi = oest.estimate(lat, th, seed=11, counter=5, nrv=3, tol=1e-13)
    G = np.linalg.inv(dense_M(lat, th))
    for k in range(3):
        assert np.allclose(xi[k], philox.draw_random_vector(11, 5, k, 4, 6))
        want = (G @ xi[k].reshape(-1)).reshape(xi[k].shape)
        assert np.max(np.abs(X[k] - want)) < 1e-10 * np.max(np.abs(want))
    # g is the mean of conj(xi_k,i) (M^{-1} xi_k)_i over k and i
    want_g = sum(np.vdot(xi[k].reshape(-1), G @ xi[k].reshape(-1)) for k in range(3)) / (3 * lat.n_sites)
    assert abs(g - want_g) < 1e-10


def test_estimate_is_unbiased_around_one_half():
    """E[g] = Tr(M^{-1}) / N, whose real part is 1/2; the per-vector estimates
    scatter with their own sample standard deviation."""
    lat = oracle.Lattice(4, 8)
    th = inputs.theta_hot(4, 8, 13)
    nrv = 200
    per = []
    for k in range(nrv):
        g_k, _, _ = oest.estimate(lat, th, seed=17, counter=1000 * k, nrv=1, tol=1e-12)
        per.append(g_k)
    per = np.array(per)
    mean, sem = per.real.mean(), per.real.std(ddof=1) / np.sqrt(nrv)
    assert abs(mean - 0.5) < 5 * sem
    assert 0 < sem < 0.05
