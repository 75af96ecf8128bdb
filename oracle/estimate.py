"""FP64 reference of the stochastic estimation of fermionic observables
(test infrastructure only).

Methods, "Stochastic estimation of fermionic observables": with random vectors
xi whose entries satisfy E[xi_i^* xi_j] = delta_ij, (M^{-1} xi)_i xi_j^* is an
unbiased estimate of (M^{-1})_ij.  M^{-1} xi is obtained as (M^dagger M)^{-1} R
with R = M^dagger xi, by CG.  The estimate kept here is the mean diagonal

    g = (1 / (n_rv N)) sum_k sum_i conj(xi_k,i) (M^{-1} xi_k)_i,

whose expectation is Tr(M^{-1}) / N.  At half filling on the bipartite
lattice the real part of every (M^{-1})_ii is exactly 1/2 (particle-hole
symmetry), whatever the gauge field, which gives the estimate a closed form to
be tested against.

The vectors are CN(0, 1) Philox draws on stream 3 (oracle/philox.py).
"""
from __future__ import annotations

import numpy as np

from . import Lattice, apply_M, cg, dot
from .philox import draw_random_vector


def estimate(lat: Lattice, theta, seed: int, counter: int, nrv: int, tol: float = 1e-10):
    """Returns (g, X, xi): the complex estimate, and the solutions M^{-1} xi_k and
    draws as arrays of shape (nrv, Ntau, L, L).  Each solve starts from the previous X."""
    xs, xis = [], []
    total = 0.0 + 0.0j
    X = None
    for k in range(nrv):
        xi = draw_random_vector(seed, counter, k, lat.L, lat.Ntau)
        R = apply_M(lat, theta, xi, dagger=True)
        X, _, _, _ = cg(lat, theta, R, x0=X, tol=tol)
        total += dot(xi, X)
        xs.append(X.copy())
        xis.append(xi)
    return total / (nrv * lat.n_sites), np.array(xs), np.array(xis)
