"""Pins of the oracle's flexible CG (oracle/fcg.py) to facts that do not go through
its own code: with one fixed Hermitian positive definite preconditioner it is
the pCG of Eq. (pCG) (same iterates, to rounding), with the identity it solves
the dense system, and with a preconditioner that changes every iteration it still
converges to the dense solution and keeps consecutive directions O-orthogonal."""
import numpy as np

import oracle
from oracle import fcg as ofcg
from oracle import precond as opc
from paper_2508_16298_gb300 import inputs
from tests.dense import dense_M


def dense_MdagM(lat, th):
    M = dense_M(lat.L, lat.Ntau, th, lat.dtau * lat.t)
    return M.conj().T @ M


def small():
    L, N = 4, 8
    lat = oracle.Lattice(L, N)
    th = inputs.theta_hot(L, N, 11)
    phi = inputs.complex_gaussian(L, N, 12)
    return lat, th, phi


def test_identity_preconditioner_solves_the_dense_system():
    lat, th, phi = small()
    O = dense_MdagM(lat, th)
    want = np.linalg.solve(O, phi.ravel()).reshape(phi.shape)
    x, n, res, status = ofcg.fcg(lat, th, phi, lambda k, r: r, tol=1e-12)
    assert status == "converged" and res <= 1e-12
    assert np.max(np.abs(x - want)) / np.max(np.abs(want)) < 1e-9


def test_fixed_hpd_preconditioner_gives_the_pcg_iterates():
    """With z = Otilde^{-1} r every iteration, Re<z_{n+1}, r_n> = 0 in exact
    arithmetic, so FCG's Polak-Ribiere coefficient is pCG's: the iterates after a
    fixed number of steps agree with oracle.precond.pcg to rounding."""
    lat, th, phi = small()
    c = opc.coefficients(lat)
    for m in (3, 10):
        xf, nf, _, _ = ofcg.fcg(lat, th, phi, lambda k, r: opc.apply(c, r), tol=1e-30, maxit=m)
        xp, npc, _ = opc.pcg(lat, th, phi, c, tol=1e-30, maxit=m)
        assert nf == npc == m
        assert np.max(np.abs(xf - xp)) / np.max(np.abs(xp)) < 1e-10


def test_variable_preconditioner_converges_and_keeps_directions_conjugate():
    """Alternating the tau-line preconditioner with a random Hermitian positive
    definite diagonal scaling: the solve reaches the dense solution, and each new
    direction is O-orthogonal to the previous one (|<d_n, O d_{n-1}>| tiny)."""
    lat, th, phi = small()
    O = dense_MdagM(lat, th)
    want = np.linalg.solve(O, phi.ravel()).reshape(phi.shape)
    c = opc.coefficients(lat)
    D = inputs.rng(13).uniform(0.5, 2.0, size=phi.shape)

    def prec(k, r):
        return opc.apply(c, r) if k % 2 else D * r

    x, n, res, status = ofcg.fcg(lat, th, phi, prec, tol=1e-12)
    assert status == "converged" and res <= 1e-12
    assert np.max(np.abs(x - want)) / np.max(np.abs(want)) < 1e-8
    # replay the first iterations to read the directions
    r = phi.copy()
    z = prec(0, r)
    d = z.copy()
    rz = ofcg.rdot(r, z)
    prev = None
    for k in range(6):
        q = oracle.apply_MdagM(lat, th, d)
        if prev is not None:
            pq = prev[1]
            assert abs(ofcg.rdot(d, pq)) < 1e-10 * np.sqrt(ofcg.rdot(d, q) * ofcg.rdot(prev[0], pq))
        a = rz / ofcg.rdot(d, q)
        r_old, r = r, r - a * q
        z = prec(k + 1, r)
        rz_new = ofcg.rdot(r, z)
        prev = (d, q)
        d = z + (rz_new - ofcg.rdot(r_old, z)) / rz * d
        rz = rz_new


def test_learned_guess_is_kept_only_if_it_helps():
    lat, th, phi = small()
    O = dense_MdagM(lat, th)
    exact = np.linalg.solve(O, phi.ravel()).reshape(phi.shape)
    x0 = np.zeros_like(phi)
    # a net that returns the exact correction is kept; one that returns -r0 * 10 is not
    x1, used = ofcg.learned_guess(lat, th, phi, x0, lambda r: exact)
    assert used and np.max(np.abs(x1 - exact)) < 1e-12
    x2, used2 = ofcg.learned_guess(lat, th, phi, x0, lambda r: -10.0 * r)
    assert not used2 and np.all(x2 == x0)
