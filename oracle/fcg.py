"""FP64 reference of flexible CG with a learned preconditioner (test infrastructure only).

Not a method of the paper: it is the solver the learned preconditioner of this
project plugs into.  The recurrence is the pCG of Eq. (pCG) with two changes
that let the preconditioner change from one iteration to the next (Notay,
"Flexible conjugate gradients", SIAM J. Sci. Comput. 22 (2000), with one kept
direction):

  * z_n = P_n(r_n) may differ for every n (here: the net on some iterations,
    the tau-line preconditioner on the others);
  * the direction update uses the Polak-Ribiere coefficient
        rho_n = Re<z_{n+1}, r_{n+1} - r_n> / Re<z_n, r_n>,
    which equals the pCG coefficient Re<r_{n+1}, z_{n+1}> / Re<r_n, z_n> when
    P_n is one fixed Hermitian positive definite operator (then
    <z_{n+1}, r_n> = 0), and keeps the new direction O-orthogonal to the
    previous one when it is not.

Inner products are real parts (complex vectors as real vectors of twice the
length; O = M^dagger M is Hermitian positive definite, so it is symmetric
positive definite on those).

The learned initial guess is the north-star's x0 = x + K(theta)(phi - O x),
kept only if its residual is smaller than that of x.

Arrays follow oracle/__init__.py; vectors are complex128 (Ntau, L, L).
"""
from __future__ import annotations

import numpy as np

from . import Lattice, apply_MdagM


def rdot(a, b) -> float:
    """Re<a, b> = Re sum conj(a) b."""
    return float(np.vdot(a, b).real)


def learned_guess(lat: Lattice, theta, phi, x, net):
    """x + K (phi - O x) if that lowers the residual, else x.  Returns (x, used)."""
    r0 = phi - apply_MdagM(lat, theta, x)
    x1 = x + net(r0)
    r1 = phi - apply_MdagM(lat, theta, x1)
    if rdot(r1, r1) < rdot(r0, r0):
        return x1, True
    return x, False


def fcg(lat: Lattice, theta, phi, precond, x0=None, tol: float = 1e-8, maxit: int = 10000):
    """Flexible CG on (M^dagger M) X = phi from X_0 = x0 (zeros if None).

    precond(n, r) returns z_n = P_n(r) for iteration n (n = 0 for the first
    direction).  Stops when ||r_n|| <= tol ||phi|| or after maxit iterations.
    Returns (X, iterations, ||phi - O X|| / ||phi||, status) with status
    "converged", "maxit" or "breakdown" (Re<r, z> <= 0 or <d, O d> <= 0)."""
    phi = np.asarray(phi, dtype=np.complex128)
    x = np.zeros_like(phi) if x0 is None else np.array(x0, dtype=np.complex128)
    bb = rdot(phi, phi)
    r = phi - apply_MdagM(lat, theta, x)
    status = "maxit"
    n = 0
    if rdot(r, r) <= tol * tol * bb:
        status = "converged"
    else:
        z = precond(0, r)
        d = z.copy()
        rz = rdot(r, z)
        while n < maxit:
            q = apply_MdagM(lat, theta, d)
            dq = rdot(d, q)
            if not (rz > 0.0 and dq > 0.0):
                status = "breakdown"
                break
            zeta = rz / dq
            x = x + zeta * d
            r_old = r
            r = r - zeta * q
            n += 1
            if rdot(r, r) <= tol * tol * bb:
                status = "converged"
                break
            z = precond(n, r)
            rz_new = rdot(r, z)
            beta = (rz_new - rdot(r_old, z)) / rz
            d = z + beta * d
            rz = rz_new
    res = phi - apply_MdagM(lat, theta, x)
    return x, n, float(np.sqrt(rdot(res, res) / bb)) if bb > 0 else 0.0, status
