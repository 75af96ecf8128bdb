"""FP64 reference of the tau-line preconditioner (test infrastructure only).

Methods, "CG method and preconditioner": the preconditioner is built once
from O = M^dagger M at the pi-flux gauge field.  The steps are an incomplete
Cholesky factor L, the Neumann series of L^{-1} cut after 20 terms, the
entries of L^{-1} below 1e-3 dropped, and Otilde^{-1} = L^{-1} L^{-dagger}.
The paper reports that the result is banded along tau, with its diagonals a
whole slice (V_s sites) apart, i.e. it couples each site only to itself on
other slices, and that its bulk entries do not depend on the lattice size.
This module takes that structure as the definition.

 1. At the pi-flux field every site is equivalent.  The same-site part of O
    couples (tau, s) to (tau +- 1, s).  It is the tau-line matrix
        T = a - b (S + S^dagger),
    with a = O_{(tau,s),(tau,s)} = 1 + sum_j |B_js|^2 and
    b = -O_{(tau,s),(tau+1,s)} = B_ss.  S is the antiperiodic shift
    (S u)_tau = u_{tau-1}, (S u)_0 = -u_{Ntau-1}.
 2. Bulk Cholesky factor of T: T = L L^dagger with L = sqrt(b/rho) (1 - rho S)
    and rho + 1/rho = a/b, 0 < rho < 1.  This is the limit that the Cholesky
    recursion of the tridiagonal T reaches away from its first row.
 3. Neumann series: L^{-1} = sqrt(rho/b) sum_{m>=0} rho^m S^m.  Its entries
    are sqrt(rho/b) rho^m, so dropping those below 1e-3 keeps m <= W.  The
    20-term cut of the paper keeps more than W terms here, so the truncation
    decides the width.
 4. Otilde^{-1} = (rho/b) F_W^dagger F_W on every site's tau line, with
    F_W = sum_{m=0}^{W} rho^m S^m (S is unitary, so the order of the two
    factors is immaterial).  It is Hermitian positive definite.

The readings (which same-site quantities enter, the bulk factor and the
unit-diagonal Neumann series) are stated here because the paper gives the
recipe but not these details.

The pCG recurrence is Eq. (pCG).  Arrays follow oracle/__init__.py.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Lattice, apply_B, apply_MdagM, dot

TRUNCATION = 1e-3  # entries of L^{-1} below this are dropped (Methods)


def pi_flux(L: int, Ntau: int) -> np.ndarray:
    """theta_y(x, y) = pi (x mod 2), theta_x = 0: flux pi through every plaquette."""
    th = np.zeros((Ntau, L, L, 2))
    th[:, :, 1::2, 1] = np.pi
    return th


@dataclass(frozen=True)
class LineCoefficients:
    a: float    # same-site diagonal of O at pi flux
    b: float    # same-site tau coupling of O at pi flux (B_ss)
    rho: float  # bulk Cholesky ratio, rho + 1/rho = a/b
    W: int      # highest power of rho S kept in L^{-1}

    @property
    def scale(self) -> float:
        """rho / b, the prefactor of F_W^dagger F_W."""
        return self.rho / self.b


def coefficients(lat: Lattice) -> LineCoefficients:
    """Steps 1-3: a and b from one column of B at pi flux, then rho and W."""
    L = lat.L
    th = pi_flux(L, 2)[0]
    e = np.zeros((L, L), dtype=np.complex128)
    e[0, 0] = 1.0
    col = apply_B(lat, th, e)  # B e_s: column s of B
    b = float(col[0, 0].real)
    a = 1.0 + float(np.sum(np.abs(col) ** 2))
    q = a / b
    rho = (q - np.sqrt(q * q - 4.0)) / 2.0
    pref = np.sqrt(rho / b)
    W = 0
    while pref * rho ** (W + 1) >= TRUNCATION:
        W += 1
    return LineCoefficients(a, b, float(rho), W)


def shift(u: np.ndarray, m: int) -> np.ndarray:
    """(S^m u)_tau = u_{tau-m} with a sign flip for every wrap through tau = 0 (m >= 0)."""
    N = u.shape[0]
    out = np.empty_like(u)
    for tau in range(N):
        src = tau - m
        sign = 1.0
        while src < 0:
            src += N
            sign = -sign
        out[tau] = sign * u[src]
    return out


def shift_adj(u: np.ndarray, m: int) -> np.ndarray:
    """(S^{dagger m} u)_tau = u_{tau+m} with a sign flip for every wrap through tau = Ntau."""
    N = u.shape[0]
    out = np.empty_like(u)
    for tau in range(N):
        src = tau + m
        sign = 1.0
        while src >= N:
            src -= N
            sign = -sign
        out[tau] = sign * u[src]
    return out


def apply_F(c: LineCoefficients, u: np.ndarray) -> np.ndarray:
    """F_W u = sum_{m=0}^{W} rho^m S^m u."""
    return sum(c.rho ** m * shift(u, m) for m in range(c.W + 1))


def apply_F_adj(c: LineCoefficients, u: np.ndarray) -> np.ndarray:
    """F_W^dagger u = sum_{m=0}^{W} rho^m S^{dagger m} u."""
    return sum(c.rho ** m * shift_adj(u, m) for m in range(c.W + 1))


def apply(c: LineCoefficients, r) -> np.ndarray:
    """Otilde^{-1} r = (rho/b) F_W^dagger F_W r, on every site's tau line."""
    r = np.asarray(r, dtype=np.complex128)
    return c.scale * apply_F_adj(c, apply_F(c, r))


def pcg(lat: Lattice, theta, phi, c: LineCoefficients, x0=None, tol: float = 1e-10, maxit: int = 100000):
    """Preconditioned CG of Eq. (pCG) on (M^dagger M) X = phi.  Stops when the
    recursive residual meets tol, then checks the true residual and restarts
    from it if the two drifted apart.  Returns (X, iterations, true relative residual)."""
    phi = np.asarray(phi, dtype=np.complex128)
    x = np.zeros_like(phi) if x0 is None else np.array(x0, dtype=np.complex128)
    bb = dot(phi, phi).real
    if bb == 0.0:
        return np.zeros_like(phi), 0, 0.0
    k = 0
    while True:
        r = phi - apply_MdagM(lat, theta, x)
        if dot(r, r).real <= tol * tol * bb or k >= maxit:
            return x, k, float(np.sqrt(dot(r, r).real / bb))
        z = apply(c, r)
        d = z.copy()
        rz = dot(r, z).real
        while k < maxit:
            q = apply_MdagM(lat, theta, d)
            zeta = rz / dot(d, q).real
            x = x + zeta * d
            r = r - zeta * q
            k += 1
            if dot(r, r).real <= tol * tol * bb:
                break
            z = apply(c, r)
            rz_new = dot(r, z).real
            d = z + (rz_new / rz) * d
            rz = rz_new
