"""The preconditioner recipe of the Methods taken literally, on small lattices
(test infrastructure only).

Methods, "CG method and preconditioner", gives the construction step by step:

 1. O = M^dagger M at a fixed field (in practice the pi-flux field);
 2. an incomplete Cholesky factor L of O (lower triangular);
 3. L^{-1} from its Neumann series 1 + (1 - L) + (1 - L)^2 + ..., 20 terms;
 4. entries below 1e-3 dropped;
 5. Otilde^{-1} = L^{-1} L^{-dagger}.

Fig. 3(a) reports the result for Ntau x L x L = 60 x 6 x 6 as banded along tau
("bandwidth 6", diagonals V_s apart).  The library uses a tau-line reading of
the same recipe (oracle/precond.py).  This module builds the recipe densely, so
that the two can be compared on the paper's own lattice: which tau offsets
survive the truncation, how far the operators are apart, and how many pCG
iterations each needs.

Readings made here (the recipe leaves them open):
  * incomplete Cholesky is IC(0): L has the sparsity of the lower triangle of
    O (its structural non-zeros, |O_ij| > 1e-14) and (L L^dagger)_ij = O_ij on
    that pattern;
  * the printed "O ~ L^dagger L" and "Otilde^{-1} = L^{-1} L^{-dagger}" are not
    consistent with each other for a lower-triangular L; the consistent pair
    O ~ L L^dagger, Otilde^{-1} = L^{-dagger} L^{-1} is used (both orders are
    available through `order`);
  * the Neumann series is evaluated as printed (`series="literal"`), in the
    unit-diagonal form L^{-1} = D^{-1} sum_k N^k with L = (1 - N) D
    (`series="unit"`), or replaced by the exact triangular inverse
    (`series="exact"`, what the series converges to when it converges);
  * the truncation acts on the approximate L^{-1} (`truncate_factor`) or on
    the assembled Otilde^{-1}.

Everything is dense numpy in FP64: 60 x 6 x 6 = 2160 unknowns.
"""
from __future__ import annotations

import numpy as np

from . import Lattice, apply_MdagM

TRUNCATION = 1e-3
NEUMANN_TERMS = 20
PATTERN_EPS = 1e-14


def dense_MdagM(lat: Lattice, theta) -> np.ndarray:
    """O = M^dagger M as a dense matrix, column by column from the matrix-free oracle."""
    n = lat.n_sites
    O = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        O[:, j] = apply_MdagM(lat, theta, e.reshape(lat.Ntau, lat.L, lat.L)).ravel()
    return O


def incomplete_cholesky(A: np.ndarray, pattern: np.ndarray | None = None) -> np.ndarray:
    """IC(0): lower-triangular L with L_ij = 0 off `pattern` (default: the
    structural non-zeros of A) and the Cholesky formula on it, column by column:
        L_jj = sqrt(A_jj - sum_{k<j} |L_jk|^2),
        L_ij = (A_ij - sum_{k<j} L_ik conj(L_jk)) / L_jj   (i > j, (i, j) in the pattern).
    Raises ValueError on a non-positive pivot."""
    n = A.shape[0]
    if pattern is None:
        pattern = np.abs(A) > PATTERN_EPS
    Lf = np.zeros_like(A, dtype=np.complex128)
    for j in range(n):
        piv = (A[j, j] - np.vdot(Lf[j, :j], Lf[j, :j])).real
        if not piv > 0.0:
            raise ValueError(f"non-positive pivot {piv} at column {j}")
        Lf[j, j] = np.sqrt(piv)
        col = (A[j + 1:, j] - Lf[j + 1:, :j] @ np.conj(Lf[j, :j])) / Lf[j, j]
        col[~pattern[j + 1:, j]] = 0.0
        Lf[j + 1:, j] = col
    return Lf


def neumann_inverse(Lf: np.ndarray, terms: int = NEUMANN_TERMS, series: str = "literal") -> np.ndarray:
    """Approximate L^{-1}.
    literal: sum_{k<terms} (1 - L)^k, as printed;
    unit:    D^{-1} sum_{k<terms} N^k with D = diag(L), N = 1 - L D^{-1} (L = (1 - N) D);
    exact:   the triangular inverse itself."""
    n = Lf.shape[0]
    eye = np.eye(n)
    if series == "exact":
        return np.linalg.inv(Lf)
    if series == "literal":
        A, post = eye - Lf, None
    elif series == "unit":
        d = Lf.diagonal()
        A, post = eye - Lf / d[None, :], 1.0 / d
    else:
        raise ValueError(series)
    S = eye.astype(np.complex128)
    P = eye.astype(np.complex128)
    for _ in range(1, terms):
        P = P @ A
        S = S + P
    return S if post is None else post[:, None] * S


def truncate(A: np.ndarray, eps: float = TRUNCATION) -> np.ndarray:
    """Entries with |A_ij| < eps set to zero."""
    return np.where(np.abs(A) >= eps, A, 0.0)


def preconditioner(Lf: np.ndarray, series: str = "exact", truncate_factor: bool = True,
                   order: str = "consistent") -> np.ndarray:
    """Otilde^{-1} from the factor: consistent = L^{-dagger} L^{-1} (O ~ L L^dagger),
    printed = L^{-1} L^{-dagger}.  The 1e-3 truncation acts on the approximate L^{-1}
    (truncate_factor) or on the product."""
    Li = neumann_inverse(Lf, series=series)
    if truncate_factor:
        Li = truncate(Li)
    P = Li.conj().T @ Li if order == "consistent" else Li @ Li.conj().T
    return P if truncate_factor else truncate(P)


def tau_profile(P: np.ndarray, lat: Lattice) -> np.ndarray:
    """max |P_ij| over pairs of sites whose slices are m apart (m = 0..Ntau/2, tau periodic)."""
    V, N = lat.V, lat.Ntau
    B = np.abs(P).reshape(N, V, N, V).max(axis=(1, 3))  # [tau_i, tau_j]
    out = np.zeros(N // 2 + 1)
    for ti in range(N):
        for tj in range(N):
            m = min((ti - tj) % N, (tj - ti) % N)
            out[m] = max(out[m], B[ti, tj])
    return out


def same_site_fraction(P: np.ndarray, lat: Lattice) -> float:
    """Fraction of the non-zero entries of P that couple a site to itself (on any slice)."""
    idx = np.argwhere(P != 0)
    return float(np.mean(idx[:, 0] % lat.V == idx[:, 1] % lat.V))


def pcg_iterations(lat: Lattice, theta, phi, apply_prec, tol: float = 1e-8, maxit: int = 5000) -> int:
    """Iterations of the pCG of Eq. (pCG) from X_0 = 0 until ||r|| <= tol ||phi||
    (recursive residual), with z = apply_prec(r) on flat vectors (None: identity).
    Returns -1 if maxit is reached or the recurrence breaks down."""
    shape = (lat.Ntau, lat.L, lat.L)
    phi = np.asarray(phi, dtype=np.complex128).ravel()
    prec = (lambda v: v) if apply_prec is None else apply_prec
    bb = np.vdot(phi, phi).real
    x = np.zeros_like(phi)
    r = phi.copy()
    z = prec(r)
    d = z.copy()
    rz = np.vdot(r, z).real
    for k in range(maxit):
        q = apply_MdagM(lat, theta, d.reshape(shape)).ravel()
        dq = np.vdot(d, q).real
        if not (dq > 0.0 and rz > 0.0):
            return -1
        zeta = rz / dq
        x = x + zeta * d
        r = r - zeta * q
        if np.vdot(r, r).real <= tol * tol * bb:
            return k + 1
        z = prec(r)
        rz_new = np.vdot(r, z).real
        d = z + (rz_new / rz) * d
        rz = rz_new
    return -1
