"""Dense brute-force constructions used to pin the oracle on tiny lattices.

Written independently of ``oracle/``: the hopping matrices are assembled entry
by entry from the bond list and exponentiated with ``scipy.linalg.expm``
(not with the closed cosh/sinh form the oracle uses), and M is assembled block by
block from the printed matrix of the Methods (Eq. (M_alpha)).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def site(L: int, x: int, y: int) -> int:
    return (x % L) + L * (y % L)


def family_of(c: int, x: int, y: int) -> int:
    """Checkerboard family of the bond leaving (x, y) in direction c (0 = x, 1 = y)."""
    if c == 0:
        return 1 if x % 2 == 0 else 2
    return 3 if y % 2 == 0 else 4


def hopping(L: int, theta_slice: np.ndarray, families=(1, 2, 3, 4)) -> np.ndarray:
    """H_ij = e^{i theta_ij}, H_ji = e^{-i theta_ij} on the bonds of the given families."""
    V = L * L
    H = np.zeros((V, V), dtype=complex)
    for y in range(L):
        for x in range(L):
            for c in range(2):
                if family_of(c, x, y) not in families:
                    continue
                i = site(L, x, y)
                j = site(L, x + 1, y) if c == 0 else site(L, x, y + 1)
                ph = np.exp(1j * theta_slice[y, x, c])
                H[i, j] += ph
                H[j, i] += np.conj(ph)
    return H


def dense_B(L: int, theta_slice: np.ndarray, a: float) -> np.ndarray:
    """e^{V4/2} e^{V3/2} e^{V2/2} e^{V1/2} e^{V1/2} e^{V2/2} e^{V3/2} e^{V4/2}, V_f = a H_f."""
    E = {f: sla.expm(0.5 * a * hopping(L, theta_slice, (f,))) for f in (1, 2, 3, 4)}
    out = np.eye(L * L, dtype=complex)
    for f in (4, 3, 2, 1, 1, 2, 3, 4):
        out = out @ E[f]
    return out


def dense_M(L: int, Ntau: int, theta: np.ndarray, a: float) -> np.ndarray:
    """Eq. (M_alpha) in 0-based slices: block (tau, tau) = 1, block (tau, tau-1) = -B_{tau-1},
    block (0, Ntau-1) = +B_{Ntau-1}."""
    V = L * L
    M = np.eye(V * Ntau, dtype=complex)
    for tau in range(Ntau):
        B = dense_B(L, theta[tau], a)
        if tau < Ntau - 1:
            M[(tau + 1) * V:(tau + 2) * V, tau * V:(tau + 1) * V] = -B
        else:
            M[0:V, tau * V:(tau + 1) * V] = B
    return M


def fermion_action_dense(L: int, Ntau: int, theta: np.ndarray, a: float, eta: np.ndarray) -> float:
    M = dense_M(L, Ntau, theta, a)
    e = eta.reshape(-1)
    return float(np.real(np.vdot(e, np.linalg.solve(M.conj().T @ M, e))))


def bosonic_action_direct(L, Ntau, theta, dtau, J, K, noncompact):
    """Straight transcription of S_B = dtau * sum_tau L_B (compact or non-compact)."""
    S = 0.0
    for tau in range(Ntau):
        tn = (tau + 1) % Ntau
        for y in range(L):
            for x in range(L):
                for c in range(2):
                    d = theta[tn, y, x, c] - theta[tau, y, x, c]
                    S += (d * d if noncompact else 1.0 - np.cos(d)) / (J * dtau * dtau) * dtau
                # plaquette with lower-left corner (x, y), counter-clockwise edges
                cu = (theta[tau, y, x, 0] + theta[tau, y, (x + 1) % L, 1]
                      - theta[tau, (y + 1) % L, x, 0] - theta[tau, y, x, 1])
                S += dtau * K * np.cos(cu)
    return S
