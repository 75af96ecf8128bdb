"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws numbers (numpy
PCG64 streams keyed by an integer seed) in the shapes of the paper's runs.

* theta: float64 (Ntau, L, L, 2), indexed [tau, y, x, c]; c = 0 the bond
  (x,y)->(x+1,y), c = 1 the bond (x,y)->(x,y+1).  "Hot start": i.i.d. uniform
  in [-pi, pi) on every spatial bond (temporal links are fixed to zero and not
  stored).
* vectors: complex128 (Ntau, L, L), indexed [tau, y, x].
* R ~ CN(0, 1): real and imaginary parts i.i.d. N(0, 1/2) (density e^{-|R|^2}).
* p ~ N(0, 1/2) per bond (density e^{-p^2}, the kinetic term sum p^2 of H).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def theta_hot(L: int, Ntau: int, seed: int) -> np.ndarray:
    return rng(seed).uniform(-np.pi, np.pi, size=(Ntau, L, L, 2))


def theta_zero(L: int, Ntau: int) -> np.ndarray:
    return np.zeros((Ntau, L, L, 2))


def theta_pi_flux(L: int, Ntau: int) -> np.ndarray:
    """theta_y(x, y) = pi * (x mod 2), theta_x = 0: flux pi through every plaquette."""
    th = np.zeros((Ntau, L, L, 2))
    th[:, :, 1::2, 1] = np.pi
    return th


def complex_gaussian(L: int, Ntau: int, seed: int) -> np.ndarray:
    g = rng(seed).standard_normal(size=(2, Ntau, L, L))
    return (g[0] + 1j * g[1]) * np.sqrt(0.5)


def momenta(L: int, Ntau: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(size=(Ntau, L, L, 2)) * np.sqrt(0.5)


def uniform01(seed: int) -> float:
    return float(rng(seed).uniform(0.0, 1.0))


def theta_warm(L: int, Ntau: int, seed: int, J: float = 1.0, dtau: float = 0.1) -> np.ndarray:
    """Gauge field smooth in imaginary time, shaped like an equilibrated configuration.

    Every bond gets a uniform angle u ~ U[-pi, pi) plus a periodic Gaussian walk
    in tau: increments d_tau ~ N(0, J*dtau/2) with their mean removed (so the
    walk closes on itself), which is the distribution of the temporal term
    (1/(J dtau)) (theta_{tau+1} - theta_tau)^2 of the bosonic action on its own.
    """
    g = rng(seed)
    u = g.uniform(-np.pi, np.pi, size=(1, L, L, 2))
    d = g.standard_normal(size=(Ntau, L, L, 2)) * np.sqrt(0.5 * J * dtau)
    d -= d.mean(axis=0, keepdims=True)
    w = np.cumsum(d, axis=0) - d[0]
    return u + w


def theta_ordered(L: int, Ntau: int, seed: int, J: float = 1.0, dtau: float = 0.1,
                  sigma_space: float = 0.3, tau_walk: float = 1.0) -> np.ndarray:
    """Gauge field near the pi-flux background that half-filled fermions favour.

    theta = pi-flux + fluctuation + random gauge transformation:
      * fluctuation: every bond gets N(0, sigma_space^2) plus a periodic Gaussian
        walk in tau with step variance tau_walk * J*dtau/2 (tau_walk = 0: the
        field does not depend on tau, a "cold" start);
      * gauge transformation: theta_ij += l_i - l_j with l ~ U[-pi, pi) per
        spatial site (the same at every tau), which changes no gauge-invariant
        quantity, so the field looks random bond by bond.
    """
    g = rng(seed)
    th = theta_pi_flux(L, Ntau)
    th += g.standard_normal(size=(1, L, L, 2)) * sigma_space
    d = g.standard_normal(size=(Ntau, L, L, 2)) * np.sqrt(0.5 * J * dtau * tau_walk)
    d -= d.mean(axis=0, keepdims=True)
    th += np.cumsum(d, axis=0) - d[0]
    lam = g.uniform(-np.pi, np.pi, size=(L, L))  # [y, x]
    th[..., 0] += lam[None, :, :] - np.roll(lam, -1, axis=1)[None, :, :]
    th[..., 1] += lam[None, :, :] - np.roll(lam, -1, axis=0)[None, :, :]
    return th
