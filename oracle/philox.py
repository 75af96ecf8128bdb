"""Philox4x32-10 counter-based generator and the HQMC Gaussian draws.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Written from the published
definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC 2011): a 4x32-bit counter and a 2x32-bit key; each of the 10 rounds
multiplies counter words 0 and 2 by the constants 0xD2511F53 and 0xCD9E8D57,
mixes the high halves with the other words and the key, and the key is advanced
by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.

The draw layout (which counter produces which variable) is the library's
documented convention, restated here independently so that GPU draws can be
reproduced on the host:

  key     = (seed & 0xffffffff, seed >> 32)
  counter = (element, stream, traj_counter & 0xffffffff, traj_counter >> 32)
  stream 0: momenta, element = site i   -> p[2i], p[2i+1]  (N(0, 1/2) each)
  stream 1: pseudofermion, element = i  -> R[i] = (g0 + i g1)/sqrt(2)  (CN(0, 1))
  stream 2: Metropolis, element 0       -> u (uniform in [0, 1))
  stream 3: stochastic-estimation vectors, element = i, traj_counter = counter + k
            -> xi_k[i] = (g0 + i g1)/sqrt(2)  (CN(0, 1))

Two uniforms per call: u_a from words (0, 1) and u_b from words (2, 3), each
((w_hi >> 5) * 2^26 + (w_lo >> 6)) * 2^-53.  Gaussians by Box-Muller:
r = sqrt(-2 log(1 - u_a)), g0 = r cos(2 pi u_b), g1 = r sin(2 pi u_b).
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """ctr: uint32 array of shape (4, n); key: two uint32 words.  Returns (4, n) uint32."""
    c = [np.asarray(ctr[k], dtype=np.uint64) for k in range(4)]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack(c).astype(np.uint32)


def _words(seed: int, stream: int, traj_counter: int, n: int) -> np.ndarray:
    ctr = np.zeros((4, n), dtype=np.uint64)
    ctr[0] = np.arange(n, dtype=np.uint64)
    ctr[1] = stream
    ctr[2] = traj_counter & 0xFFFFFFFF
    ctr[3] = (traj_counter >> 32) & 0xFFFFFFFF
    return philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))


def _u53(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    a = (hi.astype(np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (lo.astype(np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0)


def _gauss_pairs(seed: int, stream: int, traj_counter: int, n: int):
    w = _words(seed, stream, traj_counter, n)
    ua = _u53(w[0], w[1])
    ub = _u53(w[2], w[3])
    r = np.sqrt(-2.0 * np.log(1.0 - ua))
    return r * np.cos(2.0 * np.pi * ub), r * np.sin(2.0 * np.pi * ub)


def draw_momenta(seed: int, traj_counter: int, L: int, Ntau: int) -> np.ndarray:
    """p ~ N(0, 1/2) on every bond, shape (Ntau, L, L, 2)."""
    n = L * L * Ntau
    g0, g1 = _gauss_pairs(seed, 0, traj_counter, n)
    p = np.empty((n, 2))
    p[:, 0] = g0 * np.sqrt(0.5)
    p[:, 1] = g1 * np.sqrt(0.5)
    return p.reshape(Ntau, L, L, 2)


def draw_pseudofermion(seed: int, traj_counter: int, L: int, Ntau: int) -> np.ndarray:
    """R ~ CN(0, 1) on every site, shape (Ntau, L, L)."""
    n = L * L * Ntau
    g0, g1 = _gauss_pairs(seed, 1, traj_counter, n)
    return ((g0 + 1j * g1) * np.sqrt(0.5)).reshape(Ntau, L, L)


def draw_metropolis(seed: int, traj_counter: int) -> float:
    w = _words(seed, 2, traj_counter, 1)
    return float(_u53(w[0], w[1])[0])


def draw_random_vector(seed: int, counter: int, k: int, L: int, Ntau: int) -> np.ndarray:
    """xi_k ~ CN(0, 1) on every site for stochastic estimation, shape (Ntau, L, L)."""
    n = L * L * Ntau
    g0, g1 = _gauss_pairs(seed, 3, counter + k, n)
    return ((g0 + 1j * g1) * np.sqrt(0.5)).reshape(Ntau, L, L)
