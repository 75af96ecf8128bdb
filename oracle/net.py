"""FP64 reference of the learned preconditioner's network (test infrastructure only).

The network is this project's design (the paper's preconditioner is a different,
fixed operator): L layers, layer l mapping C_in to C_out complex channels by

    h'(x, c) = sum_{mu=0..6} sum_{c'} W_l[mu, c, c'] (T_mu h)(x, c'),

mu = 0 centre, 1/2 = +x/-x, 3/4 = +y/-y, 5/6 = +tau/-tau, with the parallel
transporters (T_{+x} h)(x) = e^{i theta_x(x)} h(x + x^) and
(T_{-x} h)(x) = e^{-i theta_x(x - x^)} h(x - x^) (y alike), and
(T_{+-tau} h)(x) = s h(x +- tau^) with s = -1 across the antiperiodic boundary.
Arrays: theta (Ntau, L, L, 2) [tau, y, x, c]; fields (Ntau, L, L, C) complex.
Weights are given per layer as arrays of shape (7, C_out, C_in).
"""
from __future__ import annotations

import numpy as np

OPPOSITE = (0, 2, 1, 4, 3, 6, 5)


def transport(theta: np.ndarray, h: np.ndarray, mu: int) -> np.ndarray:
    """(T_mu h) for h of shape (Ntau, L, L, C)."""
    N = h.shape[0]
    ux = np.exp(1j * theta[..., 0])[..., None]
    uy = np.exp(1j * theta[..., 1])[..., None]
    if mu == 0:
        return h.copy()
    if mu == 1:
        return ux * np.roll(h, -1, axis=2)
    if mu == 2:
        return np.roll(np.conj(ux), 1, axis=2) * np.roll(h, 1, axis=2)
    if mu == 3:
        return uy * np.roll(h, -1, axis=1)
    if mu == 4:
        return np.roll(np.conj(uy), 1, axis=1) * np.roll(h, 1, axis=1)
    sign = np.ones((N, 1, 1, 1))
    if mu == 5:
        sign[N - 1] = -1.0
        return sign * np.roll(h, -1, axis=0)
    sign[0] = -1.0
    return sign * np.roll(h, 1, axis=0)


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Nearest bfloat16 value (8-bit significand, ties to even) of each real entry,
    taken through float32 and returned as float64: the upper 16 bits of the
    float32 pattern after adding half an ulp of bfloat16 (0x7FFF plus the lowest
    kept bit, which breaks ties towards an even significand)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32)
    u = (u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return u.view(np.float32).astype(np.float64)


def layer(theta: np.ndarray, h: np.ndarray, W: np.ndarray) -> np.ndarray:
    """One layer: sum over directions of the transported field times W[mu]^T."""
    out = None
    for mu in range(7):
        t = transport(theta, h, mu) @ W[mu].T  # (..., C_in) @ (C_in, C_out)
        out = t if out is None else out + t
    return out


def apply(theta: np.ndarray, r: np.ndarray, weights, tensor_cores: bool = False) -> np.ndarray:
    """K(theta) r for r of shape (Ntau, L, L).  tensor_cores: every 16-channel
    activation is stored in bfloat16 (real and imaginary parts rounded to the
    nearest bfloat16) before the next layer reads it, the precision of layers that
    contract BF16 activations with BF16 weights in a wide accumulator; all
    arithmetic stays FP64."""
    h = r[..., None].astype(np.complex128)
    for W in weights:
        h = layer(theta, h, np.asarray(W, dtype=np.float64))
        if tensor_cores and h.shape[-1] == 16:
            h = round_bf16(h.real) + 1j * round_bf16(h.imag)
    return h[..., 0]


def loss(theta, phi, x, weights) -> float:
    e = apply(theta, phi, weights) - x
    return float(np.vdot(e, e).real / np.vdot(x, x).real)


def loss_gradient(theta, phi, x, weights):
    """Analytic d loss / d W_l (back-propagation through the linear layers)."""
    hs = [phi[..., None].astype(np.complex128)]
    for W in weights:
        hs.append(layer(theta, hs[-1], W))
    xx = np.vdot(x, x).real
    d = 2.0 * (hs[-1] - x[..., None]) / xx
    grads = [None] * len(weights)
    for l in range(len(weights) - 1, -1, -1):
        W = weights[l]
        g = np.zeros_like(W, dtype=np.float64)
        for mu in range(7):
            th = transport(theta, hs[l], mu)                      # (..., C_in)
            C_out, C_in = d.shape[-1], th.shape[-1]
            g[mu] = (np.conj(d).reshape(-1, C_out).T @ th.reshape(-1, C_in)).real  # Re conj(d_c) (T h)_d
        grads[l] = g
        if l > 0:
            # adjoint layer: sum_mu T_mu^dagger (W_mu^T d) = sum_mu T_{mu-bar}(d @ W_mu)
            nd = None
            for mu in range(7):
                t = transport(theta, d @ W[mu], OPPOSITE[mu])
                nd = t if nd is None else nd + t
            d = nd
    return grads


def identity_weights(cin_cout):
    """Weights whose composition is the identity map (centre taps c -> c)."""
    ws = []
    for ci, co in cin_cout:
        W = np.zeros((7, co, ci))
        for c in range(min(ci, co)):
            W[0, c, c] = 1.0
        ws.append(W)
    return ws


def split_flat(flat, cin_cout):
    """Flat layer-by-layer weight vector -> list of (7, C_out, C_in) arrays."""
    out, k = [], 0
    for ci, co in cin_cout:
        n = 7 * co * ci
        out.append(np.asarray(flat[k:k + n], dtype=np.float64).reshape(7, co, ci))
        k += n
    return out


LAYERS = [(1, 16), (16, 16), (16, 16), (16, 1)]
