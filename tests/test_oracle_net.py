"""Pins of the FP64 reference of the learned preconditioner's network (no GPU)."""
import numpy as np

from oracle import net
from paper_2508_16298_gb300 import inputs

SMALL = [(1, 3), (3, 3), (3, 1)]


def rand_weights(layers, seed):
    g = inputs.rng(seed)
    return [g.standard_normal((7, co, ci)) * 0.3 for ci, co in layers]


def test_identity_weights_give_identity():
    th = inputs.theta_hot(4, 6, 1)
    r = inputs.complex_gaussian(4, 6, 2)
    assert np.allclose(net.apply(th, r, net.identity_weights(net.LAYERS)), r)


def test_transport_adjoint_is_opposite_direction():
    th = inputs.theta_hot(4, 5, 3)
    g = inputs.complex_gaussian(4, 5, 4)[..., None]
    h = inputs.complex_gaussian(4, 5, 5)[..., None]
    for mu in range(7):
        lhs = np.vdot(g, net.transport(th, h, mu))
        rhs = np.vdot(net.transport(th, g, net.OPPOSITE[mu]), h)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_linear_and_gauge_covariant():
    L, N = 4, 6
    th = inputs.theta_hot(L, N, 6)
    ws = rand_weights(SMALL, 7)
    a, b = inputs.complex_gaussian(L, N, 8), inputs.complex_gaussian(L, N, 9)
    z = net.apply(th, 0.3 * a + (1 - 2j) * b, ws)
    assert np.allclose(z, 0.3 * net.apply(th, a, ws) + (1 - 2j) * net.apply(th, b, ws))
    lam = inputs.rng(10).uniform(-np.pi, np.pi, size=(L, L))
    thg = th.copy()
    thg[..., 0] += lam[None] - np.roll(lam, -1, axis=1)[None]
    thg[..., 1] += lam[None] - np.roll(lam, -1, axis=0)[None]
    D = np.exp(1j * lam)[None]
    assert np.allclose(net.apply(thg, D * a, ws), D * net.apply(th, a, ws))


def test_translation_by_a_slice_commutes_up_to_the_boundary_sign():
    """Shifting a tau-independent field's input by one slice (antiperiodically) shifts the output."""
    L, N = 4, 6
    th = np.broadcast_to(inputs.theta_hot(L, 1, 11), (N, L, L, 2)).copy()
    ws = rand_weights(SMALL, 12)
    r = inputs.complex_gaussian(L, N, 13)
    shift = lambda v: np.concatenate([-v[-1:], v[:-1]], axis=0)  # v(tau-1), antiperiodic
    assert np.allclose(net.apply(th, shift(r), ws), shift(net.apply(th, r, ws)))


def test_gradient_matches_finite_differences():
    L, N = 4, 4
    th = inputs.theta_hot(L, N, 14)
    ws = rand_weights(SMALL, 15)
    phi, x = inputs.complex_gaussian(L, N, 16), inputs.complex_gaussian(L, N, 17)
    grads = net.loss_gradient(th, phi, x, ws)
    h = 1e-6
    g = inputs.rng(18)
    for l in range(len(ws)):
        for _ in range(6):
            idx = tuple(g.integers(0, s) for s in ws[l].shape)
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[l][idx] += h
            wm[l][idx] -= h
            fd = (net.loss(th, phi, x, wp) - net.loss(th, phi, x, wm)) / (2 * h)
            assert abs(grads[l][idx] - fd) < 1e-6 * max(1.0, abs(fd)), (l, idx, grads[l][idx], fd)
