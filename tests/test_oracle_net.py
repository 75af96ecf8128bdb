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


def test_bf16_rounding_pins():
    """Hand-worked bfloat16 roundings (8-bit significand, ties to even)."""
    e = 2.0 ** -8  # half an ulp of bfloat16 at 1
    vals = np.array([1.0, 1 + e, 1 + 3 * e, -(1 + e), 1 + 1.5 * e, 3.0, 1 / 3, 2.0 ** -20 * (1 + 2 ** -7)])
    want = np.array([1.0, 1.0, 1 + 4 * e, -1.0, 1 + 2 * e, 3.0,
                     0.333984375,  # 1/3 = 0x3EAAAAAB: kept bits 0x3EAA, remainder 0xAAAB > half: 0x3EAB
                     2.0 ** -20 * (1 + 2 ** -7)])
    assert np.array_equal(net.round_bf16(vals), want)


def test_tensor_core_mode_is_exact_when_activations_are_bf16_values():
    """theta = 0, a small-integer input and weights with entries in {-1, 0, 1, 2}:
    every activation is a small integer, exactly a bfloat16 value, so storing the
    16-channel activations in bfloat16 changes nothing."""
    L, N = 4, 6
    th = np.zeros((N, L, L, 2))
    g = inputs.rng(20)
    r = g.integers(-2, 3, size=(N, L, L)) + 1j * g.integers(-2, 3, size=(N, L, L))
    ws = [g.integers(-1, 3, size=(7, co, ci)).astype(np.float64) * (g.random((7, co, ci)) < 0.06)
          for ci, co in net.LAYERS]
    h = r[..., None].astype(np.complex128)
    for W in ws[:3]:  # the 16-channel activations: integers below 2^8 in size are bfloat16 values
        h = net.layer(th, h, W)
        assert np.max(np.abs(h.real)) < 256 and np.max(np.abs(h.imag)) < 256
    assert np.max(np.abs(h)) > 8
    a = net.apply(th, r, ws, tensor_cores=True)
    b = net.apply(th, r, ws)
    assert np.array_equal(a, b)


def test_tensor_core_mode_error_bound_of_one_layer():
    """A 16 -> 1 layer fed a rounded activation: each real entry moves by at most
    2^-9 of its size, so |layer(round(h)) - layer(h)| <= 2^-9 sum_mu |W_mu| (|Re T_mu h| +
    |Im T_mu h|) entry by entry, and on random data the bound is not slack by orders
    of magnitude."""
    L, N = 4, 6
    th = inputs.theta_hot(L, N, 21)
    g = inputs.rng(22)
    h = g.standard_normal((N, L, L, 16)) + 1j * g.standard_normal((N, L, L, 16))
    W = net.round_bf16(g.standard_normal((7, 1, 16)) * 0.3)
    hr = net.round_bf16(h.real) + 1j * net.round_bf16(h.imag)
    a = net.layer(th, hr, W)
    b = net.layer(th, h, W)
    bound = sum((np.abs(net.transport(th, h, mu).real) + np.abs(net.transport(th, h, mu).imag)) @ np.abs(W[mu]).T
                for mu in range(7))
    assert np.all(np.abs(a - b) <= 2.0 ** -9 * bound * (1 + 1e-6))
    assert np.max(np.abs(a - b)) > 1e-3 * 2.0 ** -9 * np.max(bound)


def test_tensor_core_mode_touches_only_16_channel_activations():
    L, N = 4, 6
    th = inputs.theta_hot(L, N, 23)
    r = inputs.complex_gaussian(L, N, 24)
    ws = rand_weights(SMALL, 25)  # no 16-channel activation
    assert np.array_equal(net.apply(th, r, ws, tensor_cores=True), net.apply(th, r, ws))
    ws16 = rand_weights(net.LAYERS, 26)
    a = net.apply(th, r, ws16, tensor_cores=True)
    b = net.apply(th, r, ws16)
    assert 0 < np.linalg.norm(a - b) < 1e-2 * np.linalg.norm(b)
