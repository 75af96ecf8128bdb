"""The learned preconditioner's CUDA kernels (inference and training) against the
FP64 reference network of oracle/net.py, and the learned solver."""
import numpy as np
import pytest
import torch

import oracle
from oracle import net as onet
from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), kept as float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    b = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return b.view(np.float32)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def random_flat(seed, scale=0.25):
    n = sum(7 * ci * co for ci, co in onet.LAYERS)
    return bf16(inputs.rng(seed).standard_normal(n) * scale)


@pytest.mark.parametrize("L,N", [(4, 4), (8, 12), (24, 48)])
def test_net_forward_matches_reference(hq, L, N):
    """FP32 layers on CUDA cores against the FP64 reference."""
    w = random_flat(1)
    th = inputs.theta_hot(L, N, 2)
    r = inputs.complex_gaussian(L, N, 3)
    ref = onet.apply(th, r, onet.split_flat(w, onet.LAYERS))
    with hq.Config(L, N) as cfg:
        k = hq.Net(seed=0)
        k.set_weights(w)
        hq.set_preconditioner(cfg, k)  # allocates the config's net workspace
        hq.set_net_tensor_cores(cfg, False)
        z = k.apply(cfg, cuda(th), cuda(r)).cpu().numpy()
        k.close()
    assert rel(z, ref) < 1e-5


@pytest.mark.parametrize("L,N", [(4, 4), (8, 12), (24, 48), (66, 40)])
def test_tensor_core_net_matches_bf16_reference(hq, L, N):
    """Tensor-core layers (16-channel activations stored in BF16, BF16 x BF16 products
    with FP32 accumulation) against the reference that rounds the same activations to
    BF16 (oracle/net.py, tensor_cores=True): they differ only where an FP32 and an
    FP64 activation round to different BF16 neighbours and in the order of the FP32
    sums.  Against the exact reference the error is the BF16 storage itself, an order
    of magnitude larger."""
    w = random_flat(1)
    th = inputs.theta_hot(L, N, 2)
    r = inputs.complex_gaussian(L, N, 3)
    ws = onet.split_flat(w, onet.LAYERS)
    ref_tc = onet.apply(th, r, ws, tensor_cores=True)
    ref = onet.apply(th, r, ws)
    with hq.Config(L, N) as cfg:
        k = hq.Net(seed=0)
        k.set_weights(w)
        hq.set_preconditioner(cfg, k)
        hq.set_net_tensor_cores(cfg, True)
        z = k.apply(cfg, cuda(th), cuda(r)).cpu().numpy()
        k.close()
    e_tc = np.linalg.norm(z - ref_tc) / np.linalg.norm(ref_tc)
    e_exact = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    e_model = np.linalg.norm(ref_tc - ref) / np.linalg.norm(ref)
    print(f"L={L}: tensor cores vs BF16-operand reference {e_tc:.2e}, vs exact {e_exact:.2e} "
          f"(reference's own BF16 effect {e_model:.2e})")
    # an activation that rounds to the other BF16 neighbour (one ulp, 2^-8) in one layer
    # moves the next layer's sums and flips more roundings there: a few 1e-4 in norm
    assert e_tc < 5e-4
    assert e_tc < 0.15 * e_model
    assert e_exact < 1e-2


def test_net_tensor_core_switch_arguments(hq):
    with hq.Config(8, 16) as cfg:
        for bad in (-1, 2):
            assert hq._lib.hqmc_set_net_tensor_cores(cfg.handle, bad) == hq.EINVAL
        hq.set_net_tensor_cores(cfg, False)
        hq.set_net_tensor_cores(cfg, True)


@pytest.mark.parametrize("tc", [False, True])
def test_net_is_gauge_covariant(hq, tc):
    L, N = 8, 10
    th = inputs.theta_hot(L, N, 4)
    r = inputs.complex_gaussian(L, N, 5)
    lam = inputs.rng(6).uniform(-np.pi, np.pi, size=(L, L))
    thg = th.copy()
    thg[..., 0] += lam[None] - np.roll(lam, -1, axis=1)[None]
    thg[..., 1] += lam[None] - np.roll(lam, -1, axis=0)[None]
    D = np.exp(1j * lam)[None]
    with hq.Config(L, N) as cfg:
        k = hq.Net(seed=0)
        k.set_weights(random_flat(7))
        hq.set_preconditioner(cfg, k)
        hq.set_net_tensor_cores(cfg, tc)
        a = k.apply(cfg, cuda(thg), cuda(D * r)).cpu().numpy()
        b = D * k.apply(cfg, cuda(th), cuda(r)).cpu().numpy()
        k.close()
    # BF16 storage rounds the rotated activations differently: covariance holds to
    # the storage rounding (2^-9 relative per entry) instead of FP32 rounding
    assert rel(a, b) < (2e-2 if tc else 1e-5)


def test_first_adam_step_follows_the_reference_gradient(hq):
    """Adam's first step is -lr * g / (|g| + eps): each weight moves against the sign of
    its gradient.  Compare with the reference back-propagation on one triple."""
    L, N = 6, 8
    w = random_flat(8, 0.3)
    th = inputs.theta_hot(L, N, 9)
    phi, x = inputs.complex_gaussian(L, N, 10), inputs.complex_gaussian(L, N, 11)
    ws = onet.split_flat(w, onet.LAYERS)
    grads = np.concatenate([g.reshape(-1) for g in onet.loss_gradient(th, phi, x, ws)])
    with hq.Config(L, N) as cfg:
        k = hq.Net(seed=0)
        k.set_weights(w)
        hq.set_preconditioner(cfg, k)
        loss = k.train_step(cfg, cuda(th), cuda(phi), cuda(x), lr=1e-3)
        w1 = k.get_weights()
        k.close()
    assert abs(loss - onet.loss(th, phi, x, ws)) < 1e-5 * onet.loss(th, phi, x, ws)
    step = w1 - w
    big = np.abs(grads) > 1e-3 * np.max(np.abs(grads))
    assert big.sum() > 100
    assert np.all(np.sign(step[big]) == -np.sign(grads[big]))
    assert np.allclose(np.abs(step[big]), 1e-3, rtol=1e-2)


def test_training_lowers_the_loss_and_helps_the_solver(hq):
    """Train on sampler triples (theta from the field, x solved by FP64 CG) and use the
    net through the learned solver: the true residual still judges convergence."""
    L, N = 8, 40
    lat = oracle.Lattice(L, N)
    with hq.Config(L, N) as cfg:
        k = hq.Net(seed=1)
        hq.set_preconditioner(cfg, k)
        triples = []
        for s in range(6):
            th = cuda(inputs.theta_ordered(L, N, 20 + s, tau_walk=0.0))
            phi = hq.apply_M(cfg, th, cuda(inputs.complex_gaussian(L, N, 40 + s)), dagger=True)
            X, info = hq.cg_solve(cfg, th, phi, tol=1e-10)
            triples.append((th, phi, X))
        losses = []
        for epoch in range(30):
            for th, phi, X in triples:
                losses.append(k.train_step(cfg, th, phi, X, lr=3e-3))
        assert np.mean(losses[-6:]) < 0.5 * np.mean(losses[:6])
        th = cuda(inputs.theta_ordered(L, N, 99, tau_walk=0.0))
        phi = hq.apply_M(cfg, th, cuda(inputs.complex_gaussian(L, N, 98)), dagger=True)
        Xl, il = hq.cg_solve(cfg, th, phi, tol=1e-8, solver="learned")
        Xp, ip = hq.cg_solve(cfg, th, phi, tol=1e-8, solver="mixed")
        hq.set_preconditioner(cfg, None)
        k.close()
    assert il["status"] == 0 and il["true_residual"] <= 1e-8
    assert il["net_guess_used"] == 1
    r = phi.cpu().numpy() - oracle.apply_MdagM(lat, th.cpu().numpy(), Xl.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi.cpu().numpy())
    print("learned iterations", il["iterations"], "mixed iterations", ip["iterations"])


def test_net_workspace_comes_from_the_attach_call(hq):
    """hqmc_set_preconditioner allocates the net workspace; without it the net calls
    refuse (HQMC_EINVAL), and with it neither a net apply, a training step nor a
    learned solve allocates device memory."""
    L, N = 8, 16
    th = cuda(inputs.theta_hot(L, N, 12))
    r = cuda(inputs.complex_gaussian(L, N, 13))
    with hq.Config(L, N) as cfg:
        k = hq.Net(seed=0)
        with pytest.raises(hq.HQMCError) as e:
            k.apply(cfg, th, r)
        assert e.value.status == hq.EINVAL
        hq.set_preconditioner(cfg, k)
        phi = hq.apply_M(cfg, th, r, dagger=True)
        X, _ = hq.cg_solve(cfg, th, phi, tol=1e-10)
        k.apply(cfg, th, r)  # warm-up: graphs, events
        hq.cg_solve(cfg, th, phi, tol=1e-8, solver="learned")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            k.apply(cfg, th, r)
            k.train_step(cfg, th, phi, X, lr=1e-4)
            hq.cg_solve(cfg, th, phi, tol=1e-8, solver="learned")
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        hq.set_preconditioner(cfg, None)
        k.close()
