"""Flexible CG with the learned net as a variable preconditioner
(HQMC_SOLVER_FLEARNED) against the oracle's flexible CG (oracle/fcg.py) with the
FP64 reference network (oracle/net.py) and the same BF16 weights.

The GPU recurrence runs in FP32 (FP64 reliable updates every 50 iterations), the
oracle's in FP64; after three iterations the iterates agree to FP32 rounding of
the ~100 dependent operations per element of the net and the operator (bound
1e-4 of the correction, as for preconditioned CG).  Full solves are judged by
the oracle's own residual ||phi - O X|| <= 1.01e-8 ||phi||.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import fcg as ofcg
from oracle import net as onet
from oracle import precond as opc
from paper_2508_16298_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def bf16(a):
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    b = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return b.view(np.float32)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_net(th, net, tensor_cores=False):
    """The oracle network with the GPU net's BF16 weights (and, for the tensor-core
    layers, 16-channel activations stored in BF16)."""
    ws = onet.split_flat(bf16(net.get_weights()), onet.LAYERS)
    return lambda r: onet.apply(th, r, ws, tensor_cores=tensor_cores)


@pytest.mark.parametrize("tc", [False, True])
def test_three_flexible_iterations_elementwise(hq, tc):
    L, N = 8, 40
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 61, tau_walk=0.0)
    phi = inputs.complex_gaussian(L, N, 62)
    x0 = 0.05 * inputs.complex_gaussian(L, N, 63)
    c = opc.coefficients(lat)
    with hq.Config(L, N) as cfg:
        net = hq.Net(seed=4)  # near the identity map
        hq.set_preconditioner(cfg, net)
        hq.set_net_interval(cfg, 2)  # net on iterations 0 and 2, tau-line on 1
        hq.set_net_tensor_cores(cfg, tc)
        K = oracle_net(th, net, tc)
        xg, used = ofcg.learned_guess(lat, th, phi, x0, K)
        xo, n, _, status = ofcg.fcg(lat, th, phi, lambda k, r: K(r) if k % 2 == 0 else opc.apply(c, r), x0=xg,
                                    tol=1e-30, maxit=3)
        assert n == 3 and status == "maxit"
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), x=cuda(x0), tol=1e-30, maxit=3, solver="flearned",
                              raise_on_fail=False)
        hq.set_preconditioner(cfg, None)
        net.close()
    X = X.cpu().numpy()
    assert info["iterations"] == 3 and info["fcg_fallback"] == 0
    assert info["net_guess_used"] == int(used)
    err = np.max(np.abs((X - xg) - (xo - xg))) / np.max(np.abs(xo - xg))
    print("three FCG iterations, GPU vs oracle:", err, "guess used:", used, "tensor cores:", tc)
    # tensor cores: the oracle rounds the same activations to BF16, and a value on a
    # rounding boundary may round the other way (one BF16 ulp, 2^-8)
    assert err < (1e-3 if tc else 1e-4)


def train(hq, cfg, th, L, N, n=4, epochs=20):
    trips = []
    for k in range(n):
        phi = hq.apply_M(cfg, th, cuda(inputs.complex_gaussian(L, N, 70 + k)), dagger=True)
        x, _ = hq.cg_solve(cfg, th, phi, tol=1e-10, solver="pcg64")
        trips.append((phi, x))
    net = hq.Net(seed=6)
    hq.set_preconditioner(cfg, net)
    for _ in range(epochs):
        for phi, x in trips:
            net.train_step(cfg, th, phi, x, lr=2e-3, want_loss=False)
    return net


@pytest.mark.parametrize("interval", [1, 5])
def test_flexible_solve_against_oracle(hq, interval):
    L, N = 8, 40
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 64, tau_walk=0.0)
    phi = inputs.complex_gaussian(L, N, 65)
    c = opc.coefficients(lat)
    with hq.Config(L, N) as cfg:
        tht = cuda(th)
        net = train(hq, cfg, tht, L, N)
        hq.set_net_interval(cfg, interval)
        X, info = hq.cg_solve(cfg, tht, cuda(phi), tol=1e-8, solver="flearned")
        _, ip = hq.cg_solve(cfg, tht, cuda(phi), tol=1e-8, solver="pmixed")
        K = oracle_net(th, net, True)  # the config default: tensor-core layers
        hq.set_preconditioner(cfg, None)
        net.close()
    X = X.cpu().numpy()
    print(f"interval {interval}: flearned", info, "pmixed iterations", ip["iterations"])
    assert info["status"] == 0 and info["true_residual"] <= 1e-8
    r = phi - oracle.apply_MdagM(lat, th, X)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi)
    if info["fcg_fallback"] == 0:
        xg, _ = ofcg.learned_guess(lat, th, phi, np.zeros_like(phi), K)
        _, n, res, status = ofcg.fcg(lat, th, phi, lambda k, r: K(r) if k % interval == 0 else opc.apply(c, r),
                                     x0=xg, tol=1e-8)
        print("oracle FCG iterations", n, status)
        assert status == "converged"
        # the FP32 recurrence may need a few more iterations than the FP64 one to meet
        # 1e-8, and one reliable update (every 50 iterations) restarts its drift
        assert abs(info["iterations"] - n) <= max(12, 0.25 * n)


def test_a_net_that_breaks_fcg_falls_back(hq):
    """A net equal to minus the identity makes Re<r, z> < 0 at once: the solve hands
    over to the tau-line preconditioned mixed solver and still converges."""
    L, N = 8, 40
    lat = oracle.Lattice(L, N)
    th = inputs.theta_ordered(L, N, 66, tau_walk=0.0)
    phi = inputs.complex_gaussian(L, N, 67)
    ws = onet.identity_weights(onet.LAYERS)
    ws[0] = -ws[0]
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    with hq.Config(L, N) as cfg:
        net = hq.Net(seed=0)
        net.set_weights(flat)
        hq.set_preconditioner(cfg, net)
        X, info = hq.cg_solve(cfg, cuda(th), cuda(phi), tol=1e-8, solver="flearned")
        hq.set_preconditioner(cfg, None)
        net.close()
    assert info["fcg_fallback"] == 1 and info["status"] == 0 and info["true_residual"] <= 1e-8
    r = phi - oracle.apply_MdagM(lat, th, X.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(phi)
