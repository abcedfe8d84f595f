"""GPU vs the FP64 oracle for the full activation definition of Sec. 3:
hidden activation tanh, sin or cos per network (Table Table_USmap mixes tanh
and sin subdomains) and trainable layer-wise slopes Phi(n a^k z), n = 10.

Tolerances are those of the other parity tests: losses and jets 1e-5
(scaled), gradients 1e-4 per tensor, the slopes of a network being one
tensor."""
import ctypes as C

import numpy as np
import pytest

from oracle import Oracle, adam_update
from paper_2104_10013_gb300 import problems as P
from tests.cases import CASES, tiny_problem, with_activations
from tests.test_parity import RTOL_JET, assert_grads, assert_losses, assert_scaled

pytestmark = pytest.mark.gpu

ACTS3 = [P.PHI_TANH, P.PHI_SIN, P.PHI_COS]


@pytest.fixture(scope="module")
def X():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    return X


def _grad_parity(X, pb):
    s = X.Solver(pb)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()
    return g, g_ref


@pytest.mark.parametrize("pde,method", CASES)
def test_adaptive_slopes_every_pde_and_method(X, pde, method):
    """Three subdomains with tanh, sin and cos networks and trained slopes."""
    pb = with_activations(tiny_problem(pde, method, n_sub=3, n_res=37, n_data=11, n_if=9), ACTS3)
    g, _ = _grad_parity(X, pb)
    # every slope receives a gradient
    off = 0
    for s in pb.subs:
        for net in s.nets:
            off += net.n_params
            assert np.all(g[off - net.n_slopes:off] != 0)


@pytest.mark.parametrize("act", [P.PHI_SIN, P.PHI_COS])
def test_fixed_slope_sin_and_cos_networks(X, act):
    pb = with_activations(tiny_problem(P.PDE_NS, P.XPINN, n_sub=2, n_res=37, n_data=11, n_if=9), [act],
                          adaptive=False)
    assert pb.n_params == tiny_problem(P.PDE_NS, P.XPINN, n_sub=2).n_params   # no slope parameters
    _grad_parity(X, pb)


def test_initial_slopes_reproduce_the_fixed_network_on_the_gpu(X):
    """n a^k = 1/n * n = 1: the adaptive network's losses equal the fixed
    one's (to float32 rounding of the slope), and only the slope gradients
    are added."""
    pb0 = P.poisson_xpinn(n_res_range=(300, 900), n_iface=64, n_bc=40)
    pb1 = P.poisson_xpinn(n_res_range=(300, 900), n_iface=64, n_bc=40)
    import dataclasses
    for s in pb1.subs:
        s.nets = [dataclasses.replace(n, adaptive=True) for n in s.nets]
        s.slopes = []
    s0, s1 = X.Solver(pb0), X.Solver(pb1)
    l0, g0 = s0.grad()
    l1, g1 = s1.grad()
    assert_scaled(l1, l0, RTOL_JET, "losses", axis=0)
    keep = np.ones(pb1.n_params, bool)
    off = 0
    for s in pb1.subs:
        for net in s.nets:
            off += net.n_params
            keep[off - net.n_slopes:off] = False
    rel = np.linalg.norm(g1[keep] - g0) / np.linalg.norm(g0)
    assert rel <= 1e-4, rel
    s0.close(); s1.close()


@pytest.mark.parametrize("name", ["c2_mixed_tanh_sin", "c3_ns_all_three", "c4_diffusion_sin"])
def test_adaptive_slopes_on_workload_shapes(X, name):
    mk = {
        "c2_mixed_tanh_sin": lambda: with_activations(
            P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40), [P.PHI_TANH, P.PHI_SIN]),
        "c3_ns_all_three": lambda: with_activations(
            P.kovasznay_cpinn(nx=3, ny=3, n_res=1500, n_iface=96, n_bc=80), ACTS3),
        "c4_diffusion_sin": lambda: with_activations(
            P.diffusion_xpinn(n_res=1200, n_obs=100, n_iface=40, n_kbc=20, n_copies=1), [P.PHI_SIN]),
    }[name]
    _grad_parity(X, mk())


def test_adaptive_jets_parity(X):
    pb = with_activations(P.kovasznay_cpinn(nx=2, ny=2, n_res=600, n_iface=64, n_bc=40), ACTS3)
    s = X.Solver(pb)
    orc = Oracle(pb)
    theta = pb.packed_params()
    rng = np.random.default_rng(3)
    for q in range(pb.n_sub):
        x0, x1, y0, y1 = pb.subs[q].rect
        xy = np.stack([rng.uniform(x0, x1, 777), rng.uniform(y0, y1, 777)], 1).astype(np.float32)
        for order in (0, 1, 2):
            got = s.net_jets(q, 0, xy, order)
            ref = orc.net_jets(theta, q, 0, xy, (1, 3, 5)[order])
            assert_scaled(got, ref, RTOL_JET, f"q{q} order{order}", axis=(0, 1))
    s.close()


def test_adam_trains_the_slopes_like_the_oracle(X):
    pb = with_activations(tiny_problem(P.PDE_BURGERS, P.CPINN, n_sub=3, n_res=37, n_data=11, n_if=9), ACTS3)
    s = X.Solver(pb)
    orc = Oracle(pb)
    th = s.get_params().astype(np.float64)
    _, g = s.grad()
    m = np.zeros_like(th); v = np.zeros_like(th)
    lr = orc.lr_vector()
    for t in (1, 2, 3):
        s.step(1)
        th, m, v = adam_update(th, g.astype(np.float64), m, v, t, lr, orc.beta1, orc.beta2, orc.eps)
        got = s.get_params().astype(np.float64)
        assert np.all(np.abs(got - th) <= 1e-6 * lr + 1e-7 * np.abs(th)), (t, np.abs(got - th).max())
        th = got
        _, g = s.grad()
    s.close()


def test_noalloc_with_an_adaptive_sin_network(X):
    import torch
    lib = X.load()
    rng = np.random.default_rng(4)
    n = 1500
    net = P.NetSpec([2, 24, 24, 24, 1], act=P.PHI_SIN, adaptive=True)
    xy = P._f32(rng.uniform(0, 1, size=(n, 2)))
    sub = P.Subdomain(nets=[net], res_xy=xy, res_f=P._f32(rng.normal(size=n)), data=[None], w_data=[1.0],
                      w_res=0.7, rect=(0.0, 1.0, 0.0, 1.0))
    sub.params = [P.xavier_params(net, rng)]
    sub.slopes = [P._f32(rng.uniform(0.08, 0.15, size=net.n_slopes))]
    pb = P.Problem("one", P.PDE_POISSON, [sub], [], nu=0.0, re=1.0)
    s = X.Solver(pb)
    losses, g_ref = s.grad()
    s.close()
    dev = torch.device("cuda", 0)
    theta = torch.from_numpy(pb.packed_params()).to(dev)
    xy_d = torch.from_numpy(xy).to(dev)
    f_d = torch.from_numpy(sub.res_f).to(dev)
    d = X.NetDesc()
    d.n_layers = 4
    for k, w in enumerate(net.widths):
        d.widths[k] = w
    d.act, d.adaptive, d.slope_scale = P.PHI_SIN, 1, net.slope_scale
    loss = torch.full((1,), float("nan"), device=dev)
    grads = torch.full((pb.n_params,), float("nan"), device=dev)
    rc = lib.xpinn_residual_grad_noalloc(P.PDE_POISSON, C.c_float(0.0), C.c_float(1.0), C.byref(d),
                                         theta.data_ptr(), xy_d.data_ptr(), f_d.data_ptr(), n, C.c_float(0.7),
                                         loss.data_ptr(), grads.data_ptr(),
                                         torch.cuda.current_stream(dev).cuda_stream)
    assert rc == 0, lib.xpinn_last_error().decode()
    torch.cuda.synchronize()
    assert abs(float(loss.item()) - float(losses[0, 2])) <= 1e-5 * abs(float(losses[0, 2]))
    g = grads.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_fixed_tanh_and_general_networks_in_one_launch(X):
    """Subdomains alternate between fixed-slope tanh networks and trained-slope
    sin networks: one launch of the general kernel family runs both kinds of
    network passes, which share the weight buffers and their barriers."""
    import dataclasses
    pb = P.poisson_xpinn(n_res_range=(300, 1200), n_iface=64, n_bc=40)
    rng = np.random.default_rng(8)
    for q, s in enumerate(pb.subs):
        if q % 2:
            s.nets = [dataclasses.replace(n, act=P.PHI_SIN, adaptive=True) for n in s.nets]
            s.slopes = [P._f32(rng.uniform(0.08, 0.15, size=n.n_slopes)) for n in s.nets]
    _grad_parity(X, pb)
    # and the diffusion pair: a fixed tanh u-network beside a trained cos K-network
    pb2 = P.diffusion_xpinn(n_res=800, n_obs=60, n_iface=30, n_kbc=10, n_copies=1)
    for s in pb2.subs:
        s.nets = [dataclasses.replace(s.nets[0], act=P.PHI_TANH, adaptive=False),
                  dataclasses.replace(s.nets[1], act=P.PHI_COS, adaptive=True)]
        s.slopes = []
    _grad_parity(X, pb2)
