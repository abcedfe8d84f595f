"""Residual items of the training step on the tensor cores (option
train_tensor_cores): the forward jets, the reverse pass and the weight
gradients of hidden layers up to 64 wide as tcgen05 TF32 MMAs over hi/lo
splits of both operands, for tanh, sin and cos networks under Laplacian-jet
PDEs (Poisson, Navier-Stokes).

* losses (1e-5) and every gradient tensor (1e-4) match the FP64 oracle on a
  Navier-Stokes cPINN (width 64, six hidden layers, three outputs) and on a
  Poisson XPINN whose subdomains mix qualifying networks (widths 40-64,
  zero-padded to 64, two to five hidden layers) with one-hidden-layer
  networks that stay on the jet kernel in the same step; point counts leave
  ragged tiles (32 points) and ragged items;
* tanh, sin and cos hidden layers with trained or fixed slopes (the slope
  gradients included);
* the smallest network the kernel takes (one hidden-to-hidden layer of width
  33, zero-padded to 64), the deepest (seven hidden layers, every tensor-memory
  column in use) and items longer than one accumulator flush (16 tiles) on a
  large workload, sampled against the oracle;
* Adam steps follow the oracle given the gradient, repeated gradients agree
  bit for bit, and the per-subdomain loop schedule agrees within tolerance;
* the result lies within the tolerances of the FP32 jet kernel's.
"""
import numpy as np
import pytest

from oracle import Oracle, adam_update
from paper_2104_10013_gb300 import problems as P
from tests.test_parity import RTOL_GRAD, X, assert_grads, assert_losses  # noqa: F401

pytestmark = pytest.mark.gpu


def ns_small(n_res=300):
    return P.kovasznay_cpinn(nx=2, ny=2, n_res=n_res, n_iface=32, n_bc=40)


def poisson_mixed():
    return P.poisson_xpinn(nx=3, ny=2, n_res_range=(150, 700), width_range=(40, 64), depth_range=(1, 5),
                           n_iface=40, n_bc=30, seed=12)


def solver(X, pb, tc):
    s = X.Solver(pb)
    s.set_options(train_tensor_cores=tc)
    return s


@pytest.mark.parametrize("name", ["ns_w64_d6", "poisson_w40_64_mixed"])
def test_tensor_core_grad_matches_the_oracle(X, name):
    pb = ns_small() if name == "ns_w64_d6" else poisson_mixed()
    s = solver(X, pb, 64 if name == "ns_w64_d6" else 40)
    n_items, n_tc, n_tc_sub = s.plan_counts()
    depths = [len(sd.nets[0].widths) - 2 for sd in pb.subs]
    assert n_tc > 0 and n_tc_sub == sum(d >= 2 for d in depths), (n_tc, n_tc_sub, depths)
    if name != "ns_w64_d6":
        assert n_tc_sub < pb.n_sub   # some subdomains stay on the jet kernel
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


def test_tensor_core_items_are_deterministic_and_schedule_independent(X):
    """Repeated gradients agree bit for bit; the per-subdomain loop schedule
    (which cuts each subdomain's residual points into two items per SM so
    that its own launch fills the GPU) agrees within the tolerances."""
    pb = poisson_mixed()
    s = solver(X, pb, 40)
    l1, g1 = s.grad()
    l2, g2 = s.grad()
    assert np.array_equal(g1, g2) and np.array_equal(l1, l2)
    s.set_options(schedule=1)
    assert s.plan_counts()[1] > 0
    l3, g3 = s.grad()
    assert_losses(l3, l1)
    assert_grads(g3, g1.astype(np.float64), pb)
    s.close()


def test_tensor_core_grad_is_near_the_jet_kernel(X):
    pb = ns_small(n_res=700)
    a = solver(X, pb, 64)
    b = solver(X, pb, 0)
    assert a.plan_counts()[1] > 0 and b.plan_counts()[1] == 0
    la, ga = a.grad()
    lb, gb = b.grad()
    assert_losses(la, lb)
    assert_grads(ga, gb.astype(np.float64), pb, rtol=2 * RTOL_GRAD)
    a.close(); b.close()


def test_tensor_core_adam_steps_follow_the_oracle(X):
    pb = ns_small()
    s = solver(X, pb, 64)
    orc = Oracle(pb)
    th = s.get_params().astype(np.float64)
    _, g = s.grad()
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    lr = orc.lr_vector()
    for t in (1, 2, 3):
        s.step(1)
        th, m, v = adam_update(th, g.astype(np.float64), m, v, t, lr, orc.beta1, orc.beta2, orc.eps)
        got = s.get_params().astype(np.float64)
        assert np.all(np.abs(got - th) <= 1e-6 * lr + 1e-7 * np.abs(th)), (t, np.abs(got - th).max())
        th = got
        _, g = s.grad()
        terms, g_ref = orc.grad(th)
        assert_grads(g, g_ref, pb)
    s.close()


def test_narrowest_shallowest_network_on_the_tensor_cores(X):
    """2 -> 33 x 2 -> 1: one hidden-to-hidden layer, 31 zero-padded neurons."""
    pb = P.poisson_xpinn(nx=2, ny=1, n_res_range=(300, 400), width_range=(33, 33), depth_range=(2, 2),
                         n_iface=24, n_bc=20, seed=5)
    s = solver(X, pb, 33)
    assert s.plan_counts()[2] == 2
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


def test_items_longer_than_a_flush_sampled():
    """4 x 200k residual points: items of about 21 tiles, so each item's
    gradient accumulators are flushed into its slice once mid-item and once
    at its end; the oracle checks one whole subdomain."""
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as XX
    B.build()
    XX.load()
    pb = P.kovasznay_cpinn(nx=2, ny=2, n_res=200_000, n_iface=64, n_bc=40)
    s = XX.Solver(pb)
    n_items, n_tc, _ = s.plan_counts()
    assert 800_000 / n_tc > 16 * 32, n_tc   # items span more than one flush of 16 tiles
    losses, g = s.grad()
    s.close()
    terms, g_ref = Oracle(pb).grad(pb.packed_params(), subset=[1])
    assert_losses(losses[[1]], terms)
    from tests.test_parity import tensor_slices
    for name, sl in tensor_slices(pb):
        if name.startswith("q1n"):
            a, b = g[sl].astype(np.float64), g_ref[sl]
            assert np.linalg.norm(a - b) <= RTOL_GRAD * np.linalg.norm(b), name
            assert np.abs(a - b).max() <= RTOL_GRAD * np.abs(b).max(), name


def test_tensor_core_choice_per_subdomain(X):
    """With train_tensor_cores = 64, the one 64-wide subdomain of the uneven
    Poisson workload lies below the share rule; choosing the tensor-core
    kernel for it alone puts its residual items there, and the gradient still
    matches the oracle.
    Choosing the jet kernel everywhere empties the tensor-core items of the
    Navier-Stokes case."""
    pb = P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40)
    s = solver(X, pb, 64)
    assert s.plan_counts()[1] == 0 and not s.tc_subdomains().any()
    wide = [q for q, sd in enumerate(pb.subs) if max(sd.nets[0].widths[1:-1]) == 64 and len(sd.nets[0].widths) >= 4]
    assert wide
    sel = np.full(pb.n_sub, -1, np.int32)
    sel[wide] = 1
    s.set_tc_select(sel)
    assert s.plan_counts()[2] == len(wide)
    assert list(np.flatnonzero(s.tc_subdomains())) == wide
    assert list(s.tc_select()) == list(sel)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()
    t = solver(X, ns_small(), 64)
    assert t.plan_counts()[1] > 0
    t.set_tc_select(np.zeros(4, np.int32))
    assert t.plan_counts()[1] == 0
    t.close()


@pytest.mark.parametrize("acts,adaptive", [((P.PHI_SIN, P.PHI_COS, P.PHI_TANH), True),
                                           ((P.PHI_COS, P.PHI_SIN), False),
                                           ((P.PHI_TANH,), True)])
def test_general_activations_on_the_tensor_cores(X, acts, adaptive):
    """tanh, sin and cos hidden layers with trained slopes n a^k (Sec. 3) or
    fixed ones: the kernel's general rules, including every slope gradient."""
    from tests.cases import with_activations
    pb = with_activations(ns_small(), list(acts), adaptive=adaptive)
    s = solver(X, pb, 64)
    assert s.plan_counts()[2] == pb.n_sub
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


def test_default_minimum_width_takes_the_uneven_poisson_workload(X):
    """At the default train_tensor_cores (33) the subdomains of the uneven
    Poisson XPINN with hidden widths 33-64 and at least two hidden layers
    hold more than half of its residual points, so the share rule sends
    their residual items to the tensor-core kernel; the gradient matches the
    oracle."""
    pb = P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40)
    s = X.Solver(pb)
    assert s.options()["train_tensor_cores"] == 33
    want = [q for q, sd in enumerate(pb.subs)
            if all(33 <= w <= 64 for w in sd.nets[0].widths[1:-1]) and len(sd.nets[0].widths) >= 4]
    assert 2 * sum(pb.subs[q].res_xy.shape[0] for q in want) >= pb.n_res
    assert list(np.flatnonzero(s.tc_subdomains())) == want
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


def test_deepest_network_on_the_tensor_cores(X):
    """2 -> 64 x 7 -> 3: eight weight layers, every tensor-memory column in use
    (six hidden-to-hidden weight-gradient accumulators)."""
    pb = P.kovasznay_cpinn(nx=2, ny=1, n_res=300, n_iface=24, n_bc=30, depth=7)
    s = solver(X, pb, 64)
    assert s.plan_counts()[2] == pb.n_sub
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()
