"""GPU (CUDA C-ABI) vs the FP64 oracle, element by element, on the same
seeded inputs and the same float32 weights.

Tolerances (fixed here; float32 rounds each layer at about 6e-8 relative to
its activations, and the jets, losses and gradients sum tens to thousands of
such terms):
  jets, interface values, losses:  |a - b| <= 1e-5 * max(|b|, rms(b))
      where rms is taken over the compared points and, for jets, over all
      outputs of the network for the same jet component (the float32
      rounding of every output is set by the activations of the last hidden
      layer, which all outputs share: a Navier-Stokes pressure gradient of
      0.006 carries the rounding of velocity gradients of 0.3); for losses
      the rms of one term over the subdomains;
  gradients, per weight tensor W^k / b^k of every subdomain:
      ||g - g*||_2 <= 1e-4 ||g*||_2  and  max|g - g*| <= 1e-4 max|g*|;
  Adam, given the GPU's own gradient: |theta - theta*| <= 1e-6 lr.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2104_10013_gb300 import problems as P
from tests.cases import CASES, tiny_problem, with_activations

pytestmark = pytest.mark.gpu

RTOL_JET = 1e-5
RTOL_GRAD = 1e-4


@pytest.fixture(scope="module")
def X():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    return X


def assert_scaled(a, b, rtol, what, axis=0):
    """|a - b| <= rtol * max(|b|, rms of b over `axis`) elementwise."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    rms = np.sqrt(np.mean(b * b, axis=axis, keepdims=True))
    den = np.maximum(np.abs(b), rms)
    den = np.where(den == 0, 1.0, den)
    err = np.abs(a - b) / den
    i = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= rtol, f"{what}: max scaled error {err.max():.3e} at {i}: {a[i]} vs {b[i]}"


def tensor_slices(pb):
    """(name, slice) of every W^k and b^k of every subdomain in the packed layout."""
    out, off = [], 0
    for q, s in enumerate(pb.subs):
        for n, net in enumerate(s.nets):
            for k in range(1, len(net.widths)):
                no, ni = net.widths[k], net.widths[k - 1]
                out.append((f"q{q}n{n}W{k}", slice(off, off + no * ni))); off += no * ni
                out.append((f"q{q}n{n}b{k}", slice(off, off + no))); off += no
            if net.n_slopes:
                out.append((f"q{q}n{n}a", slice(off, off + net.n_slopes))); off += net.n_slopes
    return out


def assert_grads(g, g_ref, pb, rtol=RTOL_GRAD):
    g = np.asarray(g, np.float64)
    for name, sl in tensor_slices(pb):
        a, b = g[sl], g_ref[sl]
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.abs(a).max() <= 1e-30, name
            continue
        rel = np.linalg.norm(a - b) / nb
        mx = np.abs(a - b).max() / np.abs(b).max()
        assert rel <= rtol and mx <= rtol, f"{name}: rel {rel:.3e}, max {mx:.3e}"


def assert_losses(l, l_ref):
    assert_scaled(l, l_ref, RTOL_JET, "losses", axis=0)


def small_c2():
    return P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40)


def small_c3():
    return P.kovasznay_cpinn(nx=3, ny=3, n_res=1500, n_iface=96, n_bc=80)


def small_c4():
    return P.diffusion_xpinn(n_res=1200, n_obs=100, n_iface=40, n_kbc=20, n_copies=2)


WORKLOADS = {
    "c1_burgers_cpinn_full": lambda: P.burgers_cpinn(),
    "c2_poisson_xpinn_small": small_c2,
    "c3_kovasznay_cpinn_small": small_c3,
    "c4_diffusion_xpinn_small": small_c4,
    "burgers_spacetime_xpinn_4x2": lambda: P.burgers_spacetime(4, 2, n_res_total=6000),
    "burgers_cpinn_x_xpinn_t_4x4": lambda: P.burgers_spacetime(4, 4, n_res_total=6000, method_x=P.CPINN),
    # the Burgers cPINN configuration with the flux it names literally, u u_x - nu u_x
    "c1_burgers_cpinn_literal_flux": lambda: P.burgers_cpinn(flux_mode=P.FLUX_LITERAL),
}
TINY = {f"tiny_pde{p}_m{m}": (lambda p=p, m=m: tiny_problem(p, m, n_sub=3, n_res=37, n_data=11, n_if=9))
        for p, m in CASES}


def _tiny_literal():
    pb = tiny_problem(P.PDE_BURGERS, P.CPINN, n_sub=3, n_res=37, n_data=11, n_if=9)
    pb.flux_mode = P.FLUX_LITERAL
    for it in pb.ifaces:                 # both components of f . n exercised
        it.normal = (0.6, 0.8)
    return pb


TINY["tiny_pde0_m0_literal_flux"] = _tiny_literal


@pytest.mark.parametrize("name", list(WORKLOADS) + list(TINY))
def test_grad_parity(X, name):
    pb = {**WORKLOADS, **TINY}[name]()
    s = X.Solver(pb)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


@pytest.mark.parametrize("name", list(WORKLOADS) + ["tiny_pde3_m1"])
def test_jets_parity(X, name):
    pb = {**WORKLOADS, **TINY}[name]()
    s = X.Solver(pb)
    orc = Oracle(pb)
    theta = pb.packed_params()
    rng = np.random.default_rng(1)
    for q in sorted(set([0, pb.n_sub - 1, pb.n_sub // 2])):
        sd = pb.subs[q]
        x0, x1, y0, y1 = sd.rect if sd.rect is not None else (0, 1, 0, 1)
        n = 777   # several sub-tiles and a ragged tail
        xy = np.stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n)], 1).astype(np.float32)
        for net in range(len(sd.nets)):
            for order in (0, 1, 2):
                K = (1, 3, 5)[order]
                got = s.net_jets(q, net, xy, order)
                ref = orc.net_jets(theta, q, net, xy, K)
                assert_scaled(got, ref, RTOL_JET, f"{name} q{q} net{net} order{order}", axis=(0, 1))
    s.close()


@pytest.mark.parametrize("name", list(WORKLOADS) + ["tiny_pde3_m1", "tiny_pde2_m1", "tiny_pde0_m0_literal_flux"])
def test_interface_exchange_parity(X, name):
    pb = {**WORKLOADS, **TINY}[name]()
    s = X.Solver(pb)
    s.grad()
    got = s.iface_values()
    orc = Oracle(pb)
    theta = pb.packed_params()
    rows = []
    for e, it in enumerate(pb.ifaces):
        sides = []
        for side in (0, 1):
            u, qty = orc.iface_quantities(__import__("torch").tensor(theta, dtype=__import__("torch").float64), e, side)
            sides.append(np.concatenate([u.detach().numpy(), qty.detach().numpy()], 1))
        rows.append(np.stack(sides, 1))   # [n, 2, nv]
    ref = np.concatenate(rows, 0)
    assert_scaled(got.reshape(ref.shape), ref, RTOL_JET, f"{name} exchange", axis=(0, 1))
    s.close()


def test_grouped_and_loop_schedules_agree_bitwise(X):
    pb = small_c2()
    s = X.Solver(pb)
    l1, g1 = s.grad()
    s.set_options(schedule=1)
    l2, g2 = s.grad()
    assert np.array_equal(g1, g2) and np.array_equal(l1, l2)
    s.close()


def test_repeated_grad_is_bitwise_deterministic(X):
    pb = small_c3()
    s = X.Solver(pb)
    l1, g1 = s.grad()
    l2, g2 = s.grad()
    assert np.array_equal(g1, g2) and np.array_equal(l1, l2)
    s.close()


@pytest.mark.parametrize("name", ["c1_burgers_cpinn_full", "c2_poisson_xpinn_small", "tiny_pde3_m1"])
def test_adam_step_matches_oracle_given_the_gradient(X, name):
    pb = {**WORKLOADS, **TINY}[name]()
    s = X.Solver(pb)
    orc = Oracle(pb)
    theta0 = s.get_params().astype(np.float64)
    l_grad, g = s.grad()
    m = np.zeros_like(theta0)
    v = np.zeros_like(theta0)
    th = theta0
    for t in (1, 2, 3):
        l_step = s.step(1)[0]
        if t == 1:
            assert np.array_equal(l_step, l_grad)   # the step's losses are measured before its update
        th, m, v = __import__("oracle").adam_update(th, g.astype(np.float64), m, v, t, orc.lr_vector(),
                                                    orc.beta1, orc.beta2, orc.eps)
        got = s.get_params().astype(np.float64)
        lr = orc.lr_vector()
        assert np.all(np.abs(got - th) <= 1e-6 * lr + 1e-7 * np.abs(th)), (t, np.abs(got - th).max())
        th = got
        _, g = s.grad()
    s.close()


def test_checkpoint_resume_is_bitwise(X):
    pb = P.burgers_cpinn(n_res=500)
    a = X.Solver(pb)
    la = a.step(10)
    ref = a.get_params()
    b = X.Solver(pb)
    lb1 = b.step(5)
    blob = b.get_state()
    b.close()
    c = X.Solver(pb)
    c.set_state(blob)
    lb2 = c.step(5)
    assert np.array_equal(c.get_params(), ref)
    assert np.array_equal(np.concatenate([lb1, lb2]), la)
    a.close(); c.close()


def test_multi_step_graph_is_bitwise_equal_to_single_steps(X):
    """40 steps in one call replay the 16-step graph twice and the one-step
    graph 8 times; the same 40 steps without graphs, one launch sequence per
    step, give the same parameters and loss rows bit for bit."""
    pb = P.burgers_cpinn(n_res=400)
    a = X.Solver(pb)
    la = a.step(40)
    b = X.Solver(pb)
    b.set_options(use_graph=0)
    lb = np.concatenate([b.step(1) for _ in range(40)])
    assert np.array_equal(la, lb)
    assert np.array_equal(a.get_params(), b.get_params())
    a.close(); b.close()


def test_training_trajectory_follows_the_oracle(X):
    """100 Adam steps of the full Burgers cPINN problem: the loss curve stays
    within 1e-3 relative of the FP64 trajectory (float32 drift only)."""
    pb = P.burgers_cpinn()
    s = X.Solver(pb)
    lg = s.step(100)
    orc = Oracle(pb)
    th = pb.packed_params().astype(np.float64)
    m = np.zeros_like(th); v = np.zeros_like(th)
    W = orc.weights()
    for t in range(1, 101):
        terms, th, m, v = orc.step(th, m, v, t)
        J_ref = (terms * W).sum()
        J_gpu = (lg[t - 1].astype(np.float64) * W).sum()
        assert abs(J_gpu - J_ref) <= 1e-3 * J_ref, (t, J_gpu, J_ref)
    assert (lg[-1] * W).sum() < 0.5 * (lg[0] * W).sum()   # it trains
    s.close()


@pytest.mark.parametrize("order", [0, 1, 2])
def test_stitched_eval_parity(X, order):
    pb = small_c2()
    s = X.Solver(pb)
    rng = np.random.default_rng(3)
    xy = rng.random((3001, 2)).astype(np.float32)
    xc, yc = pb.meta["xcuts"], pb.meta["ycuts"]
    on_cuts = np.array([[xc[1], 0.3], [0.6, yc[2]], [xc[2], yc[1]], [xc[0], yc[0]], [1.2, 0.5]], np.float32)
    xy = np.concatenate([xy, on_cuts])
    got = s.eval(0, xy, order)
    ref = Oracle(pb).eval_stitched(pb.packed_params(), 0, xy, (1, 3, 5)[order])
    assert np.isnan(got[-1]).all() and np.isnan(ref[-1]).all()
    assert_scaled(got[:-1], ref[:-1], RTOL_JET, f"eval order {order}", axis=(0, 1))
    s.close()


def test_edge_cases_empty_and_single_point_sets(X):
    """A subdomain without residual points, one without data, an interface
    with a single point, point counts that leave ragged sub-tiles."""
    pb = tiny_problem(P.PDE_NS, P.CPINN, n_sub=3, n_res=1, n_data=1, n_if=1)
    pb.subs[1].res_xy = pb.subs[1].res_xy[:0]
    pb.subs[1].res_f = pb.subs[1].res_f[:0]
    pb.subs[2].data = [None]
    s = X.Solver(pb)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


def test_residual_points_can_be_replaced(X):
    pb = P.burgers_cpinn(n_res=300)
    s = X.Solver(pb)
    rng = np.random.default_rng(9)
    for sd in pb.subs:
        x0, x1, y0, y1 = sd.rect
        sd.res_xy = np.stack([rng.uniform(x0, x1, 300), rng.uniform(y0, y1, 300)], 1).astype(np.float32)
    xy = np.concatenate([sd.res_xy for sd in pb.subs])
    s.set_residual_points(xy, np.zeros(len(xy), np.float32))
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


def test_full_size_bench_workload_parity(X):
    """The benchmark's workload (16-subdomain XPINN Poisson at full size),
    in the launch configuration the benchmark times: every loss term and
    every gradient tensor against the oracle."""
    pb = P.poisson_xpinn()
    s = X.Solver(pb)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


def test_autotune_keeps_parity_and_state(X, tmp_path):
    pb = small_c2()
    s = X.Solver(pb)
    theta0 = s.get_params()
    cache = str(tmp_path / "tune.json")
    rec = s.autotune(steps=2, cache=cache)
    assert rec["options"]["points_per_thread"] in (1, 2) and rec["ms"] > 0
    assert np.array_equal(s.get_params(), theta0)          # tuning does not train
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s2 = X.Solver(pb)
    rec2 = s2.autotune(cache=cache)                         # served from the cache
    assert rec2 == rec and s2.options()["items_per_cta"] == rec["options"]["items_per_cta"]
    assert set(rec["class_caps"]) == {X.Solver.shape_class(sd) for sd in pb.subs}
    assert np.array_equal(s2.tile_caps(), s.tile_caps())    # per-class caps restored
    s.close(); s2.close()


def test_per_shape_tile_caps_keep_parity(X):
    """Different sub-tile caps for different shape classes in one grouped
    launch (the uneven Poisson workload: every class its own cap, cycling
    through 8..256 points): losses and gradients stay within tolerance."""
    pb = small_c2()
    s = X.Solver(pb)
    keys = sorted({X.Solver.shape_class(sd) for sd in pb.subs})
    choice = {k: (8, 32, 48, 0, 96)[i % 5] for i, k in enumerate(keys)}
    caps = [choice[X.Solver.shape_class(sd)] for sd in pb.subs]
    s.set_tile_caps(caps)
    assert np.array_equal(s.tile_caps(), caps)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()


@pytest.mark.parametrize("order", [0, 2])
def test_stitched_eval_on_voronoi_regions(X, order):
    """Eq. FSol on the irregular decomposition: points inside the polygon go to
    the region of their nearest site, points outside get NaN."""
    pb = small_c4()
    s = X.Solver(pb)
    rng = np.random.default_rng(4)
    inside = np.concatenate([sd.res_xy[rng.choice(sd.res_xy.shape[0], 150, replace=False)]
                             for sd in pb.subs[:10]])
    outside = np.array([[10.0, 10.0], [-5.0, 0.3]], np.float32)
    xy = np.concatenate([inside, outside]).astype(np.float32)
    for model in (0, 1):
        got = s.eval(model, xy, order)
        ref = Oracle(pb).eval_stitched(pb.packed_params(), model, xy, (1, 3, 5)[order])
        assert np.isnan(got[-2:]).all() and np.isnan(ref[-2:]).all()
        assert_scaled(got[:-2], ref[:-2], RTOL_JET, f"voronoi eval model {model}", axis=(0, 1))
    s.close()


def test_eval_from_workspace_is_device_planned_and_bitwise_equal(X):
    """xpinn_eval_ws with device points, output and workspace (no host round
    trip) equals xpinn_eval bit for bit and the oracle within tolerance,
    including the worst case of every point on a corner shared by four
    subdomains (the workspace bound) and points on single cuts."""
    import torch
    pb = small_c2()
    s = X.Solver(pb)
    xc, yc = pb.meta["xcuts"], pb.meta["ycuts"]
    rng = np.random.default_rng(8)
    corners = np.array([[xc[i], yc[j]] for i in range(1, 4) for j in range(1, 4)], np.float32)
    xy = np.concatenate([np.repeat(corners, 40, axis=0),                       # four boxes each
                         np.stack([np.full(200, xc[2]), rng.random(200)], 1),  # two boxes
                         rng.random((2000, 2))]).astype(np.float32)
    for order in (0, 2):
        ref_host = s.eval(0, xy, order)
        ws = torch.empty(s.eval_workspace_size(len(xy), order), dtype=torch.uint8, device="cuda")
        dxy = torch.from_numpy(xy).cuda()
        dout = torch.full(ref_host.shape, float("nan"), device="cuda")
        s.eval_ws(0, dxy, order, dout, ws)
        torch.cuda.synchronize()
        s.sync()
        got = dout.cpu().numpy()
        assert np.array_equal(got, ref_host)
        ref = Oracle(pb).eval_stitched(pb.packed_params(), 0, xy, (1, 3, 5)[order])
        assert_scaled(got, ref, RTOL_JET, f"workspace eval order {order}", axis=(0, 1))
    s.close()


def test_voronoi_routing_on_and_next_to_polygon_edges(X):
    """Points exactly on the polygon's edges (rounded to float32) and one ulp
    to either side in x and y: the GPU router and the oracle classify every one
    the same way (inside: routed and evaluated; outside: NaN), since both take
    the even-odd decision in float32 in the same operation order."""
    pb = small_c4()
    poly = np.asarray(pb.polygon, np.float32)
    rng = np.random.default_rng(11)
    on = []
    for e in range(len(poly)):
        a, b = poly[e], poly[(e + 1) % len(poly)]
        for t in rng.random(12):
            on.append(a + np.float32(t) * (b - a))
    on = np.asarray(on, np.float32)
    pts = [on]
    for axis in (0, 1):
        for direction in (np.inf, -np.inf):
            q = on.copy()
            q[:, axis] = np.nextafter(q[:, axis], np.float32(direction))
            pts.append(q)
    xy = np.concatenate(pts + [poly]).astype(np.float32)     # and the vertices themselves
    s = X.Solver(pb)
    got = s.eval(0, xy, 0)
    ref = Oracle(pb).eval_stitched(pb.packed_params(), 0, xy, 1)
    gn, rn = np.isnan(got[:, 0, 0]), np.isnan(ref[:, 0, 0])
    assert np.array_equal(gn, rn), np.nonzero(gn != rn)[0][:10]
    assert 0 < gn.sum() < len(xy)          # both outcomes occur
    assert_scaled(got[~gn], ref[~rn], RTOL_JET, "edge points", axis=(0, 1))
    s.close()


@pytest.mark.parametrize("widths,pde,method", [
    ([2] + [112] * 11 + [3], P.PDE_NS, P.CPINN),      # the largest width and depth the ABI accepts
    ([2, 1, 1, 1], P.PDE_POISSON, P.XPINN),          # one neuron per hidden layer
    ([2, 16, 3], P.PDE_NS, P.XPINN),                 # one hidden layer: no hidden-to-hidden weights
    ([2, 9, 17, 33, 1], P.PDE_BURGERS, P.XPINN),     # widths that are not multiples of the tile
])
def test_extreme_network_shapes(X, widths, pde, method):
    pb = tiny_problem(pde, method, n_sub=2, widths=widths, n_res=37, n_data=11, n_if=9)
    rng = np.random.default_rng(7)
    for sd in pb.subs:   # Xavier-scaled weights keep deep wide jets in a sane range
        sd.params = [P.xavier_params(n, rng) for n in sd.nets]
        for layers in sd.params:
            for k, (W, b) in enumerate(layers):
                layers[k] = (W, P._f32(rng.normal(size=b.shape) * 0.1))
    s = X.Solver(pb)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    xy = np.random.default_rng(2).uniform(0, 1, size=(300, 2)).astype(np.float32)
    got = s.net_jets(0, 0, xy, 2)
    ref = Oracle(pb).net_jets(pb.packed_params(), 0, 0, xy, 5)
    assert_scaled(got, ref, RTOL_JET, "jets", axis=(0, 1))
    s.close()


def test_evaluation_follows_new_parameters(X):
    """The weight images the jet kernel copies are rebuilt after set_params and
    after training steps: evaluations use the parameters of the moment."""
    pb = small_c2()
    s = X.Solver(pb)
    orc = Oracle(pb)
    xy = np.random.default_rng(5).uniform(0, 1, size=(500, 2)).astype(np.float32)
    q = 5
    x0, x1, y0, y1 = pb.subs[q].rect
    xy[:, 0] = x0 + (x1 - x0) * xy[:, 0]
    xy[:, 1] = y0 + (y1 - y0) * xy[:, 1]
    got0 = s.net_jets(q, 0, xy, 2)                    # images built from the initial parameters
    theta = pb.packed_params() * np.float32(0.9)
    s.set_params(theta)
    got1 = s.net_jets(q, 0, xy, 2)
    ref1 = orc.net_jets(theta, q, 0, xy, 5)
    assert_scaled(got1, ref1, RTOL_JET, "after set_params", axis=(0, 1))
    assert np.abs(got1 - got0).max() > 1e-3
    s.step(2)
    theta2 = s.get_params()
    got2 = s.net_jets(q, 0, xy, 2)
    ref2 = orc.net_jets(theta2, q, 0, xy, 5)
    assert_scaled(got2, ref2, RTOL_JET, "after steps", axis=(0, 1))
    s.close()


# every (points per thread, threads per CTA) instantiation the planner can
# choose, for both kernel families: the autotuner may pick any of them
KERNEL_CONFIGS = [(2, 256), (1, 256), (2, 128), (1, 128), (1, 512)]


@pytest.mark.parametrize("pt,threads", KERNEL_CONFIGS)
@pytest.mark.parametrize("family", ["tanh", "general"])
def test_every_kernel_configuration(X, pt, threads, family):
    pb = small_c2() if family == "tanh" else with_activations(small_c4(), [P.PHI_SIN, P.PHI_COS, P.PHI_TANH])
    s = X.Solver(pb)
    s.set_options(points_per_thread=pt, threads_per_cta=threads, items_per_cta=4)
    opts = s.options()
    assert opts["points_per_thread"] == pt and opts["threads_per_cta"] == threads
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert_losses(losses, terms)
    assert_grads(g, g_ref, pb)
    s.close()
