"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests reuses the oracle's own formula for the quantity it
checks: residual operators are checked on closed-form solutions of each PDE,
fluxes against the divergence identity of the conservation law, jets against
finite differences and a hand-derived one-neuron network, gradients against
central finite differences of the loss, the loss against its invariants and
special cases (one subdomain, identical neighbours, constant networks), Adam
against its closed form under a constant gradient, and the stitched solution
(Eq. FSol) against constant networks.
"""
import math

import numpy as np
import pytest
import torch

from oracle import Oracle, jets, residual, flux_normal, adam_update, route_rect, network
from paper_2104_10013_gb300 import problems as P
from tests.cases import tiny_problem as _tiny_problem, CASES

DT = torch.float64
NU = 0.01 / math.pi


def _field_jets(fn, z, K):
    """Jets [n, n_out, K] of a closed-form field fn(z) -> [n, n_out], by AD,
    kept differentiable with respect to z (for divergence checks)."""
    u = fn(z)
    comps = [u]
    g = [torch.autograd.grad(u[:, o].sum(), z, create_graph=True)[0] for o in range(u.shape[1])]
    comps.append(torch.stack([gi[:, 0] for gi in g], 1))
    comps.append(torch.stack([gi[:, 1] for gi in g], 1))
    if K > 3:
        comps.append(torch.stack([torch.autograd.grad(gi[:, 0].sum(), z, create_graph=True)[0][:, 0]
                                  for gi in g], 1))
    if K > 4:
        comps.append(torch.stack([torch.autograd.grad(gi[:, 1].sum(), z, create_graph=True)[0][:, 1]
                                  for gi in g], 1))
    return torch.stack(comps, 2)


def _pts(n, lo, hi, seed=0):
    r = np.random.default_rng(seed)
    z = lo + (np.asarray(hi) - np.asarray(lo)) * r.random((n, 2))
    return torch.tensor(z, dtype=DT, requires_grad=True)


# ---------------------------------------------------------------- residuals

def test_burgers_residual_vanishes_on_travelling_wave():
    # u = c - a tanh(a (x - c t) / (2 nu)) solves u_t + u u_x = nu u_xx exactly.
    a, c = 0.7, 0.3
    z = _pts(200, (-1, 0), (1, 1))
    fn = lambda z: (c - a * torch.tanh(a * (z[:, 0] - c * z[:, 1]) / (2 * NU)))[:, None]
    J = _field_jets(fn, z, 4)
    r = residual(P.PDE_BURGERS, [J], torch.zeros(200, dtype=DT), NU, 1.0)
    scale = J.abs().max().item()
    assert r.abs().max().item() < 1e-11 * scale ** 2


def test_burgers_residual_detects_non_solution():
    # the same wave with the wrong speed is not a solution: the operator must see it
    a, c = 0.7, 0.3
    z = _pts(200, (-1, 0), (1, 1))
    fn = lambda z: (c - a * torch.tanh(a * (z[:, 0] - 1.5 * c * z[:, 1]) / (2 * NU)))[:, None]
    J = _field_jets(fn, z, 4)
    r = residual(P.PDE_BURGERS, [J], torch.zeros(200, dtype=DT), NU, 1.0)
    assert r.abs().max().item() > 1e-2


def test_poisson_residual_vanishes_on_manufactured_solution():
    z = _pts(300, (0, 0), (1, 1), seed=1)
    pi = math.pi
    fn = lambda z: (torch.sin(2 * pi * z[:, 0]) * torch.sin(3 * pi * z[:, 1])
                    + 0.1 * torch.sin(20 * pi * z[:, 0] * z[:, 1]))[:, None]
    J = _field_jets(fn, z, 5)
    zz = z.detach().numpy()
    f = torch.tensor(P.poisson_forcing(zz[:, 0], zz[:, 1]), dtype=DT)
    r = residual(P.PDE_POISSON, [J], f, 0.0, 1.0)
    assert r.abs().max().item() < 1e-9 * f.abs().max().item()


def test_navier_stokes_residual_vanishes_on_kovasznay():
    re = 40.0
    lam = re / 2 - math.sqrt(re * re / 4 + 4 * math.pi ** 2)
    z = _pts(300, (-0.5, -0.5), (1.0, 1.5), seed=2)

    def fn(z):
        e = torch.exp(lam * z[:, 0])
        u = 1 - e * torch.cos(2 * math.pi * z[:, 1])
        v = lam / (2 * math.pi) * e * torch.sin(2 * math.pi * z[:, 1])
        p = 0.5 * (1 - torch.exp(2 * lam * z[:, 0]))
        return torch.stack([u, v, p], 1)
    J = _field_jets(fn, z, 5)
    r = residual(P.PDE_NS, [J], torch.zeros(300, dtype=DT), 0.0, re)
    assert r.abs().max().item() < 1e-11
    # and the closed form of the generator is the same field
    zz = z.detach().numpy()
    assert np.allclose(P.kovasznay_exact(zz[:, 0], zz[:, 1], re), fn(z).detach().numpy(), atol=1e-14)
    # a wrong Reynolds number breaks it
    r_bad = residual(P.PDE_NS, [J], torch.zeros(300, dtype=DT), 0.0, 2 * re)
    assert r_bad.abs().max().item() > 1e-2


def test_diffusion_residual_vanishes_on_manufactured_pair():
    z = _pts(300, (-1, -1), (2, 2), seed=3)
    fu = lambda z: (20 * torch.exp(-0.1 * z[:, 1]))[:, None]
    fk = lambda z: (1 + 0.5 * torch.sin(math.pi * z[:, 0]) * torch.cos(math.pi * z[:, 1]))[:, None]
    Ju, Jk = _field_jets(fu, z, 5), _field_jets(fk, z, 3)
    zz = z.detach().numpy()
    f = torch.tensor(P.diffusion_forcing(zz[:, 0], zz[:, 1]), dtype=DT)
    r = residual(P.PDE_DIFFUSION, [Ju, Jk], f, 0.0, 1.0)
    assert r.abs().max().item() < 1e-12
    assert np.allclose(P.diffusion_exact_u(zz[:, 0], zz[:, 1]), fu(z).detach().numpy()[:, 0])
    assert np.allclose(P.diffusion_exact_k(zz[:, 0], zz[:, 1]), fk(z).detach().numpy()[:, 0])


# ---------------------------------------------------------------- fluxes

def _divergence(pde, fn, z, K, Kk=None, nu=0.0, re=1.0, mode=P.FLUX_CONSERVATIVE):
    """div f of the oracle's flux, by AD of f . e_x and f . e_y."""
    J = [_field_jets(fn[0], z, K)] + ([_field_jets(fn[1], z, Kk)] if Kk else [])
    fx = flux_normal(pde, J, (1.0, 0.0), nu, re, mode)
    fy = flux_normal(pde, J, (0.0, 1.0), nu, re, mode)
    div = []
    for c in range(fx.shape[1]):
        gx = torch.autograd.grad(fx[:, c].sum(), z, create_graph=True)[0][:, 0]
        gy = torch.autograd.grad(fy[:, c].sum(), z, create_graph=True)[0][:, 1]
        div.append(gx + gy)
    return torch.stack(div, 1)


def _smooth(seed, n_out):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(n_out, 4, 2, generator=g, dtype=DT)
    B = torch.randn(n_out, 4, generator=g, dtype=DT)
    return lambda z: torch.stack([torch.tanh(z @ A[o].T + B[o]).sum(1) for o in range(n_out)], 1)


def test_flux_divergence_is_the_conservation_law():
    """For a conservation law div f = L(u): the flux of each PDE must have the
    residual (plus the forcing) as its divergence, for any smooth field."""
    z = _pts(100, (-1, -1), (1, 1), seed=4)
    zero = torch.zeros(100, dtype=DT)
    # Burgers in (x, t): d/dx (u^2/2 - nu u_x) + d/dt u = u_t + u u_x - nu u_xx
    fu = _smooth(0, 1)
    div = _divergence(P.PDE_BURGERS, [fu], z, 4, nu=NU)
    r = residual(P.PDE_BURGERS, [_field_jets(fu, z, 4)], zero, NU, 1.0)
    assert torch.allclose(div, r, atol=1e-12)
    # Poisson: div(-grad u) = -lap u
    div = _divergence(P.PDE_POISSON, [fu], z, 5)
    r = residual(P.PDE_POISSON, [_field_jets(fu, z, 5)], zero, 0.0, 1.0)
    assert torch.allclose(div, r, atol=1e-12)
    # diffusion: div(K grad u) = K lap u + grad K . grad u
    fk = _smooth(1, 1)
    div = _divergence(P.PDE_DIFFUSION, [fu, fk], z, 5, Kk=3)
    r = residual(P.PDE_DIFFUSION, [_field_jets(fu, z, 5), _field_jets(fk, z, 3)], zero, 0.0, 1.0)
    assert torch.allclose(div, r, atol=1e-12)
    # Navier-Stokes, Table flux-table: the conservative momentum fluxes differ
    # from the convective form by u * div(u), the mass flux is div(u) itself
    re = 40.0
    fns = _smooth(2, 3)
    J = _field_jets(fns, z, 5)
    div = _divergence(P.PDE_NS, [fns], z, 5, re=re)
    r = residual(P.PDE_NS, [J], zero, 0.0, re)
    u, v = J[:, 0, 0], J[:, 1, 0]
    assert torch.allclose(div[:, 0], r[:, 0] + u * r[:, 2], atol=1e-11)
    assert torch.allclose(div[:, 1], r[:, 1] + v * r[:, 2], atol=1e-11)
    assert torch.allclose(div[:, 2], r[:, 2], atol=1e-12)


# ---------------------------------------------------------------- jets

def test_one_neuron_network_closed_form():
    # u = w2 tanh(w1 . z + b1) + b2: u_i = w2 w1_i (1 - t^2), u_ii = -2 w2 w1_i^2 t (1 - t^2)
    w1 = np.array([[0.7, -1.3]]); b1 = np.array([0.2]); w2 = np.array([[1.9]]); b2 = np.array([-0.4])
    layers = [(torch.tensor(w1), torch.tensor(b1)), (torch.tensor(w2), torch.tensor(b2))]
    z = np.random.default_rng(5).normal(size=(50, 2))
    J = jets(layers, torch.tensor(z), P.ACT_IDENTITY, 5).detach().numpy()[:, 0, :]
    t = np.tanh(z @ w1[0] + b1[0])
    s = 1 - t * t
    ref = np.stack([w2[0, 0] * t + b2[0],
                    w2[0, 0] * w1[0, 0] * s, w2[0, 0] * w1[0, 1] * s,
                    -2 * w2[0, 0] * w1[0, 0] ** 2 * t * s, -2 * w2[0, 0] * w1[0, 1] ** 2 * t * s], 1)
    assert np.allclose(J, ref, rtol=1e-13, atol=1e-13)


def test_one_neuron_softplus_closed_form():
    # y = softplus(a), a = w . z + b: y_i = sig(a) w_i, y_ii = sig(a)(1 - sig(a)) w_i^2
    w = np.array([[0.8, -0.6]]); b = np.array([0.3])
    layers = [(torch.tensor(w), torch.tensor(b))]
    z = np.random.default_rng(6).normal(size=(40, 2)) * 3
    J = jets(layers, torch.tensor(z), P.ACT_SOFTPLUS, 5).detach().numpy()[:, 0, :]
    a = z @ w[0] + b[0]
    sg = 1 / (1 + np.exp(-a))
    ref = np.stack([np.log1p(np.exp(a)), sg * w[0, 0], sg * w[0, 1],
                    sg * (1 - sg) * w[0, 0] ** 2, sg * (1 - sg) * w[0, 1] ** 2], 1)
    assert np.allclose(J, ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("out_act", [P.ACT_IDENTITY, P.ACT_SOFTPLUS])
def test_jets_match_central_differences(out_act):
    net = P.NetSpec([2, 7, 6, 5, 2], out_act)
    layers = [(torch.tensor(W, dtype=DT) * 1.5, torch.tensor(np.random.default_rng(k).normal(size=b.shape)))
              for k, (W, b) in enumerate(P.xavier_params(net, np.random.default_rng(7)))]
    z = np.random.default_rng(8).uniform(-1, 1, size=(30, 2))
    J = jets(layers, torch.tensor(z), out_act, 5).detach().numpy()
    f = lambda zz: network(layers, torch.tensor(zz), out_act).detach().numpy()
    u0 = f(z)
    assert np.allclose(J[:, :, 0], u0, atol=1e-15)
    for i in range(2):
        e = np.zeros(2); e[i] = 1.0
        h1, h2 = 1e-5, 1e-3
        d1 = (f(z + h1 * e) - f(z - h1 * e)) / (2 * h1)
        d2 = (f(z + h2 * e) - 2 * u0 + f(z - h2 * e)) / (h2 * h2)
        assert np.allclose(J[:, :, 1 + i], d1, atol=1e-8)
        assert np.allclose(J[:, :, 3 + i], d2, atol=2e-6)


# ---------------------------------------------------------------- losses


@pytest.mark.parametrize("pde,method", CASES)
def test_gradient_matches_central_differences(pde, method):
    """dJ(Theta_q)/dTheta_q with neighbours held constant, against central FD
    of J_q alone (the neighbours' values do not depend on Theta_q)."""
    _check_gradient_by_central_differences(_tiny_problem(pde, method))


def test_gradient_matches_central_differences_literal_burgers_flux():
    """The same check with the literal Burgers flux u u_x - nu u_x on the
    cPINN interfaces (the form the Burgers cPINN configuration names)."""
    pb = _tiny_problem(P.PDE_BURGERS, P.CPINN)
    pb.flux_mode = P.FLUX_LITERAL
    _check_gradient_by_central_differences(pb)


def _check_gradient_by_central_differences(pb):
    orc = Oracle(pb)
    theta = pb.packed_params().astype(np.float64)
    W = orc.weights()
    _, g = orc.grad(theta)
    owner = np.concatenate([np.full(s.n_params, q) for q, s in enumerate(pb.subs)])
    rng = np.random.default_rng(0)
    idx = rng.choice(theta.size, size=min(40, theta.size), replace=False)
    h = 1e-6
    for i in idx:
        q = owner[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h; tm[i] -= h
        with torch.no_grad():
            pass
        Jp = (orc.loss_terms(torch.tensor(tp)).detach().numpy()[q] * W[q]).sum()
        Jm = (orc.loss_terms(torch.tensor(tm)).detach().numpy()[q] * W[q]).sum()
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


@pytest.mark.parametrize("pde", [P.PDE_BURGERS, P.PDE_POISSON, P.PDE_NS, P.PDE_DIFFUSION])
def test_single_subdomain_is_vanilla_pinn(pde):
    """N_sd = 1: no interface terms remain (Eq. p-loss), the MSEs are means
    (invariant when every point is duplicated), and for the zero network the
    data term is mean |g|^2 and, for Poisson, the residual term is mean f^2."""
    pb = _tiny_problem(pde, P.XPINN, n_sub=1)
    orc = Oracle(pb)
    theta = pb.packed_params().astype(np.float64)
    t1 = orc.loss_terms(torch.tensor(theta)).detach().numpy()[0]
    assert t1[3] == 0.0 and t1[4] == 0.0
    s = pb.subs[0]
    s.res_xy = np.concatenate([s.res_xy, s.res_xy]); s.res_f = np.concatenate([s.res_f, s.res_f])
    s.data = [P.DataSet(np.concatenate([d.xy, d.xy]), np.concatenate([d.val, d.val])) for d in s.data]
    t2 = Oracle(pb).loss_terms(torch.tensor(theta)).detach().numpy()[0]
    assert np.allclose(t1, t2, rtol=1e-13)
    zero = np.zeros_like(theta)
    if pde == P.PDE_DIFFUSION:
        return  # softplus(0) != 0
    t0 = Oracle(pb).loss_terms(torch.tensor(zero)).detach().numpy()[0]
    assert np.isclose(t0[0], (s.data[0].val.astype(np.float64) ** 2).sum(1).mean(), rtol=1e-13)
    if pde == P.PDE_POISSON:
        assert np.isclose(t0[2], (s.res_f.astype(np.float64) ** 2).mean(), rtol=1e-13)


@pytest.mark.parametrize("pde,method", CASES)
def test_identical_neighbours_give_zero_interface_terms(pde, method):
    pb = _tiny_problem(pde, method, n_sub=3)
    for s in pb.subs[1:]:
        s.params = pb.subs[0].params
    orc = Oracle(pb)
    theta = pb.packed_params().astype(np.float64)
    terms, g = orc.grad(theta)
    assert np.abs(terms[:, 3:]).max() < 1e-24
    for s in pb.subs:
        s.w_avg = 0.0; s.w_iface = 0.0
    _, g0 = Oracle(pb).grad(theta)
    assert np.allclose(g, g0, rtol=0, atol=1e-13)


def test_constant_networks_interface_terms_closed_form():
    """u_q = b, u_q+ = c everywhere: MSE_uavg = ((b - c) / 2)^2 (the average
    {{u}} includes u_q) and, for the Burgers flux u^2/2 - nu u_x across x-cuts,
    MSE_flux = (b^2/2 - c^2/2)^2; q's two interfaces add up."""
    pb = _tiny_problem(P.PDE_BURGERS, P.CPINN, n_sub=3)
    consts = [0.4, -1.1, 2.0]
    for s, c in zip(pb.subs, consts):
        s.params = [[(np.zeros_like(W), np.zeros_like(b)) for W, b in s.params[0]]]
        s.params[0][-1] = (s.params[0][-1][0], np.full_like(s.params[0][-1][1], c))
    terms = Oracle(pb).loss_terms(torch.tensor(pb.packed_params().astype(np.float64))).detach().numpy()
    c = [np.float64(np.float32(x)) for x in consts]
    avg = lambda a, b: ((a - b) / 2) ** 2
    flux = lambda a, b: (a * a / 2 - b * b / 2) ** 2
    assert np.isclose(terms[0, 3], avg(c[0], c[1]), rtol=1e-13)
    assert np.isclose(terms[1, 3], avg(c[1], c[0]) + avg(c[1], c[2]), rtol=1e-13)
    assert np.isclose(terms[1, 4], flux(c[1], c[0]) + flux(c[1], c[2]), rtol=1e-13)
    assert np.isclose(terms[2, 4], flux(c[2], c[1]), rtol=1e-13)


def test_literal_burgers_flux_closed_form_on_one_neuron_networks():
    """Literal cPINN flux of the Burgers configuration, f = (u u_x - nu u_x, u)
    in (x, t), on one-neuron networks u = w2 tanh(a x + c t + b1) + b2 whose
    u_x = w2 a (1 - tanh^2) is written out by hand: MSE_flux of each side is
    the mean over the interface points of (f_q . n - f_q+ . n)^2, with a
    normal that has both components so that both parts of f are exercised.
    A dropped u u_x or nu u_x term, a wrong sign, or the conservative u^2/2
    in its place fails it."""
    pb = _tiny_problem(P.PDE_BURGERS, P.CPINN, n_sub=2, widths=[2, 1, 1])
    pb.flux_mode = P.FLUX_LITERAL
    normal = (0.6, 0.8)
    pb.ifaces[0].normal = normal
    prm = [(0.7, -0.4, 0.2, 1.3, -0.5), (-1.1, 0.9, -0.3, 0.6, 0.25)]   # a, c, b1, w2, b2
    for s, (a, c, b1, w2, b2) in zip(pb.subs, prm):
        s.params = [[(np.array([[a, c]], np.float32), np.array([b1], np.float32)),
                     (np.array([[w2]], np.float32), np.array([b2], np.float32))]]
    terms = Oracle(pb).loss_terms(torch.tensor(pb.packed_params().astype(np.float64))).detach().numpy()
    nu = np.float64(np.float32(pb.nu))
    n0, n1 = (np.float64(np.float32(v)) for v in normal)
    xy = pb.ifaces[0].xy.astype(np.float64)

    def f_dot_n(a, c, b1, w2, b2):
        a, c, b1, w2, b2 = (np.float64(np.float32(v)) for v in (a, c, b1, w2, b2))
        t = np.tanh(a * xy[:, 0] + c * xy[:, 1] + b1)
        u = w2 * t + b2
        ux = w2 * a * (1 - t * t)
        return n0 * (u * ux - nu * ux) + n1 * u

    f0, f1 = f_dot_n(*prm[0]), f_dot_n(*prm[1])
    want = np.mean((f0 - f1) ** 2)
    assert np.isclose(terms[0, 4], want, rtol=1e-12, atol=0)
    assert np.isclose(terms[1, 4], want, rtol=1e-12, atol=0)
    # the conservative form differs on the same networks
    pb.flux_mode = P.FLUX_CONSERVATIVE
    t2 = Oracle(pb).loss_terms(torch.tensor(pb.packed_params().astype(np.float64))).detach().numpy()
    assert not np.isclose(t2[0, 4], want, rtol=1e-3)


# ---------------------------------------------------------------- Adam

def test_adam_first_step_and_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every step, so every step moves theta by -lr g / (|g| + eps)."""
    g = np.array([1e-3, -2.0, 5e-9, 0.0, 7.5])
    lr, eps = np.array([1e-3, 1e-3, 2e-3, 1e-3, 5e-4]), 1e-8
    th, m, v = np.ones(5), np.zeros(5), np.zeros(5)
    for t in range(1, 6):
        th_new, m, v = adam_update(th, g, m, v, t, lr, 0.9, 0.999, eps)
        assert np.allclose(th_new - th, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-18)
        th = th_new


# ---------------------------------------------------------------- stitching

def test_stitched_solution_averages_on_interfaces():
    """Eq. FSol: inside Omega_q the value of net q, on an interface shared by
    S subdomains the mean of their S values, outside every subdomain NaN."""
    pb = P.poisson_xpinn(nx=2, ny=2, n_res_range=(5, 5), depth_range=(1, 1), width_range=(2, 2),
                         n_iface=2, n_bc=2)
    consts = [1.0, 2.0, 4.0, 8.0]
    for s, c in zip(pb.subs, consts):
        s.params = [[(np.zeros_like(W), np.full_like(b, c if k == len(s.params[0]) - 1 else 0.0))
                     for k, (W, b) in enumerate(s.params[0])]]
    xc, yc = pb.meta["xcuts"], pb.meta["ycuts"]
    xs = [0.5 * (xc[0] + xc[1]), xc[1], 0.5 * (xc[1] + xc[2])]
    ys = [0.5 * (yc[0] + yc[1]), yc[1], 0.5 * (yc[1] + yc[2])]
    pts = np.array([[x, y] for y in ys for x in xs] + [[2.0, 0.5]])
    out = Oracle(pb).eval_stitched(pb.packed_params(), 0, pts, 1)[:, 0, 0]
    want = [1, 1.5, 2, 2.5, 3.75, 5, 4, 6, 8, np.nan]
    assert np.allclose(out, want, equal_nan=True)
    memb = route_rect([s.rect for s in pb.subs], pts)
    assert [len(m) for m in memb] == [1, 2, 1, 2, 4, 2, 1, 2, 1, 0]


def test_voronoi_routing_polygon_membership_by_hand():
    """The even-odd rule on an L-shaped (non-convex) polygon with one site:
    points inside the L route to the site, points in the notch or outside the
    bounding box route nowhere (membership read off the drawing)."""
    from oracle import route_voronoi
    L = [(0, 0), (2, 0), (2, 1), (1, 1), (1, 2), (0, 2)]
    pts = np.array([[0.5, 0.5], [1.5, 0.5], [0.5, 1.5], [1.5, 1.5], [2.5, 0.5], [-0.1, 1.0], [0.5, 2.1]],
                   np.float32)
    got = route_voronoi([(0.5, 0.5)], L, pts)
    assert got == [[0], [0], [0], [], [], [], []]


def test_voronoi_routing_on_symmetric_sites():
    """Sites at (-1, 0), (1, 0), (0, 2) in a square: a point on the y axis
    below the third site's cell is equidistant (exactly, in float32) from the
    first two and shared by both; points near a site belong to it; points
    outside the polygon belong to none."""
    from oracle import route_voronoi
    sites = [(-1.0, 0.0), (1.0, 0.0), (0.0, 2.0)]
    square = [(-3, -3), (3, -3), (3, 3), (-3, 3)]
    pts = [(0.0, -0.5), (-0.9, 0.1), (1.2, -0.3), (0.1, 2.2), (4.0, 0.0), (0.0, 0.25)]
    memb = route_voronoi(sites, square, pts)
    assert memb == [[0, 1], [0], [1], [2], [], [0, 1]]


@pytest.mark.parametrize("act", [P.PHI_TANH, P.PHI_SIN, P.PHI_COS])
def test_one_neuron_with_slope_closed_form(act):
    # u = w2 phi(s (w1 . z + b1)) + b2: u_i = w2 s w1_i phi', u_ii = w2 s^2 w1_i^2 phi''
    w1 = np.array([[0.7, -1.3]]); b1 = np.array([0.2]); w2 = np.array([[1.9]]); b2 = np.array([-0.4])
    n, a = 10.0, 0.137
    s = n * a
    layers = [(torch.tensor(w1), torch.tensor(b1)), (torch.tensor(w2), torch.tensor(b2))]
    z = np.random.default_rng(9).normal(size=(40, 2))
    J = jets(layers, torch.tensor(z), P.ACT_IDENTITY, 5, act, torch.tensor([a], dtype=torch.float64), n).detach().numpy()[:, 0, :]
    v = s * (z @ w1[0] + b1[0])
    f, d1, d2 = {P.PHI_TANH: (np.tanh(v), 1 - np.tanh(v) ** 2, -2 * np.tanh(v) * (1 - np.tanh(v) ** 2)),
                 P.PHI_SIN: (np.sin(v), np.cos(v), -np.sin(v)),
                 P.PHI_COS: (np.cos(v), -np.sin(v), -np.cos(v))}[act]
    ref = np.stack([w2[0, 0] * f + b2[0],
                    w2[0, 0] * s * w1[0, 0] * d1, w2[0, 0] * s * w1[0, 1] * d1,
                    w2[0, 0] * s * s * w1[0, 0] ** 2 * d2, w2[0, 0] * s * s * w1[0, 1] ** 2 * d2], 1)
    assert np.allclose(J, ref, rtol=1e-12, atol=1e-12)


def test_initial_slopes_give_the_fixed_network():
    """n a^k = 1 at initialisation (Sec. 3): an adaptive network with its
    initial slopes computes exactly what the fixed-slope network does."""
    pb = _tiny_problem(P.PDE_NS, P.CPINN, n_sub=2)
    pa = _tiny_problem(P.PDE_NS, P.CPINN, n_sub=2, adaptive=True)
    for s in pa.subs:
        s.slopes = []                        # initial slopes 1/n
    for sa, sb in zip(pa.subs, pb.subs):
        sa.params = sb.params
    ta = Oracle(pa).loss_terms(torch.tensor(pa.packed_params().astype(np.float64))).detach().numpy()
    tb = Oracle(pb).loss_terms(torch.tensor(pb.packed_params().astype(np.float64))).detach().numpy()
    assert np.allclose(ta, tb, rtol=1e-6)     # 1/n is rounded to float32 in the packed vector


@pytest.mark.parametrize("pde,method,act", [(P.PDE_BURGERS, P.CPINN, P.PHI_TANH),
                                            (P.PDE_POISSON, P.XPINN, P.PHI_SIN),
                                            (P.PDE_DIFFUSION, P.XPINN, P.PHI_COS)])
def test_gradient_with_slopes_matches_central_differences(pde, method, act):
    pb = _tiny_problem(pde, method, act=act, adaptive=True)
    orc = Oracle(pb)
    theta = pb.packed_params().astype(np.float64)
    W = orc.weights()
    _, g = orc.grad(theta)
    owner = np.concatenate([np.full(s.n_params, q) for q, s in enumerate(pb.subs)])
    # every slope, plus some weights
    slope_idx, off = [], 0
    for s in pb.subs:
        for net in s.nets:
            off += net.n_params
            slope_idx += list(range(off - net.n_slopes, off))
    idx = slope_idx + list(np.random.default_rng(1).choice(theta.size, 10, replace=False))
    h = 1e-6
    for i in idx:
        q = owner[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h; tm[i] -= h
        Jp = (orc.loss_terms(torch.tensor(tp)).detach().numpy()[q] * W[q]).sum()
        Jm = (orc.loss_terms(torch.tensor(tm)).detach().numpy()[q] * W[q]).sum()
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def _taylor_forward(layers, z, out_act, act, slopes, scale):
    """Second-order forward-mode (truncated Taylor) arithmetic written out
    here: every quantity carries (value, d/dz0, d/dz1, d2/dz0^2, d2/dz1^2)
    and each operation applies its chain rule.  Independent of the oracle,
    which takes its derivatives by reverse-mode autograd."""
    def lin(W, b, H):            # H: [n_in, 5, npts] -> [n_out, 5, npts]
        out = np.einsum("oi,icp->ocp", W, H)
        out[:, 0, :] += b[:, None]
        return out

    def unary(f, f1, f2, Z):     # elementwise phi with its first two derivatives
        v, d0, d1, dd0, dd1 = Z[:, 0], Z[:, 1], Z[:, 2], Z[:, 3], Z[:, 4]
        return np.stack([f(v), f1(v) * d0, f1(v) * d1, f1(v) * dd0 + f2(v) * d0 ** 2,
                         f1(v) * dd1 + f2(v) * d1 ** 2], 1)

    phis = {P.PHI_TANH: (np.tanh, lambda v: 1 - np.tanh(v) ** 2,
                         lambda v: -2 * np.tanh(v) * (1 - np.tanh(v) ** 2)),
            P.PHI_SIN: (np.sin, np.cos, lambda v: -np.sin(v)),
            P.PHI_COS: (np.cos, lambda v: -np.sin(v), lambda v: -np.cos(v))}
    npts = z.shape[0]
    H = np.zeros((2, 5, npts))
    H[:, 0, :] = z.T
    H[0, 1, :] = 1.0
    H[1, 2, :] = 1.0
    for k, (W, b) in enumerate(layers):
        if k > 0:
            s = 1.0 if slopes is None else scale * slopes[k - 1]
            f, f1, f2 = phis[act]
            H = unary(lambda v: f(s * v), lambda v: s * f1(s * v), lambda v: s * s * f2(s * v), H)
        H = lin(W, b, H)
    if out_act == P.ACT_SOFTPLUS:
        sig = lambda v: 1 / (1 + np.exp(-v))
        H = unary(lambda v: np.log1p(np.exp(v)), sig, lambda v: sig(v) * (1 - sig(v)), H)
    return np.transpose(H, (2, 0, 1))       # [npts, n_out, 5]


@pytest.mark.parametrize("act,adaptive,out_act", [(P.PHI_TANH, False, P.ACT_IDENTITY),
                                                  (P.PHI_SIN, True, P.ACT_IDENTITY),
                                                  (P.PHI_COS, True, P.ACT_SOFTPLUS)])
def test_jets_match_forward_mode_taylor_arithmetic(act, adaptive, out_act):
    rng = np.random.default_rng(11)
    net = P.NetSpec([2, 6, 5, 4, 2], out_act, act=act, adaptive=adaptive)
    layers = [(rng.normal(size=(net.widths[k], net.widths[k - 1])) * 0.8, rng.normal(size=net.widths[k]) * 0.3)
              for k in range(1, len(net.widths))]
    slopes = rng.uniform(0.08, 0.15, size=net.n_slopes) if adaptive else None
    z = rng.normal(size=(25, 2))
    ref = _taylor_forward(layers, z, out_act, act, slopes, 10.0)
    got = jets([(torch.tensor(W), torch.tensor(b)) for W, b in layers], torch.tensor(z), out_act, 5, act,
               None if slopes is None else torch.tensor(slopes), 10.0).detach().numpy()
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-10)
