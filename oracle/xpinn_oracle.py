"""FP64 CPU oracle: cPINN / XPINN losses, gradients, Adam and stitched eval.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Jet component order used throughout (K = number of components kept):
    0: u,  1: d u / d z0,  2: d u / d z1,  3: d2 u / d z0^2,  4: d2 u / d z1^2
where z = (x, y) for steady problems and z = (x, t) for Burgers.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_2104_10013_gb300 import problems as P

DT = torch.float64


def _t(a) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=DT)


def _r32(x) -> float:
    """A scalar as the float32 value the problem description carries."""
    return float(np.float32(x))


# --------------------------------------------------------------------------
# Network (Sec. 3)
# --------------------------------------------------------------------------

def softplus(z: torch.Tensor) -> torch.Tensor:
    """log(1 + e^z), written in a form without overflow for large z."""
    return torch.clamp(z, min=0.0) + torch.log1p(torch.exp(-torch.abs(z)))


def phi(act: int, v: torch.Tensor) -> torch.Tensor:
    """Hidden activation Phi: tanh, sin or cos (Table Table_USmap)."""
    if act == P.PHI_SIN:
        return torch.sin(v)
    if act == P.PHI_COS:
        return torch.cos(v)
    return torch.tanh(v)


def network(layers, z: torch.Tensor, out_act: int, act: int = P.PHI_TANH, slopes=None,
            scale: float = 1.0) -> torch.Tensor:
    """N^1 = W^1 z + b^1, N^k = W^k Phi(n a^{k-1} N^{k-1}) + b^k (2 <= k <= L),
    Sec. 3: with `slopes` the layer-wise slopes a^1..a^{L-1} and scale n,
    otherwise n a^k fixed at its initial value 1.  The last layer is the
    identity, or a softplus for a strictly positive field."""
    h = z
    for k, (W, b) in enumerate(layers):
        if k > 0:
            s = 1.0 if slopes is None else scale * slopes[k - 1]
            h = phi(act, s * h)
        h = h @ W.T + b
    if out_act == P.ACT_SOFTPLUS:
        h = softplus(h)
    return h


def _grad(y: torch.Tensor, z: torch.Tensor) -> torch.Tensor:
    g = torch.autograd.grad(y.sum(), z, create_graph=True, allow_unused=True)[0]
    return torch.zeros_like(z) if g is None else g


def jets(layers, z: torch.Tensor, out_act: int, K: int, act: int = P.PHI_TANH, slopes=None,
         scale: float = 1.0) -> torch.Tensor:
    """Network output and its input derivatives at every point, by reverse-mode
    AD (Sec. 4.1): returns [n, D_out, K] in the component order above.  The
    result stays differentiable with respect to the weights and slopes."""
    z = z.detach().clone().requires_grad_(True)
    u = network(layers, z, out_act, act, slopes, scale)
    comps = [u]
    if K > 1:
        g = [_grad(u[:, o], z) for o in range(u.shape[1])]
        comps.append(torch.stack([gi[:, 0] for gi in g], 1))
        if K > 2:
            comps.append(torch.stack([gi[:, 1] for gi in g], 1))
        if K > 3:
            comps.append(torch.stack([_grad(gi[:, 0], z)[:, 0] for gi in g], 1))
        if K > 4:
            comps.append(torch.stack([_grad(gi[:, 1], z)[:, 1] for gi in g], 1))
    return torch.stack(comps, dim=2)


# --------------------------------------------------------------------------
# PDE residuals and interface fluxes (Sec. 2, Sec. 7)
# --------------------------------------------------------------------------

# jet components needed at residual points, per PDE and per net
K_RES = {P.PDE_BURGERS: (4,), P.PDE_POISSON: (5,), P.PDE_NS: (5,), P.PDE_DIFFUSION: (5, 3)}


def K_IFACE(pde: int, method: int) -> tuple:
    """Jet components needed at interface points: first derivatives for the
    cPINN flux, the residual's components for XPINN residual continuity."""
    if method == P.XPINN:
        return K_RES[pde]
    if pde == P.PDE_BURGERS:
        return (2,)
    return (3, 3) if pde == P.PDE_DIFFUSION else (3,)


def n_eq(pde: int) -> int:
    return 3 if pde == P.PDE_NS else 1


def n_out_total(problem) -> int:
    return sum(n.widths[-1] for n in problem.subs[0].nets)


def residual(pde: int, J: list, f: torch.Tensor, nu: float, re: float) -> torch.Tensor:
    """F(u) = L_x(u) - f (Sec. 2) from the jets J (one [n, D_out, K] tensor per
    net); returns [n, n_eq].
      Burgers (Eq. BE, z = (x, t)):   u_t + u u_x - nu u_xx
      Poisson:                        -(u_xx + u_yy) - f
      Navier-Stokes (Eq. NSEq):       u.grad u + grad p - lap u / Re, div u
                                      (no forcing term; f is ignored)
      inverse diffusion (Eq. heq):    K lap u + grad K . grad u - f
    """
    Ju = J[0]
    if pde == P.PDE_BURGERS:
        u, ux, ut, uxx = Ju[:, 0, 0], Ju[:, 0, 1], Ju[:, 0, 2], Ju[:, 0, 3]
        return (ut + u * ux - nu * uxx - f)[:, None]
    if pde == P.PDE_POISSON:
        return (-(Ju[:, 0, 3] + Ju[:, 0, 4]) - f)[:, None]
    if pde == P.PDE_NS:
        u, v, p = Ju[:, 0], Ju[:, 1], Ju[:, 2]
        r1 = u[:, 0] * u[:, 1] + v[:, 0] * u[:, 2] + p[:, 1] - (u[:, 3] + u[:, 4]) / re
        r2 = u[:, 0] * v[:, 1] + v[:, 0] * v[:, 2] + p[:, 2] - (v[:, 3] + v[:, 4]) / re
        r3 = u[:, 1] + v[:, 2]
        return torch.stack([r1, r2, r3], 1)
    if pde == P.PDE_DIFFUSION:
        Jk = J[1]
        u, k = Ju[:, 0], Jk[:, 0]
        r = k[:, 0] * (u[:, 3] + u[:, 4]) + k[:, 1] * u[:, 1] + k[:, 2] * u[:, 2] - f
        return r[:, None]
    raise ValueError(pde)


def flux_normal(pde: int, J: list, normal, nu: float, re: float, flux_mode: int) -> torch.Tensor:
    """Normal flux f . n at interface points (cPINN, Eq. cPINNLoss), one
    column per conservation law; returns [n, n_eq].
      Burgers, conservative form u_t + (u^2/2 - nu u_x)_x = 0 in (x, t):
          f = (u^2/2 - nu u_x, u); the literal mode uses u u_x - nu u_x.
      Poisson -div(grad u) = f:   f = -grad u.
      Navier-Stokes: Table flux-table (x-momentum, y-momentum, mass).
      Diffusion div(K grad u) = f: f = K grad u.
    """
    n0, n1 = float(normal[0]), float(normal[1])
    Ju = J[0]
    if pde == P.PDE_BURGERS:
        u, ux = Ju[:, 0, 0], Ju[:, 0, 1]
        fx = u * u / 2 - nu * ux if flux_mode == P.FLUX_CONSERVATIVE else u * ux - nu * ux
        return (n0 * fx + n1 * u)[:, None]
    if pde == P.PDE_POISSON:
        return (-(n0 * Ju[:, 0, 1] + n1 * Ju[:, 0, 2]))[:, None]
    if pde == P.PDE_NS:
        u, v, p = Ju[:, 0], Ju[:, 1], Ju[:, 2]
        fxm = (u[:, 0] ** 2 + p[:, 0] - u[:, 1] / re, u[:, 0] * v[:, 0] - u[:, 2] / re)
        fym = (u[:, 0] * v[:, 0] - v[:, 1] / re, v[:, 0] ** 2 + p[:, 0] - v[:, 2] / re)
        fma = (u[:, 0], v[:, 0])
        return torch.stack([n0 * a + n1 * b for a, b in (fxm, fym, fma)], 1)
    if pde == P.PDE_DIFFUSION:
        k = J[1][:, 0, 0]
        return (k * (n0 * Ju[:, 0, 1] + n1 * Ju[:, 0, 2]))[:, None]
    raise ValueError(pde)


# --------------------------------------------------------------------------
# Adam (Sec. 6) and routing (Eq. FSol)
# --------------------------------------------------------------------------

def adam_update(theta, g, m, v, t: int, lr, b1: float, b2: float, eps: float):
    """One bias-corrected Adam step (Kingma & Ba), per subdomain learning rate
    `lr` (scalar or per-parameter array).  Returns (theta, m, v)."""
    theta, g, m, v, lr = (np.asarray(a, dtype=np.float64) for a in (theta, g, m, v, lr))
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def route_rect(rects, xy) -> list:
    """For each point, the subdomains whose closed rectangle contains it; a
    point on a common interface of S subdomains belongs to all S of them."""
    xy = np.asarray(xy, dtype=np.float64)
    out = []
    for x, y in xy:
        out.append([q for q, (x0, x1, y0, y1) in enumerate(rects)
                    if x0 <= x <= x1 and y0 <= y <= y1])
    return out


def route_voronoi(sites, polygon, xy) -> list:
    """Irregular regions (Sec. 7.6): a point inside the polygon (even-odd
    rule) belongs to the Voronoi cell of its nearest site; the sites at exactly
    the same float32 distance ((dx*dx) + (dy*dy), each operation rounded to
    float32) share it.  Points outside the polygon belong to no region.  The
    even-odd test decides in float32 too, with the crossing abscissa of an
    edge rounded as ax + ((y - ay) * (bx - ax)) / (by - ay), operation by
    operation: points on or within rounding of an edge are an integer decision
    taken in the precision of the data, the same on every implementation."""
    f32 = np.float32
    poly = np.asarray(polygon, dtype=np.float32)
    xy = np.asarray(xy)
    out = []
    s32 = np.asarray(sites, dtype=np.float32)
    for z in xy:
        x, y = f32(z[0]), f32(z[1])
        inside = False
        for e in range(len(poly)):
            (ax, ay), (bx, by) = poly[e], poly[(e + 1) % len(poly)]
            if (ay > y) != (by > y):
                t = f32(f32(y - ay) * f32(bx - ax))
                xc = f32(ax + f32(t / f32(by - ay)))
                if x < xc:
                    inside = not inside
        if not inside:
            out.append([])
            continue
        z32 = np.asarray(z, dtype=np.float32)
        dx = z32[0] - s32[:, 0]
        dy = z32[1] - s32[:, 1]
        d = (dx * dx) + (dy * dy)          # float32 arithmetic, no fused multiply-add
        out.append([int(q) for q in np.nonzero(d == d.min())[0]])
    return out


# --------------------------------------------------------------------------
# The training step (Algorithm 1)
# --------------------------------------------------------------------------

class Oracle:
    """Loss terms, gradients and Adam steps of a cPINN/XPINN problem."""

    def __init__(self, problem: P.Problem):
        self.pb = problem
        self.offsets = []
        off = 0
        for s in problem.subs:
            self.offsets.append(off)
            off += s.n_params
        self.n_params = off
        # scalars exactly as the float32 problem description carries them
        self.nu, self.re = _r32(problem.nu), _r32(problem.re)
        self.beta1, self.beta2, self.eps = _r32(problem.beta1), _r32(problem.beta2), _r32(problem.eps)

    # -- parameters --------------------------------------------------------
    def _layers(self, flat: torch.Tensor, q: int) -> list:
        """Views of the packed parameter vector: per net, [(W^k, b^k), ...]."""
        return [layers for layers, _ in self._nets(flat, q)]

    def _nets(self, flat: torch.Tensor, q: int) -> list:
        """Per net: ([(W^k, b^k), ...], slopes a^1..a^{L-1} or None)."""
        off = self.offsets[q]
        nets = []
        for net in self.pb.subs[q].nets:
            layers = []
            for k in range(1, len(net.widths)):
                no, ni = net.widths[k], net.widths[k - 1]
                W = flat[off:off + no * ni].view(no, ni); off += no * ni
                b = flat[off:off + no]; off += no
                layers.append((W, b))
            a = None
            if net.adaptive:
                a = flat[off:off + net.n_slopes]; off += net.n_slopes
            nets.append((layers, a))
        return nets

    def _net_fn(self, flat, q, n):
        """The network n of subdomain q as a function of the points."""
        net = self.pb.subs[q].nets[n]
        layers, a = self._nets(flat, q)[n]
        scale = _r32(net.slope_scale)
        return layers, a, scale, net

    def _jets(self, flat, q, xy, Ks) -> list:
        s = self.pb.subs[q]
        z = _t(xy)
        out = []
        for n, K in enumerate(Ks):
            layers, a, scale, net = self._net_fn(flat, q, n)
            out.append(jets(layers, z, net.out_act, K, net.act, a, scale))
        return out

    def net_jets(self, flat, q: int, net: int, xy, K: int) -> np.ndarray:
        """Jets [n, D_out, K] of network `net` of subdomain q at points xy."""
        layers, a, scale, nd = self._net_fn(_t(flat), q, net)
        return jets(layers, _t(xy), nd.out_act, K, nd.act, a, scale).detach().numpy()

    # -- interface quantities (Algorithm 1, computation stage) -------------
    def iface_quantities(self, flat, e: int, side: int):
        """Side `side` (0: q, 1: q+) of interface e: the solution vector u
        (all outputs of all nets) and the exchanged quantity, the normal flux
        f . n (cPINN) or the residual F (XPINN), at the interface points."""
        pb = self.pb
        it = pb.ifaces[e]
        q = it.q if side == 0 else it.qp
        J = self._jets(flat, q, it.xy, K_IFACE(pb.pde, it.method))
        uvec = torch.cat([j[:, :, 0] for j in J], 1)
        if it.method == P.CPINN:
            normal = (_r32(it.normal[0]), _r32(it.normal[1]))
            qty = flux_normal(pb.pde, J, normal, self.nu, self.re, pb.flux_mode)
        else:
            # the forcing is the same on both sides of a common point, so it
            # cancels in F_q - F_q+; it is left out of the exchanged residual
            zero_f = torch.zeros(it.xy.shape[0], dtype=DT)
            qty = residual(pb.pde, J, zero_f, self.nu, self.re)
        return uvec, qty

    # -- loss (Eqs. cPINNLoss / XPINNLoss) ---------------------------------
    def loss_terms(self, flat: torch.Tensor, subset=None) -> torch.Tensor:
        """[n_sub, 5] tensor of MSE terms (data net 0, data net 1, residual,
        average solution, flux or residual continuity), differentiable with
        respect to `flat` through each subdomain's own parameters only.
        With `subset`, only the rows of those subdomains (in that order)."""
        pb = self.pb
        qs = list(range(pb.n_sub)) if subset is None else list(subset)
        rows = []
        # values exchanged across every interface, held constant (stop-gradient)
        recv = {}
        for e, it in enumerate(pb.ifaces):
            if it.q not in qs and it.qp not in qs:
                continue
            for side in (0, 1):
                u, qty = self.iface_quantities(flat, e, side)
                recv[(e, side)] = (u.detach(), qty.detach())
        for q in qs:
            s = pb.subs[q]
            terms = [torch.zeros((), dtype=DT) for _ in range(P.N_TERMS)]
            # data mismatch MSE_u per net
            for ni, ds in enumerate(s.data):
                if ds is None or ds.xy.shape[0] == 0:
                    continue
                layers, a, scale, nd = self._net_fn(flat, q, ni)
                u = network(layers, _t(ds.xy), nd.out_act, nd.act, a, scale)
                terms[ni] = ((u - _t(ds.val)) ** 2).sum(1).mean()
            # residual MSE_F
            if s.res_xy.shape[0] > 0:
                J = self._jets(flat, q, s.res_xy, K_RES[pb.pde])
                r = residual(pb.pde, J, _t(s.res_f), self.nu, self.re)
                terms[2] = (r ** 2).sum(1).mean()
            # interface terms: sum over neighbours of per-interface means
            for e, it in enumerate(pb.ifaces):
                if q not in (it.q, it.qp):
                    continue
                side = 0 if it.q == q else 1
                u, qty = self.iface_quantities(flat, e, side)
                u_o, qty_o = recv[(e, 1 - side)]
                uavg = (u + u_o) / 2
                terms[3] = terms[3] + ((u - uavg) ** 2).sum(1).mean()
                terms[4] = terms[4] + ((qty - qty_o) ** 2).sum(1).mean()
            rows.append(torch.stack(terms))
        return torch.stack(rows)

    def weights(self) -> np.ndarray:
        """[n_sub, 5] loss weights W_u(net 0), W_u(net 1), W_F, W_I, W_flux|W_IF."""
        W = np.zeros((self.pb.n_sub, P.N_TERMS))
        for q, s in enumerate(self.pb.subs):
            for ni, w in enumerate(s.w_data):
                W[q, ni] = w
            W[q, 2:] = (s.w_res, s.w_avg, s.w_iface)
        return W.astype(np.float32).astype(np.float64)

    def grad(self, flat_np, subset=None):
        """Loss terms [n_sub, 5] and the packed gradient of every J(Theta_q)
        with respect to its own Theta_q (with `subset`: those subdomains'
        rows, and a gradient that is zero elsewhere)."""
        flat = _t(flat_np).requires_grad_(True)
        terms = self.loss_terms(flat, subset)
        W = self.weights() if subset is None else self.weights()[list(subset)]
        J = (terms * _t(W)).sum()
        (g,) = torch.autograd.grad(J, flat, allow_unused=True)
        g = torch.zeros_like(flat) if g is None else g
        return terms.detach().numpy(), g.detach().numpy()

    def lr_vector(self) -> np.ndarray:
        return np.concatenate([np.full(s.n_params, _r32(s.lr)) for s in self.pb.subs])

    def step(self, flat, m, v, t: int):
        """One training step of Algorithm 1: losses, gradients, then an
        independent Adam update of every subdomain.  t is the 1-based step
        number after the update.  Returns (terms, theta, m, v)."""
        terms, g = self.grad(flat)
        pb = self.pb
        theta, m, v = adam_update(flat, g, m, v, t, self.lr_vector(), self.beta1, self.beta2, self.eps)
        return terms, theta, m, v

    # -- stitched prediction (Eq. FSol) --------------------------------------
    def eval_stitched(self, flat, model: int, xy, K: int) -> np.ndarray:
        """u(z) = sum_q u_q(z) 1_{Omega_q}(z), the indicator being 1/S on a
        common interface of S subdomains; jets [n, D_out_total, K].  Points
        outside every subdomain give NaN."""
        pb = self.pb
        spm = pb.subs_per_model or pb.n_sub
        qs = list(range(model * spm, (model + 1) * spm))
        if pb.subs[qs[0]].region_kind == P.REGION_VORONOI:
            memb = route_voronoi([pb.subs[q].site for q in qs], pb.polygon, xy)
        else:
            memb = route_rect([pb.subs[q].rect for q in qs], xy)
        flat = _t(flat)
        dout = n_out_total(pb)
        out = np.zeros((len(xy), dout, K))
        for li, q in enumerate(qs):
            idx = [i for i, m in enumerate(memb) if li in m]
            if not idx:
                continue
            pts = np.asarray(xy)[idx]
            J = np.concatenate([
                jets(layers, _t(pts), nd.out_act, K, nd.act, a, scale).detach().numpy()
                for layers, a, scale, nd in (self._net_fn(flat, q, n) for n in range(len(pb.subs[q].nets)))],
                axis=1)
            S = np.array([len(memb[i]) for i in idx], dtype=np.float64)
            out[idx] += J / S[:, None, None]
        out[[i for i, m in enumerate(memb) if not m]] = np.nan
        return out
