"""Seeded synthetic problem generators for domain-decomposed PINNs.

This module builds the *inputs* of a cPINN / XPINN training problem: the
decomposition of the domain into subdomains, the residual, data and interface
point sets sampled in each of them, the forcing term and the boundary data of
the PDE, and the initial network weights.  It holds none of the method's
arithmetic (no network evaluation, no residual, no loss, no optimiser): it is
shared, unchanged, by the FP64 oracle and by the CUDA path, which both read
the float32 arrays it produces.

Pre-processing follows Sec. 5.1 / Algorithm 1 (pre-processing stage): the
domain is split into non-overlapping subdomains, and training, residual and
interface points are sampled i.i.d. per subdomain.  Points are drawn uniformly
in each subdomain (the paper's "N(0, sigma^2)" is not meaningful on a bounded
subdomain).  Every float array is rounded to float32 here, so that both sides
consume bit-identical inputs.

PDE ids: 0 Burgers (Sec. 7.3 / 7.5), 1 Poisson, 2 steady incompressible
Navier-Stokes (Eq. NSEq, Sec. 7.4), 3 inverse diffusion (Eq. heq, Sec. 7.6).
Interface methods: 0 cPINN (Eq. cPINNLoss), 1 XPINN (Eq. XPINNLoss).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PDE_BURGERS, PDE_POISSON, PDE_NS, PDE_DIFFUSION = 0, 1, 2, 3
CPINN, XPINN = 0, 1
ACT_IDENTITY, ACT_SOFTPLUS = 0, 1
PHI_TANH, PHI_SIN, PHI_COS = 0, 1, 2      # hidden activation Phi (Table Table_USmap)
REGION_BOX, REGION_VORONOI = 0, 1
FLUX_CONSERVATIVE, FLUX_LITERAL = 0, 1

# number of loss terms reported per subdomain:
#   0 MSE_u of data set of net 0, 1 MSE_u of data set of net 1, 2 MSE_F,
#   3 MSE_uavg, 4 MSE_flux (cPINN) or MSE_R (XPINN)
N_TERMS = 5


@dataclass
class NetSpec:
    """One fully connected network (Sec. 3): widths = [N_0, ..., N_L], hidden
    activation Phi (tanh, sin or cos).  With `adaptive`, hidden layer k uses
    Phi(n a^k z) with a trainable slope a^k and scale n (= slope_scale), one
    slope per hidden layer, appended after the network's layers."""
    widths: list
    out_act: int = ACT_IDENTITY
    act: int = PHI_TANH
    adaptive: bool = False
    slope_scale: float = 10.0

    @property
    def n_slopes(self) -> int:
        return len(self.widths) - 2 if self.adaptive else 0

    @property
    def n_params(self) -> int:
        return sum(self.widths[k] * self.widths[k - 1] + self.widths[k]
                   for k in range(1, len(self.widths))) + self.n_slopes


@dataclass
class DataSet:
    """Training data of one network: points [n, 2] and targets [n, D_out]."""
    xy: np.ndarray
    val: np.ndarray


@dataclass
class Subdomain:
    nets: list                      # [NetSpec], one or two networks
    res_xy: np.ndarray              # float32 [n_F, 2] residual points
    res_f: np.ndarray               # float32 [n_F] forcing f at residual points
    data: list                      # per net: DataSet or None
    w_data: list                    # per net: W_u
    w_res: float = 1.0              # W_F
    w_avg: float = 1.0              # W_I
    w_iface: float = 1.0            # W_I,flux (cPINN) or W_I,F (XPINN)
    lr: float = 1e-3
    rect: tuple | None = None       # (x0, x1, y0, y1) closed rectangle, for routing
    params: list = field(default_factory=list)  # per net: [(W[N_k,N_k-1], b[N_k]) ...]
    region_kind: int = 0            # REGION_BOX, or REGION_VORONOI: polygon cell of `site`
    site: tuple | None = None
    slopes: list = field(default_factory=list)  # per net: a^1..a^{L-1} (adaptive nets) or None

    @property
    def n_params(self) -> int:
        return sum(n.n_params for n in self.nets)


@dataclass
class Interface:
    """A common interface between subdomains q and qp, with its own points.
    remote: only side q belongs to this problem (one rank's part of a
    distributed decomposition); side qp is another rank's."""
    q: int
    qp: int
    method: int
    normal: tuple
    xy: np.ndarray                  # float32 [n_I, 2]
    remote: bool = False


@dataclass
class Problem:
    name: str
    pde: int
    subs: list
    ifaces: list
    nu: float = 0.0
    re: float = 1.0
    flux_mode: int = FLUX_CONSERVATIVE
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    subs_per_model: int = 0         # subdomains per independent copy (0: all)
    meta: dict = field(default_factory=dict)
    polygon: np.ndarray | None = None   # domain polygon [n, 2] for Voronoi regions

    @property
    def n_sub(self) -> int:
        return len(self.subs)

    @property
    def n_models(self) -> int:
        spm = self.subs_per_model or self.n_sub
        return self.n_sub // spm

    def packed_params(self) -> np.ndarray:
        """All parameters in the packed layout: per subdomain, per net, per
        layer k = 1..L: W^k row-major [N_k][N_{k-1}] followed by b^k; then,
        for an adaptive net, its slopes a^1..a^{L-1} (initially 1/n, so that
        n a^k = 1 as in Sec. 3)."""
        out = []
        for s in self.subs:
            for n, (net, net_params) in enumerate(zip(s.nets, s.params)):
                for W, b in net_params:
                    out.append(W.reshape(-1))
                    out.append(b.reshape(-1))
                if net.adaptive:
                    a = s.slopes[n] if n < len(s.slopes) and s.slopes[n] is not None else None
                    out.append(np.full(net.n_slopes, 1.0 / net.slope_scale) if a is None else np.asarray(a))
        return np.concatenate(out).astype(np.float32)

    def unpack_params(self, flat: np.ndarray) -> list:
        """Inverse of packed_params: per subdomain, per net, ([(W, b), ...],
        slopes or None)."""
        flat = np.asarray(flat)
        res, off = [], 0
        for s in self.subs:
            sp = []
            for net in s.nets:
                layers = []
                for k in range(1, len(net.widths)):
                    no, ni = net.widths[k], net.widths[k - 1]
                    W = flat[off:off + no * ni].reshape(no, ni); off += no * ni
                    b = flat[off:off + no]; off += no
                    layers.append((W, b))
                a = None
                if net.adaptive:
                    a = flat[off:off + net.n_slopes]; off += net.n_slopes
                sp.append((layers, a))
            res.append(sp)
        assert off == flat.size
        return res

    @property
    def n_params(self) -> int:
        return sum(s.n_params for s in self.subs)

    @property
    def n_res(self) -> int:
        return sum(s.res_xy.shape[0] for s in self.subs)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _cuts32(c) -> np.ndarray:
    """Cut coordinates rounded to float32 values, so that subdomain boxes,
    interface points and query points on a cut agree on both sides."""
    return np.asarray(c, dtype=np.float64).astype(np.float32).astype(np.float64)


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.default_rng([int(seed)] + [int(k) for k in key])


def xavier_params(net: NetSpec, rng: np.random.Generator) -> list:
    """Xavier-normal weights (std = sqrt(2 / (fan_in + fan_out))), zero biases."""
    layers = []
    for k in range(1, len(net.widths)):
        no, ni = net.widths[k], net.widths[k - 1]
        W = rng.normal(0.0, math.sqrt(2.0 / (ni + no)), size=(no, ni))
        layers.append((_f32(W), np.zeros(no, np.float32)))
    return layers


def _uniform_rect(rng, n, x0, x1, y0, y1) -> np.ndarray:
    u = rng.random((n, 2))
    return np.stack([x0 + (x1 - x0) * u[:, 0], y0 + (y1 - y0) * u[:, 1]], axis=1)


def _segment_points(rng, n, a, b) -> np.ndarray:
    """n uniform points on the segment from a to b."""
    s = rng.random(n)
    a, b = np.asarray(a, float), np.asarray(b, float)
    return a[None, :] + s[:, None] * (b - a)[None, :]


def _split_counts(n, lengths) -> list:
    """Split n points over pieces proportionally to their lengths."""
    lengths = np.asarray(lengths, float)
    if lengths.sum() <= 0:
        return [0] * len(lengths)
    raw = n * lengths / lengths.sum()
    cnt = np.floor(raw).astype(int)
    for i in np.argsort(-(raw - cnt))[: n - cnt.sum()]:
        cnt[i] += 1
    return cnt.tolist()


def _rect_boundary_pieces(rect, domain) -> list:
    """Edges of a rectangle that lie on the boundary of the rectangular domain."""
    x0, x1, y0, y1 = rect
    X0, X1, Y0, Y1 = domain
    pieces = []
    if abs(x0 - X0) < 1e-12:
        pieces.append(((x0, y0), (x0, y1)))
    if abs(x1 - X1) < 1e-12:
        pieces.append(((x1, y0), (x1, y1)))
    if abs(y0 - Y0) < 1e-12:
        pieces.append(((x0, y0), (x1, y0)))
    if abs(y1 - Y1) < 1e-12:
        pieces.append(((x0, y1), (x1, y1)))
    return pieces


def _grid_interfaces(xc, yc, rng_for, n_iface, method) -> list:
    """Interfaces of a tensor grid with cell (i, j) -> subdomain i + nx*j."""
    nx, ny = len(xc) - 1, len(yc) - 1
    out = []
    e = 0
    for j in range(ny):            # vertical cuts x = xc[i], i = 1..nx-1
        for i in range(1, nx):
            q, qp = (i - 1) + nx * j, i + nx * j
            xy = _segment_points(rng_for(e), n_iface, (xc[i], yc[j]), (xc[i], yc[j + 1]))
            out.append(Interface(q, qp, method, (1.0, 0.0), _f32(xy)))
            e += 1
    for j in range(1, ny):         # horizontal cuts y = yc[j]
        for i in range(nx):
            q, qp = i + nx * (j - 1), i + nx * j
            xy = _segment_points(rng_for(e), n_iface, (xc[i], yc[j]), (xc[i + 1], yc[j]))
            out.append(Interface(q, qp, method, (0.0, 1.0), _f32(xy)))
            e += 1
    return out


# ---------------------------------------------------------------------------
# Exact solutions / forcing terms (problem data, not method arithmetic)
# ---------------------------------------------------------------------------

def poisson_exact(x, y):
    """Manufactured u* = sin(2 pi x) sin(3 pi y) + 0.1 sin(20 pi x y)."""
    return np.sin(2 * np.pi * x) * np.sin(3 * np.pi * y) + 0.1 * np.sin(20 * np.pi * x * y)


def poisson_forcing(x, y):
    """f = -lap u* for poisson_exact (derived by hand)."""
    return (13 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.sin(3 * np.pi * y)
            + 40 * np.pi ** 2 * (x ** 2 + y ** 2) * np.sin(20 * np.pi * x * y))


def kovasznay_lambda(re):
    return re / 2 - math.sqrt(re * re / 4 + 4 * math.pi ** 2)


def kovasznay_exact(x, y, re):
    """Kovasznay flow (u, v, p), a closed-form solution of steady NS."""
    lam = kovasznay_lambda(re)
    e = np.exp(lam * x)
    u = 1 - e * np.cos(2 * np.pi * y)
    v = lam / (2 * np.pi) * e * np.sin(2 * np.pi * y)
    p = 0.5 * (1 - np.exp(2 * lam * x))
    return np.stack([u, v, p], axis=-1)


def diffusion_exact_u(x, y):
    """Temperature field of Sec. 7.6: T = 20 exp(-0.1 y)."""
    return 20.0 * np.exp(-0.1 * y)


def diffusion_exact_k(x, y):
    """Synthetic conductivity K* = 1 + 0.5 sin(pi x) cos(pi y)."""
    return 1.0 + 0.5 * np.sin(np.pi * x) * np.cos(np.pi * y)


def diffusion_forcing(x, y):
    """f = div(K* grad u*) for the two fields above (derived by hand)."""
    return np.exp(-0.1 * y) * (0.2 + 0.1 * np.sin(np.pi * x) * np.cos(np.pi * y)
                               + np.pi * np.sin(np.pi * x) * np.sin(np.pi * y))


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def burgers_cpinn(n_sub=4, n_res=1000, n_iface=100, n_bc=50, hidden=(20, 20, 20),
                  lr=1e-3, seed=0, flux_mode=FLUX_CONSERVATIVE, nu=0.01 / math.pi) -> Problem:
    """1D viscous Burgers u_t + u u_x = nu u_xx on x in [-1,1], t in [0,1]
    (Sec. 7.3, Eq. BE), u(x,0) = -sin(pi x), u(+-1,t) = 0; n_sub equal x-slabs
    coupled by cPINN (flux + average continuity).  Inputs are (x, t)."""
    xc = _cuts32(np.linspace(-1.0, 1.0, n_sub + 1))
    net = NetSpec([2, *hidden, 1])
    subs = []
    for q in range(n_sub):
        x0, x1 = xc[q], xc[q + 1]
        rng = _rng(seed, 1, q)
        res = _uniform_rect(rng, n_res, x0, x1, 0.0, 1.0)
        # initial / boundary data spread over the subdomain's boundary pieces
        pieces = [((x0, 0.0), (x1, 0.0))]
        if q == 0:
            pieces.append(((-1.0, 0.0), (-1.0, 1.0)))
        if q == n_sub - 1:
            pieces.append(((1.0, 0.0), (1.0, 1.0)))
        lens = [math.dist(a, b) for a, b in pieces]
        cnt = _split_counts(n_bc, lens)
        rb = _rng(seed, 2, q)
        bxy = np.concatenate([_segment_points(rb, c, a, b) for (a, b), c in zip(pieces, cnt)])
        bval = np.where(np.abs(bxy[:, 1]) < 1e-12, -np.sin(np.pi * bxy[:, 0]), 0.0)
        sub = Subdomain(nets=[net], res_xy=_f32(res), res_f=np.zeros(n_res, np.float32),
                        data=[DataSet(_f32(bxy), _f32(bval[:, None]))], w_data=[1.0],
                        lr=lr, rect=(x0, x1, 0.0, 1.0))
        sub.params = [xavier_params(net, _rng(seed, 3, q))]
        subs.append(sub)
    ifaces = _grid_interfaces(xc, np.array([0.0, 1.0]), lambda e: _rng(seed, 4, e), n_iface, CPINN)
    return Problem("burgers_cpinn", PDE_BURGERS, subs, ifaces, nu=nu, flux_mode=flux_mode,
                   meta=dict(xcuts=xc.tolist(), ycuts=[0.0, 1.0]))


def poisson_xpinn(nx=4, ny=4, n_res_range=(2000, 20000), depth_range=(4, 6), width_range=(20, 80),
                  n_iface=200, n_bc=100, lr=1e-3, seed=0, min_cell=0.1) -> Problem:
    """2D Poisson -lap u = f on the unit square, manufactured solution
    poisson_exact, XPINN on an uneven nx x ny tensor grid.  Each subdomain draws
    its residual-point count, depth (hidden layers) and width from the seed."""
    g = _rng(seed, 10)

    def cuts(n):
        while True:
            c = np.sort(g.random(n - 1))
            full = np.concatenate([[0.0], c, [1.0]])
            if np.all(np.diff(full) >= min_cell):
                return _cuts32(full)
    xc, yc = cuts(nx), cuts(ny)
    subs = []
    for j in range(ny):
        for i in range(nx):
            q = i + nx * j
            hp = _rng(seed, 11, q)
            n_res = int(hp.integers(n_res_range[0], n_res_range[1] + 1))
            depth = int(hp.integers(depth_range[0], depth_range[1] + 1))
            width = int(hp.integers(width_range[0], width_range[1] + 1))
            net = NetSpec([2] + [width] * depth + [1])
            rect = (xc[i], xc[i + 1], yc[j], yc[j + 1])
            rng = _rng(seed, 12, q)
            res = _f32(_uniform_rect(rng, n_res, *rect))
            pieces = _rect_boundary_pieces(rect, (0.0, 1.0, 0.0, 1.0))
            rb = _rng(seed, 13, q)
            data = None
            if pieces:
                bxy = _f32(np.concatenate([_segment_points(rb, n_bc, a, b) for a, b in pieces]))
                data = DataSet(bxy, _f32(poisson_exact(bxy[:, 0].astype(np.float64),
                                                       bxy[:, 1].astype(np.float64))[:, None]))
            f = poisson_forcing(res[:, 0].astype(np.float64), res[:, 1].astype(np.float64))
            sub = Subdomain(nets=[net], res_xy=res, res_f=_f32(f), data=[data], w_data=[1.0],
                            lr=lr, rect=rect)
            sub.params = [xavier_params(net, _rng(seed, 14, q))]
            subs.append(sub)
    ifaces = _grid_interfaces(xc, yc, lambda e: _rng(seed, 15, e), n_iface, XPINN)
    return Problem("poisson_xpinn", PDE_POISSON, subs, ifaces,
                   meta=dict(xcuts=xc.tolist(), ycuts=yc.tolist()))


def kovasznay_cpinn(nx=8, ny=8, n_res=50000, n_iface=256, n_bc=80, width=64, depth=6, re=40.0,
                    lr=6e-4, seed=0) -> Problem:
    """2D steady incompressible NS (Eq. NSEq), Kovasznay flow at Re on
    [-0.5,1] x [-0.5,1.5], cPINN on an equal nx x ny grid; each boundary
    subdomain gets n_bc Dirichlet points for (u, v, p)."""
    dom = (-0.5, 1.0, -0.5, 1.5)
    xc = _cuts32(np.linspace(dom[0], dom[1], nx + 1))
    yc = _cuts32(np.linspace(dom[2], dom[3], ny + 1))
    net = NetSpec([2] + [width] * depth + [3])
    subs = []
    for j in range(ny):
        for i in range(nx):
            q = i + nx * j
            rect = (xc[i], xc[i + 1], yc[j], yc[j + 1])
            res = _f32(_uniform_rect(_rng(seed, 21, q), n_res, *rect))
            pieces = _rect_boundary_pieces(rect, dom)
            data = None
            if pieces:
                cnt = _split_counts(n_bc, [math.dist(a, b) for a, b in pieces])
                rb = _rng(seed, 22, q)
                bxy = _f32(np.concatenate([_segment_points(rb, c, a, b)
                                           for (a, b), c in zip(pieces, cnt)]))
                data = DataSet(bxy, _f32(kovasznay_exact(bxy[:, 0].astype(np.float64),
                                                         bxy[:, 1].astype(np.float64), re)))
            sub = Subdomain(nets=[net], res_xy=res, res_f=np.zeros(n_res, np.float32),
                            data=[data], w_data=[1.0], lr=lr, rect=rect)
            sub.params = [xavier_params(net, _rng(seed, 23, q))]
            subs.append(sub)
    ifaces = _grid_interfaces(xc, yc, lambda e: _rng(seed, 24, e), n_iface, CPINN)
    return Problem("kovasznay_cpinn", PDE_NS, subs, ifaces, re=re,
                   meta=dict(xcuts=xc.tolist(), ycuts=yc.tolist()))


# ---------------------------------------------------------------------------
# Irregular geometry: a star polygon split into clipped Voronoi regions
# ---------------------------------------------------------------------------

def star_polygon(rng, n_vert=14, r_min=0.55, r_max=1.0, center=(1.0, 1.0)):
    """Vertices (counter-clockwise) of a seeded star-shaped, usually
    non-convex polygon."""
    ang = np.sort(rng.uniform(0, 2 * np.pi, n_vert))
    rad = rng.uniform(r_min, r_max, n_vert)
    return np.stack([center[0] + rad * np.cos(ang), center[1] + rad * np.sin(ang)], 1)


def in_polygon(xy, poly) -> np.ndarray:
    """Even-odd rule point-in-polygon test for points xy [n, 2]."""
    x, y = xy[:, 0][:, None], xy[:, 1][:, None]
    x0, y0 = poly[:, 0][None, :], poly[:, 1][None, :]
    x1, y1 = np.roll(poly[:, 0], -1)[None, :], np.roll(poly[:, 1], -1)[None, :]
    cond = (y0 > y) != (y1 > y)
    with np.errstate(divide="ignore", invalid="ignore"):
        xc = x0 + (y - y0) * (x1 - x0) / (y1 - y0)
    return (np.sum(cond & (x < xc), axis=1) % 2) == 1


def nearest_site(xy, sites) -> np.ndarray:
    d = ((xy[:, None, :] - sites[None, :, :]) ** 2).sum(-1)
    return np.argmin(d, axis=1)


def _bisector_pieces(poly, sites, i, j):
    """Pieces (a, b) of the common Voronoi edge of sites i and j inside the polygon."""
    si, sj = sites[i], sites[j]
    m = 0.5 * (si + sj)
    nrm = sj - si
    d = np.array([-nrm[1], nrm[0]]) / np.linalg.norm(nrm)
    lo, hi = -1e3, 1e3
    for k in range(len(sites)):
        if k in (i, j):
            continue
        # |x - s_i|^2 <= |x - s_k|^2  <=>  2 x.(s_k - s_i) <= |s_k|^2 - |s_i|^2, x = m + t d
        g = 2 * (sites[k] - si)
        c = sites[k] @ sites[k] - si @ si - g @ m
        a = g @ d
        if abs(a) < 1e-14:
            if c < 0:
                return []
            continue
        if a > 0:
            hi = min(hi, c / a)
        else:
            lo = max(lo, c / a)
    if hi <= lo:
        return []
    # crossings with the polygon boundary
    ts = [lo, hi]
    n = len(poly)
    for e in range(n):
        p, q = poly[e], poly[(e + 1) % n]
        M = np.array([d, p - q]).T
        if abs(np.linalg.det(M)) < 1e-14:
            continue
        t, s = np.linalg.solve(M, p - m)
        if 0 <= s <= 1 and lo < t < hi:
            ts.append(t)
    ts = np.sort(np.array(ts))
    pieces = []
    for a, b in zip(ts[:-1], ts[1:]):
        mid = m + 0.5 * (a + b) * d
        if b - a > 1e-9 and in_polygon(mid[None, :], poly)[0]:
            pieces.append((m + a * d, m + b * d))
    return pieces


def _sample_region(rng, poly, sites, q, n, batch=200000):
    lo, hi = poly.min(0), poly.max(0)
    out, have = [], 0
    while have < n:
        z = lo + (hi - lo) * rng.random((batch, 2))
        z = z[in_polygon(z, poly)]
        z = z[nearest_site(z, sites) == q]
        out.append(z)
        have += len(z)
    return np.concatenate(out)[:n]


def diffusion_xpinn(n_regions=10, n_res=30000, n_obs=500, n_iface=100, n_kbc=50, n_copies=256,
                    u_hidden=(40,) * 5, k_hidden=(20,) * 4, noise=0.01, seed=0,
                    acts=(PHI_TANH, PHI_SIN, PHI_COS), adaptive=True) -> Problem:
    """Inverse diffusion div(K grad u) = f (Eq. heq) with unknown K, on a seeded
    non-convex star polygon split into the clipped Voronoi regions of
    n_regions seeded sites; two networks per region, u and K (softplus
    output).  Data: n_obs noisy observations of u* = 20 exp(-0.1 y) per region
    (noise sigma = `noise` x rms of the observed values), n_kbc values of
    K* = 1 + 0.5 sin(pi x) cos(pi y) on the polygon boundary per boundary
    region, n_iface points on every common Voronoi edge (XPINN).  n_copies
    independent copies share the points and differ in initial weights,
    learning rate (log-uniform in [1e-4, 1e-2]) and the weights W_I, W_F
    (log-uniform in [0.1, 10]).  Region q uses the hidden activation
    acts[q % len(acts)] with trainable slopes (initially n a^k = 1): with the
    defaults tanh, sin, cos, tanh, ... as in Table Table_USmap."""
    g = _rng(seed, 40)
    poly = star_polygon(g)
    sites = []
    while len(sites) < n_regions:
        z = poly.min(0) + (poly.max(0) - poly.min(0)) * g.random((64, 2))
        sites.extend(z[in_polygon(z, poly)].tolist())
    sites = np.array(sites[:n_regions]).astype(np.float32).astype(np.float64)
    poly = poly.astype(np.float32).astype(np.float64)
    sites32 = sites
    # boundary points for K data: uniform in arc length, assigned to the nearest site
    edges = [(poly[e], poly[(e + 1) % len(poly)]) for e in range(len(poly))]
    lens = np.array([math.dist(a, b) for a, b in edges])
    gb = _rng(seed, 41)
    cnt = _split_counts(20 * n_kbc * n_regions, lens)
    bpts = np.concatenate([_segment_points(gb, c, a, b) for (a, b), c in zip(edges, cnt)])
    bown = nearest_site(bpts, sites)
    u_nets = [NetSpec([2, *u_hidden, 1], act=acts[q % len(acts)], adaptive=adaptive) for q in range(n_regions)]
    k_nets = [NetSpec([2, *k_hidden, 1], ACT_SOFTPLUS, act=acts[q % len(acts)], adaptive=adaptive)
              for q in range(n_regions)]
    region_pts = []
    for q in range(n_regions):
        rng = _rng(seed, 42, q)
        res = _f32(_sample_region(rng, poly, sites, q, n_res))
        f = _f32(diffusion_forcing(res[:, 0].astype(np.float64), res[:, 1].astype(np.float64)))
        obs = _sample_region(rng, poly, sites, q, n_obs)
        uo = diffusion_exact_u(obs[:, 0], obs[:, 1])
        uo = uo + noise * np.sqrt(np.mean(uo ** 2)) * rng.normal(size=uo.shape)
        kb = bpts[bown == q][:n_kbc]
        kd = DataSet(_f32(kb), _f32(diffusion_exact_k(kb[:, 0], kb[:, 1])[:, None])) if len(kb) else None
        region_pts.append((res, f, DataSet(_f32(obs), _f32(uo[:, None])), kd))
    iface_geo = []
    for i in range(n_regions):
        for j in range(i + 1, n_regions):
            pieces = _bisector_pieces(poly, sites, i, j)
            if not pieces:
                continue
            plen = np.array([math.dist(a, b) for a, b in pieces])
            if plen.sum() < 1e-6:
                continue
            ge = _rng(seed, 43, i, j)
            c = _split_counts(n_iface, plen)
            xy = np.concatenate([_segment_points(ge, cc, a, b) for (a, b), cc in zip(pieces, c)])
            nrm = (sites[j] - sites[i]) / np.linalg.norm(sites[j] - sites[i])
            iface_geo.append((i, j, (float(nrm[0]), float(nrm[1])), _f32(xy)))
    subs, ifaces = [], []
    for cp in range(n_copies):
        hp = _rng(seed, 44, cp)
        lr = float(10 ** hp.uniform(-4, -2))
        w_i = float(10 ** hp.uniform(-1, 1))
        w_f = float(10 ** hp.uniform(-1, 1))
        for q in range(n_regions):
            res, f, du, dk = region_pts[q]
            u_net, k_net = u_nets[q], k_nets[q]
            sub = Subdomain(nets=[u_net, k_net], res_xy=res, res_f=f, data=[du, dk], w_data=[1.0, 1.0],
                            w_res=w_f, w_avg=w_i, w_iface=w_i, lr=lr)
            lo, hi = poly.min(0), poly.max(0)
            sub.rect = (float(lo[0]), float(hi[0]), float(lo[1]), float(hi[1]))
            sub.region_kind = REGION_VORONOI
            sub.site = (float(sites32[q, 0]), float(sites32[q, 1]))
            sub.params = [xavier_params(u_net, _rng(seed, 45, cp, q, 0)),
                          xavier_params(k_net, _rng(seed, 45, cp, q, 1))]
            subs.append(sub)
        for (i, j, nrm, xy) in iface_geo:
            ifaces.append(Interface(cp * n_regions + i, cp * n_regions + j, XPINN, nrm, xy))
    return Problem("diffusion_xpinn", PDE_DIFFUSION, subs, ifaces, subs_per_model=n_regions,
                   meta=dict(polygon=poly.tolist(), sites=sites.tolist(), n_copies=n_copies),
                   polygon=_f32(poly))


def burgers_spacetime(nx=4, nt=2, n_res_total=80000, n_iface=20, n_bc=50, hidden=(20,) * 5, lr=8e-4,
                      method_x=XPINN, method_t=XPINN, seed=0, nu=0.01 / math.pi) -> Problem:
    """Viscous Burgers (Eq. BE1, Sec. 7.5) on x in [-1,1], t in [0,1] split
    into nx x nt space-time subdomains (Table TableVB): residual points spread
    uniformly over the subdomains, n_iface points on every interface, initial
    data on t = 0 and boundary data on x = +-1.  Interfaces across x-cuts use
    method_x, across t-cuts method_t (XPINN by default; cPINN in space with
    XPINN in time is the combination suggested in Sec. 7.7)."""
    xc = _cuts32(np.linspace(-1.0, 1.0, nx + 1))
    tc = _cuts32(np.linspace(0.0, 1.0, nt + 1))
    net = NetSpec([2, *hidden, 1])
    n_sub = nx * nt
    per = n_res_total // n_sub
    subs = []
    for j in range(nt):
        for i in range(nx):
            q = i + nx * j
            rect = (xc[i], xc[i + 1], tc[j], tc[j + 1])
            res = _f32(_uniform_rect(_rng(seed, 51, q), per, *rect))
            pieces = []
            if j == 0:
                pieces.append(((xc[i], 0.0), (xc[i + 1], 0.0)))
            if i == 0:
                pieces.append(((-1.0, tc[j]), (-1.0, tc[j + 1])))
            if i == nx - 1:
                pieces.append(((1.0, tc[j]), (1.0, tc[j + 1])))
            data = None
            if pieces:
                cnt = _split_counts(n_bc, [math.dist(a, b) for a, b in pieces])
                rb = _rng(seed, 52, q)
                bxy = np.concatenate([_segment_points(rb, c, a, b) for (a, b), c in zip(pieces, cnt)])
                bval = np.where(np.abs(bxy[:, 1]) < 1e-12, -np.sin(np.pi * bxy[:, 0]), 0.0)
                data = DataSet(_f32(bxy), _f32(bval[:, None]))
            sub = Subdomain(nets=[net], res_xy=res, res_f=np.zeros(per, np.float32), data=[data],
                            w_data=[1.0], lr=lr, rect=rect)
            sub.params = [xavier_params(net, _rng(seed, 53, q))]
            subs.append(sub)
    ifaces = _grid_interfaces(xc, tc, lambda e: _rng(seed, 54, e), n_iface, method_x)
    n_xcuts = (nx - 1) * nt
    for it in ifaces[n_xcuts:]:
        it.method = method_t
    return Problem("burgers_spacetime", PDE_BURGERS, subs, ifaces, nu=nu,
                   meta=dict(xcuts=xc.tolist(), ycuts=tc.tolist()))
