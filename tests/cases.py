"""Problem builders shared by the oracle pins and the GPU parity tests."""
import math

import numpy as np

from paper_2104_10013_gb300 import problems as P

NU = 0.01 / math.pi

CASES = [(P.PDE_BURGERS, P.CPINN), (P.PDE_BURGERS, P.XPINN), (P.PDE_POISSON, P.XPINN),
         (P.PDE_POISSON, P.CPINN), (P.PDE_NS, P.CPINN), (P.PDE_NS, P.XPINN),
         (P.PDE_DIFFUSION, P.XPINN), (P.PDE_DIFFUSION, P.CPINN)]


def tiny_problem(pde, method, n_sub=2, widths=None, n_res=7, n_data=5, n_if=4, seed=0, act=P.PHI_TANH,
                 adaptive=False):
    """Two (or more) subdomains side by side on [0, n_sub] x [0, 1] with tiny
    networks, random targets and forcing; every loss term is active."""
    rng = np.random.default_rng(seed)
    kw = dict(act=act, adaptive=adaptive)
    nets = {P.PDE_BURGERS: [P.NetSpec(widths or [2, 3, 3, 1], **kw)],
            P.PDE_POISSON: [P.NetSpec(widths or [2, 3, 3, 1], **kw)],
            P.PDE_NS: [P.NetSpec(widths or [2, 3, 3, 3], **kw)],
            P.PDE_DIFFUSION: [P.NetSpec(widths or [2, 3, 3, 1], **kw),
                              P.NetSpec([2, 3, 1], P.ACT_SOFTPLUS, **kw)]}[pde]
    subs = []
    for q in range(n_sub):
        res = rng.uniform((q, 0), (q + 1, 1), size=(n_res, 2))
        data = []
        for n in nets:
            dxy = rng.uniform((q, 0), (q + 1, 1), size=(n_data, 2))
            data.append(P.DataSet(P._f32(dxy), P._f32(rng.normal(size=(n_data, n.widths[-1])))))
        s = P.Subdomain(nets=nets, res_xy=P._f32(res), res_f=P._f32(rng.normal(size=n_res)),
                        data=data, w_data=[1.3, 0.7][:len(nets)], w_res=0.9, w_avg=1.1,
                        w_iface=0.8, lr=1e-3 * (q + 1), rect=(q, q + 1, 0.0, 1.0))
        s.params = [[(P._f32(rng.normal(size=W.shape)), P._f32(rng.normal(size=b.shape) * 0.3))
                     for W, b in P.xavier_params(n, rng)] for n in nets]
        if adaptive:   # slopes away from their initial 1/n, so that their gradients are exercised
            srng = np.random.default_rng(1000 + seed + q)   # own stream: the other draws stay as without slopes
            s.slopes = [P._f32(srng.uniform(0.05, 0.2, size=n.n_slopes)) for n in nets]
        subs.append(s)
    ifaces = [P.Interface(q, q + 1, method, (1.0, 0.0),
                          P._f32(np.stack([np.full(n_if, q + 1.0), rng.random(n_if)], 1)))
              for q in range(n_sub - 1)]
    return P.Problem("tiny", pde, subs, ifaces, nu=NU, re=7.0)




def with_activations(pb, acts, adaptive=True, seed=0):
    """The problem with hidden activation acts[q % len(acts)] in subdomain q
    (as in Table Table_USmap, where tanh and sin networks sit side by side)
    and, with `adaptive`, trainable slopes drawn in [0.08, 0.15] (n a^k in
    [0.8, 1.5] for n = 10) so that their gradients are exercised."""
    import dataclasses
    rng = np.random.default_rng(500 + seed)
    for q, s in enumerate(pb.subs):
        s.nets = [dataclasses.replace(n, act=acts[q % len(acts)], adaptive=adaptive) for n in s.nets]
        s.slopes = [P._f32(rng.uniform(0.08, 0.15, size=n.n_slopes)) for n in s.nets] if adaptive else []
    return pb
