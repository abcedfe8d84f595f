"""The torch.autograd.Function front end: its backward is the library's
hand-written jet reverse pass.  Checked against the FP64 oracle's gradient
and against central finite differences of each subdomain's own loss J_q
(the neighbours held constant, Algorithm 1), both through the GPU library."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2104_10013_gb300 import problems as P
from tests.cases import tiny_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pde,method", [(P.PDE_NS, P.CPINN), (P.PDE_DIFFUSION, P.XPINN),
                                        (P.PDE_BURGERS, P.CPINN)])
def test_autograd_backward_is_the_jet_reverse_pass(pde, method):
    import torch
    from paper_2104_10013_gb300 import autograd as AG
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    pb = tiny_problem(pde, method, n_sub=3, n_res=64, n_data=16, n_if=16, widths=None)
    s = X.Solver(pb)
    dev = torch.device("cuda", 0)
    theta0 = torch.from_numpy(pb.packed_params()).to(dev)
    theta = theta0.clone().requires_grad_(True)
    W = AG.loss_weights(pb, dev)
    J = AG.xpinn_loss(theta, s, W)
    (g,) = torch.autograd.grad(J, theta)
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    J_ref = (terms * Oracle(pb).weights()).sum()
    assert abs(J.item() - J_ref) <= 1e-5 * abs(J_ref)
    gn = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gn - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    # central differences of J_q alone (owner of each parameter), in float32
    owner = np.concatenate([np.full(sd.n_params, q) for q, sd in enumerate(pb.subs)])
    Wn = W.cpu().numpy().astype(np.float64)
    idx = np.argsort(-np.abs(g_ref))[:6]
    for i in idx:
        q = owner[i]
        h = 1e-2 * max(1.0, abs(float(theta0[i])))
        vals = []
        for sgn in (1, -1):
            t = theta0.clone()
            t[i] += sgn * h
            s.set_params(t)
            losses, _ = s.grad()
            vals.append((losses[q].astype(np.float64) * Wn[q]).sum())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gn[i]) <= 2e-2 * abs(gn[i]) + 1e-4, (i, fd, gn[i])
    s.close()
