"""The torch.autograd.Function front end: its forward is the library's
objective J = sum_q J(Theta_q) (weighted in the library), its backward the
library's hand-written jet reverse pass.  Checked against the FP64 oracle's
objective and gradient, and against central finite differences of each
subdomain's own J(Theta_q) as the library reports it (the neighbours held
constant, Algorithm 1)."""
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
    J = AG.xpinn_loss(theta, s)
    (g,) = torch.autograd.grad(J, theta)
    orc = Oracle(pb)
    terms, g_ref = orc.grad(pb.packed_params())
    Jq_ref = (terms * orc.weights()).sum(1)
    assert abs(J.item() - Jq_ref.sum()) <= 1e-5 * abs(Jq_ref.sum())
    _, J_sub, _, _ = s.objective()
    assert np.all(np.abs(J_sub - Jq_ref) <= 1e-5 * np.maximum(np.abs(Jq_ref), np.sqrt(np.mean(Jq_ref ** 2))))
    gn = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gn - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    # fourth-order central differences (h and 2h) of J(Theta_q) of the
    # parameter's owner, from the library's float32 objective
    owner = np.concatenate([np.full(sd.n_params, q) for q, sd in enumerate(pb.subs)])
    idx = np.argsort(-np.abs(g_ref))[:6]
    for i in idx:
        q = owner[i]
        h = 1e-2 * max(1.0, abs(float(theta0[i])))
        vals = {}
        for m in (2, 1, -1, -2):
            t = theta0.clone()
            t[i] += m * h
            s.set_params(t)
            vals[m] = float(s.objective()[1][q])
        fd = (8 * (vals[1] - vals[-1]) - (vals[2] - vals[-2])) / (12 * h)
        assert abs(fd - gn[i]) <= 5e-3 * abs(gn[i]) + 1e-4, (i, fd, gn[i])
    s.close()


def test_objective_is_bitwise_reproducible_and_matches_grad():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    pb = tiny_problem(P.PDE_POISSON, P.XPINN, n_sub=3, n_res=64, n_data=16, n_if=16)
    s = X.Solver(pb)
    J1, Js1, l1, g1 = s.objective()
    J2, Js2, l2, g2 = s.objective()
    lg, gg = s.grad()
    assert np.array_equal(J1, J2) and np.array_equal(Js1, Js2) and np.array_equal(g1, g2)
    assert np.array_equal(l1, lg) and np.array_equal(g1, gg)
    s.close()
