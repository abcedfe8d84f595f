"""Training on a private fork (xpinn_fork_step): a subset S of a model's
subdomains trained on the request's own residual points, starting from the
model's parameters, Adam moments and step count, with the interface
neighbours outside S held at the model's parameters (Algorithm 1).

Checked: the first step's loss terms of S against the FP64 oracle on the
same problem with S's residual points replaced by the request's; the
parameters after one step against a whole handle stepping that problem (the
same first update of S, summed in another item order); the model's own
parameters unchanged; a fork repeated is bitwise the same.
"""
import copy

import numpy as np
import pytest

from oracle import Oracle
from paper_2104_10013_gb300 import problems as P
from tests.test_parity import RTOL_JET, assert_scaled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    return X


def request_points(pb, sel, counts, seed=5):
    rng = np.random.default_rng(seed)
    xy, f = [], []
    for q, n in zip(sel, counts):
        x0, x1, y0, y1 = pb.subs[q].rect
        pts = np.stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n)], 1).astype(np.float32)
        xy.append(pts)
        f.append((rng.normal(size=n) if pb.pde == P.PDE_POISSON else np.zeros(n)).astype(np.float32))
    return xy, f


def with_points(pb, sel, xy, f):
    pb2 = copy.deepcopy(pb)
    for q, a, b in zip(sel, xy, f):
        pb2.subs[q].res_xy = a
        pb2.subs[q].res_f = b
    return pb2


@pytest.mark.parametrize("name,sel,counts", [
    ("poisson_xpinn", [5, 6, 9], [1000, 2500, 777]),     # interior subdomains, neighbours outside S
    ("burgers_cpinn", [0, 3], [1500, 640]),              # end slabs, cPINN fluxes
    ("kovasznay_cpinn", [4], [3000]),                    # one subdomain, four neighbours
])
def test_fork_first_step_matches_oracle_and_full_handle(X, name, sel, counts):
    pb = {"poisson_xpinn": lambda: P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40),
          "burgers_cpinn": lambda: P.burgers_cpinn(n_res=500),
          "kovasznay_cpinn": lambda: P.kovasznay_cpinn(nx=3, ny=3, n_res=1500, n_iface=96, n_bc=80)}[name]()
    xy, f = request_points(pb, sel, counts)
    s = X.Solver(pb)
    theta0 = s.get_params()
    losses, fparams = s.fork_step(sel, xy, f, n_steps=1)
    assert np.array_equal(s.get_params(), theta0)             # the model is untouched
    pb2 = with_points(pb, sel, xy, f)
    terms, _ = Oracle(pb2).grad(pb2.packed_params(), subset=sel)
    assert_scaled(losses[0], terms, RTOL_JET, "fork losses", axis=0)
    # one step of the whole problem with S's points replaced: S's blocks take the same update
    s2 = X.Solver(pb2)
    s2.step(1)
    th2 = s2.get_params()
    offs = np.cumsum([0] + [sd.n_params for sd in pb.subs])
    want = np.concatenate([th2[offs[q]:offs[q + 1]] for q in sel])
    start = np.concatenate([theta0[offs[q]:offs[q + 1]] for q in sel])
    d_fork, d_full = fparams - start, want - start
    assert np.linalg.norm(d_fork - d_full) <= 1e-3 * np.linalg.norm(d_full)
    s.close(); s2.close()


def test_fork_is_deterministic_and_continues_adam(X):
    """Four fork steps from a model that has trained 3 steps (Adam moments
    and t = 3 carried over): a repeated fork is bitwise the same, and its loss
    rows and final parameters follow the FP64 oracle's Adam trajectory from
    the model's saved state, with S's parameters evolving and the neighbours'
    held at the model's values (float32 drift only over the 4 steps)."""
    import struct
    from oracle import adam_update
    pb = P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40)
    s = X.Solver(pb)
    s.step(3)                                                  # Adam moments and t > 0
    blob = s.get_state()
    t0 = struct.unpack_from("<i", blob, 12)[0]                 # header: magic[8], version, step_t
    n = pb.n_params
    theta, m, v = (np.frombuffer(blob, np.float32, n, 32 + k * 4 * n).astype(np.float64) for k in range(3))
    assert t0 == 3
    sel = [2, 7]
    xy, f = request_points(pb, sel, [900, 1300], seed=9)
    l1, p1 = s.fork_step(sel, xy, f, n_steps=4)
    l2, p2 = s.fork_step(sel, xy, f, n_steps=4)
    assert np.array_equal(l1, l2) and np.array_equal(p1, p2)
    assert l1.shape == (4, 2, P.N_TERMS)
    pb2 = with_points(pb, sel, xy, f)
    orc = Oracle(pb2)
    offs = np.cumsum([0] + [sd.n_params for sd in pb.subs])
    mask = np.zeros(n, bool)
    for q in sel:
        mask[offs[q]:offs[q + 1]] = True
    th = theta.copy()
    lr = orc.lr_vector()
    for k in range(4):
        terms, g = orc.grad(th, subset=sel)                   # S's rows; neighbours at th (model values)
        assert_scaled(l1[k], terms, 1e-4, f"fork step {k} losses", axis=0)
        th_new, m_new, v_new = adam_update(th, g, m, v, t0 + k + 1, lr, orc.beta1, orc.beta2, orc.eps)
        th = np.where(mask, th_new, th)
        m = np.where(mask, m_new, m)
        v = np.where(mask, v_new, v)
    want = np.concatenate([th[offs[q]:offs[q + 1]] for q in sel])
    start = np.concatenate([theta[offs[q]:offs[q + 1]] for q in sel])
    assert np.linalg.norm(p1 - want) <= 1e-3 * np.linalg.norm(want - start)
    assert np.array_equal(s.get_state(), blob)                 # the model is untouched
    s.close()


def test_fork_rejects_bad_requests(X):
    pb = P.burgers_cpinn(n_res=200)
    s = X.Solver(pb)
    xy = [np.zeros((4, 2), np.float32)] * 2
    with pytest.raises(X.XpinnError):
        s.fork_step([1, 1], xy)                               # repeated subdomain
    with pytest.raises(X.XpinnError):
        s.fork_step([9], xy[:1])                              # out of range
    s.close()


def test_fork_edge_cases(X):
    """Zero steps return the model's own parameters of the selection; a
    selected subdomain given no residual points trains on its data and
    interface terms only (its residual term is 0), against the oracle."""
    pb = P.poisson_xpinn(n_res_range=(300, 1500), n_iface=64, n_bc=40)
    s = X.Solver(pb)
    offs = np.cumsum([0] + [sd.n_params for sd in pb.subs])
    theta = s.get_params()
    sel = [3, 12]
    xy, f = request_points(pb, sel, [500, 0])
    l0, p0 = s.fork_step(sel, xy, f, n_steps=0)
    assert l0.shape == (0, 2, P.N_TERMS)
    assert np.array_equal(p0, np.concatenate([theta[offs[q]:offs[q + 1]] for q in sel]))
    l1, _ = s.fork_step(sel, xy, f, n_steps=1)
    pb2 = with_points(pb, sel, xy, f)
    terms, _ = Oracle(pb2).grad(pb2.packed_params(), subset=sel)
    assert terms[1, 2] == 0 and l1[0, 1, 2] == 0
    assert_scaled(l1[0], terms, RTOL_JET, "fork losses", axis=0)
    s.close()
