"""The continuous-batching server (xpinn_server_*): every request's result is
the same alone and in a mix (bitwise): evaluations equal xpinn_eval, whole-
model step requests equal xpinn_step, training requests on a subdomain
subset with their own points (forks) equal xpinn_fork_step; requests are
admitted by their footprint in the server's preallocated pools (a small pool
makes them queue, and every result is still right), and a request larger
than a pool is refused up front."""
import numpy as np
import pytest

from paper_2104_10013_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    return X


def requests(pb, rng, n_req):
    out = []
    x0, x1 = pb.meta["xcuts"][0], pb.meta["xcuts"][-1]
    y0, y1 = pb.meta["ycuts"][0], pb.meta["ycuts"][-1]
    for _ in range(n_req):
        n = int(10 ** rng.uniform(0, 3.5))
        xy = np.stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n)], 1).astype(np.float32)
        out.append((xy, int(rng.integers(0, 3))))
    return out


def test_results_are_the_same_alone_and_in_the_mix(X):
    rng = np.random.default_rng(0)
    pb2 = P.poisson_xpinn(n_res_range=(300, 600), n_iface=32, n_bc=20)
    pb1 = P.burgers_cpinn(n_res=300)
    m0, m1 = X.Solver(pb2), X.Solver(pb1)
    ma, mb = X.Solver(pb1), X.Solver(pb1)      # identical models for step requests
    reqs = [(0, xy, o) for xy, o in requests(pb2, rng, 12)] + [(1, xy, o) for xy, o in requests(pb1, rng, 12)]
    # fork requests on model 0: subdomain subsets with their own residual points
    forks = []
    for sel, counts in (([5, 6], [1200, 800]), ([0], [3000]), ([9, 10, 13], [500, 700, 900])):
        xy_l, f_l = [], []
        for q, n in zip(sel, counts):
            x0, x1, y0, y1 = pb2.subs[q].rect
            xy_l.append(np.stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n)], 1).astype(np.float32))
            f_l.append(rng.normal(size=n).astype(np.float32))
        forks.append((sel, xy_l, f_l))
    srv = X.Server([m0, m1, ma], hbm_budget=1 << 28)
    alone = []
    for m, xy, o in reqs:
        r = srv.wait(srv.submit_eval(m, xy, o))
        assert r["status"] == 0, r["error"]
        alone.append(r["out"].copy())
    step_alone = srv.wait(srv.submit_step(2, 3))["out"].copy()
    fork_alone = []
    for sel, xy_l, f_l in forks:
        r = srv.wait(srv.submit_fork(0, sel, xy_l, f_l, n_steps=2))
        assert r["status"] == 0, r["error"]
        fork_alone.append(tuple(a.copy() for a in r["out"]))
    srv.close()
    # the same requests as one burst, interleaved with step requests on another model and forks
    srv = X.Server([m0, m1, mb], hbm_budget=1 << 28)
    order = rng.permutation(len(reqs))
    tickets = {}
    st = None
    ft = []
    for k, i in enumerate(order):
        m, xy, o = reqs[i]
        tickets[i] = srv.submit_eval(m, xy, o)
        if k == len(order) // 2:
            st = srv.submit_step(2, 3)
        if k % 8 == 3:
            sel, xy_l, f_l = forks[len(ft)]
            ft.append(srv.submit_fork(0, sel, xy_l, f_l, n_steps=2))
    res = {i: srv.wait(t) for i, t in tickets.items()}
    step_mix = srv.wait(st)["out"]
    fork_mix = [srv.wait(t) for t in ft]
    srv.close()
    assert max(r["batch"] for r in res.values()) > 1          # continuous batching happened
    assert max(r["tick_requests"] for r in res.values()) > 1
    for (sel, xy_l, f_l), a, r in zip(forks, fork_alone, fork_mix):
        assert r["status"] == 0, r["error"]
        assert np.array_equal(r["out"][0], a[0]) and np.array_equal(r["out"][1], a[1])
        direct = m0.fork_step(sel, xy_l, f_l, n_steps=2)
        assert np.array_equal(direct[0], a[0]) and np.array_equal(direct[1], a[1])
    for i, (m, xy, o) in enumerate(reqs):
        assert res[i]["status"] == 0 and res[i]["latency_ms"] > 0, res[i]["error"]
        assert np.array_equal(res[i]["out"], alone[i], equal_nan=True), i
        direct = [m0, m1][m].eval(0, xy, o)
        assert np.array_equal(direct, alone[i], equal_nan=True), i
    assert np.array_equal(step_alone, step_mix)
    assert np.array_equal(ma.get_params(), mb.get_params())


def test_request_larger_than_budget_is_refused(X):
    pb1 = P.burgers_cpinn(n_res=100)
    m = X.Solver(pb1)
    srv = X.Server([m], hbm_budget=1 << 16)
    xy = np.zeros((100000, 2), np.float32)
    with pytest.raises(X.XpinnError) as e:
        srv.submit_eval(0, xy, 0)
    assert e.value.code == -2
    t = srv.submit_eval(0, xy[:10] + 0.1, 0)
    assert srv.wait(t)["status"] == 0
    with pytest.raises(X.XpinnError) as e:                     # a fork of a subdomain that does not exist
        srv.submit_fork(0, [7], [np.zeros((10, 2), np.float32)])
    assert e.value.code == -1
    srv.close()


def test_small_pool_makes_requests_queue_and_results_stay_right(X):
    """A 16 MiB device pool holds only a few of these evaluations' workspaces
    at a time: the rest wait in the queue and are admitted as ticks complete
    and free the pool (no allocation per request); every result equals
    xpinn_eval."""
    rng = np.random.default_rng(1)
    pb1 = P.burgers_cpinn(n_res=300)
    m = X.Solver(pb1)
    reqs = []
    for _ in range(40):
        n = int(rng.integers(5000, 20000))
        xy = np.stack([rng.uniform(-1, 1, n), rng.uniform(0, 1, n)], 1).astype(np.float32)
        reqs.append((xy, int(rng.integers(0, 3))))
    srv = X.Server([m], hbm_budget=16 << 20)
    tickets = [srv.submit_eval(0, xy, o) for xy, o in reqs]
    res = [srv.wait(t) for t in tickets]
    srv.close()
    assert max(r["queue_ms"] for r in res) > 0
    for (xy, o), r in zip(reqs, res):
        assert r["status"] == 0, r["error"]
        assert np.array_equal(r["out"], m.eval(0, xy, o), equal_nan=True)
    m.close()
