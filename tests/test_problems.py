"""The seeded input generators: geometry and data they promise."""
import numpy as np

from paper_2104_10013_gb300 import problems as P


def test_burgers_initial_and_boundary_data():
    pb = P.burgers_cpinn(n_res=10, n_iface=5, n_bc=30)
    for s in pb.subs:
        xy, v = s.data[0].xy.astype(np.float64), s.data[0].val[:, 0]
        ic = np.abs(xy[:, 1]) < 1e-12
        assert np.allclose(v[ic], -np.sin(np.pi * xy[ic, 0]), atol=1e-6)
        assert np.allclose(np.abs(xy[~ic, 0]), 1.0) and np.allclose(v[~ic], 0.0)
    assert len(pb.ifaces) == 3 and all(np.allclose(it.xy[:, 0], it.xy[0, 0]) for it in pb.ifaces)


def test_grid_interfaces_lie_on_shared_edges():
    pb = P.poisson_xpinn(n_res_range=(50, 60), n_iface=20, n_bc=10)
    assert len(pb.ifaces) == 24
    for it in pb.ifaces:
        a, b = pb.subs[it.q].rect, pb.subs[it.qp].rect
        for (x, y) in it.xy.astype(np.float64):
            for r in (a, b):
                assert r[0] <= x <= r[1] and r[2] <= y <= r[3]
    for s in pb.subs:
        x0, x1, y0, y1 = s.rect
        assert np.all((s.res_xy[:, 0] >= x0) & (s.res_xy[:, 0] <= x1))
        assert np.all((s.res_xy[:, 1] >= y0) & (s.res_xy[:, 1] <= y1))


def test_voronoi_regions_and_edges():
    pb = P.diffusion_xpinn(n_res=500, n_obs=50, n_iface=40, n_kbc=20, n_copies=2)
    poly = np.array(pb.meta["polygon"])
    sites = np.array(pb.meta["sites"])
    n = len(sites)
    assert pb.n_sub == 2 * n and pb.subs_per_model == n
    for q in range(n):
        s = pb.subs[q]
        xy = s.res_xy.astype(np.float64)
        assert P.in_polygon(xy, poly).all()
        assert (P.nearest_site(xy, sites) == q).all()
        assert s.nets[1].out_act == P.ACT_SOFTPLUS
    for it in pb.ifaces[: len(pb.ifaces) // 2]:
        xy = it.xy.astype(np.float64)
        di = np.linalg.norm(xy - sites[it.q], axis=1)
        dj = np.linalg.norm(xy - sites[it.qp], axis=1)
        dmin = np.linalg.norm(xy[:, None, :] - sites[None], axis=2).min(1)
        assert np.allclose(di, dj, atol=1e-5) and np.allclose(di, dmin, atol=1e-5)
        assert P.in_polygon(xy, poly).mean() > 0.95   # float32 rounding at the boundary
    # the two copies share points and geometry but not weights or learning rates
    assert pb.subs[0].res_xy is pb.subs[n].res_xy
    assert pb.subs[0].lr != pb.subs[n].lr
    assert not np.array_equal(pb.subs[0].params[0][0][0], pb.subs[n].params[0][0][0])


def test_spacetime_burgers_interfaces():
    pb = P.burgers_spacetime(4, 2, n_res_total=800, method_x=P.CPINN)
    assert pb.n_sub == 8 and len(pb.ifaces) == 3 * 2 + 4 * 1
    for it in pb.ifaces:
        if it.normal == (1.0, 0.0):
            assert it.method == P.CPINN and np.allclose(it.xy[:, 0], it.xy[0, 0])
        else:
            assert it.method == P.XPINN and np.allclose(it.xy[:, 1], it.xy[0, 1])
    ic = [s for s in pb.subs if s.rect[2] == 0.0]
    assert len(ic) == 4 and all(s.data[0] is not None for s in ic)


def test_inverse_diffusion_uses_the_table_activations():
    """Table Table_USmap: region activations tanh, sin, cos, tanh, ... with
    trainable slopes, initialised to n a^k = 1."""
    pb = P.diffusion_xpinn(n_res=200, n_obs=20, n_iface=10, n_kbc=5, n_copies=1)
    want = [P.PHI_TANH, P.PHI_SIN, P.PHI_COS] * 4
    for q, s in enumerate(pb.subs):
        for net in s.nets:
            assert net.act == want[q] and net.adaptive and net.slope_scale == 10.0
    theta = pb.packed_params()
    off = 0
    for s in pb.subs:
        for net in s.nets:
            off += net.n_params
            assert np.all(theta[off - net.n_slopes:off] * net.slope_scale == np.float32(0.1) * 10)
