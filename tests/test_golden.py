"""Generators and oracle settings against values the paper prints, kept as
text fixtures under tests/golden/ (each file states the passage it copies)."""
import math
import os

import numpy as np

from paper_2104_10013_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _keys(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split("=", 1)
                out[k.strip()] = v.strip()
    return out


def test_burgers_problem_as_printed():
    """Sec. 7.3 Eq. BE / Sec. 7.5 Eq. BE1: nu, domain, initial and boundary
    data of both Burgers generators."""
    g = _keys("burgers_eq_BE.txt")
    nu = eval(g["nu"], {"math": math})
    x_min, x_max = float(g["x_min"]), float(g["x_max"])
    for pb in (P.burgers_cpinn(n_res=50, n_iface=5, n_bc=40), P.burgers_spacetime(4, 2, n_res_total=800)):
        assert pb.nu == np.float32(nu) or abs(pb.nu - nu) < 1e-12
        for s in pb.subs:
            assert np.all((s.res_xy[:, 0] >= x_min) & (s.res_xy[:, 0] <= x_max) & (s.res_xy[:, 1] >= 0))
            if not s.data or s.data[0] is None:
                continue
            xy, v = s.data[0].xy.astype(np.float64), s.data[0].val[:, 0].astype(np.float64)
            ic = np.abs(xy[:, 1]) < 1e-12
            want_ic = np.array([eval(g["initial"], {"math": math, "x": x}) for x in xy[ic, 0]])
            assert np.allclose(v[ic], want_ic, atol=1e-6)
            bc = ~ic
            assert np.allclose(np.abs(xy[bc, 0]), max(abs(x_min), abs(x_max)))
            assert np.allclose(v[bc], float(g["boundary"]))


def test_inverse_diffusion_activations_follow_table_usmap():
    """Table Table_USmap: the activation of every region's networks, with
    trainable slopes (the table's column is the adaptive activation)."""
    rows = _rows("table_usmap.txt")
    pb = P.diffusion_xpinn(n_res=200, n_obs=20, n_iface=10, n_kbc=5, n_copies=1)
    names = {"tanh": P.PHI_TANH, "sin": P.PHI_SIN, "cos": P.PHI_COS}
    assert pb.n_sub == len(rows)
    for (idx, _n_res, act), s in zip(rows, pb.subs):
        for net in s.nets:
            assert net.act == names[act] and net.adaptive, (idx, act)


def test_space_time_burgers_partitions_of_table_tablevb():
    """Table TableVB and Sec. 7.5: 80k residual points spread over the
    subdomains, 20 points per interface, 5 x 20 tanh networks, lr 8e-4;
    cPINN partitions only x, XPINN partitions x and t."""
    for nx, nt, method in _rows("table_tablevb.txt"):
        nx, nt = int(nx), int(nt)
        m = P.CPINN if method == "cPINN" else P.XPINN
        pb = P.burgers_spacetime(nx, nt, method_x=m, method_t=P.XPINN)
        assert pb.n_sub == nx * nt
        assert sum(s.res_xy.shape[0] for s in pb.subs) == 80000
        assert all(s.res_xy.shape[0] == 80000 // (nx * nt) for s in pb.subs)
        assert all(it.xy.shape[0] == 20 for it in pb.ifaces)
        assert all(it.method == m for it in pb.ifaces) if nt == 1 else True
        for s in pb.subs:
            assert s.nets[0].widths == [2] + [20] * 5 + [1] and s.nets[0].act == P.PHI_TANH
            assert abs(s.lr - 8e-4) < 1e-12
