"""Host arithmetic of bench.py's roofline lines (no GPU): the algorithmic
FLOP count of 6 K M per residual point, over all subdomains or the ones the
tensor-core kernel trains, and that kernel's executed tensor work at the
padded width."""
import numpy as np

import bench
from paper_2104_10013_gb300 import problems as P


def test_algorithmic_flops_counts_each_network_once_per_point():
    pb = P.kovasznay_cpinn(nx=2, ny=1, n_res=100, n_iface=8, n_bc=10)
    # 2 -> 64 x 6 -> 3: M = 5 x 64 x 64 + 3 x 64, K = 4 Laplacian-jet components
    m = 5 * 64 * 64 + 3 * 64
    assert bench.algorithmic_flops(pb) == 6 * 4 * m * pb.n_res
    assert bench.algorithmic_flops(pb, {1}) == 6 * 4 * m * pb.subs[1].res_xy.shape[0]
    assert bench.algorithmic_flops(pb, set()) == 0


def test_inverse_diffusion_counts_both_networks():
    pb = P.diffusion_xpinn(n_res=50, n_obs=5, n_iface=4, n_kbc=3, n_copies=1)
    per_pt = 6 * 4 * (4 * 40 * 40 + 40) + 6 * 3 * (3 * 20 * 20 + 20)   # u-net K = 4, K-net K = 3
    assert bench.algorithmic_flops(pb) == per_pt * pb.n_res


class _FakeSolver:
    """plan_counts / tc_subdomains / tc_kernel_ms of a Solver whose
    tensor-core kernel trains subdomains `on` in `ms` milliseconds."""

    def __init__(self, on, ms):
        self.on = np.asarray(on, np.int32)
        self.tc_ms = [ms]

    def plan_counts(self):
        return 10, 4, int(self.on.sum())

    def tc_subdomains(self):
        return self.on


def test_tensor_core_roofline_counts_only_its_subdomains():
    pb = P.poisson_xpinn(nx=2, ny=2, n_res_range=(100, 200), width_range=(40, 64), depth_range=(2, 4),
                         n_iface=8, n_bc=10, seed=3)
    on = [1, 0, 1, 0]
    r = bench.roofline_tc(pb, _FakeSolver(on, 2.0), 4.0)
    assert r["flop_per_launch"] == bench.algorithmic_flops(pb, {0, 2})
    assert r["achieved"] == r["flop_per_launch"] / 2e-3 / 1e12
    assert r["kernel_share_of_step"] == 0.5
    # executed: the hidden-to-hidden layers at width 64, 10/3 of 6 K (64 x 64) per layer and point
    ex = sum(10.0 / 3.0 * 6 * 4 * (len(pb.subs[q].nets[0].widths) - 3) * 64 * 64 * pb.subs[q].res_xy.shape[0]
             for q in (0, 2))
    assert np.isclose(r["executed_tensor_flop_per_launch"], ex)
    assert bench.roofline_tc(pb, type("S", (), {"plan_counts": lambda self: (10, 0, 0)})(), 4.0) is None
