"""Evaluation on the tensor cores (option eval_tensor_cores): the forward
jets of Eq. FSol's stitched solution with the hidden-to-hidden contractions
as tcgen05 TF32 MMAs over a hi/lo split of both operands.

* every order (u; u, u_x, u_y; u, u_x, u_y, u_xx, u_yy) matches the FP64
  oracle within the jet tolerance, for hidden widths 32, 64 and 80, two to
  five hidden-to-hidden layers, tanh with fixed slopes and tanh/sin/cos with
  trained slopes, at point counts that leave ragged tiles, on the cuts
  between subdomains (1/S averages) and outside the domain (NaN);
* the result is deterministic and within twice the tolerance of the FP32 jet
  kernel's;
* models that do not qualify (several widths, two networks, a softplus
  output) are evaluated by the jet kernel, bit for bit as without the option;
* the images follow the parameters after training steps;
* the workspace entry point with device buffers gives the same bits.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2104_10013_gb300 import problems as P
from tests.cases import with_activations
from tests.test_parity import RTOL_JET, X, assert_scaled, small_c2, small_c4  # noqa: F401

pytestmark = pytest.mark.gpu


def kovasznay(width, depth, acts=None, adaptive=True, seed=0):
    pb = P.kovasznay_cpinn(nx=3, ny=2, n_res=400, n_iface=32, n_bc=40, width=width, depth=depth, seed=seed)
    if acts:
        pb = with_activations(pb, acts, adaptive=adaptive, seed=seed)
    return pb


def query_points(pb, n=2037, seed=5):
    rng = np.random.default_rng(seed)
    x0, x1, y0, y1 = -0.5, 1.0, -0.5, 1.5
    xy = np.stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n)], 1)
    xc, yc = pb.meta["xcuts"], pb.meta["ycuts"]
    cuts = np.array([[xc[1], 0.1], [0.2, yc[1]], [xc[1], yc[1]], [xc[2], yc[1]]])
    return np.concatenate([xy, cuts, [[7.0, 7.0]]]).astype(np.float32)


def tc_eval(s, xy, order, on=1):
    s.set_options(eval_tensor_cores=on)
    out = s.eval(0, xy, order)
    s.sync()
    return out


CASES_TC = {
    "w64_d6_tanh_fixed": dict(width=64, depth=6, acts=None),
    "w32_d3_sin_cos_tanh_trained": dict(width=32, depth=3, acts=[P.PHI_SIN, P.PHI_COS, P.PHI_TANH]),
    "w80_d4_tanh_sin_trained": dict(width=80, depth=4, acts=[P.PHI_TANH, P.PHI_SIN]),
}


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("case", list(CASES_TC))
def test_tensor_core_eval_matches_the_oracle(X, case, order):
    pb = kovasznay(**CASES_TC[case])
    s = X.Solver(pb)
    xy = query_points(pb)
    got = tc_eval(s, xy, order)
    ref = Oracle(pb).eval_stitched(pb.packed_params(), 0, xy, (1, 3, 5)[order])
    assert np.isnan(got[-1]).all() and np.isnan(ref[-1]).all()
    assert_scaled(got[:-1], ref[:-1], RTOL_JET, f"tensor-core eval {case} order {order}", axis=(0, 1))
    s.close()


def test_tensor_core_eval_is_deterministic_and_near_the_jet_kernel(X):
    pb = kovasznay(64, 5, acts=[P.PHI_TANH, P.PHI_COS])
    s = X.Solver(pb)
    xy = query_points(pb, n=5001)
    for order in (0, 1, 2):
        a = tc_eval(s, xy, order)
        b = tc_eval(s, xy, order)
        assert np.array_equal(a, b, equal_nan=True)
        simt = tc_eval(s, xy, order, on=0)
        assert_scaled(a[:-1], simt[:-1], 2 * RTOL_JET, f"tensor cores vs jet kernel, order {order}", axis=(0, 1))
    s.close()


@pytest.mark.parametrize("name", ["poisson_uneven_widths", "diffusion_two_networks"])
def test_models_that_do_not_qualify_keep_the_jet_kernel(X, name):
    pb = {"poisson_uneven_widths": small_c2, "diffusion_two_networks": small_c4}[name]()
    s = X.Solver(pb)
    rng = np.random.default_rng(2)
    lo = np.min([sd.res_xy.min(0) for sd in pb.subs], 0)
    hi = np.max([sd.res_xy.max(0) for sd in pb.subs], 0)
    xy = rng.uniform(lo, hi, (1500, 2)).astype(np.float32)
    for order in (0, 2):
        off = tc_eval(s, xy, order, on=0)
        on = tc_eval(s, xy, order, on=1)
        assert np.array_equal(off, on, equal_nan=True)
    s.close()


def test_tensor_core_eval_follows_training(X):
    pb = kovasznay(64, 4, acts=[P.PHI_SIN, P.PHI_TANH])
    s = X.Solver(pb)
    xy = query_points(pb, n=800)
    tc_eval(s, xy, 2)                       # images built for the initial parameters
    s.step(3)
    got = tc_eval(s, xy, 2)
    theta = s.get_params().astype(np.float32)
    assert not np.array_equal(theta, pb.packed_params())
    ref = Oracle(pb).eval_stitched(theta, 0, xy, 5)
    assert_scaled(got[:-1], ref[:-1], RTOL_JET, "tensor-core eval after training", axis=(0, 1))
    s.close()


def test_tensor_core_eval_from_workspace_is_bitwise_equal(X):
    import torch
    pb = kovasznay(80, 3)
    s = X.Solver(pb)
    xy = query_points(pb, n=3000)
    s.set_options(eval_tensor_cores=1)
    for order in (0, 1, 2):
        ref_host = s.eval(0, xy, order)
        ws = torch.empty(s.eval_workspace_size(len(xy), order), dtype=torch.uint8, device="cuda")
        dxy = torch.from_numpy(xy).cuda()
        dout = torch.full(ref_host.shape, float("nan"), device="cuda")
        s.eval_ws(0, dxy, order, dout, ws)
        torch.cuda.synchronize()
        s.sync()
        assert np.array_equal(dout.cpu().numpy(), ref_host, equal_nan=True)
    s.close()
