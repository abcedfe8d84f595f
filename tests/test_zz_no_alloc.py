"""The allocation-free entry point, xpinn_residual_grad_noalloc.

It exists for callers that may not allocate device memory (a host framework
that owns the allocator, a fixed memory budget, a region that must not
allocate): their working memory comes from a fixed array built into the
library.  Its result must be the residual part of the ordinary gradient:
here it is compared, on two calls in a row (the second reuses the array the
first left behind), with xpinn_grad on a one-subdomain problem that has only
residual points, within the tolerances of the parity tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2104_10013_gb300 import problems as P

pytestmark = pytest.mark.gpu


def one_subdomain(pde, widths, n, seed=0):
    rng = np.random.default_rng(seed)
    net = P.NetSpec(widths)
    xy = P._f32(rng.uniform(0, 1, size=(n, 2)))
    f = P._f32(rng.normal(size=n)) if pde == P.PDE_POISSON else np.zeros(n, np.float32)
    sub = P.Subdomain(nets=[net], res_xy=xy, res_f=f, data=[None], w_data=[1.0], w_res=0.7,
                      rect=(0.0, 1.0, 0.0, 1.0))
    sub.params = [[(W * 1.3, P._f32(rng.normal(size=b.shape) * 0.2))
                   for W, b in P.xavier_params(net, rng)]]
    return P.Problem("one", pde, [sub], [], nu=0.01 / np.pi, re=40.0)


def net_desc(X, widths):
    d = X.NetDesc()
    d.n_layers = len(widths) - 1
    for k, w in enumerate(widths):
        d.widths[k] = w
    d.out_act = P.ACT_IDENTITY
    return d


@pytest.mark.parametrize("pde,widths,n", [
    (P.PDE_POISSON, [2, 40, 40, 40, 40, 1], 3001),
    (P.PDE_NS, [2, 64, 64, 64, 3], 2049),
    (P.PDE_BURGERS, [2, 20, 20, 20, 1], 777),
    # 6 x 64 at 50k points: its working set at one CTA per SM exceeds the
    # 32 MiB array, so the call runs on fewer CTAs
    (P.PDE_NS, [2, 64, 64, 64, 64, 64, 64, 3], 50000),
])
def test_noalloc_matches_grad_on_two_calls_in_a_row(pde, widths, n):
    import torch
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    lib = X.load()
    pb = one_subdomain(pde, widths, n)
    s = X.Solver(pb)
    losses, g_ref = s.grad()
    s.close()
    loss_ref = float(losses[0, 2])
    dev = torch.device("cuda", 0)
    theta = torch.from_numpy(pb.packed_params()).to(dev)
    xy = torch.from_numpy(pb.subs[0].res_xy).to(dev)
    f = torch.from_numpy(pb.subs[0].res_f).to(dev)
    desc = net_desc(X, widths)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        loss = torch.full((1,), float("nan"), device=dev)
        grads = torch.full((pb.n_params,), float("nan"), device=dev)
        rc = lib.xpinn_residual_grad_noalloc(pde, C.c_float(pb.nu), C.c_float(pb.re), C.byref(desc),
                                             theta.data_ptr(), xy.data_ptr(), f.data_ptr(), n,
                                             C.c_float(0.7), loss.data_ptr(), grads.data_ptr(), stream)
        assert rc == 0, lib.xpinn_last_error().decode()
        torch.cuda.synchronize()
        g = grads.cpu().numpy().astype(np.float64)
        l = float(loss.item())
        assert abs(l - loss_ref) <= 1e-5 * abs(loss_ref), (call, l, loss_ref)
        rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
        mx = np.abs(g - g_ref).max() / np.abs(g_ref).max()
        assert rel <= 1e-4 and mx <= 1e-4, (call, rel, mx)


def test_noalloc_rejects_bad_requests_before_launching():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    lib = X.load()
    desc = net_desc(X, [2, 16, 16, 1])
    buf = (C.c_float * 8)()
    p = C.cast(buf, C.c_void_p)
    # NULL output
    assert lib.xpinn_residual_grad_noalloc(1, 0.0, 1.0, C.byref(desc), p, p, p, 4, 1.0, None, p, None) == -1
    # two-network PDE is outside what the entry point covers
    assert lib.xpinn_residual_grad_noalloc(3, 0.0, 1.0, C.byref(desc), p, p, p, 4, 1.0, p, p, None) == -6
    assert lib.xpinn_last_error()
    # width beyond the limit
    bad = net_desc(X, [2, 500, 1])
    assert lib.xpinn_residual_grad_noalloc(1, 0.0, 1.0, C.byref(bad), p, p, p, 4, 1.0, p, p, None) == -1


def _call(lib, X, pde, desc, theta, xy, f, n, loss, grads, stream, nu=0.0, re=40.0):
    return lib.xpinn_residual_grad_noalloc(pde, C.c_float(nu), C.c_float(re), C.byref(desc),
                                           theta.data_ptr(), xy.data_ptr(), f.data_ptr(), n,
                                           C.c_float(0.7), loss.data_ptr(), grads.data_ptr(), stream)


def test_noalloc_with_no_points_gives_zero_loss_and_gradient():
    import torch
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    lib = X.load()
    widths = [2, 16, 16, 1]
    pb = one_subdomain(P.PDE_POISSON, widths, 4)
    dev = torch.device("cuda", 0)
    theta = torch.from_numpy(pb.packed_params()).to(dev)
    xy = torch.zeros((1, 2), device=dev)
    f = torch.zeros((1,), device=dev)
    loss = torch.full((1,), float("nan"), device=dev)
    grads = torch.full((pb.n_params,), float("nan"), device=dev)
    rc = _call(lib, X, P.PDE_POISSON, net_desc(X, widths), theta, xy, f, 0, loss, grads,
               torch.cuda.current_stream(dev).cuda_stream)
    assert rc == 0, lib.xpinn_last_error().decode()
    torch.cuda.synchronize()
    assert float(loss.item()) == 0.0 and bool((grads == 0).all())


def test_noalloc_device_error_gives_nan_outputs_and_the_next_call_recovers():
    """The device error word is preset (testing hook) as if a bounded wait
    had given up: the asynchronous call cannot return the error, so its loss
    and gradient come out NaN; the next call, without the preset, is right."""
    import torch
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    lib = X.load()
    widths = [2, 24, 24, 1]
    n = 500
    pb = one_subdomain(P.PDE_POISSON, widths, n)
    s = X.Solver(pb)
    losses, g_ref = s.grad()
    s.close()
    dev = torch.device("cuda", 0)
    theta = torch.from_numpy(pb.packed_params()).to(dev)
    xy = torch.from_numpy(pb.subs[0].res_xy).to(dev)
    f = torch.from_numpy(pb.subs[0].res_f).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    desc = net_desc(X, widths)
    for preset in (-4, 0):
        lib.xpinn_noalloc_debug_preset_error(preset)
        loss = torch.zeros((1,), device=dev)
        grads = torch.zeros((pb.n_params,), device=dev)
        assert _call(lib, X, P.PDE_POISSON, desc, theta, xy, f, n, loss, grads, stream) == 0
        torch.cuda.synchronize()
        if preset:
            assert bool(torch.isnan(loss).all()) and bool(torch.isnan(grads).all())
        else:
            g = grads.cpu().numpy().astype(np.float64)
            assert abs(float(loss.item()) - float(losses[0, 2])) <= 1e-5 * abs(float(losses[0, 2]))
            assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
