"""Why the tensor-core kernels take three TF32 products per term: a CPU
emulation of the forward jet contraction of the Navier-Stokes workload's
network (2 -> 64 x 6 -> 3, Laplacian jets; the widest uniform layers of the
five workloads) with float32 accumulation in the kernel's order, against the
FP64 oracle in the jet parity metric (1e-5 of max(|b|, RMS over the points
and outputs)).  One TF32 product per term misses the tolerance by two orders
of magnitude; three products over a hi/lo split of both operands (the form
the evaluation and training kernels use) meet it, as plain FP32 does."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2104_10013_gb300 import problems as P

RTOL_JET = 1e-5


def _tf32(a):
    """Round float32 to TF32 (10 explicit mantissa bits), to nearest even."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0xFFF + ((u >> 13) & 1)) & ~np.uint64(0x1FFF)
    return u.astype(np.uint32).view(np.float32)


def _contract(H, W, mode):
    """[n, K, j] x [o, j] -> [n, K, o], float32 sums in j order."""
    if mode == "fp32":
        terms = [(H, W)]
    elif mode == "tf32":
        terms = [(_tf32(H), _tf32(W))]
    else:
        Hh, Wh = _tf32(H), _tf32(W)
        terms = [(Hh, Wh), (Hh, _tf32(W - Wh)), (_tf32(H - Hh), Wh)]
    acc = np.zeros(H.shape[:2] + (W.shape[0],), np.float32)
    for j in range(W.shape[1]):
        for h, w in terms:
            acc = acc + h[:, :, j:j + 1] * w[None, None, :, j]
    return acc


def _jets(layers, xy, mode):
    W, b = layers[0]
    z = xy @ W.T + b
    Z = np.stack([z, np.broadcast_to(W[:, 0], z.shape), np.broadcast_to(W[:, 1], z.shape),
                  np.zeros_like(z)], 1).astype(np.float32)
    for W, b in layers[1:]:
        t = np.tanh(Z[:, 0])
        s = 1 - t * t
        H = np.stack([t, s * Z[:, 1], s * Z[:, 2], s * Z[:, 3] - 2 * t * s * (Z[:, 1] ** 2 + Z[:, 2] ** 2)], 1)
        Z = _contract(H.astype(np.float32), W.astype(np.float32), mode)
        Z[:, 0] += b
    return Z.transpose(0, 2, 1)   # [n, out, (u, u_x, u_y, lap u)]


@pytest.fixture(scope="module")
def case():
    pb = P.kovasznay_cpinn(nx=3, ny=3, n_res=200, n_iface=16, n_bc=16)
    q = 4
    x0, x1, y0, y1 = pb.subs[q].rect
    rng = np.random.default_rng(1)
    xy = np.stack([rng.uniform(x0, x1, 600), rng.uniform(y0, y1, 600)], 1).astype(np.float32)
    ref = Oracle(pb).net_jets(pb.packed_params(), q, 0, xy, 5)      # u, u_x, u_y, u_xx, u_yy
    ref = np.concatenate([ref[:, :, :3], (ref[:, :, 3] + ref[:, :, 4])[:, :, None]], 2)
    return pb.subs[q].params[0], xy, ref


def _scaled_error(a, ref):
    rms = np.sqrt((ref ** 2).mean(axis=(0, 1), keepdims=True))
    return float((np.abs(a - ref) / np.maximum(np.abs(ref), rms)).max())


def test_tf32_rounding_is_exact_on_tf32_values_and_halves_to_even():
    x = np.array([1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11], np.float32)
    assert np.array_equal(_tf32(x), np.array([1.0, 1.0 + 2.0 ** -10, 1.0, 1.0 + 2.0 ** -9], np.float32))


@pytest.mark.parametrize("mode,ok", [("fp32", True), ("tf32", False), ("3xtf32", True)])
def test_contraction_precision_against_the_jet_tolerance(case, mode, ok):
    layers, xy, ref = case
    e = _scaled_error(_jets(layers, xy, mode), ref)
    if ok:
        assert e <= RTOL_JET, e
    else:
        assert e >= 20 * RTOL_JET, e
