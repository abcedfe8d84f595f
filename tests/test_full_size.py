"""Full-size workloads in the benchmark's launch configuration (grouped;
the inverse-diffusion headline with the autotuned options the benchmark
picks): the GPU computes every subdomain; the FP64 oracle, which
cannot do the whole problem in seconds, checks a sample of whole subdomains
(their loss terms and every gradient tensor), chosen to include interior and
boundary subdomains and, for the copies, the first and last copy."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2104_10013_gb300 import problems as P
from tests.test_parity import RTOL_GRAD, RTOL_JET, assert_scaled, tensor_slices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    return X


def check_sample(X, pb, sample, autotune=False):
    s = X.Solver(pb)
    if autotune:            # the tile options the benchmark times
        s.autotune(steps=1)
    losses, g = s.grad()
    s.close()
    orc = Oracle(pb)
    terms, g_ref = orc.grad(pb.packed_params(), subset=sample)
    # losses of the sampled subdomains; scale: rms of each term over the sample
    assert_scaled(losses[sample], terms, RTOL_JET, "losses", axis=0)
    slices = dict(tensor_slices(pb))
    for q in sample:
        for name, sl in slices.items():
            if not name.startswith(f"q{q}n"):
                continue
            a, b = g[sl].astype(np.float64), g_ref[sl]
            nb = np.linalg.norm(b)
            rel = np.linalg.norm(a - b) / nb
            mx = np.abs(a - b).max() / np.abs(b).max()
            assert rel <= RTOL_GRAD and mx <= RTOL_GRAD, (name, rel, mx)


def test_kovasznay_full_size_sampled():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    pb = P.kovasznay_cpinn()
    assert pb.n_res == 3_200_000
    check_sample(X, pb, [0, 27, 63])


def test_inverse_diffusion_256_copies_sampled():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    pb = P.diffusion_xpinn()
    assert pb.n_sub == 2560 and pb.n_params == 256 * (80620 + 10 * (5 + 4))   # weights, biases; slopes
    check_sample(X, pb, [3, 1234, 2559], autotune=True)


def test_kovasznay_gradient_against_central_differences_at_step_0():
    """The Navier-Stokes cPINN workload's weight gradients from the GPU at the
    initial parameters, against FP64 central differences of J_q (neighbours'
    networks unchanged) for sampled weights of every layer of two subdomains:
    the check the Navier-Stokes configuration asks for, without the oracle's
    own gradient in between."""
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    import torch
    B.build()
    X.load()
    pb = P.kovasznay_cpinn(nx=3, ny=3, n_res=400, n_iface=48, n_bc=40)
    s = X.Solver(pb)
    _, g = s.grad()
    s.close()
    orc = Oracle(pb)
    W = orc.weights()
    theta = pb.packed_params().astype(np.float64)
    rng = np.random.default_rng(3)
    slices = tensor_slices(pb)
    h = 1e-6
    for q in (0, 4):
        gq = np.concatenate([g[sl] for name, sl in slices if name.startswith(f"q{q}n")])
        scale = np.abs(gq).max()
        for name, sl in slices:
            if not name.startswith(f"q{q}n"):
                continue
            for i in rng.choice(np.arange(sl.start, sl.stop), 2, replace=False):
                tp, tm = theta.copy(), theta.copy()
                tp[i] += h
                tm[i] -= h
                jp = (orc.loss_terms(torch.tensor(tp), subset=[q]).detach().numpy()[0] * W[q]).sum()
                jm = (orc.loss_terms(torch.tensor(tm), subset=[q]).detach().numpy()[0] * W[q]).sum()
                fd = (jp - jm) / (2 * h)
                assert abs(g[i] - fd) <= 1e-4 * scale, (name, i, g[i], fd)
