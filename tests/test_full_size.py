"""Full-size workloads in the benchmark's launch configuration (grouped,
autotuned defaults): the GPU computes every subdomain; the FP64 oracle, which
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


def check_sample(X, pb, sample):
    s = X.Solver(pb)
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
    check_sample(X, pb, [3, 1234, 2559])
