"""Failure detection without faulting the GPU.

* The in-kernel wait for the interface exchange is bounded: with the fault
  injected (it waits for one exchange item more than exists, a counter that
  nothing completes) it gives up after about a second, the call returns
  XPINN_ERR_TIMEOUT, and the same handle then computes the correct gradient.
* A loss that becomes non-finite during training is reported as
  XPINN_ERR_NONFINITE, not silently returned.
"""
import time

import numpy as np
import pytest

from oracle import Oracle
from paper_2104_10013_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2104_10013_gb300 import build as B
    from paper_2104_10013_gb300 import xpinn as X
    B.build()
    X.load()
    return X


def test_exchange_wait_times_out_and_the_handle_recovers(X):
    pb = P.burgers_cpinn(n_res=200, n_iface=20, n_bc=20)
    s = X.Solver(pb)
    s.set_options(inject_fault=1)
    t0 = time.perf_counter()
    with pytest.raises(X.XpinnError) as e:
        s.grad()
    assert e.value.code == -4                      # XPINN_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30
    s.set_options(inject_fault=0)
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    s.close()


def test_nonfinite_loss_is_reported(X):
    pb = P.burgers_cpinn(n_res=200, n_iface=20, n_bc=20)
    s = X.Solver(pb)
    theta = pb.packed_params()
    theta[:] = 3e19                                 # squares overflow float32
    s.set_params(theta)
    with pytest.raises(X.XpinnError) as e:
        s.step(1)
    assert e.value.code == -5                      # XPINN_ERR_NONFINITE
    s.close()
