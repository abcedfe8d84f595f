"""Failure detection without faulting the GPU.

* The in-kernel wait for the interface exchange is bounded: with the fault
  injected (it waits for one exchange item more than exists, a counter that
  nothing completes) it gives up after about a second, the call returns
  XPINN_ERR_TIMEOUT, and the same handle then computes the correct gradient.
* A loss that becomes non-finite during training is reported as
  XPINN_ERR_NONFINITE, not silently returned.
* Steps queued without host losses (NULL or device buffers) do not
  synchronise; a timeout or a non-finite loss among them is kept in the
  handle's device status word and returned by the next synchronising call
  (xpinn_sync), after which the handle works again.
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


def test_async_step_timeout_is_reported_by_the_next_sync(X):
    pb = P.burgers_cpinn(n_res=200, n_iface=20, n_bc=20)
    s = X.Solver(pb)
    s.set_options(inject_fault=1)
    assert s.step(1, losses=None) is None           # queued; returns without waiting
    with pytest.raises(X.XpinnError) as e:
        s.sync()
    assert e.value.code == -4                       # XPINN_ERR_TIMEOUT
    s.sync()                                        # read once, then cleared
    s.set_options(inject_fault=0)
    s.set_params(pb.packed_params())
    losses, g = s.grad()
    terms, g_ref = Oracle(pb).grad(pb.packed_params())
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    s.close()


def test_async_step_timeout_with_device_losses(X):
    import torch
    pb = P.burgers_cpinn(n_res=200, n_iface=20, n_bc=20)
    s = X.Solver(pb)
    s.set_options(inject_fault=1)
    dl = torch.zeros((1, pb.n_sub, P.N_TERMS), dtype=torch.float32, device="cuda")
    s.step(1, losses=dl)
    with pytest.raises(X.XpinnError) as e:
        s.sync(torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -4
    s.close()


def test_nonfinite_loss_of_async_steps_is_reported_by_sync(X):
    pb = P.burgers_cpinn(n_res=200, n_iface=20, n_bc=20)
    s = X.Solver(pb)
    theta = pb.packed_params()
    theta[:] = 3e19                                 # squares overflow float32
    s.set_params(theta)
    s.step(2, losses=None)
    with pytest.raises(X.XpinnError) as e:
        s.sync()
    assert e.value.code == -5                       # XPINN_ERR_NONFINITE
    s.set_params(pb.packed_params())
    s.sync()
    assert np.all(np.isfinite(s.step(1)))
    s.close()
