"""Failure detection without a GPU fault: the bounded device wait that guards
every TMA tile copy gives up after its time limit, the kernel records it in
the error flags and returns, ap_dvm_sync_status reports AP_DVM_ERR_TIMEOUT
once, and the context stays usable (ap_dvm_check_wait_timeout waits on an
mbarrier that nothing completes; no copy is in flight)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_19847_gb300 import api, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_the_context_stays_usable():
    n = 64
    X0 = W.random_moment_state(n, n, seed=61, amp=0.3)
    p = api.default_params(n, n, eps=1e-2, dt=0.01)
    s = api.Solver(p)
    s.set_state(torch.from_numpy(X0).cuda())
    t0 = time.perf_counter()
    s.check_wait_timeout(50_000_000)                  # 50 ms
    with pytest.raises(api.ApDvmError) as e:
        s.sync_status()
    assert e.value.status == 6                          # AP_DVM_ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.05
    s.sync_status()                                     # reported once, then cleared
    s.step(3)
    s.sync_status()
    ref = api.Solver(p)
    ref.set_state(torch.from_numpy(X0).cuda())
    ref.step(3)
    assert np.array_equal(s.get_state().cpu().numpy(), ref.get_state().cpu().numpy())


def test_wait_limit_is_validated():
    s = api.Solver(api.default_params(32, 32, eps=1e-2, dt=0.01))
    for bad in (0, 999, 10_000_000_001):
        with pytest.raises(api.ApDvmError):
            s.check_wait_timeout(bad)
    s.sync_status()
