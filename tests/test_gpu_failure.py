"""Failure detection without a GPU fault: a device-side wait on a barrier that nothing
completes gives up after its bound and reports AZ_ETIMEOUT to the host, the context stays
usable, and the same wait with the barrier completed reports AZ_OK.  The wait is the
bounded mbarrier wait every staged kernel of the library uses."""
import numpy as np
import pytest

from gpu_common import Case, api, needs_gpu, rel_err, small_workload

pytestmark = [pytest.mark.gpu, needs_gpu]

AZ_OK, AZ_ETIMEOUT = 0, -7


def test_wait_that_nothing_completes_times_out():
    # about 1 ms of SM clock: the wait gives up and says so
    assert api().selftest_wait(arrive=False, limit_cycles=2_000_000) == AZ_ETIMEOUT


def test_completed_wait_succeeds():
    assert api().selftest_wait(arrive=True, limit_cycles=2_000_000) == AZ_OK


def test_context_usable_after_a_timeout():
    assert api().selftest_wait(arrive=False, limit_cycles=1_000_000) == AZ_ETIMEOUT
    w = small_workload(64, 80, npt=40, seed=21)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp64")
    for got, ref in zip(res, c.oracle()):
        per, norm = rel_err(got.cpu().numpy(), ref)
        assert per <= 1e-12 and norm <= 1e-12
    assert gpu.status() == AZ_OK
