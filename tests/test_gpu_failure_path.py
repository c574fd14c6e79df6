"""The device-side failure path, exercised without any GPU fault: a wait on
a barrier that nothing completes gives up after its limit and reports
MBAR_ETIMEOUT; afterwards the device and a new context work normally."""
import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports_a_timeout():
    status, waited = M.selftest_wait_timeout(50_000)
    assert status == "MBAR_ETIMEOUT"
    assert 0.05 <= waited < 1.0
    assert "gave up" in M.lib().mbar_last_error().decode()


def test_the_device_is_usable_after_a_timeout():
    M.selftest_wait_timeout(20_000)
    p = W.harmonic(K=6, d=3, N_k=500, seed=1)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_FP64)
    ctx.solve()
    f = ctx.free_energies()
    ctx.close()
    assert np.max(np.abs(f - O.solve_mbar(p.u_kn, p.N_k))) < 1e-8


def test_limit_is_validated():
    status, _ = M.selftest_wait_timeout(0)
    assert status == "MBAR_EINVAL"
