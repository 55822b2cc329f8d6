"""Failure detection without a GPU fault: the cluster solve's exchange waits
are bounded; a wait on a barrier that nothing arrives on gives up after its
limit, sets the error bit that epd_lb_sync reports as EPD_LB_ETIMEOUT, and
leaves the context usable."""
import numpy as np
import pytest

import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_exchange_wait_gives_up_and_the_context_stays_usable():
    assert P.binding.selftest_bounded_wait(50) is True
    # the same device keeps working: a cluster-solve step and its densities
    r = W.with_(W.plain_small(), nx=64, ny=64, ns=16, precision=P.MIXED_FP32, f0=2.0)
    h = P.EpdLb([r])
    assert h.tiles(0)["path"] == 2
    h.step(2)
    h.sync()
    phi, q = h.densities(0)
    assert np.isfinite(phi).all() and q[0] > 0
    h.close()


def test_selftest_arguments_are_checked():
    with pytest.raises(P.EpdLbError):
        P.binding.selftest_bounded_wait(0)
    with pytest.raises(P.EpdLbError):
        P.binding.selftest_bounded_wait(5000)
