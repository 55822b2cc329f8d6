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


@pytest.mark.parametrize("prec,shape", [(P.PLAIN_FP64, (32, 64)), (P.MIXED_FP32, (64, 64)), (P.MIXED_FP32, (64, 1024))])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_field_is_reported_by_sync(prec, shape, bad):
    # a failure made on the host: one non-finite omega value handed in through
    # epd_lb_set_state makes the next solve's Q non-finite, which the device
    # error word carries to epd_lb_sync as EPD_LB_ENONFINITE (streaming FP64,
    # cluster-resident and radix-8 streaming solves)
    ny, nx = shape
    r = W.with_(W.plain_small(), nx=nx, ny=ny, ns=8, precision=prec, f0=2.0)
    h = P.EpdLb([r])
    h.step(1)
    h.sync()
    om, pop, vel = h.get_state(0)
    om[1, ny // 3, nx // 5] = bad
    h.set_state(0, om, pop, vel)
    h.step(1)
    with pytest.raises(P.EpdLbError) as ei:
        h.sync()
    assert ei.value.code == -4
    h.close()
    # the context stays usable: a fresh handle steps cleanly
    h2 = P.EpdLb([r])
    h2.step(1)
    h2.sync()
    h2.close()


def test_short_workspace_is_refused():
    # EPD_LB_ENOMEM for a caller workspace one byte short or misaligned; the
    # library checks before touching the memory
    import ctypes

    import torch

    runs = [W.with_(W.plain_small(), nx=32, ny=32, ns=8, precision=P.MIXED_FP32)]
    need = P.binding.epd_lb_workspace_bytes(runs)
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) & ~255
    st = torch.cuda.Stream()
    h = ctypes.c_void_p()
    arr = P.binding._params_array(runs)
    lib = P.lib()
    assert lib.epd_lb_init(arr, 1, base, need - 1, st.cuda_stream, ctypes.byref(h)) == -2
    assert lib.epd_lb_init(arr, 1, base + 8, need, st.cuda_stream, ctypes.byref(h)) == -2
    assert lib.epd_lb_init(arr, 1, base, need, st.cuda_stream, ctypes.byref(h)) == 0
    lib.epd_lb_step(h, 1)
    assert lib.epd_lb_sync(h) == 0
    lib.epd_lb_destroy(h)
