"""The allocation-free single-chain solve (epd_prop_solve_noalloc) against the
workspace entry point (epd_prop_solve).

epd_prop_solve_noalloc serves callers that cannot allocate device memory at
the time of the call (inside a host framework that owns the device's memory,
in allocation-free real-time loops);
its scratch is a fixed array inside the library.  The test calls it twice in
a row through the C ABI (the second call reuses the scratch left by the
first) and compares both results with epd_prop_solve, within the tolerances
of the other GPU tests.  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest

import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {P.PLAIN_FP64: 1e-10, P.MIXED_FP32: 2e-6}


def _solve_with_workspace(torch, r, om_d):
    nb = P.epd_prop_solve_workspace_bytes(r)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wptr = (ws.data_ptr() + 255) & ~255
    phi = torch.empty_like(om_d)
    q = torch.empty(2, dtype=torch.float64, device="cuda")
    P.epd_prop_solve(r, om_d.data_ptr(), phi.data_ptr(), q.data_ptr(), wptr, nb, 0)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), q.cpu().numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
@pytest.mark.parametrize("ny,nx,ns", [(64, 128, 16), (128, 128, 64)])
def test_noalloc_matches_workspace_solve_twice(prec, ny, nx, ns):
    torch = pytest.importorskip("torch")
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=prec, f_a=0.4, phi_p=0.2)
    om_d = torch.from_numpy(W.random_omega(ny, nx, seed=ny + ns)).cuda()
    ref_phi, ref_q = _solve_with_workspace(torch, r, om_d)
    torch.cuda.synchronize()
    mem = None
    for _ in range(2):
        phi = torch.full_like(om_d, float("nan"))
        q = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
        P.epd_prop_solve_noalloc(r, om_d.data_ptr(), phi.data_ptr(), q.data_ptr(), 0)
        torch.cuda.synchronize()
        after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
        # torch's pool is untouched, and from the second call on (the first may
        # load the library's device image) the device's free memory too
        assert after[1] == before[1]
        if mem is not None:
            assert after[0] == before[0]
        mem = after[0]
        assert _rel(phi.cpu().numpy(), ref_phi) < TOL[prec]
        assert _rel(q.cpu().numpy(), ref_q) < TOL[prec]


def test_noalloc_rejects_problems_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    r = P.RunParams(nx=512, ny=256, ns=64, precision=P.MIXED_FP32)
    om_d = torch.zeros((3, 256, 512), dtype=torch.float64, device="cuda")
    phi = torch.empty_like(om_d)
    q = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.EpdLbError) as ei:
        P.epd_prop_solve_noalloc(r, om_d.data_ptr(), phi.data_ptr(), q.data_ptr(), 0)
    assert ei.value.code == -8
