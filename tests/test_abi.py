"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/epd_lb.h declares; parameter checks need no device."""
import os
import re

import pytest

import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "epd_lb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(epd_\w+)\s*\(", txt)))


def test_header_declares_binding_symbols():
    assert sorted(P.SYMBOLS) == declared_symbols()


def test_library_exports_every_declared_symbol():
    L = P.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_workspace_sizes_without_gpu():
    small = P.epd_lb_workspace_bytes([W.plain_small()])
    assert small > 0 and small % 256 == 0
    # the 4-run channel batch needs about 4x one run
    one = P.epd_lb_workspace_bytes(W.channel_256x512()[:1])
    four = P.epd_lb_workspace_bytes(W.channel_256x512())
    assert 3.5 * one < four < 4.5 * one


def test_mixed_radix_grids_accepted():
    # even lengths of the form 2^a 3^b 5^c: the paper's own 150 x 150 grid
    for nx, ny in ((150, 150), (96, 60), (30, 20), (2048, 1536)):
        assert P.epd_lb_workspace_bytes([W.with_(W.plain_small(), nx=nx, ny=ny)]) > 0
    # odd N_s (the paper's N_s = N = 17) on the radix-2 streaming solve
    assert P.epd_lb_workspace_bytes(W.paper_150(P.MIXED_FP32)) > 0
    assert P.epd_lb_workspace_bytes([W.with_(W.plain_small(), ns=17)]) > 0


@pytest.mark.parametrize("bad", [dict(nx=14), dict(nx=75), dict(ny=4), dict(ns=7, precision=1), dict(ns=0), dict(precision=2),
                                 dict(phi_p=1.0), dict(gamma_s=1.0), dict(dx=0.0), dict(nx=4096), dict(ny=2250)])
def test_invalid_parameters_rejected(bad):
    p = W.with_(W.plain_small(), **bad)
    with pytest.raises(P.EpdLbError) as ei:
        P.epd_lb_workspace_bytes([p])
    assert ei.value.code == -1
