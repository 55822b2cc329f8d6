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
                                 dict(phi_p=1.0), dict(gamma_s=1.0), dict(dx=0.0), dict(nx=4096), dict(ny=2250),
                                 dict(junction_rule=2), dict(junction_rule=-1)])
def test_invalid_parameters_rejected(bad):
    p = W.with_(W.plain_small(), **bad)
    with pytest.raises(P.EpdLbError) as ei:
        P.epd_lb_workspace_bytes([p])
    assert ei.value.code == -1


def _rc(fn, *args):
    return getattr(P.lib(), fn)(*args)


def test_empty_and_null_arguments_rejected():
    import ctypes

    n = ctypes.c_size_t(7)
    one = P.binding._params_array([W.plain_small()])
    assert _rc("epd_lb_workspace_bytes", one, 0, ctypes.byref(n)) == -1
    assert _rc("epd_lb_workspace_bytes", None, 1, ctypes.byref(n)) == -1
    assert _rc("epd_lb_workspace_bytes", one, 1, None) == -1
    assert n.value == 7  # nothing written on failure
    h = ctypes.c_void_p(0)
    assert _rc("epd_lb_init", one, 0, None, 0, None, ctypes.byref(h)) == -1 and not h.value
    assert _rc("epd_lb_init", None, 1, None, 0, None, ctypes.byref(h)) == -1 and not h.value
    assert _rc("epd_lb_init", one, 1, None, 0, None, None) == -1
    c = W.plain_small().c()
    assert _rc("epd_prop_solve_workspace_bytes", None, ctypes.byref(n)) == -1
    assert _rc("epd_prop_solve_workspace_bytes", ctypes.byref(c), None) == -1
    # the stateless solve checks its pointers before touching the device
    assert _rc("epd_prop_solve", ctypes.byref(c), None, None, None, None, 0, None) == -1
    assert _rc("epd_sur_workspace_bytes", 32, 64, 0, 0, ctypes.byref(n)) == -1
    assert _rc("epd_sur_workspace_bytes", 32, 40, 1, 0, ctypes.byref(n)) == -1
    assert _rc("epd_sur_workspace_bytes", 36, 64, 1, 0, ctypes.byref(n)) == -1
    assert _rc("epd_sur_workspace_bytes", 24, 64, 1, 0, ctypes.byref(n)) == -1  # ny a multiple of 16
    assert _rc("epd_sur_workspace_bytes", 32, 64, 1, 0, None) == -1
    assert _rc("epd_lb_surrogate_workspace_bytes", None, ctypes.byref(n)) == -1
    assert n.value == 7


def test_mach_preflight_refuses_before_any_device_call():
    import ctypes

    h = ctypes.c_void_p(0)
    fast = P.binding._params_array([W.with_(W.plain_small(), f0=1e9)])
    assert _rc("epd_lb_init", fast, 1, None, 0, None, ctypes.byref(h)) == -5 and not h.value


def test_box_rules_of_the_3d_entry_points():
    run = W.with_(W.plain_small(), nx=32, ny=32, ns=8)
    solve = P.epd_prop_solve3d_workspace_bytes(run, 16)
    # the coupled 3D step holds the solve's workspace and more
    import ctypes

    n = ctypes.c_size_t()
    assert _rc("epd_step3d_workspace_bytes", ctypes.byref(run.c()), 16, ctypes.byref(n)) == 0
    assert n.value > solve > 0
    assert P.epd_prop_solve3d_workspace_bytes(W.with_(run, nx=30, ny=20), 12) > 0  # mixed radix
    for nz in (0, 7, 14, 4096):  # odd, not 2^a 3^b 5^c, beyond the longest axis
        with pytest.raises(P.EpdLbError):
            P.epd_prop_solve3d_workspace_bytes(run, nz)
    with pytest.raises(P.EpdLbError):  # 2^23 sites: beyond the 2^22-site limit
        P.epd_prop_solve3d_workspace_bytes(W.with_(run, nx=256, ny=256), 128)
    assert _rc("epd_step3d_workspace_bytes", ctypes.byref(run.c()), 7, ctypes.byref(n)) == -1
    assert _rc("epd_prop_solve3d_workspace_bytes", None, 16, ctypes.byref(n)) == -1


def test_runs_group_by_everything_but_f0_seed_and_noise():
    # the workspace of separate groups adds up (one head shared), while runs
    # of one group share their tables: grouping is visible without a device
    a = W.with_(W.plain_small(), precision=P.MIXED_FP32)
    ws = P.epd_lb_workspace_bytes
    b = W.with_(a, ns=24)
    c = W.with_(a, phi_p=0.25)
    head = ws([a]) + ws([b]) - ws([a, b])
    assert head > 0 and head % 256 == 0
    assert ws([a]) + ws([c]) - ws([a, c]) == head
    for field in ("chi_bs", "kappa_h", "d_p", "inv_beta_v", "gamma_s", "dt", "f_a", "precision", "junction_rule"):
        v = getattr(a, field)
        other = W.with_(a, **{field: P.PLAIN_FP64 if field == "precision" else
                              (1 if field == "junction_rule" else (0.5 * v if v else 0.1))})
        assert ws([a]) + ws([other]) - ws([a, other]) == head, field
    for field, value in (("f0", 3.0), ("seed", 99), ("noise_amp", 2e-3)):
        same = W.with_(a, **{field: value})
        assert ws([a, same]) < 2 * ws([a]) - head, field


def test_error_codes_match_the_header():
    txt = open(os.path.join(ROOT, "include", "epd_lb.h")).read()
    codes = {int(v): k for k, v in re.findall(r"\b(EPD_LB_E\w+)\s*=\s*(-\d+)", txt)}
    assert codes == P.binding.ERRORS
    assert re.search(r"\bEPD_LB_OK\s*=\s*0\b", txt) and P.binding.EPD_LB_OK == 0


def test_params_struct_matches_the_header():
    # field names, order and types of epd_lb_params against the ctypes mirror
    import ctypes

    txt = open(os.path.join(ROOT, "include", "epd_lb.h")).read()
    body = re.search(r"typedef struct epd_lb_params \{(.*?)\} epd_lb_params;", txt, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    ctype = {"int32_t": ctypes.c_int32, "double": ctypes.c_double, "uint64_t": ctypes.c_uint64}
    want = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        t, names = decl.split(None, 1)
        want += [(n.strip(), ctype[t]) for n in names.split(",")]
    assert [(n, t) for n, t in P.binding.CParams._fields_] == want


def test_binding_signatures_match_the_header():
    # every prototype's parameter count and kinds (pointer or the scalar
    # type) against the argtypes and restype the binding declares
    import ctypes

    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "epd_lb.h")).read(), flags=re.S)
    protos = re.findall(r"(int32_t|int|void|const char\s*\*)\s*(epd_\w+)\s*\(([^)]*)\)\s*;", txt)
    assert len(protos) == len(declared_symbols())
    scalar = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "size_t": ctypes.c_size_t,
              "double": ctypes.c_double, "float": ctypes.c_float}
    L = P.lib()
    for ret, name, params in protos:
        fn = getattr(L, name)
        params = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        assert len(fn.argtypes) == len(params), name
        for p, a in zip(params, fn.argtypes):
            if "*" in p:
                assert a in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(a, "_type_") and issubclass(a, ctypes._Pointer), (name, p, a)
            else:
                base = p.split()[0]
                assert ctypes.sizeof(a) == ctypes.sizeof(scalar[base]) and (a in (ctypes.c_double, ctypes.c_float)) == (base in ("double", "float")), (name, p, a)
        if ret == "void":
            assert fn.restype is None, name
        elif "char" in ret:
            assert fn.restype is ctypes.c_char_p, name
        else:
            assert ctypes.sizeof(fn.restype) == 4, name
