"""The input recipe of the paper's own system against the values Sec. 3
prints (tests/golden/paper_system.txt): the default run parameters and the
150 x 150 ensemble workload."""
import os

import pytest

from paper_1804_02883_gb300 import binding as B
from paper_1804_02883_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_system.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_default_parameters_are_the_papers():
    g = _golden()
    r = B.RunParams()
    assert r.n_seg == g["n_seg"] and r.kappa_h == g["kappa_h"]
    assert (r.chi_ab, r.chi_as, r.chi_bs) == (g["chi_ab"], g["chi_as"], g["chi_bs_droplet"])
    assert r.d_p / r.d_s == pytest.approx(g["d_p_over_d_s"], rel=1e-15)
    assert r.dx / r.rg == pytest.approx(g["dx_over_rg"], rel=1e-15) and r.dt == g["dt_over_tau"]
    # R_g / c, c = dx / dt the lattice velocity: about 0.006 tau
    assert r.rg / (r.dx / r.dt) == pytest.approx(g["rg_over_c"], abs=5e-4)


def test_paper_ensemble_workload():
    g = _golden()
    runs = W.paper_150(B.MIXED_FP32)
    assert g["box_over_rg"] / g["dx_over_rg"] == pytest.approx(g["sites_per_axis"])
    assert {(r.nx, r.ny) for r in runs} == {(int(g["sites_per_axis"]),) * 2}
    assert all(r.ns == g["n_seg"] and r.n_seg == g["n_seg"] for r in runs)
    assert all(r.f_a == g["q_a"] and r.phi_p == g["mean_phi_p"] for r in runs)
    chis = sorted({r.chi_bs for r in runs})
    assert chis == [g["chi_bs_vesicle"], g["chi_bs_droplet"]]
    assert sum(r.chi_bs == g["chi_bs_droplet"] for r in runs) == len(runs) // 2
    assert len({r.seed for r in runs}) == len(runs)  # the noise differs from run to run
