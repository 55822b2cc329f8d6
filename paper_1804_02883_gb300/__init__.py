"""GB300 (sm_103a) hybrid Lattice-Boltzmann / External-Potential-Dynamics
time stepper (Heuser, Sevink and Schmid, arXiv:1804.02883).

The compute path is the CUDA library ``libepd_lb.so`` behind the C ABI of
``include/epd_lb.h``; this package is its ctypes binding plus the workload
presets.  PyTorch provides device memory and streams only.

    import paper_1804_02883_gb300 as P
    from paper_1804_02883_gb300 import workloads as W

    h = P.EpdLb(W.channel_256x512(P.MIXED_FP32))  # 4 runs, one batch
    h.step(100)                                   # graph-captured steps
    phi, q = h.densities(0)                       # Phi_{A,B,S}, (Q_P, Q_S)
    u = h.velocity(0)                             # LB velocity (lattice units)
    h.set_inversion(100, 1e-8)                    # the exact step of App. C
    h.step(1)
    count, stats, _ = h.particles(0, 0.5)         # clusters of Phi_P >= 0.5
    h.close()
"""
from .binding import (  # noqa: F401
    MIXED_FP32,
    PLAIN_FP64,
    SYMBOLS,
    EpdLb,
    EpdLbError,
    RunParams,
    epd_lb_workspace_bytes,
    epd_prop_solve,
    epd_prop_solve_noalloc,
    epd_prop_solve_workspace_bytes,
    epd_prop_solve3d_workspace_bytes,
    lb3d_step,
    lib,
    prop_solve3d,
    step3d,
)
