"""GB300 (sm_103a) hybrid Lattice-Boltzmann / External-Potential-Dynamics
time stepper (Heuser, Sevink and Schmid, arXiv:1804.02883).

The compute path is the CUDA library ``libepd_lb.so`` behind the C ABI of
``include/epd_lb.h``; this package is its ctypes binding plus the workload
presets.  PyTorch provides device memory and streams only.
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
