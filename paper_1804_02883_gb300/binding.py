"""Thin ctypes binding of ``include/epd_lb.h`` (libepd_lb.so).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory (the workspace) and the stream.  There is no
CPU fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, fields

import numpy as np

from . import build as _build

EPD_LB_OK = 0
ERRORS = {
    -1: "EPD_LB_EINVAL",
    -2: "EPD_LB_ENOMEM",
    -3: "EPD_LB_ECUDA",
    -4: "EPD_LB_ENONFINITE",
    -5: "EPD_LB_EUNSTABLE",
    -6: "EPD_LB_ETIMEOUT",
    -7: "EPD_LB_ENOTCONV",
    -8: "EPD_LB_ETOOLARGE",
}
PLAIN_FP64 = 0
MIXED_FP32 = 1

# Exported symbols declared in include/epd_lb.h.
SYMBOLS = (
    "epd_lb_workspace_bytes", "epd_lb_init", "epd_lb_step", "epd_lb_sync", "epd_lb_densities",
    "epd_lb_velocity", "epd_lb_set_omega_async", "epd_lb_densities_async", "epd_lb_densities_dev",
    "epd_lb_velocity_dev", "epd_lb_get_state",
    "epd_lb_set_state", "epd_lb_solve", "epd_lb_observables", "epd_lb_save", "epd_lb_load",
    "epd_lb_last_error", "epd_lb_destroy", "epd_prop_solve_workspace_bytes", "epd_prop_solve",
    "epd_lb_enable_timing", "epd_lb_kernel_times", "epd_prop_solve_noalloc", "epd_lb_tiles",
    "epd_sur_num_params", "epd_sur_workspace_bytes", "epd_sur_forward", "epd_sur_tangent", "epd_sur_gradients",
    "epd_sur_train_step",
    "epd_lb_surrogate_workspace_bytes", "epd_lb_set_surrogate", "epd_lb_surrogate_stats", "epd_lb_fields_dev",
    "epd_lb_step_fields_dev",
    "epd_lb_set_inversion", "epd_lb_inversion_stats", "epd_lb_sigma_delta", "epd_lb_width", "epd_lb_particles",
    "epd_prop_solve3d_workspace_bytes", "epd_prop_solve3d", "epd_lb3d_step", "epd_step3d_workspace_bytes",
    "epd_step3d", "epd_selftest_bounded_wait",
)


class CParams(ctypes.Structure):
    """Mirror of ``epd_lb_params``."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("ns", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("rg", ctypes.c_double), ("n_seg", ctypes.c_double),
        ("f_a", ctypes.c_double), ("phi_p", ctypes.c_double), ("chi_ab", ctypes.c_double),
        ("chi_as", ctypes.c_double), ("chi_bs", ctypes.c_double), ("kappa_h", ctypes.c_double),
        ("d_s", ctypes.c_double), ("d_p", ctypes.c_double), ("inv_beta_v", ctypes.c_double),
        ("gamma_s", ctypes.c_double), ("gamma_b", ctypes.c_double), ("gamma_g", ctypes.c_double),
        ("f0", ctypes.c_double), ("noise_amp", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("junction_rule", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


@dataclass
class RunParams:
    """Parameters of one run (see ``epd_lb_params``).  Defaults: the paper's
    model set of Sec. 3 (N = 17, kappa_H = 1.176, chi_AB = 1.05,
    chi_AS = 1.20, chi_BS = 0.75, D_S = 1, D_P = D_S/N, dx = R_G/3,
    dt = 0.002 tau), LB relaxation 0 (BGK tau = 1), f0 in units of f*."""
    nx: int = 64
    ny: int = 64
    ns: int = 32
    precision: int = PLAIN_FP64
    dx: float = 1.0 / 3.0
    dt: float = 0.002
    rg: float = 1.0
    n_seg: float = 17.0
    f_a: float = 0.5
    phi_p: float = 0.3
    chi_ab: float = 1.05
    chi_as: float = 1.20
    chi_bs: float = 0.75
    kappa_h: float = 1.176
    d_s: float = 1.0
    d_p: float = 1.0 / 17.0
    inv_beta_v: float = 1.0
    gamma_s: float = 0.0
    gamma_b: float = 0.0
    gamma_g: float = 0.0
    f0: float = 0.0
    noise_amp: float = 1e-3
    seed: int = 1
    junction_rule: int = 0  # 0 literal, 1 segment-symmetric (see epd_lb_params)

    def c(self) -> CParams:
        p = CParams()
        for f in fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p

    @property
    def n(self) -> int:
        return self.nx * self.ny


_lib = None


def lib():
    """Load libepd_lb.so (building it if the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(CParams)
        vp, dp, i32, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int64
        szp = ctypes.POINTER(ctypes.c_size_t)
        sig = {
            "epd_lb_workspace_bytes": (ctypes.c_int, [P, i32, szp]),
            "epd_lb_init": (ctypes.c_int, [P, i32, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
            "epd_lb_step": (ctypes.c_int, [vp, i64]),
            "epd_lb_sync": (ctypes.c_int, [vp]),
            "epd_lb_densities": (ctypes.c_int, [vp, i32, vp, vp]),
            "epd_lb_velocity": (ctypes.c_int, [vp, i32, vp]),
            "epd_lb_set_omega_async": (ctypes.c_int, [vp, i32, vp]),
            "epd_lb_densities_async": (ctypes.c_int, [vp, i32, vp, vp]),
            "epd_lb_densities_dev": (ctypes.c_int, [vp, i32, vp, vp]),
            "epd_lb_velocity_dev": (ctypes.c_int, [vp, i32, vp]),
            "epd_lb_get_state": (ctypes.c_int, [vp, i32, vp, vp, vp]),
            "epd_lb_set_state": (ctypes.c_int, [vp, i32, vp, vp, vp]),
            "epd_lb_solve": (ctypes.c_int, [vp, i32, vp, vp, vp]),
            "epd_lb_observables": (ctypes.c_int, [vp, i32, vp]),
            "epd_lb_save": (ctypes.c_int, [vp, vp, szp]),
            "epd_lb_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
            "epd_lb_last_error": (ctypes.c_char_p, [vp]),
            "epd_lb_destroy": (None, [vp]),
            "epd_prop_solve_workspace_bytes": (ctypes.c_int, [P, szp]),
            "epd_prop_solve": (ctypes.c_int, [P, vp, vp, vp, vp, ctypes.c_size_t, vp]),
            "epd_prop_solve3d_workspace_bytes": (ctypes.c_int, [P, i32, szp]),
            "epd_prop_solve3d": (ctypes.c_int, [P, i32, vp, vp, vp, vp, ctypes.c_size_t, vp]),
            "epd_lb3d_step": (ctypes.c_int, [P, i32, vp, vp, vp, vp, vp]),
            "epd_step3d_workspace_bytes": (ctypes.c_int, [P, i32, szp]),
            "epd_selftest_bounded_wait": (ctypes.c_int, [i32, vp, vp]),
            "epd_step3d": (ctypes.c_int, [P, i32, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]),
            "epd_lb_enable_timing": (ctypes.c_int, [vp, i32]),
            "epd_lb_kernel_times": (ctypes.c_int, [vp, vp]),
            "epd_lb_tiles": (ctypes.c_int, [vp, ctypes.c_int32, vp]),
            "epd_prop_solve_noalloc": (ctypes.c_int, [P, vp, vp, vp, vp]),
            "epd_sur_num_params": (ctypes.c_int32, []),
            "epd_sur_workspace_bytes": (ctypes.c_int, [i32, i32, i32, i32, szp]),
            "epd_sur_forward": (ctypes.c_int, [P, i32, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp, ctypes.c_size_t, vp]),
            "epd_sur_tangent": (ctypes.c_int, [P, i32, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp, vp, ctypes.c_size_t,
                                               vp]),
            "epd_sur_gradients": (ctypes.c_int, [P, i32, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp, vp,
                                                 ctypes.c_size_t, vp]),
            "epd_sur_train_step": (ctypes.c_int, [P, i32, vp, vp, vp, i32, ctypes.c_float, ctypes.c_double, ctypes.c_double,
                                                  vp, vp, vp, vp, ctypes.c_size_t, vp]),
            "epd_lb_surrogate_workspace_bytes": (ctypes.c_int, [vp, szp]),
            "epd_lb_set_surrogate": (ctypes.c_int, [vp, vp, ctypes.c_double, ctypes.c_double, i32, ctypes.c_double, i32,
                                                    vp, ctypes.c_size_t]),
            "epd_lb_surrogate_stats": (ctypes.c_int, [vp, vp]),
            "epd_lb_fields_dev": (ctypes.c_int, [vp, i32, vp, vp]),
            "epd_lb_step_fields_dev": (ctypes.c_int, [vp, i32, vp, vp]),
            "epd_lb_set_inversion": (ctypes.c_int, [vp, i32, ctypes.c_double]),
            "epd_lb_inversion_stats": (ctypes.c_int, [vp, i32, vp]),
            "epd_lb_sigma_delta": (ctypes.c_int, [vp, i32, i32, vp]),
            "epd_lb_width": (ctypes.c_int, [vp, i32, vp]),
            "epd_lb_particles": (ctypes.c_int, [vp, i32, ctypes.c_double, i32, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class EpdLbError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        super().__init__(f"{where}: {ERRORS.get(code, code)} {msg}".strip())
        self.code = code


def _params_array(runs):
    arr = (CParams * len(runs))()
    for i, r in enumerate(runs):
        arr[i] = r.c()
    return arr


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --- C-ABI names -----------------------------------------------------------

def epd_lb_workspace_bytes(runs) -> int:
    n = ctypes.c_size_t()
    rc = lib().epd_lb_workspace_bytes(_params_array(runs), len(runs), ctypes.byref(n))
    if rc:
        raise EpdLbError(rc, "epd_lb_workspace_bytes")
    return n.value


def epd_prop_solve_workspace_bytes(run: RunParams) -> int:
    n = ctypes.c_size_t()
    rc = lib().epd_prop_solve_workspace_bytes(ctypes.byref(run.c()), ctypes.byref(n))
    if rc:
        raise EpdLbError(rc, "epd_prop_solve_workspace_bytes")
    return n.value


def epd_prop_solve(run: RunParams, omega_dev: int, phi_dev: int, q_dev: int, workspace_dev: int,
                   workspace_bytes: int, stream: int = 0) -> None:
    rc = lib().epd_prop_solve(ctypes.byref(run.c()), omega_dev, phi_dev, q_dev, workspace_dev, workspace_bytes, stream)
    if rc:
        raise EpdLbError(rc, "epd_prop_solve")


def epd_prop_solve3d_workspace_bytes(run: RunParams, nz: int) -> int:
    n = ctypes.c_size_t()
    rc = lib().epd_prop_solve3d_workspace_bytes(ctypes.byref(run.c()), int(nz), ctypes.byref(n))
    if rc:
        raise EpdLbError(rc, "epd_prop_solve3d_workspace_bytes")
    return n.value


def prop_solve3d(run: RunParams, omega):
    """Single-chain solve on an nz x ny x nx box (omega: (3, nz, ny, nx) host
    array): (Phi (3, nz, ny, nx), (Q_P, Q_S)).  Device memory from torch,
    synchronous."""
    import torch

    om = np.ascontiguousarray(omega, dtype=np.float64)
    nz = om.shape[1]
    assert om.shape == (3, nz, run.ny, run.nx)
    nb = epd_prop_solve3d_workspace_bytes(run, nz)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wptr = (ws.data_ptr() + 255) & ~255
    od = torch.from_numpy(om).cuda()
    pd = torch.empty_like(od)
    qd = torch.empty(2, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    rc = lib().epd_prop_solve3d(ctypes.byref(run.c()), nz, od.data_ptr(), pd.data_ptr(), qd.data_ptr(), wptr, nb,
                                st.cuda_stream)
    if rc:
        raise EpdLbError(rc, "epd_prop_solve3d")
    st.synchronize()
    return pd.cpu().numpy(), qd.cpu().numpy()


def lb3d_step(run: RunParams, pop, force):
    """One D3Q19 collide-stream on an nz x ny x nx box (pop (19, nz, ny, nx),
    force (3, nz, ny, nx), host arrays): (populations at t + 1, velocity at
    the collision).  Device memory from torch, synchronous."""
    import torch

    pin = torch.from_numpy(np.ascontiguousarray(pop, dtype=np.float64)).cuda()
    nz = pin.shape[1]
    assert pin.shape == (19, nz, run.ny, run.nx)
    fd = torch.from_numpy(np.ascontiguousarray(force, dtype=np.float64)).cuda()
    assert fd.shape == (3, nz, run.ny, run.nx)
    pout = torch.empty_like(pin)
    vel = torch.empty_like(fd)
    st = torch.cuda.current_stream()
    rc = lib().epd_lb3d_step(ctypes.byref(run.c()), nz, pin.data_ptr(), fd.data_ptr(), pout.data_ptr(), vel.data_ptr(),
                             st.cuda_stream)
    if rc:
        raise EpdLbError(rc, "epd_lb3d_step")
    st.synchronize()
    return pout.cpu().numpy(), vel.cpu().numpy()


def step3d(run: RunParams, omega, pop, vel, nsteps: int = 1):
    """nsteps coupled steps on an nz x ny x nx box from host state omega
    (3, nz, ny, nx), pop (19, nz, ny, nx, pre-collision), vel (3, nz, ny, nx):
    (omega, pop, vel, phi, q, force) after the last step.  Synchronous."""
    import torch

    om = torch.from_numpy(np.ascontiguousarray(omega, dtype=np.float64)).cuda()
    nz = om.shape[1]
    assert om.shape == (3, nz, run.ny, run.nx)
    pd = torch.from_numpy(np.ascontiguousarray(pop, dtype=np.float64)).cuda()
    vd = torch.from_numpy(np.ascontiguousarray(vel, dtype=np.float64)).cuda()
    assert pd.shape == (19, nz, run.ny, run.nx) and vd.shape == (3, nz, run.ny, run.nx)
    phi = torch.empty_like(om)
    force = torch.empty_like(vd)
    q = torch.empty(2, dtype=torch.float64, device="cuda")
    nb = ctypes.c_size_t()
    rc = lib().epd_step3d_workspace_bytes(ctypes.byref(run.c()), nz, ctypes.byref(nb))
    if rc:
        raise EpdLbError(rc, "epd_step3d_workspace_bytes")
    ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
    wptr = (ws.data_ptr() + 255) & ~255
    st = torch.cuda.current_stream()
    for _ in range(nsteps):
        rc = lib().epd_step3d(ctypes.byref(run.c()), nz, om.data_ptr(), pd.data_ptr(), vd.data_ptr(), phi.data_ptr(),
                              q.data_ptr(), force.data_ptr(), wptr, nb.value, st.cuda_stream)
        if rc:
            raise EpdLbError(rc, "epd_step3d")
    st.synchronize()
    return tuple(t.cpu().numpy() for t in (om, pd, vd, phi, q, force))


def selftest_bounded_wait(limit_ms: int = 50) -> bool:
    """Whether the cluster solve's bounded exchange wait gives up (and reports
    it) on a barrier nothing arrives on."""
    import torch

    out = np.zeros(1, dtype=np.int32)
    rc = lib().epd_selftest_bounded_wait(int(limit_ms), torch.cuda.current_stream().cuda_stream,
                                         out.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise EpdLbError(rc, "epd_selftest_bounded_wait")
    return bool(out[0])


def epd_prop_solve_noalloc(run: RunParams, omega_dev: int, phi_dev: int, q_dev: int, stream: int = 0) -> None:
    """The single-chain solve of epd_prop_solve without a workspace: its scratch
    is a fixed array inside the library (for callers that cannot allocate device
    memory at that point; see include/epd_lb.h for the size limit and the rule
    that overlapping calls race)."""
    rc = lib().epd_prop_solve_noalloc(ctypes.byref(run.c()), omega_dev, phi_dev, q_dev, stream)
    if rc:
        raise EpdLbError(rc, "epd_prop_solve_noalloc")


class EpdLb:
    """Handle over ``epd_lb_*``: a batch of runs stepped on one GPU.

    The workspace is a torch uint8 tensor on the device and the handle's
    calls are ordered on a dedicated torch stream."""

    def __init__(self, runs, device: str = "cuda"):
        import torch

        if isinstance(runs, RunParams):
            runs = [runs]
        self.runs = list(runs)
        self.torch = torch
        nbytes = epd_lb_workspace_bytes(self.runs)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = torch.cuda.Stream(device=device)
        h = ctypes.c_void_p()
        rc = lib().epd_lb_init(_params_array(self.runs), len(self.runs), aligned, nbytes,
                               self.stream.cuda_stream, ctypes.byref(h))
        if rc:
            raise EpdLbError(rc, "epd_lb_init")
        self.h = h

    # -- checked call ------------------------------------------------------
    def _ck(self, rc: int, where: str):
        if rc:
            msg = lib().epd_lb_last_error(self.h)
            raise EpdLbError(rc, where, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            lib().epd_lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n(self, run: int = 0) -> int:
        return self.runs[run].n

    def shape(self, run: int = 0):
        return self.runs[run].ny, self.runs[run].nx

    # -- the C-ABI calls ----------------------------------------------------
    def step(self, nsteps: int = 1):
        self._ck(lib().epd_lb_step(self.h, nsteps), "epd_lb_step")

    def sync(self):
        self._ck(lib().epd_lb_sync(self.h), "epd_lb_sync")

    def densities(self, run: int = 0):
        ny, nx = self.shape(run)
        phi = np.empty((3, ny, nx))
        q = np.empty(2)
        self._ck(lib().epd_lb_densities(self.h, run, _ptr(phi), _ptr(q)), "epd_lb_densities")
        return phi, q

    def velocity(self, run: int = 0):
        ny, nx = self.shape(run)
        v = np.empty((2, ny, nx))
        self._ck(lib().epd_lb_velocity(self.h, run, _ptr(v)), "epd_lb_velocity")
        return v

    def fields_dev(self, run: int, omega_dev=None, phi_dev=None):
        """omega and Phi of a run into device tensors (3, ny, nx) FP64, on the
        handle's stream."""
        self._ck(lib().epd_lb_fields_dev(self.h, run, None if omega_dev is None else omega_dev.data_ptr(),
                                         None if phi_dev is None else phi_dev.data_ptr()), "epd_lb_fields_dev")

    def step_fields_dev(self, run: int, omega_tilde_dev=None, phi_tilde_dev=None):
        """omega~ and Phi~ of the last step of a run into device tensors
        (3, ny, nx) FP64, on the handle's stream."""
        self._ck(lib().epd_lb_step_fields_dev(self.h, run, None if omega_tilde_dev is None else omega_tilde_dev.data_ptr(),
                                              None if phi_tilde_dev is None else phi_tilde_dev.data_ptr()),
                 "epd_lb_step_fields_dev")

    def densities_dev(self, run: int, phi_dev, q_dev):
        self._ck(lib().epd_lb_densities_dev(self.h, run, phi_dev.data_ptr(), q_dev.data_ptr()), "epd_lb_densities_dev")

    def velocity_dev(self, run: int, v_dev):
        self._ck(lib().epd_lb_velocity_dev(self.h, run, v_dev.data_ptr()), "epd_lb_velocity_dev")

    def get_state(self, run: int = 0):
        ny, nx = self.shape(run)
        om = np.empty((3, ny, nx))
        pop = np.empty((9, ny, nx))
        vel = np.empty((2, ny, nx))
        self._ck(lib().epd_lb_get_state(self.h, run, _ptr(om), _ptr(pop), _ptr(vel)), "epd_lb_get_state")
        return om, pop, vel

    def set_state(self, run: int, omega=None, pop=None, vel=None):
        """Replace omega, pre-collision populations and/or velocity (None keeps)."""
        args = []
        for a, k in ((omega, 3), (pop, 9), (vel, 2)):
            if a is None:
                args.append(None)
            else:
                a = np.ascontiguousarray(a, dtype=np.float64)
                assert a.size == k * self.n(run)
                args.append(a)
        ptrs = [None if a is None else _ptr(a) for a in args]
        self._ck(lib().epd_lb_set_state(self.h, run, *ptrs), "epd_lb_set_state")

    def set_state_ptr(self, run: int, omega_ptr: int, pop_ptr: int, vel_ptr: int):
        """set_state from raw host pointers (e.g. pinned torch tensors)."""
        self._ck(lib().epd_lb_set_state(self.h, run, omega_ptr, pop_ptr, vel_ptr), "epd_lb_set_state")

    def densities_ptr(self, run: int, phi_ptr: int, q_ptr: int):
        self._ck(lib().epd_lb_densities(self.h, run, phi_ptr, q_ptr), "epd_lb_densities")

    def set_omega_async(self, run: int, omega_ptr: int):
        """Enqueue omega of `run` from a host pointer (page-locked for overlap);
        the buffer must stay untouched until sync()."""
        self._ck(lib().epd_lb_set_omega_async(self.h, run, omega_ptr), "epd_lb_set_omega_async")

    def densities_async(self, run: int, phi_ptr: int, q_ptr: int):
        """Enqueue the read of Phi and Q of `run` into host pointers; valid
        after sync()."""
        self._ck(lib().epd_lb_densities_async(self.h, run, phi_ptr, q_ptr), "epd_lb_densities_async")

    def solve(self, run: int, omega):
        ny, nx = self.shape(run)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        phi = np.empty((3, ny, nx))
        q = np.empty(2)
        self._ck(lib().epd_lb_solve(self.h, run, _ptr(om), _ptr(phi), _ptr(q)), "epd_lb_solve")
        return phi, q

    def observables(self, run: int = 0) -> dict:
        out = np.empty(8)
        self._ck(lib().epd_lb_observables(self.h, run, _ptr(out)), "epd_lb_observables")
        keys = ("mean_phi_a", "mean_phi_b", "mean_phi_s", "sigma", "lb_mass", "max_u", "q_p", "q_s")
        return dict(zip(keys, out.tolist()))

    def enable_timing(self, on: bool = True):
        self._ck(lib().epd_lb_enable_timing(self.h, int(on)), "epd_lb_enable_timing")

    def kernel_times(self) -> dict:
        """Durations (ms) inside the last step: the propagator kernels of the
        second solve (the cluster-resident launch, or the row pass storing
        history, the row pass accumulating contour sums and a column pass) and
        the LB collide-stream."""
        out = np.empty(5)
        self._ck(lib().epd_lb_kernel_times(self.h, _ptr(out)), "epd_lb_kernel_times")
        if out[4] == 1.0:
            return {"prop_cluster": float(out[0]), "lb_collide_stream": float(out[3])}
        return dict(zip(("prop_row_store", "prop_row_accumulate", "prop_col", "lb_collide_stream"), out[:4].tolist()))

    def tiles(self, run: int) -> dict:
        """Launch configuration of a run's group: solve path (0 streaming
        radix-2, 1 streaming radix-8, 2 cluster), CTAs per cluster, the
        autotuned column tile widths (EPD passes; streaming propagator
        passes), whether the differential second solve is used, and the
        chain-kernel launches per cluster solve."""
        out = np.zeros(6, dtype=np.int32)
        self._ck(lib().epd_lb_tiles(self.h, run, out.ctypes.data_as(ctypes.c_void_p)), "epd_lb_tiles")
        return {"path": int(out[0]), "cluster_ctas": int(out[1]), "column_tile": int(out[2]), "differential": bool(out[3]),
                "stream_column_tile": int(out[4]), "chain_launches": int(out[5])}

    def set_surrogate(self, params, s_in: float, s_out: float, exact_every: int = 8, residual_tol: float = 0.2,
                      hold_force: bool = False):
        """Attach the learned surrogate (FP32 parameters, host array or torch
        tensor) with its workspace on the device; exact_every = 0 detaches.
        residual_tol: relative to the exact density fluctuations; hold_force:
        surrogate steps keep the last exact step's polymer force."""
        torch = self.torch
        if exact_every <= 0:
            self._ck(lib().epd_lb_set_surrogate(self.h, None, 0.0, 0.0, 0, 0.0, 0, None, 0), "epd_lb_set_surrogate")
            return
        nb = ctypes.c_size_t()
        self._ck(lib().epd_lb_surrogate_workspace_bytes(self.h, ctypes.byref(nb)), "epd_lb_surrogate_workspace_bytes")
        self.sur_workspace = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.workspace.device)
        ptr = (self.sur_workspace.data_ptr() + 255) & ~255
        hp = np.ascontiguousarray(params.detach().cpu().numpy() if hasattr(params, "detach") else params, dtype=np.float32)
        self._ck(lib().epd_lb_set_surrogate(self.h, hp.ctypes.data_as(ctypes.c_void_p), s_in, s_out, exact_every,
                                            residual_tol, int(hold_force), ptr, nb.value), "epd_lb_set_surrogate")

    def set_inversion(self, max_iter: int, tol: float = 1e-8):
        """Exact step of App. C: Fletcher-Reeves inversion of the convected
        densities with at most max_iter iterations per step down to the RMS
        residual tol (0: exactly max_iter); max_iter = 0 restores the
        truncated step."""
        self._ck(lib().epd_lb_set_inversion(self.h, int(max_iter), float(tol)), "epd_lb_set_inversion")

    def inversion_stats(self, run: int = 0) -> dict:
        """Iterations and residuals (before, after) of the last exact step."""
        out = np.empty(3)
        self._ck(lib().epd_lb_inversion_stats(self.h, run, _ptr(out)), "epd_lb_inversion_stats")
        return {"iterations": int(out[0]), "residual0": float(out[1]), "residual": float(out[2])}

    def sigma_delta(self, run_a: int, run_b: int) -> float:
        """sigma_Delta of Eq. (22) between two runs on the same grid."""
        out = np.empty(1)
        self._ck(lib().epd_lb_sigma_delta(self.h, run_a, run_b, _ptr(out)), "epd_lb_sigma_delta")
        return float(out[0])

    def width(self, run: int = 0) -> float:
        """Y_2^P of Eq. (30)."""
        out = np.empty(1)
        self._ck(lib().epd_lb_width(self.h, run, _ptr(out)), "epd_lb_width")
        return float(out[0])

    PARTICLE_FIELDS = ("sites", "content", "cx", "cy", "gxx", "gxy", "gyy", "R", "c", "c_rel")

    def particles(self, run: int = 0, threshold: float = 0.5, max_particles: int = 4096, labels: bool = False):
        """(count, stats (min(count, max_particles), 10), labels (ny, nx) or
        None) of the clusters with Phi_P >= threshold; columns as in
        PARTICLE_FIELDS."""
        ny, nx = self.shape(run)
        cnt = np.zeros(1, dtype=np.int32)
        st = np.zeros((max(max_particles, 1), 10))
        lab = np.empty((ny, nx), dtype=np.int32) if labels else None
        self._ck(lib().epd_lb_particles(self.h, run, float(threshold), int(max_particles),
                                        cnt.ctypes.data_as(ctypes.c_void_p), st.ctypes.data_as(ctypes.c_void_p),
                                        None if lab is None else lab.ctypes.data_as(ctypes.c_void_p)),
                 "epd_lb_particles")
        c = int(cnt[0])
        return c, st[: min(c, max_particles)].copy(), lab

    def surrogate_stats(self) -> dict:
        out = np.empty(6)
        self._ck(lib().epd_lb_surrogate_stats(self.h, _ptr(out)), "epd_lb_surrogate_stats")
        keys = ("steps", "exact", "surrogate", "forced_exact", "last_residual", "falling_back")
        return dict(zip(keys, out.tolist()))

    def save(self) -> bytes:
        n = ctypes.c_size_t()
        self._ck(lib().epd_lb_save(self.h, None, ctypes.byref(n)), "epd_lb_save")
        buf = ctypes.create_string_buffer(n.value)
        self._ck(lib().epd_lb_save(self.h, buf, ctypes.byref(n)), "epd_lb_save")
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._ck(lib().epd_lb_load(self.h, buf, len(blob)), "epd_lb_load")
