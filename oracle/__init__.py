"""FP64 CPU oracle for the hybrid LB/EPD time step -- TEST INFRASTRUCTURE ONLY.

This package wraps ``epd_lb_oracle.c`` (plain C, FP64) with ctypes.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product path (``paper_1804_02883_gb300``) never does, and the
oracle imports nothing from the product.

Each function cites the passage of Heuser, Sevink and Schmid, arXiv:1804.02883
that it restates; the readings taken where the paper is silent are documented
in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epd_lb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libepd_lb_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no SIMD flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("ns", ctypes.c_int32), ("junction_rule", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("rg", ctypes.c_double),
        ("n_seg", ctypes.c_double), ("f_a", ctypes.c_double), ("phi_p", ctypes.c_double),
        ("chi_ab", ctypes.c_double), ("chi_as", ctypes.c_double), ("chi_bs", ctypes.c_double),
        ("kappa_h", ctypes.c_double), ("d_s", ctypes.c_double), ("d_p", ctypes.c_double),
        ("inv_beta_v", ctypes.c_double), ("gamma_s", ctypes.c_double), ("gamma_b", ctypes.c_double),
        ("gamma_g", ctypes.c_double), ("f0", ctypes.c_double), ("noise_amp", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


@dataclass
class Params:
    """Problem parameters; defaults are the paper's set (Sec. 3): N = 17,
    kappa_H = 1.176, chi_AB = 1.05, chi_AS = 1.20, chi_BS = 0.75, D_S = 1,
    D_P = D_S/N, dx = R_G/3, dt = 0.002 tau.  LB in lattice units with
    gamma_s = gamma_b = gamma_g = 0; f0 in units of f* = rho R_G / tau^2."""
    nx: int = 64
    ny: int = 64
    ns: int = 32
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
    # field at the A/B junction node: 0 literal (node j carries omega_A iff
    # j < N_A), 1 segment-symmetric (both half-steps of an interval use its
    # block's field)
    junction_rule: int = 0

    def c(self) -> _Params:
        p = _Params()
        for f in fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p

    @property
    def n(self) -> int:
        return self.nx * self.ny


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        P = ctypes.POINTER(_Params)
        sig = {
            "or_dft_naive": (None, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
            "or_fft1d": (None, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
            "or_fft2d": (None, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "or_spectral_op": (None, [P, _DP, _DP, ctypes.c_int, ctypes.c_int]),
            "or_n_a": (ctypes.c_int, [P]),
            "or_propagate": (None, [P, _DP, _DP, _DP, _DP, _DP]),
            "or_solve": (None, [P, _DP, _DP, _DP]),
            "or_mu": (None, [P, _DP, _DP, _DP]),
            "or_aux_convection": (None, [P, _DP, _DP, _DP]),
            "or_diffusion_update": (None, [P, _DP, _DP, _DP]),
            "or_fstar_lattice": (ctypes.c_double, [P]),
            "or_force": (None, [P, _DP, _DP]),
            "or_poiseuille_force": (ctypes.c_double, [P, ctypes.c_int]),
            "or_eta": (ctypes.c_double, [P]),
            "or_lb_step": (None, [P, _DP, _DP, _DP]),
            "or_splitmix64": (ctypes.c_uint64, [ctypes.c_uint64]),
            "or_noise": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_uint64]),
            "or_flow_profile": (ctypes.c_double, [P, ctypes.c_double]),
            "or_discrete_profile": (ctypes.c_double, [P, ctypes.c_int]),
            "or_init": (None, [P, _DP, _DP, _DP]),
            "or_step": (None, [P, _DP, _DP, _DP, _DP, _DP, _DP, _DP]),
            "or_sigma": (ctypes.c_double, [P, _DP]),
            "or_convect_phi": (None, [P, _DP, _DP, _DP]),
            "or_invert": (ctypes.c_int, [P, _DP, _DP, _DP, _DP, ctypes.c_int, ctypes.c_double, _DP]),
            "or_step_exact": (None, [P, _DP, _DP, _DP, _DP, _DP, _DP, ctypes.c_int, ctypes.c_double, _DP]),
            "or_sigma_delta": (ctypes.c_double, [P, _DP, _DP]),
            "or_fft3d": (None, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "or_solve3d": (None, [P, ctypes.c_int, _DP, _DP, _DP]),
            "or_lb3d_step": (None, [P, ctypes.c_int, _DP, _DP, _DP]),
            "or_spectral_op3d": (None, [P, ctypes.c_int, _DP, _DP, ctypes.c_int]),
            "or_force3d": (None, [P, ctypes.c_int, _DP, _DP]),
            "or_step3d": (None, [P, ctypes.c_int, _DP, _DP, _DP, _DP, _DP, _DP]),
            "or_width": (ctypes.c_double, [P, _DP]),
            "or_particles": (ctypes.c_int, [P, _DP, ctypes.c_double, ctypes.POINTER(ctypes.c_int), _DP, ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --- FFT ------------------------------------------------------------------

def fft1d(x, sign: int = -1) -> np.ndarray:
    """Radix-2 FFT (no normalisation); sign -1 forward, +1 backward."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    lib().or_fft1d(a.ctypes.data, a.size, sign)
    return a


def dft_naive(x, sign: int = -1) -> np.ndarray:
    """O(n^2) DFT summed in long double."""
    a = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(a)
    lib().or_dft_naive(a.ctypes.data, out.ctypes.data, a.size, sign)
    return out


def fft2d(x, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    lib().or_fft2d(a.ctypes.data, a.shape[0], a.shape[1], sign)
    return a


def spectral_op(p: Params, f, axis: int, order: int) -> np.ndarray:
    """axis 0/1 with order 1: d/dx, d/dy; order 2: second derivative;
    axis 2: Laplacian.  Spectral, continuum wavenumbers."""
    f = _f64(f).reshape(p.ny, p.nx)
    out = np.empty_like(f)
    lib().or_spectral_op(ctypes.byref(p.c()), _d(f), _d(out), axis, order)
    return out


# --- single-chain statistics (Sec. 2, Eqs. (6)-(11)) -----------------------

def n_a(p: Params) -> int:
    return lib().or_n_a(ctypes.byref(p.c()))


def propagate(p: Params, w_a, w_b, g0=None):
    """Histories (ns+1, ny, nx) of g (Eq. (6)) and g' (Eq. (7))."""
    w_a = _f64(w_a).reshape(p.ny, p.nx)
    w_b = _f64(w_b).reshape(p.ny, p.nx)
    g = np.empty((p.ns + 1, p.ny, p.nx))
    gp = np.empty_like(g)
    g0p = None if g0 is None else _d(_f64(g0).reshape(p.ny, p.nx))
    lib().or_propagate(ctypes.byref(p.c()), _d(w_a), _d(w_b), g0p, _d(g), _d(gp))
    return g, gp


def solve(p: Params, omega):
    """Densities Phi (3, ny, nx) and (Q_P, Q_S) for fields omega (3, ny, nx)."""
    omega = _f64(omega).reshape(3, p.ny, p.nx)
    phi = np.empty_like(omega)
    q = np.empty(2)
    lib().or_solve(ctypes.byref(p.c()), _d(omega), _d(phi), _d(q))
    return phi, q


def fft3d(x, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    nz, ny, nx = a.shape
    lib().or_fft3d(a.ctypes.data_as(ctypes.c_void_p), nz, ny, nx, sign)
    return a


def solve3d(p: Params, nz: int, omega):
    """Densities Phi (3, nz, ny, nx) and (Q_P, Q_S) of the 3D single-chain
    solve for fields omega (3, nz, ny, nx)."""
    omega = _f64(omega).reshape(3, nz, p.ny, p.nx)
    phi = np.empty_like(omega)
    q = np.empty(2)
    lib().or_solve3d(ctypes.byref(p.c()), int(nz), _d(omega), _d(phi), _d(q))
    return phi, q


# --- EPD dynamics (Sec. 2, Eqs. (1), (5); App. C) --------------------------

def mu(p: Params, phi, omega) -> np.ndarray:
    phi = _f64(phi).reshape(3, p.ny, p.nx)
    omega = _f64(omega).reshape(3, p.ny, p.nx)
    out = np.empty_like(phi)
    lib().or_mu(ctypes.byref(p.c()), _d(phi), _d(omega), _d(out))
    return out


def aux_convection(p: Params, omega, vel_lat) -> np.ndarray:
    omega = _f64(omega).reshape(3, p.ny, p.nx)
    vel = _f64(vel_lat).reshape(2, p.ny, p.nx)
    out = np.empty_like(omega)
    lib().or_aux_convection(ctypes.byref(p.c()), _d(omega), _d(vel), _d(out))
    return out


def diffusion_update(p: Params, omega_tilde, mu_) -> np.ndarray:
    wt = _f64(omega_tilde).reshape(3, p.ny, p.nx)
    m = _f64(mu_).reshape(3, p.ny, p.nx)
    out = np.empty_like(wt)
    lib().or_diffusion_update(ctypes.byref(p.c()), _d(wt), _d(m), _d(out))
    return out


def fstar_lattice(p: Params) -> float:
    return lib().or_fstar_lattice(ctypes.byref(p.c()))


def force(p: Params, dphi) -> np.ndarray:
    """Polymer force (2, ny, nx) in lattice units from dPhi^D (3, ny, nx)."""
    dphi = _f64(dphi).reshape(3, p.ny, p.nx)
    out = np.empty((2, p.ny, p.nx))
    lib().or_force(ctypes.byref(p.c()), _d(dphi), _d(out))
    return out


# --- LB (Sec. 2, Eqs. (12), (14)-(16)) -------------------------------------

def poiseuille_force(p: Params, y: int) -> float:
    return lib().or_poiseuille_force(ctypes.byref(p.c()), y)


def eta(p: Params) -> float:
    return lib().or_eta(ctypes.byref(p.c()))


def lb_step(p: Params, pop, force_total):
    """One collide+stream.  Returns (new populations, velocity at collision)."""
    pop = _f64(pop).reshape(9, p.ny, p.nx).copy()
    f = _f64(force_total).reshape(2, p.ny, p.nx)
    vel = np.empty((2, p.ny, p.nx))
    lib().or_lb_step(ctypes.byref(p.c()), _d(pop), _d(f), _d(vel))
    return pop, vel


D3Q19_C = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
                    (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
D3Q19_W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def lb3d_step(p: Params, nz: int, pop, force_total):
    """One D3Q19 collide+stream on an nz x ny x nx box: (populations at t+1
    (19, nz, ny, nx), velocity at the collision (3, nz, ny, nx))."""
    pop = _f64(pop).reshape(19, nz, p.ny, p.nx).copy()
    f = _f64(force_total).reshape(3, nz, p.ny, p.nx)
    vel = np.empty((3, nz, p.ny, p.nx))
    lib().or_lb3d_step(ctypes.byref(p.c()), int(nz), _d(pop), _d(f), _d(vel))
    return pop, vel


def spectral_op3d(p: Params, nz: int, f, op: int) -> np.ndarray:
    """op 0, 1, 2: d/dx, d/dy, d/dz; op 3: the Laplacian, of a real (nz, ny, nx) field."""
    f = _f64(f).reshape(nz, p.ny, p.nx)
    out = np.empty_like(f)
    lib().or_spectral_op3d(ctypes.byref(p.c()), int(nz), _d(f), _d(out), int(op))
    return out


def force3d(p: Params, nz: int, dphi) -> np.ndarray:
    dphi = _f64(dphi).reshape(3, nz, p.ny, p.nx)
    out = np.empty((3, nz, p.ny, p.nx))
    lib().or_force3d(ctypes.byref(p.c()), int(nz), _d(dphi), _d(out))
    return out


def step3d(p: Params, nz: int, omega, pop, vel):
    """One coupled step on the 3D box: (omega, pop, vel, phi, q, force), all new arrays."""
    omega = _f64(omega).reshape(3, nz, p.ny, p.nx).copy()
    pop = _f64(pop).reshape(19, nz, p.ny, p.nx).copy()
    vel = _f64(vel).reshape(3, nz, p.ny, p.nx).copy()
    phi = np.empty_like(omega)
    force = np.empty_like(vel)
    q = np.empty(2)
    lib().or_step3d(ctypes.byref(p.c()), int(nz), _d(omega), _d(pop), _d(vel), _d(phi), _d(q), _d(force))
    return omega, pop, vel, phi, q, force


def flow_profile(p: Params, y: float) -> float:
    return lib().or_flow_profile(ctypes.byref(p.c()), float(y))


def discrete_profile(p: Params, y: int) -> float:
    return lib().or_discrete_profile(ctypes.byref(p.c()), int(y))


# --- initial state and the coupled step (Sec. 3, Sec. 4, App. C) -----------

def splitmix64(x: int) -> int:
    return lib().or_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF))


def noise(seed: int, counter: int) -> float:
    return lib().or_noise(seed, counter)


def init(p: Params):
    """(omega (3,ny,nx), pre-collision populations (9,ny,nx), velocity (2,ny,nx))."""
    omega = np.empty((3, p.ny, p.nx))
    pop = np.empty((9, p.ny, p.nx))
    vel = np.empty((2, p.ny, p.nx))
    lib().or_init(ctypes.byref(p.c()), _d(omega), _d(pop), _d(vel))
    return omega, pop, vel


@dataclass
class State:
    omega: np.ndarray
    pop: np.ndarray
    vel: np.ndarray
    phi: np.ndarray
    q: np.ndarray
    force: np.ndarray


def initial_state(p: Params) -> State:
    omega, pop, vel = init(p)
    phi, q = solve(p, omega)
    return State(omega, pop, vel, phi, q, np.zeros((2, p.ny, p.nx)))


def step(p: Params, st: State, nsteps: int = 1, phi_tilde_out: bool = False):
    """Advance the coupled EPD/LB state in place by nsteps steps."""
    pt = np.empty((3, p.ny, p.nx)) if phi_tilde_out else None
    for _ in range(nsteps):
        lib().or_step(ctypes.byref(p.c()), _d(st.omega), _d(st.pop), _d(st.vel), _d(st.phi),
                      _d(st.q), _d(st.force), None if pt is None else _d(pt))
    return pt


# --- the exact step: convection of Phi and the CG inversion (App. C) ------

def convect_phi(p: Params, phi, vel_lat) -> np.ndarray:
    """Phi~ = Phi - dt div(v Phi) (3, ny, nx), v = u_lat dx/dt."""
    phi = _f64(phi).reshape(3, p.ny, p.nx)
    vel = _f64(vel_lat).reshape(2, p.ny, p.nx)
    out = np.empty_like(phi)
    lib().or_convect_phi(ctypes.byref(p.c()), _d(phi), _d(vel), _d(out))
    return out


def invert(p: Params, phi_target, omega0, max_iter: int = 50, tol: float = 1e-8):
    """Fletcher-Reeves inversion Phi(omega) = phi_target from omega0.
    Returns (omega, Phi(omega), (Q_P, Q_S), iterations, residual before, after)."""
    target = _f64(phi_target).reshape(3, p.ny, p.nx)
    omega = _f64(omega0).reshape(3, p.ny, p.nx).copy()
    phi = np.empty_like(omega)
    q = np.empty(2)
    stats = np.empty(2)
    it = lib().or_invert(ctypes.byref(p.c()), _d(target), _d(omega), _d(phi), _d(q), int(max_iter), float(tol),
                         _d(stats))
    return omega, phi, q, it, stats[0], stats[1]


def step_exact(p: Params, st: State, nsteps: int = 1, max_iter: int = 50, tol: float = 1e-8):
    """Advance by nsteps exact steps (the inversion of App. C).  st.phi must
    hold Phi(t) on entry.  Returns the per-step (iterations, residual before,
    residual after) as an array (nsteps, 3)."""
    out = np.empty((nsteps, 3))
    for k in range(nsteps):
        stats = np.empty(3)
        lib().or_step_exact(ctypes.byref(p.c()), _d(st.omega), _d(st.pop), _d(st.vel), _d(st.phi), _d(st.q),
                            _d(st.force), int(max_iter), float(tol), _d(stats))
        out[k] = stats
    return out


def sigma(p: Params, phi) -> float:
    phi = _f64(phi).reshape(3, p.ny, p.nx)
    return lib().or_sigma(ctypes.byref(p.c()), _d(phi))


# --- analysis of Phi_P (Sec. 3, Sec. 4) ------------------------------------

def sigma_delta(p: Params, phi_a, phi_b) -> float:
    a = _f64(phi_a).reshape(3, p.ny, p.nx)
    b = _f64(phi_b).reshape(3, p.ny, p.nx)
    return lib().or_sigma_delta(ctypes.byref(p.c()), _d(a), _d(b))


def width(p: Params, phi) -> float:
    """Y_2^P of Eq. (30) (channel centres at L_y/4 and 3 L_y/4)."""
    phi = _f64(phi).reshape(3, p.ny, p.nx)
    return lib().or_width(ctypes.byref(p.c()), _d(phi))


PARTICLE_FIELDS = ("sites", "content", "cx", "cy", "gxx", "gxy", "gyy", "R", "c", "c_rel")


def particles(p: Params, phi, threshold: float = 0.5, max_out: int = 4096):
    """(labels (ny, nx) int, stats (count, 10)) of the clusters with
    Phi_P >= threshold; stats columns as in PARTICLE_FIELDS."""
    phi = _f64(phi).reshape(3, p.ny, p.nx)
    labels = np.empty((p.ny, p.nx), dtype=np.int32)
    stats = np.zeros((max_out, 10))
    cnt = lib().or_particles(ctypes.byref(p.c()), _d(phi), float(threshold),
                             labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(stats), int(max_out))
    return labels, stats[: min(cnt, max_out)].copy(), cnt
