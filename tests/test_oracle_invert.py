"""Pins of the oracle's exact step of App. C: the convection of the
composition fields (the convective part of Eq. (2)), the Fletcher-Reeves
inversion omega = Phi^{-1}(Phi~) (Sec. 2, the integrator paragraph; App. C,
items 2 and 3) and the step built from them."""
import numpy as np

import oracle as O


def _grid(p):
    x = np.arange(p.nx) * p.dx
    y = np.arange(p.ny) * p.dx
    return x[None, :], y[:, None]


def test_convect_phi_uniform_flow_of_a_mode(oracle_lib):
    # uniform v: div(v Phi) = v . grad Phi, closed form for a Fourier mode
    p = O.Params(nx=16, ny=8)
    x, y = _grid(p)
    kx = 2 * np.pi * 3 / (p.nx * p.dx)
    ky = 2 * np.pi * 2 / (p.ny * p.dx)
    th = kx * x + ky * y
    amp = np.array([1e-3, -2e-3, 5e-4])
    phi = np.stack([0.1 + a * np.cos(th) for a in amp])
    ux, uy = 0.02, -0.01
    vel = np.stack([np.full((p.ny, p.nx), ux), np.full((p.ny, p.nx), uy)])
    out = O.convect_phi(p, phi, vel)
    vs = p.dx / p.dt
    for s, a in enumerate(amp):
        want = phi[s] + p.dt * a * vs * (ux * kx + uy * ky) * np.sin(th)
        assert np.abs(out[s] - want).max() < 1e-15 * 100


def test_convect_phi_is_the_flux_form(oracle_lib):
    # a compressible flow v_x = b cos(q x) over Phi(y): the advective form
    # v . grad Phi vanishes, the flux form leaves Phi div v
    p = O.Params(nx=16, ny=16)
    x, y = _grid(p)
    q = 2 * np.pi * 2 / (p.nx * p.dx)
    k = 2 * np.pi * 1 / (p.ny * p.dx)
    b = 0.01
    phi = np.stack([0.2 + 1e-3 * np.cos(k * y) + 0 * x] * 3)
    vel = np.stack([b * np.cos(q * x) + 0 * y, np.zeros((p.ny, p.nx))])
    out = O.convect_phi(p, phi, vel)
    vs = p.dx / p.dt
    want = phi + p.dt * vs * b * q * np.sin(q * x) * phi
    assert np.abs(out - want).max() < 1e-14


def test_convect_phi_conserves_each_species(oracle_lib):
    p = O.Params(nx=16, ny=32)
    rng = np.random.default_rng(3)
    phi = 0.2 + 1e-3 * rng.standard_normal((3, p.ny, p.nx))
    vel = 0.05 * rng.standard_normal((2, p.ny, p.nx))
    out = O.convect_phi(p, phi, vel)
    assert np.abs(out.mean(axis=(1, 2)) - phi.mean(axis=(1, 2))).max() < 1e-15
    assert np.abs(out - phi).max() > 1e-4  # and it does move material


def _smooth_field(p, rng, amp, modes=3):
    x, y = _grid(p)
    f = np.zeros((p.ny, p.nx))
    for _ in range(modes):
        mx, my = rng.integers(-3, 4, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        f += amp * np.cos(2 * np.pi * (mx * x / (p.nx * p.dx) + my * y / (p.ny * p.dx)) + ph)
    return f


def test_invert_recovers_the_fields_up_to_species_constants(oracle_lib):
    # Phi is unchanged by a constant shift of omega_A, omega_B or omega_S
    # alone (Q and I absorb it), and G is convex: the inverse of Phi(omega*) is
    # omega* up to those three constants
    p = O.Params(nx=16, ny=16, ns=8, phi_p=0.2)
    rng = np.random.default_rng(5)
    w_star = np.stack([_smooth_field(p, rng, 0.05) for _ in range(3)])
    phi_star, _ = O.solve(p, w_star)
    w0 = w_star + np.stack([_smooth_field(p, rng, 0.01) + c for c in (0.3, -0.2, 0.1)])
    w, phi, q, it, r0, r1 = O.invert(p, phi_star, w0, max_iter=400, tol=1e-13)
    # conjugate directions: 53 iterations here, steepest descent with the same
    # line search takes 145
    assert r0 > 1e-4 and r1 < 1e-13 and 0 < it <= 70
    dw = w - w_star
    dw -= dw.mean(axis=(1, 2), keepdims=True)
    assert np.abs(dw).max() < 1e-9
    assert np.abs(phi - phi_star).max() < 1e-12


def test_invert_at_the_solution_takes_no_iteration(oracle_lib):
    p = O.Params(nx=8, ny=8, ns=8)
    rng = np.random.default_rng(6)
    w = 0.01 * rng.standard_normal((3, p.ny, p.nx))
    phi, _ = O.solve(p, w)
    w1, phi1, q, it, r0, r1 = O.invert(p, phi, w, max_iter=10, tol=1e-8)
    assert it == 0 and r0 == 0.0 and np.array_equal(w1, w) and np.array_equal(phi1, phi)


def test_invert_with_zero_tolerance_runs_max_iter(oracle_lib):
    p = O.Params(nx=8, ny=8, ns=8)
    rng = np.random.default_rng(7)
    w = 0.01 * rng.standard_normal((3, p.ny, p.nx))
    phi, _ = O.solve(p, w)
    w0 = w + 0.001 * rng.standard_normal((3, p.ny, p.nx))
    *_, it, r0, r1 = O.invert(p, phi, w0, max_iter=3, tol=0.0)
    assert it == 3 and r1 < r0


def test_mismatch_is_the_gradient_of_the_convex_function(oracle_lib):
    # G(omega) = <sum_I omega_I Phi~_I> + (phi_p/N) ln Q_P + (1 - phi_p) ln Q_S;
    # its directional derivative along v is <(Phi~ - Phi(omega)) . v>.  Exact for
    # the solvent; for the polymer up to the split of the junction node between
    # the A and B trapezoids (a fraction of order 1/N_s of the contour sum).
    p = O.Params(nx=8, ny=8, ns=32, phi_p=0.2)
    rng = np.random.default_rng(8)
    w = 0.05 * rng.standard_normal((3, p.ny, p.nx))
    target = 0.2 + 0.01 * rng.standard_normal((3, p.ny, p.nx))

    def G(om):
        _, q = O.solve(p, om)
        return np.mean(np.sum(om * target, axis=0)) + p.phi_p / p.n_seg * np.log(q[0]) + (1 - p.phi_p) * np.log(q[1])

    phi, _ = O.solve(p, w)
    for species, tol in ((2, 1e-8), (0, 0.05), (1, 0.05)):
        v = np.zeros_like(w)
        v[species] = rng.standard_normal((p.ny, p.nx))
        h = 1e-5
        num = (G(w + h * v) - G(w - h * v)) / (2 * h)
        ana = np.mean(np.sum((target - phi) * v, axis=0))
        assert abs(num - ana) <= tol * abs(ana), (species, num, ana)


def test_exact_step_without_iterations_is_the_truncated_step(oracle_lib):
    p = O.Params(nx=16, ny=16, ns=8, f0=1e-5)
    a = O.initial_state(p)
    b = O.initial_state(p)
    for _ in range(2):
        O.step(p, a)
        st = O.step_exact(p, b, max_iter=0)
        assert st[0, 0] == 0
    for f in ("omega", "pop", "vel", "phi", "q", "force"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_exact_step_converges_and_keeps_masses(oracle_lib):
    # the first step's flow is the x-independent channel profile, which the
    # auxiliary convection of omega follows almost exactly; the second step
    # carries the polymer-driven flow and needs the iteration
    p = O.Params(nx=32, ny=32, ns=16, phi_p=0.2, f0=5e-4, noise_amp=0.05)
    st = O.initial_state(p)
    stats = O.step_exact(p, st, nsteps=2, max_iter=50, tol=1e-8)
    assert np.all(stats[:, 2] < 1e-8) and np.all(stats[:, 0] < 50)
    it, r0, r1 = stats[1]
    assert r0 > 1e-6 and it >= 3
    na = O.n_a(p)
    means = st.phi.mean(axis=(1, 2))
    assert abs(means[0] - p.phi_p * na / p.ns) < 1e-14
    assert abs(means[1] - p.phi_p * (1 - na / p.ns)) < 1e-14
    assert abs(means[2] - (1 - p.phi_p)) < 1e-14
