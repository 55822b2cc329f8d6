"""Pins of the two readings of the field at the A/B junction node (Sec. 2:
omega_A for s < q_A, omega_B otherwise; the split step of Eq. (8)).

junction_rule 0 (literal): node j carries omega_A iff j < N_A.
junction_rule 1 (segment-symmetric): both half-steps of the interval
[s_j, s_{j+1}] use the field of its block, A iff j < N_A.

Pinned here: the segment-symmetric rule is exactly symmetric under reversing
the chain (A <-> B with q_A -> 1 - q_A), which the literal rule is not; for
fields uniform within each block it gives the continuum propagator at every
node; both rules keep the contour-split invariance (T4) and the exact mass
(T5); and a dense-matrix brute force with the per-interval fields."""
import numpy as np
import pytest
import scipy.linalg

import oracle as O


def fields(ny, nx, seed, amp=0.3):
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((3, ny, nx))


@pytest.mark.parametrize("ns,f_a", [(16, 0.25), (12, 0.5), (17, 0.882)])
def test_segment_symmetric_rule_is_exactly_chain_reversal_symmetric(oracle_lib, ns, f_a):
    # Reversing the chain swaps the blocks: (omega_A, omega_B, q_A) ->
    # (omega_B, omega_A, 1 - q_A) must give Phi_A <-> Phi_B and the same Q.
    # N_A' = N_s - N_A must hold for the mirrored parameter set.
    p = O.Params(nx=16, ny=8, ns=ns, f_a=f_a, phi_p=0.2, junction_rule=1)
    pm = O.Params(**{**p.__dict__, "f_a": 1.0 - f_a})
    assert O.n_a(pm) == ns - O.n_a(p)
    om = fields(p.ny, p.nx, seed=ns)
    phi, q = O.solve(p, om)
    phim, qm = O.solve(pm, om[[1, 0, 2]])
    assert abs(q[0] / qm[0] - 1) < 1e-13
    assert np.abs(phi[0] - phim[1]).max() < 1e-13 * np.abs(phi[0]).max()
    assert np.abs(phi[1] - phim[0]).max() < 1e-13 * np.abs(phi[1]).max()


def test_literal_rule_breaks_chain_reversal_symmetry(oracle_lib):
    # the same mirror test under the literal rule differs at the junction term
    p = O.Params(nx=16, ny=8, ns=16, f_a=0.25, phi_p=0.2, junction_rule=0)
    pm = O.Params(**{**p.__dict__, "f_a": 0.75})
    om = fields(p.ny, p.nx, seed=3)
    phi, _ = O.solve(p, om)
    phim, _ = O.solve(pm, om[[1, 0, 2]])
    assert np.abs(phi[0] - phim[1]).max() > 1e-6 * np.abs(phi[0]).max()


def test_segment_symmetric_block_uniform_fields_continuum(oracle_lib):
    # omega uniform within each block: the Laplacian factor is the identity
    # and the segment-symmetric rule gives the continuum propagator
    # g(s) = exp(-N int_0^s omega) at every node, junction node included
    p = O.Params(nx=8, ny=8, ns=12, f_a=0.5, phi_p=0.25, junction_rule=1)
    wa_c, wb_c = 0.31, -0.17
    wa = np.full((p.ny, p.nx), wa_c)
    wb = np.full((p.ny, p.nx), wb_c)
    g, gp = O.propagate(p, wa, wb)
    na, ds = O.n_a(p), 1.0 / p.ns
    for j in range(p.ns + 1):
        s, qa = j * ds, na * ds
        expo = wa_c * min(s, qa) + wb_c * max(0.0, s - qa)
        assert np.allclose(g[j], np.exp(-p.n_seg * expo), rtol=1e-13, atol=0)
        sp = j * ds  # g' from the B end
        expo_p = wb_c * min(sp, 1 - qa) + wa_c * max(0.0, sp - (1 - qa))
        assert np.allclose(gp[j], np.exp(-p.n_seg * expo_p), rtol=1e-13, atol=0)
    # and the literal rule does not, at and after the junction node
    g0, _ = O.propagate(O.Params(**{**p.__dict__, "junction_rule": 0}), wa, wb)
    assert abs(g0[na][0, 0] / g[na][0, 0] - 1) > 1e-3


@pytest.mark.parametrize("rule", [0, 1])
def test_split_invariance_and_mass_under_both_rules(oracle_lib, rule):
    # T4 and T5 are exact for either reading
    p = O.Params(nx=16, ny=32, ns=20, f_a=0.35, phi_p=0.15, junction_rule=rule)
    om = fields(p.ny, p.nx, seed=5, amp=0.2)
    g, gp = O.propagate(p, om[0], om[1])
    qp = g[-1].mean()
    for j in range(p.ns + 1):
        assert abs((g[j] * gp[p.ns - j]).mean() / qp - 1) < 1e-13
    phi, q = O.solve(p, om)
    assert abs(phi[0].mean() + phi[1].mean() - p.phi_p) < 1e-14
    assert abs(phi[2].mean() - (1 - p.phi_p)) < 1e-14


def test_rules_differ_only_through_the_junction(oracle_lib):
    # with omega_A = omega_B the junction node's field does not matter
    p0 = O.Params(nx=8, ny=16, ns=10, f_a=0.4, junction_rule=0)
    p1 = O.Params(**{**p0.__dict__, "junction_rule": 1})
    om = fields(p0.ny, p0.nx, seed=9)
    om[1] = om[0]
    a, qa = O.solve(p0, om)
    b, qb = O.solve(p1, om)
    assert np.abs(a - b).max() == 0 and np.all(qa == qb)
    om = fields(p0.ny, p0.nx, seed=9)
    a, _ = O.solve(p0, om)
    b, _ = O.solve(p1, om)
    assert np.abs(a - b).max() > 1e-6


@pytest.mark.parametrize("f_a", [0.5, 0.25])
def test_segment_symmetric_dense_matrix_brute_force(oracle_lib, f_a):
    # dense Laplacian from the DFT definition, exp(R_G^2 ds L) by expm, the
    # recursion with one field per interval, trapezoid sums
    p = O.Params(nx=8, ny=4, ns=4, f_a=f_a, phi_p=0.2, rg=0.9, junction_rule=1)
    n = p.n
    om = fields(p.ny, p.nx, seed=8, amp=0.4)

    def k_axis(m, nn):
        mm = m if m <= nn // 2 else m - nn
        return 2 * np.pi * mm / (nn * p.dx)

    ys, xs = np.divmod(np.arange(n), p.nx)
    lap = np.zeros((n, n))
    for my in range(p.ny):
        for mx in range(p.nx):
            kk = k_axis(mx, p.nx) ** 2 + k_axis(my, p.ny) ** 2
            ph = np.exp(2j * np.pi * (mx * xs / p.nx + my * ys / p.ny))
            lap += (-kk * np.outer(ph, ph.conj())).real / n
    ds = 1 / p.ns
    T = scipy.linalg.expm(p.rg ** 2 * ds * lap)
    na = O.n_a(p)
    wa, wb = om[0].ravel(), om[1].ravel()
    intervals = [wa if j < na else wb for j in range(p.ns)]  # of g

    def chain(flds):
        g = [np.ones(n)]
        for w in flds:
            e = np.exp(-p.n_seg * w * ds / 2)
            g.append(e * (T @ (e * g[-1])))
        return g

    g, gp = chain(intervals), chain(intervals[::-1])
    qp = g[-1].mean()
    ia = sum((0.5 if j in (0, na) else 1.0) * ds * g[j] * gp[p.ns - j] for j in range(na + 1))
    ib = sum((0.5 if j in (na, p.ns) else 1.0) * ds * g[j] * gp[p.ns - j] for j in range(na, p.ns + 1))
    phi, q = O.solve(p, om)
    assert abs(q[0] / qp - 1) < 1e-13
    assert np.abs(phi[0].ravel() - p.phi_p * ia / qp).max() < 1e-13
    assert np.abs(phi[1].ravel() - p.phi_p * ib / qp).max() < 1e-13
