"""Pins of the Newmark-beta oracle and of the oracle's inertia term (Sec. 4.1.2)
against closed forms."""
import dataclasses

import numpy as np

from fixtures import artery_layers, artery_tube
from oracle import newmark as N
from oracle import solid as O


def test_average_acceleration_conserves_the_oscillator_energy():
    """beta = 1/4, gamma = 1/2 on m u'' + k u = 0: 1/2 m v^2 + 1/2 k u^2 is
    invariant, even at omega dt = 2."""
    m, k = 2.0, 8.0                       # omega = 2
    _, _, e = N.sdof(m, k, 0.3, -0.7, 1.0, 1000, 0.25, 0.5)
    assert np.abs(e - e[0]).max() <= 1e-12 * e[0]


def test_average_acceleration_is_second_order():
    """Error of u(T) against u0 cos(w T) + v0 / w sin(w T) falls by ~4 when dt halves."""
    m, k, u0, v0, T = 1.0, 4.0, 1.0, 0.5, 3.0
    w = np.sqrt(k / m)
    exact = u0 * np.cos(w * T) + v0 / w * np.sin(w * T)
    errs = []
    for n in (200, 400, 800):
        u, _, _ = N.sdof(m, k, u0, v0, T / n, n, 0.25, 0.5)
        errs.append(abs(u[-1] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2


def _amplification(beta, gamma, w_dt):
    """One-step map (u, v) -> (u', v') of the oscillator (m = 1, k = w^2, dt = 1);
    the acceleration is fixed by equilibrium at every step."""
    cols = []
    for u0, v0 in ((1.0, 0.0), (0.0, 1.0)):
        u, v, _ = N.sdof(1.0, w_dt * w_dt, u0, v0, 1.0, 1, beta, gamma)
        cols.append([u[1], v[1]])
    return np.array(cols).T


def test_spectral_radius_of_the_step():
    """Unconditional stability and dissipation: rho(A) = 1 for beta = 1/4,
    gamma = 1/2; rho(A) < 1 for the paper's beta = 0.625, gamma = 1
    (gamma > 1/2, beta >= (gamma + 1/2)^2 / 4) at every omega dt."""
    for w_dt in (0.1, 1.0, 10.0, 100.0):
        r_avg = np.abs(np.linalg.eigvals(_amplification(0.25, 0.5, w_dt))).max()
        r_pap = np.abs(np.linalg.eigvals(_amplification(0.625, 1.0, w_dt))).max()
        assert abs(r_avg - 1.0) <= 1e-12
        assert r_pap < 1.0
    # and the criterion has teeth: beta = 0.05 < (gamma + 1/2)^2 / 4 with
    # gamma = 1/2 is only conditionally stable and blows up at omega dt = 10
    assert np.abs(np.linalg.eigvals(_amplification(0.05, 0.5, 10.0))).max() > 1.0


def test_the_papers_parameters_damp_the_oscillator():
    """beta = 0.625, gamma = 1: after 400 steps the energy has dropped (the
    kinetic + potential energy need not fall at every step at large omega dt)."""
    for dt in (0.05, 5.0):
        _, _, e = N.sdof(1.0, 4.0, 1.0, 0.0, dt, 400, 0.625, 1.0)
        assert e[-1] < 0.5 * e[0]


def test_update_reproduces_the_displacement_recurrence():
    """The a_n and v_n returned satisfy the Newmark displacement recurrence
    d_n = d_(n-1) + dt v_(n-1) + dt^2/2 ((1 - 2 beta) a_(n-1) + 2 beta a_n)."""
    rng = np.random.default_rng(0)
    d0, v0, a0, d1 = (rng.standard_normal(50) for _ in range(4))
    beta, gamma, dt = 0.625, 1.0, 0.01
    a1, v1, h1 = N.newmark_update(d1, d0, v0, a0, beta, gamma, dt)
    assert np.allclose(d0 + dt * v0 + 0.5 * dt * dt * ((1 - 2 * beta) * a0 + 2 * beta * a1), d1, rtol=0, atol=1e-13)
    assert np.allclose(v1, v0 + dt * ((1 - gamma) * a0 + gamma * a1), rtol=0, atol=1e-12)
    # the next step's inertia: c d_2 - h_1 is the acceleration a_2 of the recurrence
    d2 = rng.standard_normal(50)
    a2, _, _ = N.newmark_update(d2, d1, v1, a1, beta, gamma, dt)
    assert np.allclose(d2 / (beta * dt * dt) - h1, a2, rtol=1e-12, atol=1e-9)


def _translation(mesh, t):
    s = np.zeros((mesh.n_nodes, 4))
    s[:, :3] = t
    return s


def test_inertia_of_a_rigid_translation():
    """F = I and p = 0: only the inertia term acts.  With history h = c d the
    acceleration vanishes and so does the whole residual; with h = 0 the nodal
    inertial forces add up to rho c V_total t (the consistent mass matrix has
    total mass rho V)."""
    mesh = artery_tube(n_theta=16, n_z=2, length=0.125, materials=artery_layers(1.0e3, rho=1.2))
    c = 1.0 / (0.625 * 0.01 ** 2)
    P = O.Problem(mesh, O.Options(inertia_coef=c))
    t = np.array([0.01, -0.02, 0.005])
    s = _translation(mesh, t)
    R0 = P.residual(s, hist=np.tile(c * t, (mesh.n_nodes, 1)))
    assert np.abs(R0).max() <= 1e-9 * c * np.abs(t).max()
    # without Dirichlet rows every nodal force counts
    Pfree = O.Problem(dataclasses.replace(mesh, dir_mask=np.zeros_like(mesh.dir_mask)), O.Options(inertia_coef=c))
    tot = Pfree.residual(s, hist=np.zeros((mesh.n_nodes, 3)))[:, :3].sum(axis=0)
    assert np.allclose(tot, 1.2 * c * Pfree.V.sum() * t, rtol=1e-12, atol=0)
